// decode.cu -- the steps just upstream of the march that turn decoder output into
// march inputs, and their gradients: the opacity fade factor (Sec. 3.1.3), the
// assembly of a view's payload from view-dependent colour and opacity (Sec. 3.1.3),
// rotations from axis-angle (Rodrigues) vectors (Sec. 3.1.2), and the volume
// minimisation prior (Sec. 3.3).
#include "pack.cuh"

namespace mvp {

// Opacity fade W(x,y,z) = exp(-alpha (x^beta + y^beta + z^beta)) at voxel (i, j, l) of an
// M^3 payload, (x, y, z) = 2 (i, j, l)/(M - 1) - 1 (corner-aligned voxel coordinates).
// Integer beta >= 0 is applied by repeated squaring.
__device__ __forceinline__ float ipow(float x, int b) {
  float r = 1.0f;
  while (b > 0) {
    if (b & 1) r *= x;
    x *= x;
    b >>= 1;
  }
  return r;
}

// W at voxel position v of an M^3 grid.
__device__ __forceinline__ float fade_weight(int v, int M, float alpha, int beta) {
  const int x = v % M, y = (v / M) % M, z = v / (M * M);
  const float h = 2.0f / (float)(M - 1);
  const float fx = fmaf((float)x, h, -1.0f), fy = fmaf((float)y, h, -1.0f), fz = fmaf((float)z, h, -1.0f);
  return expf(-alpha * (ipow(fx, beta) + ipow(fy, beta) + ipow(fz, beta)));
}

// Voxel i of a payload in type DT (round to nearest even).
template <int DT>
__device__ __forceinline__ void store_voxel(void *dst, int64_t i, float4 c) {
  if (DT == MVP_F32) {
    reinterpret_cast<float4 *>(dst)[i] = c;
  } else if (DT == MVP_BF16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(c.x, c.y), b = __floats2bfloat162_rn(c.z, c.w);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t *>(&a);
    o.y = *reinterpret_cast<uint32_t *>(&b);
    reinterpret_cast<uint2 *>(dst)[i] = o;
  } else {
    __half2 a = __floats2half2_rn(c.x, c.y), b = __floats2half2_rn(c.z, c.w);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t *>(&a);
    o.y = *reinterpret_cast<uint32_t *>(&b);
    reinterpret_cast<uint2 *>(dst)[i] = o;
  }
}

// One thread per voxel position v of the M^3 grid (blockIdx.x) computes W once and
// applies it to voxel v of primitives blockIdx.y, blockIdx.y + gridDim.y, ... src and
// dst may be the same buffer (dst FP32): each element is read, then written, by one
// thread.
template <int DT>
__global__ void __launch_bounds__(256) k_fade(const float4 *src, void *dst, int64_t n_prims, int M, float alpha,
                                              int beta) {
  const int M3 = M * M * M;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= M3) return;
  const float w = fade_weight(v, M, alpha, beta);
  for (int64_t k = blockIdx.y; k < n_prims; k += gridDim.y) {
    const int64_t i = k * M3 + v;
    float4 c = src[i];
    c.w *= w;
    store_voxel<DT>(dst, i, c);
  }
}

// A view's payload: voxel i = (rgb[i], alpha[i] W) from the view-dependent colour
// [n][M^3][3] and the view-independent opacity [n][M^3], same grid as k_fade.
template <int DT>
__global__ void __launch_bounds__(256) k_assemble(const float *__restrict__ rgb, const float *__restrict__ op,
                                                  void *__restrict__ dst, int64_t n_prims, int M, float alpha,
                                                  int beta) {
  const int M3 = M * M * M;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= M3) return;
  const float w = fade_weight(v, M, alpha, beta);
  for (int64_t k = blockIdx.y; k < n_prims; k += gridDim.y) {
    const int64_t i = k * M3 + v;
    const float4 c = make_float4(__ldg(rgb + 3 * i), __ldg(rgb + 3 * i + 1), __ldg(rgb + 3 * i + 2), __ldg(op + i) * w);
    store_voxel<DT>(dst, i, c);
  }
}

// sin(theta/2)/theta and (d/dtheta of it)/theta, with series near 0.
__device__ __forceinline__ void rodrigues_terms(float th2, float &c, float &f, float &g) {
  const float th = sqrtf(th2);
  if (th < 1.0e-3f) {
    c = 1.0f - th2 * 0.125f;
    f = 0.5f - th2 * (1.0f / 48.0f);
    g = -1.0f / 24.0f + th2 * (1.0f / 960.0f);
  } else {
    float sh, ch;
    sincosf(0.5f * th, &sh, &ch);
    c = ch;
    f = sh / th;
    g = (0.5f * th * ch - sh) / (th2 * th);
  }
}

// q = (cos(theta/2), sin(theta/2) r/theta), theta = |r|.
__global__ void k_aa_to_quat(const float *__restrict__ r, int n, float *__restrict__ q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float rx = r[3 * k], ry = r[3 * k + 1], rz = r[3 * k + 2];
  float c, f, g;
  rodrigues_terms(rx * rx + ry * ry + rz * rz, c, f, g);
  q[4 * k] = c;
  q[4 * k + 1] = f * rx;
  q[4 * k + 2] = f * ry;
  q[4 * k + 3] = f * rz;
}

// g_r += (dq/dr)^T g_q: dq_w/dr = -(f/2) r, dq_v/dr = f I + g r r^T.
__global__ void k_aa_vjp(const float *__restrict__ r, const float *__restrict__ gq, int n, float *__restrict__ gr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float rx = r[3 * k], ry = r[3 * k + 1], rz = r[3 * k + 2];
  float c, f, g;
  rodrigues_terms(rx * rx + ry * ry + rz * rz, c, f, g);
  const float gw = gq[4 * k], gx = gq[4 * k + 1], gy = gq[4 * k + 2], gz = gq[4 * k + 3];
  const float dot = gx * rx + gy * ry + gz * rz;
  const float a = -0.5f * f * gw + g * dot;
  gr[3 * k] += a * rx + f * gx;
  gr[3 * k + 1] += a * ry + f * gy;
  gr[3 * k + 2] += a * rz + f * gz;
}

// L_vol = lambda sum_k prod_j (2 s_kj) (side lengths = twice the half extents);
// dL/ds_kj = 2 lambda prod_{m != j} (2 s_km).
__global__ void __launch_bounds__(256) k_volume_prior(const float *__restrict__ s, int n, float lambda,
                                                      float *__restrict__ loss, float *__restrict__ gs) {
  __shared__ float part[8];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.0f;
  if (k < n) {
    const float a = 2.0f * s[3 * k], b = 2.0f * s[3 * k + 1], c = 2.0f * s[3 * k + 2];
    v = lambda * a * b * c;
    if (gs) {
      gs[3 * k] += 2.0f * lambda * b * c;
      gs[3 * k + 1] += 2.0f * lambda * a * c;
      gs[3 * k + 2] += 2.0f * lambda * a * b;
    }
  }
  if (!loss) return;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float w = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
    w = warp_sum(w);
    if (threadIdx.x == 0) atomicAdd(loss, w);
  }
}

// Voxel-position blocks in x; enough blocks in y to fill the GPU several times over,
// each looping over primitives.
static dim3 voxel_grid(int64_t n_prims, int M) {
  const int M3 = M * M * M;
  const unsigned gx = (unsigned)((M3 + 255) / 256);
  const int64_t want = (4 * 152 * 8 + gx - 1) / gx;
  return dim3(gx, (unsigned)(n_prims < want ? n_prims : (want > 65535 ? 65535 : want)));
}

cudaError_t launch_fade(const float *src, void *dst, int64_t n_prims, int M, int dtype, float alpha, int beta,
                        cudaStream_t st) {
  if (n_prims <= 0) return cudaSuccess;
  const dim3 grid = voxel_grid(n_prims, M);
  const float4 *s4 = reinterpret_cast<const float4 *>(src);
  if (dtype == MVP_F32) k_fade<MVP_F32><<<grid, 256, 0, st>>>(s4, dst, n_prims, M, alpha, beta);
  else if (dtype == MVP_BF16) k_fade<MVP_BF16><<<grid, 256, 0, st>>>(s4, dst, n_prims, M, alpha, beta);
  else k_fade<MVP_F16><<<grid, 256, 0, st>>>(s4, dst, n_prims, M, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const float *rgb, const float *op, void *dst, int64_t n_prims, int M, int dtype,
                            float alpha, int beta, cudaStream_t st) {
  if (n_prims <= 0) return cudaSuccess;
  const dim3 grid = voxel_grid(n_prims, M);
  if (dtype == MVP_F32) k_assemble<MVP_F32><<<grid, 256, 0, st>>>(rgb, op, dst, n_prims, M, alpha, beta);
  else if (dtype == MVP_BF16) k_assemble<MVP_BF16><<<grid, 256, 0, st>>>(rgb, op, dst, n_prims, M, alpha, beta);
  else k_assemble<MVP_F16><<<grid, 256, 0, st>>>(rgb, op, dst, n_prims, M, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_aa_to_quat(const float *r, int n, float *q, cudaStream_t st) {
  if (n > 0) k_aa_to_quat<<<(n + 255) / 256, 256, 0, st>>>(r, n, q);
  return cudaGetLastError();
}

cudaError_t launch_aa_vjp(const float *r, const float *gq, int n, float *gr, cudaStream_t st) {
  if (n > 0) k_aa_vjp<<<(n + 255) / 256, 256, 0, st>>>(r, gq, n, gr);
  return cudaGetLastError();
}

cudaError_t launch_volume_prior(const float *s, int n, float lambda, float *loss, float *gs, cudaStream_t st) {
  if (n > 0) k_volume_prior<<<(n + 255) / 256, 256, 0, st>>>(s, n, lambda, loss, gs);
  return cudaGetLastError();
}

}  // namespace mvp
