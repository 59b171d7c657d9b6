// bvh.cu -- per-frame LBVH over oriented primitives (Sec. 3.2.1: the paper rebuilds
// a data-parallel BVH every frame because the primitives move; it cites Karras'
// construction from sorted Morton codes).
//
// Steps, all on one stream without host synchronisation:
//   1. k_bounds   : min/max of the centres (one block; exact).
//   2. k_prims    : rotation, membership pose, march transform, oriented-box world
//                   bounds, 30-bit Morton code of the centre.
//   3. radix sort : stable LSD sort of the 30-bit codes with the primitive index as
//                   value (4 passes of 8 bits: count, scan, scatter).
//   4. k_hierarchy: leaves and internal nodes of the binary radix tree over the
//                   unique keys (morton << 32 | k), one thread per node.
//   5. k_refit    : bottom-up union of child boxes with per-node arrival counters.
#include "bvh.cuh"

namespace mvp {

// ------------------------------------------------------------------ 1. bounds
__global__ void __launch_bounds__(1024) k_bounds(const float *__restrict__ t, int n, float *__restrict__ scene) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float v = t[3 * k + j];
      lo[j] = fminf(lo[j], v);
      hi[j] = fmaxf(hi[j], v);
    }
  }
  __shared__ float s[32][6];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lo[j] = warp_min(lo[j]);
    hi[j] = warp_max(hi[j]);
  }
  if (lane == 0)
    for (int j = 0; j < 3; ++j) { s[warp][j] = lo[j]; s[warp][3 + j] = hi[j]; }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float a = lane < nw ? s[lane][j] : INFINITY;
      float b = lane < nw ? s[lane][3 + j] : -INFINITY;
      a = warp_min(a);
      b = warp_max(b);
      if (lane == 0) { scene[j] = a; scene[3 + j] = b; }
    }
  }
}

// ------------------------------------------------------------------ 2. primitives
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Quantise one axis: u = (v - lo)/(hi - lo) (0 if hi == lo), q = min(floor(u*1024), 1023).
__device__ __forceinline__ uint32_t quant10(float v, float lo, float hi) {
  float ext = __fsub_rn(hi, lo);
  float u = ext > 0.0f ? __fdiv_rn(__fsub_rn(v, lo), ext) : 0.0f;
  float f = floorf(__fmul_rn(u, 1024.0f));
  if (f > 1023.0f) f = 1023.0f;
  return (uint32_t)f;
}

__global__ void k_prims(const float *__restrict__ t, const float *__restrict__ q, const float *__restrict__ s,
                        int n, int M, const float *__restrict__ scene, Pose *__restrict__ pose,
                        Xform *__restrict__ xf, float4 *__restrict__ pbox, uint32_t *__restrict__ keys,
                        int *__restrict__ vals) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float tx = t[3 * k], ty = t[3 * k + 1], tz = t[3 * k + 2];
  float sx = s[3 * k], sy = s[3 * k + 1], sz = s[3 * k + 2];
  float R[9];
  rot_spec(q[4 * k], q[4 * k + 1], q[4 * k + 2], q[4 * k + 3], R);
  Pose P;
  P.p0 = make_float4(R[0], R[1], R[2], R[3]);
  P.p1 = make_float4(R[4], R[5], R[6], R[7]);
  P.p2 = make_float4(R[8], tx, ty, tz);
  P.p3 = make_float4(__frcp_rn(sx), __frcp_rn(sy), __frcp_rn(sz), 0.0f);
  pose[k] = P;
  // u = diag(h/s) R^T (x - t) + h as rows {M_j0, M_j1, M_j2, c_j}, fixed rounding:
  // hs_j = h / s_j, M_jm = hs_j * R_mj, c_j = ((h - M_j0 t0) - M_j1 t1) - M_j2 t2.
  // Per sample the kernels evaluate u_j = fma(M_j0, x0, fma(M_j1, x1, fma(M_j2, x2, c_j)))
  // with x = fma(t_i, d, o); the voxel cell floor(u) is decided by these FP32 values.
  float h = 0.5f * (float)(M - 1);
  float hs[3] = {__fdiv_rn(h, sx), __fdiv_rn(h, sy), __fdiv_rn(h, sz)};
  float tt[3] = {tx, ty, tz};
  float rows[3][4];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float c = h;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      rows[j][m] = __fmul_rn(hs[j], R[3 * m + j]);
      c = __fsub_rn(c, __fmul_rn(rows[j][m], tt[m]));
    }
    rows[j][3] = c;
  }
  Xform X;
  X.r0 = make_float4(rows[0][0], rows[0][1], rows[0][2], rows[0][3]);
  X.r1 = make_float4(rows[1][0], rows[1][1], rows[1][2], rows[1][3]);
  X.r2 = make_float4(rows[2][0], rows[2][1], rows[2][2], rows[2][3]);
  xf[k] = X;
  // world bounds of the oriented box: t +- |R| s, inflated so that no point the
  // FP32 membership test can accept falls outside
  float lo[3], hi[3];
  float ss[3] = {sx, sy, sz};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float e = fabsf(R[3 * i]) * ss[0] + fabsf(R[3 * i + 1]) * ss[1] + fabsf(R[3 * i + 2]) * ss[2];
    float pad = 1.0e-5f * (fabsf(tt[i]) + e) + 1.0e-30f;
    lo[i] = tt[i] - e - pad;
    hi[i] = tt[i] + e + pad;
  }
  pbox[2 * k] = make_float4(lo[0], lo[1], lo[2], 0.0f);
  pbox[2 * k + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
  uint32_t qx = quant10(tx, scene[0], scene[3]);
  uint32_t qy = quant10(ty, scene[1], scene[4]);
  uint32_t qz = quant10(tz, scene[2], scene[5]);
  keys[k] = (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
  vals[k] = k;
}

// ------------------------------------------------------------------ 3. radix sort
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
static_assert(SORT_TILE == BVH_SORT_TILE, "BVH_SORT_TILE sizes the digit-count buffers");

__global__ void __launch_bounds__(SORT_THREADS) k_sort_count(const uint32_t *__restrict__ keys, int n, int shift,
                                                             int nblocks, int *__restrict__ counts) {
  __shared__ int hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * SORT_TILE;
#pragma unroll
  for (int c = 0; c < SORT_ITEMS; ++c) {
    int i = base + c * SORT_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  counts[threadIdx.x * nblocks + blockIdx.x] = hist[threadIdx.x];
}

// Exclusive scan of `total` ints in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_excl(int *__restrict__ a, int total) {
  __shared__ int wsum[32];
  int per = (total + blockDim.x - 1) / blockDim.x;
  int begin = threadIdx.x * per, end = min(begin + per, total);
  int local = 0;
  for (int i = begin; i < end; ++i) local += a[i];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = wsum[lane];
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(FULL, iv, o);
      if (lane >= o) iv += u;
    }
    wsum[lane] = iv - v;
  }
  __syncthreads();
  int run = wsum[warp] + incl - local;
  for (int i = begin; i < end; ++i) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const uint32_t *__restrict__ kin,
                                                               const int *__restrict__ vin, int n, int shift,
                                                               int nblocks, const int *__restrict__ offsets,
                                                               uint32_t *__restrict__ kout, int *__restrict__ vout) {
  constexpr int NW = SORT_THREADS / 32;
  __shared__ int base[256];
  __shared__ int wcnt[NW][256];
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offsets[tid * nblocks + blockIdx.x];
  unsigned lt = (1u << lane) - 1u;
  int tile = blockIdx.x * SORT_TILE;
  for (int c = 0; c < SORT_ITEMS; ++c) {
    int i = tile + c * SORT_THREADS + tid;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    int val = valid ? vin[i] : 0;
    int d = valid ? (int)((key >> shift) & 255u) : 256 + lane;
#pragma unroll
    for (int w = 0; w < NW; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(FULL, d);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    int sum = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      int v = wcnt[w][tid];
      wcnt[w][tid] = sum;
      sum += v;
    }
    __syncthreads();
    if (valid) {
      int pos = base[d] + wcnt[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    base[tid] += sum;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ 4. hierarchy
__device__ __forceinline__ int delta(const uint32_t *__restrict__ km, const int *__restrict__ kv, int n, int i,
                                     int j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = ((uint64_t)km[i] << 32) | (uint32_t)kv[i];
  uint64_t b = ((uint64_t)km[j] << 32) | (uint32_t)kv[j];
  return __clzll(a ^ b);
}

__global__ void k_hierarchy(const uint32_t *__restrict__ km, const int *__restrict__ kv, int n,
                            const float4 *__restrict__ pbox, Node *__restrict__ nodes, int *__restrict__ parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // leaf i: node n-1+i
  {
    int k = kv[i];
    float4 lo = pbox[2 * k], hi = pbox[2 * k + 1];
    Node L;
    L.lox = lo.x; L.loy = lo.y; L.loz = lo.z; L.left = -1 - k;
    L.hix = hi.x; L.hiy = hi.y; L.hiz = hi.z; L.right = 0;
    nodes[n - 1 + i] = L;
  }
  if (i == 0) parent[0] = -1;
  if (i >= n - 1) return;
  // internal node i: direction of its range, its other end j, and the split
  int d = (delta(km, kv, n, i, i + 1) - delta(km, kv, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(km, kv, n, i, i - d);
  int lmax = 2;
  while (delta(km, kv, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int step = lmax >> 1; step >= 1; step >>= 1)
    if (delta(km, kv, n, i, i + (l + step) * d) > dmin) l += step;
  int j = i + l * d;
  int dnode = delta(km, kv, n, i, j);
  int sgap = 0;
  for (int div = 2;; div <<= 1) {
    int step = (l + div - 1) / div;
    if (delta(km, kv, n, i, i + (sgap + step) * d) > dnode) sgap += step;
    if (step == 1) break;
  }
  int g = i + sgap * d + min(d, 0);
  int lc = (min(i, j) == g) ? (n - 1 + g) : g;
  int rc = (max(i, j) == g + 1) ? (n - 1 + g + 1) : g + 1;
  Node N;
  N.lox = N.loy = N.loz = 0.0f;
  N.hix = N.hiy = N.hiz = 0.0f;
  N.left = lc;
  N.right = rc;
  nodes[i] = N;
  parent[lc] = i;
  parent[rc] = i;
}

// ------------------------------------------------------------------ 5. refit
__global__ void k_refit(Node *nodes, const int *__restrict__ parent, int *flags, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int node = parent[n - 1 + i];
  while (node >= 0) {
    __threadfence();
    if (atomicAdd(&flags[node], 1) == 0) return;  // the sibling subtree is not done yet
    __threadfence();
    int l = __ldcg(&nodes[node].left), r = __ldcg(&nodes[node].right);
    const float4 *L = reinterpret_cast<const float4 *>(&nodes[l]);
    const float4 *Rr = reinterpret_cast<const float4 *>(&nodes[r]);
    float4 a0 = __ldcg(L), a1 = __ldcg(L + 1), b0 = __ldcg(Rr), b1 = __ldcg(Rr + 1);
    float4 *D = reinterpret_cast<float4 *>(&nodes[node]);
    __stcg(D, make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), __int_as_float(l)));
    __stcg(D + 1, make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), __int_as_float(r)));
    node = parent[node];
  }
}

// ------------------------------------------------------------------ host side
static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

cudaError_t bvh_reserve(BvhBuffers &b, int n) {
  if (n <= b.cap && b.base) return cudaSuccess;
  if (b.base) {
    cudaFree(b.base);
    b.base = nullptr;
    b.cap = 0;
  }
  int cap = n < 64 ? 64 : n;
  int G = (cap + SORT_TILE - 1) / SORT_TILE;
  size_t off = 0;
  size_t o_scene = off; off = align_up(off + 6 * sizeof(float));
  size_t o_pose = off; off = align_up(off + (size_t)cap * sizeof(Pose));
  size_t o_xf = off; off = align_up(off + (size_t)cap * sizeof(Xform));
  size_t o_pbox = off; off = align_up(off + (size_t)cap * 2 * sizeof(float4));
  size_t o_ka = off; off = align_up(off + (size_t)cap * sizeof(uint32_t));
  size_t o_kb = off; off = align_up(off + (size_t)cap * sizeof(uint32_t));
  size_t o_va = off; off = align_up(off + (size_t)cap * sizeof(int));
  size_t o_vb = off; off = align_up(off + (size_t)cap * sizeof(int));
  size_t o_cnt = off; off = align_up(off + (size_t)256 * G * sizeof(int));
  size_t o_nodes = off; off = align_up(off + (size_t)(2 * cap) * sizeof(Node));
  size_t o_par = off; off = align_up(off + (size_t)(2 * cap) * sizeof(int));
  size_t o_flags = off; off = align_up(off + (size_t)cap * sizeof(int));
  size_t o_gmc = off; off = align_up(off + (size_t)cap * 12 * sizeof(float));
  char *p = nullptr;
  cudaError_t e = cudaMalloc(&p, off);
  if (e != cudaSuccess) return e;
  b.base = p;
  b.bytes = off;
  b.cap = cap;
  b.scene = reinterpret_cast<float *>(p + o_scene);
  b.pose = reinterpret_cast<Pose *>(p + o_pose);
  b.xf = reinterpret_cast<Xform *>(p + o_xf);
  b.pbox = reinterpret_cast<float4 *>(p + o_pbox);
  b.keys_a = reinterpret_cast<uint32_t *>(p + o_ka);
  b.keys_b = reinterpret_cast<uint32_t *>(p + o_kb);
  b.vals_a = reinterpret_cast<int *>(p + o_va);
  b.vals_b = reinterpret_cast<int *>(p + o_vb);
  b.counts = reinterpret_cast<int *>(p + o_cnt);
  b.nodes = reinterpret_cast<Node *>(p + o_nodes);
  b.parent = reinterpret_cast<int *>(p + o_par);
  b.flags = reinterpret_cast<int *>(p + o_flags);
  b.gmc = reinterpret_cast<float *>(p + o_gmc);
  return cudaSuccess;
}

void bvh_release(BvhBuffers &b) {
  if (b.base) cudaFree(b.base);
  b = BvhBuffers();
}

cudaError_t bvh_build(BvhBuffers &b, const float *t, const float *q, const float *s, int n, int M,
                      cudaStream_t st) {
  b.n = n;
  b.M = M;
  if (n == 0) return cudaGetLastError();
  k_bounds<<<1, 1024, 0, st>>>(t, n, b.scene);
  k_prims<<<(n + 255) / 256, 256, 0, st>>>(t, q, s, n, M, b.scene, b.pose, b.xf, b.pbox, b.keys_a, b.vals_a);
  int G = (n + SORT_TILE - 1) / SORT_TILE;
  uint32_t *kin = b.keys_a, *kout = b.keys_b;
  int *vin = b.vals_a, *vout = b.vals_b;
  for (int pass = 0; pass < 4; ++pass) {
    int shift = 8 * pass;
    k_sort_count<<<G, SORT_THREADS, 0, st>>>(kin, n, shift, G, b.counts);
    k_scan_excl<<<1, 1024, 0, st>>>(b.counts, 256 * G);
    k_sort_scatter<<<G, SORT_THREADS, 0, st>>>(kin, vin, n, shift, G, b.counts, kout, vout);
    uint32_t *tk = kin; kin = kout; kout = tk;
    int *tv = vin; vin = vout; vout = tv;
  }
  // four passes: the sorted data is back in keys_a / vals_a
  k_hierarchy<<<(n + 255) / 256, 256, 0, st>>>(b.keys_a, b.vals_a, n, b.pbox, b.nodes, b.parent);
  if (n > 1) {
    cudaMemsetAsync(b.flags, 0, sizeof(int) * (size_t)(n - 1), st);
    k_refit<<<(n + 255) / 256, 256, 0, st>>>(b.nodes, b.parent, b.flags, n);
  }
  return cudaGetLastError();
}

__global__ void k_export_keys(const uint32_t *__restrict__ km, const int *__restrict__ kv, int n,
                              uint64_t *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ((uint64_t)km[i] << 32) | (uint32_t)kv[i];
}

__global__ void k_export_nodes(const Node *__restrict__ nodes, int n, int32_t *__restrict__ children,
                               float *__restrict__ bounds) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n - 1) return;
  Node N = nodes[i];
  if (children && i < n - 1) {
    children[2 * i] = N.left;
    children[2 * i + 1] = N.right;
  }
  if (bounds) {
    bounds[6 * i + 0] = N.lox; bounds[6 * i + 1] = N.loy; bounds[6 * i + 2] = N.loz;
    bounds[6 * i + 3] = N.hix; bounds[6 * i + 4] = N.hiy; bounds[6 * i + 5] = N.hiz;
  }
}

cudaError_t bvh_export(const BvhBuffers &b, uint64_t *keys, int32_t *children, float *bounds, float *scene,
                       cudaStream_t st) {
  int n = b.n;
  if (n == 0) return cudaSuccess;
  if (keys) k_export_keys<<<(n + 255) / 256, 256, 0, st>>>(b.keys_a, b.vals_a, n, keys);
  if (children || bounds) k_export_nodes<<<(2 * n + 254) / 256, 256, 0, st>>>(b.nodes, n, children, bounds);
  if (scene) cudaMemcpyAsync(scene, b.scene, 6 * sizeof(float), cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

}  // namespace mvp
