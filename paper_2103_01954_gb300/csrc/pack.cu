// pack.cu -- payload precision conversion and pinhole camera rays.
#include "pack.cuh"
#include "camera.cuh"

namespace mvp {

// FP32 -> BF16 / FP16, round to nearest even, 4 values (one RGBA voxel) per thread.
template <int DT>
__global__ void k_pack(const float *__restrict__ src, void *__restrict__ dst, int64_t n) {
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i >= n) return;
  if (i + 4 <= n && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && ((reinterpret_cast<uintptr_t>(dst) & 7) == 0)) {
    float4 v = *reinterpret_cast<const float4 *>(src + i);
    uint2 o;
    if (DT == MVP_BF16) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
      o.x = *reinterpret_cast<uint32_t *>(&a);
      o.y = *reinterpret_cast<uint32_t *>(&b);
    } else {
      __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
      o.x = *reinterpret_cast<uint32_t *>(&a);
      o.y = *reinterpret_cast<uint32_t *>(&b);
    }
    *reinterpret_cast<uint2 *>(reinterpret_cast<uint16_t *>(dst) + i) = o;
  } else {
    for (int64_t j = i; j < n && j < i + 4; ++j) {
      if (DT == MVP_BF16)
        reinterpret_cast<__nv_bfloat16 *>(dst)[j] = __float2bfloat16_rn(src[j]);
      else
        reinterpret_cast<__half *>(dst)[j] = __float2half_rn(src[j]);
    }
  }
}

cudaError_t launch_pack(const float *src, void *dst, int64_t n, int dtype, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (dtype == MVP_F32) return cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  int64_t threads = (n + 3) / 4;
  unsigned blocks = (unsigned)((threads + 255) / 256);
  if (dtype == MVP_BF16) k_pack<MVP_BF16><<<blocks, 256, 0, st>>>(src, dst, n);
  else k_pack<MVP_F16><<<blocks, 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// Pinhole rays of a W x H image, row-major (camera_ray in camera.cuh).
__global__ void k_camera(Cam c, float *__restrict__ o, float *__restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)c.width * c.height;
  if (i >= n) return;
  int row = (int)(i / c.width), col = (int)(i - (int64_t)row * c.width);
  float oo[3], dd[3];
  camera_ray(c.m, c.focal, c.width, c.height, row, col, oo, dd);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    o[3 * i + j] = oo[j];
    d[3 * i + j] = dd[j];
  }
}

cudaError_t launch_camera(const Cam &c, float *o, float *d, cudaStream_t st) {
  int64_t n = (int64_t)c.width * c.height;
  if (n <= 0) return cudaSuccess;
  k_camera<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, o, d);
  return cudaGetLastError();
}

}  // namespace mvp
