// probe.cu -- the gather and scatter ceilings of the march's voxel access pattern.
//
// No counterpart in the paper: a measurement of the GPU, the denominator of the
// march's and the adjoint's roofline fractions. Per (sample, primitive) evaluation the
// march reads the 8 corner voxels of one cell (voxel offsets 0, 1, M, M+1, M^2,
// M^2+1, M^2+M, M^2+M+1 from the cell's first voxel) and the adjoint adds a float4 to
// each of them. This kernel issues exactly those accesses with none of the rest of
// the work, in the march's coherence pattern: a warp is an 8x4 pixel tile whose lanes
// sit a quarter voxel apart in the primitive's grid (the paper-scale frame's pixel
// footprint: 4096 boxes of 16^3 voxels seen at 1024 px focal length), and consecutive
// samples of a lane lie two thirds of a voxel apart along its ray (dt = 0.005). Its
// rate is therefore what the load (or reduction) path sustains for that pattern when
// nothing else competes for issue slots: the ceiling the fused kernels are held to.
//
// footprint 0: each SM gathers inside one primitive of its own (chosen by its SM id),
// so after the first touch every access hits L1. footprint 1: each warp moves to
// another primitive every 16 samples, over all n primitives, so a footprint larger
// than L1 and smaller than L2 is served by L2. The loads' sum goes to a one-float
// sink, which keeps every load alive.
#include "march.cuh"

namespace mvp {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_RUN = 16;  // samples a warp spends in one primitive (footprint 1)

__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Cell coordinate in [0, M-2] of a lane's sample: the warp tile's origin plus the
// lane's offset, advancing along the ray, wrapped inside the grid.
__device__ __forceinline__ int cell(float base, float step, float lane_off, int i, int M) {
  const float span = (float)(M - 1);
  float u = base + lane_off + step * (float)i;
  u = u - span * floorf(u / span);  // in [0, M-1)
  const int c = (int)u;
  return c < 0 ? 0 : (c > M - 2 ? M - 2 : c);
}

template <int DT, bool SCATTER>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(const void *payload, float4 *grad, int n, int M,
                                                         int footprint, int steps, float *sink) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
  const float lx = 0.25f * (float)(lane & 7), ly = 0.25f * (float)(lane >> 3);
  const int64_t M3 = (int64_t)M * M * M;
  const int64_t o1 = 1, oM = M, oM2 = (int64_t)M * M;
  float acc0 = 0.0f, acc1 = 0.0f;
  int k = footprint == 0 ? (int)(sm_id() % (unsigned)n) : 0;
  float bx = 0.0f, by = 0.0f, bz = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.67f;
  for (int i = 0; i < steps; ++i) {
    if (i % PROBE_RUN == 0) {  // a new warp tile / primitive: origin and ray direction
      const uint32_t h = mix32(warp * 0x9e3779b9U + (uint32_t)(i / PROBE_RUN) * 0x85ebca6bU + 1U);
      if (footprint != 0) k = (int)(mix32(h) % (uint32_t)n);
      bx = (float)(h & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      by = (float)((h >> 8) & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      bz = (float)((h >> 16) & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      sx = 0.67f * 0.3f * ((float)((h >> 24) & 0xf) * (1.0f / 8.0f) - 1.0f);
      sy = 0.67f * 0.3f * ((float)((h >> 28) & 0xf) * (1.0f / 8.0f) - 1.0f);
      sz = 0.67f * 0.9f;
    }
    const int j = i % PROBE_RUN;
    const int cx = cell(bx, sx, lx, j, M), cy = cell(by, sy, ly, j, M), cz = cell(bz, sz, 0.0f, j, M);
    const int64_t v = (int64_t)k * M3 + ((int64_t)cz * M + cy) * M + cx;
    if (SCATTER) {
      const float4 g = make_float4(1e-3f, 2e-3f, 3e-3f, 4e-3f);
      atomicAdd(grad + v, g);
      atomicAdd(grad + v + o1, g);
      atomicAdd(grad + v + oM, g);
      atomicAdd(grad + v + oM + o1, g);
      atomicAdd(grad + v + oM2, g);
      atomicAdd(grad + v + oM2 + o1, g);
      atomicAdd(grad + v + oM2 + oM, g);
      atomicAdd(grad + v + oM2 + oM + o1, g);
    } else {
      const float4 a = Voxel<DT>::load(payload, v), b = Voxel<DT>::load(payload, v + o1);
      const float4 c = Voxel<DT>::load(payload, v + oM), d = Voxel<DT>::load(payload, v + oM + o1);
      const float4 e = Voxel<DT>::load(payload, v + oM2), f = Voxel<DT>::load(payload, v + oM2 + o1);
      const float4 g = Voxel<DT>::load(payload, v + oM2 + oM), h = Voxel<DT>::load(payload, v + oM2 + oM + o1);
      // consume every channel (packed adds) so no load is dropped
      float2 s0 = __fadd2_rn(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(lo2(c), lo2(d)));
      float2 s1 = __fadd2_rn(__fadd2_rn(lo2(e), lo2(f)), __fadd2_rn(lo2(g), lo2(h)));
      float2 s2 = __fadd2_rn(__fadd2_rn(hi2(a), hi2(b)), __fadd2_rn(hi2(c), hi2(d)));
      float2 s3 = __fadd2_rn(__fadd2_rn(hi2(e), hi2(f)), __fadd2_rn(hi2(g), hi2(h)));
      const float2 s = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
      acc0 += s.x;
      acc1 += s.y;
    }
  }
  if (!SCATTER) {
    const float w = warp_sum(acc0 + acc1);
    if (lane == 0) atomicAdd(sink, w);
  }
}

template <int DT, bool SCATTER>
cudaError_t launch_probe_t(const void *payload, float4 *grad, int n, int M, int footprint, int steps, float *sink,
                           int grid, cudaStream_t st) {
  k_probe<DT, SCATTER><<<grid, PROBE_THREADS, 0, st>>>(payload, grad, n, M, footprint, steps, sink);
  return cudaGetLastError();
}

}  // namespace
}  // namespace mvp

extern "C" mvp_status mvp_gather_probe(const void *payload, int32_t dtype, int32_t n, int32_t M, int32_t mode,
                                       int32_t footprint, int32_t steps, float *grad, float *sink, int64_t *accesses,
                                       mvp_stream stream) {
  using namespace mvp;
  if (n < 1 || M < 2 || M > MVP_MAX_M || steps < 1 || (mode != 0 && mode != 1) || (footprint != 0 && footprint != 1))
    return record_error("mvp_gather_probe: bad n, M, steps, mode or footprint"), MVP_ERR_INVALID_ARG;
  if (mode == 0 && (!payload || !sink || (dtype != MVP_F32 && dtype != MVP_BF16 && dtype != MVP_F16)))
    return record_error("mvp_gather_probe: loads need a payload, a sink and a payload dtype"), MVP_ERR_INVALID_ARG;
  if (mode == 1 && !grad) return record_error("mvp_gather_probe: reductions need grad"), MVP_ERR_INVALID_ARG;
  const uintptr_t al = mode == 1 ? 16 : (dtype == MVP_F32 ? 16 : 8);
  if (reinterpret_cast<uintptr_t>(mode == 1 ? (const void *)grad : payload) % al)
    return record_error("mvp_gather_probe: misaligned array"), MVP_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return record_error("mvp_gather_probe: no device"), MVP_ERR_CUDA;
  const void *k = mode == 1 ? reinterpret_cast<const void *>(k_probe<MVP_F32, true>)
                            : dtype == MVP_F32 ? reinterpret_cast<const void *>(k_probe<MVP_F32, false>)
                            : dtype == MVP_BF16 ? reinterpret_cast<const void *>(k_probe<MVP_BF16, false>)
                                                : reinterpret_cast<const void *>(k_probe<MVP_F16, false>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PROBE_THREADS, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int grid = sms * per_sm;  // every SM full, one wave
  cudaStream_t st = (cudaStream_t)stream;
  float4 *g4 = reinterpret_cast<float4 *>(grad);
  cudaError_t e;
  if (mode == 1) e = launch_probe_t<MVP_F32, true>(nullptr, g4, n, M, footprint, steps, nullptr, grid, st);
  else if (dtype == MVP_F32) e = launch_probe_t<MVP_F32, false>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
  else if (dtype == MVP_BF16) e = launch_probe_t<MVP_BF16, false>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
  else e = launch_probe_t<MVP_F16, false>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
  if (e != cudaSuccess) return record_error("mvp_gather_probe: launch failed"), MVP_ERR_CUDA;
  if (accesses) *accesses = (int64_t)grid * PROBE_THREADS * steps * 8;
  return MVP_OK;
}
