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
#include <type_traits>

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

// 32 bytes with one 256-bit load (read-only path).
__device__ __forceinline__ uint4 ld32_lo(const void *p, uint4 &hi) {
  uint4 lo;
  asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
               : "l"(p));
  return lo;
}

__device__ __forceinline__ float4 widen(uint2 r, int dt) {
  if (dt == MVP_F16) {
    __half2 a = *reinterpret_cast<__half2 *>(&r.x), b = *reinterpret_cast<__half2 *>(&r.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                     __uint_as_float(r.y & 0xffff0000u));
}

// The voxels of `per` consecutive voxel slots of element e of a layout whose
// elements hold `per` voxels (1: one voxel; 2: a voxel and its +x neighbour; 4: a
// voxel, +x, +y, +x+y), summed channel-pair-wise into s.
template <int DT, int PER>
__device__ __forceinline__ void load_elem(const void *base, int64_t e, float2 &s) {
  if (DT == MVP_F32) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + e * PER;
    if (PER == 1) {
      const float4 a = __ldg(p);
      s = __fadd2_rn(s, __fadd2_rn(lo2(a), hi2(a)));
    } else {
#pragma unroll
      for (int h = 0; h < PER / 2; ++h) {
        uint4 hi;
        const uint4 lo = ld32_lo(p + 2 * h, hi);
        const float4 a = make_float4(__uint_as_float(lo.x), __uint_as_float(lo.y), __uint_as_float(lo.z),
                                     __uint_as_float(lo.w));
        const float4 b = make_float4(__uint_as_float(hi.x), __uint_as_float(hi.y), __uint_as_float(hi.z),
                                     __uint_as_float(hi.w));
        s = __fadd2_rn(s, __fadd2_rn(__fadd2_rn(lo2(a), hi2(a)), __fadd2_rn(lo2(b), hi2(b))));
      }
    }
  } else {
    const uint2 *p = reinterpret_cast<const uint2 *>(base) + e * PER;
    if (PER == 1) {
      const float4 a = widen(__ldg(p), DT);
      s = __fadd2_rn(s, __fadd2_rn(lo2(a), hi2(a)));
    } else if (PER == 2) {
      const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
      const float4 a = widen(make_uint2(r.x, r.y), DT), b = widen(make_uint2(r.z, r.w), DT);
      s = __fadd2_rn(s, __fadd2_rn(__fadd2_rn(lo2(a), hi2(a)), __fadd2_rn(lo2(b), hi2(b))));
    } else {
      uint4 hi;
      const uint4 lo = ld32_lo(p, hi);
      const float4 a = widen(make_uint2(lo.x, lo.y), DT), b = widen(make_uint2(lo.z, lo.w), DT);
      const float4 c = widen(make_uint2(hi.x, hi.y), DT), d = widen(make_uint2(hi.z, hi.w), DT);
      s = __fadd2_rn(s, __fadd2_rn(__fadd2_rn(__fadd2_rn(lo2(a), hi2(a)), __fadd2_rn(lo2(b), hi2(b))),
                                   __fadd2_rn(__fadd2_rn(lo2(c), hi2(c)), __fadd2_rn(lo2(d), hi2(d)))));
    }
  }
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

// RES: launched at a fixed residency (128-thread blocks, see mvp_gather_probe); a
// separate instance, so its shared-memory carveout leaves the full-occupancy one alone.
template <int DT, bool SCATTER, int PER = 1, bool RES = false>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(const void *payload, float4 *grad, int n, int M,
                                                         int footprint, int steps, float *sink) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
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
    } else if (PER == 1) {
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
    } else {
      // duplicated layouts: the element of a voxel holds PER of its cell's corners
      float2 s = make_float2(0.0f, 0.0f);
      load_elem<DT, PER>(payload, v, s);
      load_elem<DT, PER>(payload, v + oM2, s);
      if (PER == 2) {
        load_elem<DT, PER>(payload, v + oM, s);
        load_elem<DT, PER>(payload, v + oM2 + oM, s);
      }
      acc0 += s.x;
      acc1 += s.y;
    }
  }
  if (!SCATTER) {
    const float w = warp_sum(acc0 + acc1);
    if (lane == 0) atomicAdd(sink, w);
  }
}

// Mode 4: the same gathers staged through shared memory. Per chunk of 4 samples the
// warp finds the box of voxels its lanes' cells span (integer warp min/max), copies it
// into its slice of shared memory in rows along x (coalesced), and reads the 8
// corners of each lane's cells from there; a box larger than STAGE_VOXELS falls back
// to global loads.
constexpr int STAGE_VOXELS = 256;
constexpr int STAGE_CHUNK = 4;

template <int DT>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_staged(const void *payload, int n, int M, int footprint,
                                                                int steps, float *sink) {
  using V = typename std::conditional<DT == MVP_F32, float4, uint2>::type;
  extern __shared__ __align__(16) unsigned char probe_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  V *stage = reinterpret_cast<V *>(probe_smem) + wib * STAGE_VOXELS;
  const V *src = reinterpret_cast<const V *>(payload);
  const uint32_t warp = (blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
  const float lx = 0.25f * (float)(lane & 7), ly = 0.25f * (float)(lane >> 3);
  const int64_t M3 = (int64_t)M * M * M;
  float2 acc = make_float2(0.0f, 0.0f);
  int k = footprint == 0 ? (int)(sm_id() % (unsigned)n) : 0;
  float bx = 0.0f, by = 0.0f, bz = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.67f;
  for (int i0 = 0; i0 < steps; i0 += STAGE_CHUNK) {
    if (i0 % PROBE_RUN == 0) {
      const uint32_t h = mix32(warp * 0x9e3779b9U + (uint32_t)(i0 / PROBE_RUN) * 0x85ebca6bU + 1U);
      if (footprint != 0) k = (int)(mix32(h) % (uint32_t)n);
      bx = (float)(h & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      by = (float)((h >> 8) & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      bz = (float)((h >> 16) & 0xff) * (1.0f / 256.0f) * (float)(M - 1);
      sx = 0.67f * 0.3f * ((float)((h >> 24) & 0xf) * (1.0f / 8.0f) - 1.0f);
      sy = 0.67f * 0.3f * ((float)((h >> 28) & 0xf) * (1.0f / 8.0f) - 1.0f);
      sz = 0.67f * 0.9f;
    }
    const int nj = min(STAGE_CHUNK, steps - i0);
    int cx[STAGE_CHUNK], cy[STAGE_CHUNK], cz[STAGE_CHUNK];
    int lo_x = M, lo_y = M, lo_z = M, hi_x = 0, hi_y = 0, hi_z = 0;
#pragma unroll
    for (int q = 0; q < STAGE_CHUNK; ++q) {
      const int j = (i0 + q) % PROBE_RUN;
      cx[q] = cell(bx, sx, lx, j, M);
      cy[q] = cell(by, sy, ly, j, M);
      cz[q] = cell(bz, sz, 0.0f, j, M);
      if (q < nj) {
        lo_x = min(lo_x, cx[q]), lo_y = min(lo_y, cy[q]), lo_z = min(lo_z, cz[q]);
        hi_x = max(hi_x, cx[q] + 1), hi_y = max(hi_y, cy[q] + 1), hi_z = max(hi_z, cz[q] + 1);
      }
    }
    lo_x = __reduce_min_sync(FULL, lo_x), lo_y = __reduce_min_sync(FULL, lo_y), lo_z = __reduce_min_sync(FULL, lo_z);
    hi_x = __reduce_max_sync(FULL, hi_x), hi_y = __reduce_max_sync(FULL, hi_y), hi_z = __reduce_max_sync(FULL, hi_z);
    const int dx = hi_x - lo_x + 1, dy = hi_y - lo_y + 1, dz = hi_z - lo_z + 1;
    const int nvox = dx * dy * dz;
    const int64_t kb = (int64_t)k * M3;
    if (nvox <= STAGE_VOXELS) {
      __syncwarp();
      for (int q = lane; q < nvox; q += 32) {
        const int x = q % dx, yz = q / dx, y = yz % dy, z = yz / dy;
        stage[q] = __ldg(src + kb + ((int64_t)(lo_z + z) * M + (lo_y + y)) * M + (lo_x + x));
      }
      __syncwarp();
      const int sdy = dx * dy;
#pragma unroll
      for (int q = 0; q < STAGE_CHUNK; ++q) {
        if (q < nj) {
        const int b = ((cz[q] - lo_z) * dy + (cy[q] - lo_y)) * dx + (cx[q] - lo_x);
#define MVP_STAGED(o)                                                                   \
  {                                                                                     \
    float4 v;                                                                           \
    if (DT == MVP_F32) v = reinterpret_cast<const float4 *>(stage)[b + (o)];            \
    else v = widen(reinterpret_cast<const uint2 *>(stage)[b + (o)], DT);                \
    acc = __fadd2_rn(acc, __fadd2_rn(lo2(v), hi2(v)));                                  \
  }
        MVP_STAGED(0) MVP_STAGED(1) MVP_STAGED(dx) MVP_STAGED(dx + 1)
        MVP_STAGED(sdy) MVP_STAGED(sdy + 1) MVP_STAGED(sdy + dx) MVP_STAGED(sdy + dx + 1)
        }
#undef MVP_STAGED
      }
    } else {
      const int64_t oM = M, oM2 = (int64_t)M * M;
#pragma unroll
      for (int q = 0; q < STAGE_CHUNK; ++q) {
        if (q < nj) {
        const int64_t v = kb + ((int64_t)cz[q] * M + cy[q]) * M + cx[q];
#define MVP_DIRECT(o)                                                                   \
  {                                                                                     \
    const float4 w = Voxel<DT>::load(payload, v + (o));                                 \
    acc = __fadd2_rn(acc, __fadd2_rn(lo2(w), hi2(w)));                                  \
  }
        MVP_DIRECT(0) MVP_DIRECT(1) MVP_DIRECT(oM) MVP_DIRECT(oM + 1)
        MVP_DIRECT(oM2) MVP_DIRECT(oM2 + 1) MVP_DIRECT(oM2 + oM) MVP_DIRECT(oM2 + oM + 1)
        }
#undef MVP_DIRECT
      }
    }
  }
  const float w = warp_sum(acc.x + acc.y);
  if (lane == 0) atomicAdd(sink, w);
}

template <int DT, bool SCATTER, int PER>
cudaError_t launch_probe_t(const void *payload, float4 *grad, int n, int M, int footprint, int steps, float *sink,
                           int grid, cudaStream_t st) {
  k_probe<DT, SCATTER, PER><<<grid, PROBE_THREADS, 0, st>>>(payload, grad, n, M, footprint, steps, sink);
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_staged(const void *payload, int n, int M, int footprint, int steps, float *sink, int sms,
                          cudaStream_t st) {
  const size_t smem = (size_t)(PROBE_THREADS / 32) * STAGE_VOXELS * (DT == MVP_F32 ? 16 : 8);
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(k_probe_staged<DT>), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_staged<DT>, PROBE_THREADS, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  k_probe_staged<DT><<<sms * per_sm, PROBE_THREADS, smem, st>>>(payload, n, M, footprint, steps, sink);
  return cudaGetLastError();
}

// The kernels of the frame march and the adjoint run 4-warp blocks holding
// sizeof(TileShared<MARCH_CAP>) x 4 bytes of shared memory each, `blocks` of them per SM
// (registers allow no more). This launches the probe the same way: 128-thread blocks
// with that much dynamic shared memory and a carveout that holds exactly `blocks` of
// them, so the probe sees the same warps per SM and the same L1 size. Returns
// cudaErrorInvalidConfiguration if the device does not give that residency.
template <int DT, bool SCATTER>
cudaError_t launch_resident(const void *payload, float4 *grad, int n, int M, int footprint, int steps, float *sink,
                            int blocks, int sms, int smem_per_sm, cudaStream_t st) {
  auto k = k_probe<DT, SCATTER, 1, true>;
  const size_t smem = sizeof(TileShared<MARCH_CAP>) * TILE_WARPS;
  const int need = (int)(blocks * (smem + 1024));  // 1 KB per block is the driver's
  const int pct = (need * 100 + smem_per_sm - 1) / smem_per_sm;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem)) != cudaSuccess) return e;
  if (per_sm != blocks) return cudaErrorInvalidConfiguration;
  k<<<sms * blocks, 128, smem, st>>>(payload, grad, n, M, footprint, steps, sink);
  return cudaGetLastError();
}

template <int PER>
cudaError_t launch_loads(int dtype, const void *payload, int n, int M, int footprint, int steps, float *sink,
                         int grid, cudaStream_t st) {
  if (dtype == MVP_F32) return launch_probe_t<MVP_F32, false, PER>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
  if (dtype == MVP_BF16) return launch_probe_t<MVP_BF16, false, PER>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
  return launch_probe_t<MVP_F16, false, PER>(payload, nullptr, n, M, footprint, steps, sink, grid, st);
}

}  // namespace
}  // namespace mvp

extern "C" mvp_status mvp_gather_probe(const void *payload, int32_t dtype, int32_t n, int32_t M, int32_t mode,
                                       int32_t footprint, int32_t steps, float *grad, float *sink, int64_t *accesses,
                                       mvp_stream stream) {
  using namespace mvp;
  // bits 0-7: the access mode; bits 8-15: 4-warp blocks per SM (0: every SM full)
  const int blocks = (mode >> 8) & 0xff;
  const bool bad_mode = mode < 0 || (mode >> 16) != 0 || (mode & 0xff) > 4 || blocks > 16 ||
                        (blocks > 0 && (mode & 0xff) > 1);
  if (n < 1 || M < 2 || M > MVP_MAX_M || steps < 1 || bad_mode || (footprint != 0 && footprint != 1))
    return record_error("mvp_gather_probe: bad n, M, steps, mode or footprint"), MVP_ERR_INVALID_ARG;
  mode &= 0xff;
  if (mode != 1 && (!payload || !sink || (dtype != MVP_F32 && dtype != MVP_BF16 && dtype != MVP_F16)))
    return record_error("mvp_gather_probe: loads need a payload, a sink and a payload dtype"), MVP_ERR_INVALID_ARG;
  if (mode == 1 && !grad) return record_error("mvp_gather_probe: reductions need grad"), MVP_ERR_INVALID_ARG;
  const int per = mode == 2 ? 2 : (mode == 3 ? 4 : 1);
  const uintptr_t al = mode == 1 ? 16 : (uintptr_t)(dtype == MVP_F32 ? 16 : 8) * per;
  if (reinterpret_cast<uintptr_t>(mode == 1 ? (const void *)grad : payload) % al)
    return record_error("mvp_gather_probe: misaligned array"), MVP_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return record_error("mvp_gather_probe: no device"), MVP_ERR_CUDA;
  const void *k = mode == 1 ? reinterpret_cast<const void *>(k_probe<MVP_F32, true>)
                            : reinterpret_cast<const void *>(k_probe<MVP_F32, false>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PROBE_THREADS, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int grid = sms * per_sm;  // every SM full, one wave
  cudaStream_t st = (cudaStream_t)stream;
  float4 *g4 = reinterpret_cast<float4 *>(grad);
  cudaError_t e;
  if (blocks > 0) {
    int smem_per_sm = 0;
    if (cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        smem_per_sm <= 0)
      return record_error("mvp_gather_probe: no device"), MVP_ERR_CUDA;
    if (mode == 1) e = launch_resident<MVP_F32, true>(nullptr, g4, n, M, footprint, steps, nullptr, blocks, sms, smem_per_sm, st);
    else if (dtype == MVP_F32) e = launch_resident<MVP_F32, false>(payload, nullptr, n, M, footprint, steps, sink, blocks, sms, smem_per_sm, st);
    else if (dtype == MVP_BF16) e = launch_resident<MVP_BF16, false>(payload, nullptr, n, M, footprint, steps, sink, blocks, sms, smem_per_sm, st);
    else e = launch_resident<MVP_F16, false>(payload, nullptr, n, M, footprint, steps, sink, blocks, sms, smem_per_sm, st);
    if (e == cudaErrorInvalidConfiguration) {
      cudaGetLastError();
      return record_error("mvp_gather_probe: the device does not give that residency"), MVP_ERR_INVALID_ARG;
    }
    if (e != cudaSuccess) return record_error("mvp_gather_probe: launch failed"), MVP_ERR_CUDA;
    if (accesses) *accesses = (int64_t)sms * blocks * 128 * steps * 8;
    return MVP_OK;
  }
  if (mode == 1) e = launch_probe_t<MVP_F32, true, 1>(nullptr, g4, n, M, footprint, steps, nullptr, grid, st);
  else if (mode == 0) e = launch_loads<1>(dtype, payload, n, M, footprint, steps, sink, grid, st);
  else if (mode == 2) e = launch_loads<2>(dtype, payload, n, M, footprint, steps, sink, grid, st);
  else if (mode == 3) e = launch_loads<4>(dtype, payload, n, M, footprint, steps, sink, grid, st);
  else if (dtype == MVP_F32) e = launch_staged<MVP_F32>(payload, n, M, footprint, steps, sink, sms, st);
  else if (dtype == MVP_BF16) e = launch_staged<MVP_BF16>(payload, n, M, footprint, steps, sink, sms, st);
  else e = launch_staged<MVP_F16>(payload, n, M, footprint, steps, sink, sms, st);
  if (e != cudaSuccess) return record_error("mvp_gather_probe: launch failed"), MVP_ERR_CUDA;
  if (mode == 4) {  // the staged kernel's own grid
    int per_sm4 = 0;
    const size_t smem = (size_t)(PROBE_THREADS / 32) * STAGE_VOXELS * (dtype == MVP_F32 ? 16 : 8);
    const void *k4 = dtype == MVP_F32 ? reinterpret_cast<const void *>(k_probe_staged<MVP_F32>)
                   : dtype == MVP_BF16 ? reinterpret_cast<const void *>(k_probe_staged<MVP_BF16>)
                                       : reinterpret_cast<const void *>(k_probe_staged<MVP_F16>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm4, k4, PROBE_THREADS, smem) != cudaSuccess || per_sm4 < 1)
      per_sm4 = 1;
    if (accesses) *accesses = (int64_t)sms * per_sm4 * PROBE_THREADS * steps * 8;
  } else if (accesses) {
    *accesses = (int64_t)grid * PROBE_THREADS * steps * 8;
  }
  return MVP_OK;
}
