// march.cu -- the frame kernel of the fused traversal + march + composite
// (march_tile.cuh), the evaluation-count variant, and per-ray hit-list export.
#include "march_tile.cuh"

namespace mvp {

template <int DT, int CAP, bool COUNT, int MT, bool SEQ = false>
__global__ void __launch_bounds__(TILE_WARPS * 32, MVP_MARCH_MINB) k_march(MarchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<CAP> &sh = reinterpret_cast<TileShared<CAP> *>(smem_raw)[warp];
  pdl_wait();  // whatever ran before (the BVH refit, usually) is complete and visible
  const int64_t slot = (int64_t)blockIdx.x * TILE_WARPS + warp;
  if (slot >= a.geom.n_warp_tiles) return;
  int64_t wt = slot;
  if (a.order) {  // heaviest tiles of the last frame first, so that none starts late
    const int o = __ldg(a.order + slot);
    if (o >= 0 && o < a.geom.n_warp_tiles) wt = o;
  }
  LaneRay L;
  load_lane_ray(L, a.o, a.d, tile_ray(a.geom, wt, lane));
  if (__ballot_sync(FULL, L.r >= 0) == 0) return;
  if (lane == 0) sh.clk = (unsigned int)clock();  // kept in shared memory, not in a register
  march_tile<DT, CAP, COUNT, MT, SEQ>(sh, a, L);
  if (a.cost) {
    __syncwarp();
    if (lane == 0) {
      int64_t t = slot;  // the tile, found again rather than held through the march
      if (a.order) {
        const int o = __ldg(a.order + slot);
        if (o >= 0 && o < a.geom.n_warp_tiles) t = o;
      }
      a.cost[t] = (unsigned int)clock() - sh.clk;  // cycles on this SM (modulo 2^32)
    }
  }
}


// ----------------------------------------------------------------------------
// Hit lists: each lane emits its ray's (primitive, tin, tout). Passes over the
// depth range in windows; a hit belongs to the window that holds its tin, so a
// window split after an overflow never emits a hit twice. FILL = false counts.
template <bool FILL>
__global__ void __launch_bounds__(TILE_WARPS * 32) k_hits(HitArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<1> &sh = reinterpret_cast<TileShared<1> *>(smem_raw)[warp];
  const int64_t wt = (int64_t)blockIdx.x * TILE_WARPS + warp;
  if (wt >= a.geom.n_warp_tiles) return;
  LaneRay L;
  load_lane_ray(L, a.o, a.d, tile_ray(a.geom, wt, lane));
  const bool valid = L.r >= 0;
  if (__ballot_sync(FULL, valid) == 0) return;
  make_packet(sh.pk, valid, L.o, L.d, a.t_far);
  int64_t count = 0;
  const int64_t base = (FILL && valid) ? a.offs[L.r] : 0;
  float ta = a.t_near, span = a.t_far - a.t_near;
  int guard = 0;
  while (ta <= a.t_far && guard < 4096) {
    ++guard;
    float tb = fminf(ta + span, a.t_far);
    bool last = tb >= a.t_far;
    int64_t c0 = count;
    auto emit = [&](int nc) -> bool {
      for (int c = 0; c < nc; ++c) {
        int k = sh.cand[c];
        if (!valid) continue;
        const float4 *pp = reinterpret_cast<const float4 *>(a.pose + k);
        Pose Pk;
        Pk.p0 = __ldg(pp);
        Pk.p1 = __ldg(pp + 1);
        Pk.p2 = __ldg(pp + 2);
        Pk.p3 = __ldg(pp + 3);
        float tin, tout;
        if (slab_spec(Pk, L.o[0], L.o[1], L.o[2], L.d[0], L.d[1], L.d[2], a.t_near, a.t_far, tin, tout) &&
            tin >= ta && (last ? tin <= tb : tin < tb)) {
          if (FILL) {
            int64_t w = base + count;
            if (w < a.cap) {
              a.ids[w] = k;
              a.tin[w] = tin;
              a.tout[w] = tout;
            }
          }
          ++count;
        }
      }
      return true;
    };
    float slack = 1.0e-5f * (fabsf(ta) + fabsf(tb)) + 1.0e-30f;
    bool ok = traverse_tile(sh, a.nodes, a.n_prims, ta - slack, tb + slack, emit, a.status);
    __syncwarp();
    if (!ok) {
      count = c0;  // drop this window's partial output and retry a narrower one
      span *= 0.5f;
      if (!(span > 1.0e-6f * (fabsf(ta) + 1.0f))) {
        if (lane == 0) atomicOr(a.status, STATUS_CAPACITY);
        break;
      }
      continue;
    }
    if (last) break;
    ta = tb;
    span = fminf(span * 2.0f, a.t_far - a.t_near);
  }
  if (!FILL && valid) a.counts[L.r] = count;
}

// Inclusive prefix sum of counts into offs[1..n], offs[0] = 0 (single block).
__global__ void __launch_bounds__(1024) k_offsets(const int64_t *__restrict__ counts, int64_t n,
                                                  int64_t *__restrict__ offs) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n ? counts[i] : 0;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int64_t w = wsum[lane];
      int64_t iw = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(FULL, iw, o);
        if (lane >= o) iw += u;
      }
      wsum[lane] = iw - w;
    }
    __syncthreads();
    if (i < n) offs[i + 1] = carry + wsum[warp] + incl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) offs[0] = 0;
}

// ----------------------------------------------------------------------------
template <int DT, int CAP, bool COUNT, int MT, bool SEQ = false>
static cudaError_t launch_march_t(const MarchArgs &a, cudaStream_t st) {
  size_t smem = sizeof(TileShared<CAP>) * TILE_WARPS;
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(k_march<DT, CAP, COUNT, MT, SEQ>), smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (a.geom.n_warp_tiles + TILE_WARPS - 1) / TILE_WARPS;
  if (blocks == 0) return cudaSuccess;
  return pdl_launch(k_march<DT, CAP, COUNT, MT, SEQ>, dim3((unsigned)blocks), dim3(TILE_WARPS * 32), smem, st, a);
}

template <int DT, bool COUNT>
static cudaError_t launch_march_m(const MarchArgs &a, cudaStream_t st) {
  // paper-literal blending of saturating samples: the paper's voxel size and a generic-M
  // kernel per payload type (evaluation counts do not depend on the blending rule)
  if (!COUNT && a.sequential)
    return a.M == 16 ? launch_march_t<DT, MARCH_CAP, false, 16, true>(a, st)
                     : launch_march_t<DT, MARCH_CAP, false, 0, true>(a, st);
  switch (a.M) {
    case 8: return launch_march_t<DT, march_cap<8>(), COUNT, 8>(a, st);
    case 16: return launch_march_t<DT, march_cap<16>(), COUNT, 16>(a, st);
    case 32: return launch_march_t<DT, march_cap<32>(), COUNT, 32>(a, st);
    default: return launch_march_t<DT, march_cap<0>(), COUNT, 0>(a, st);
  }
}

template <bool COUNT>
static cudaError_t launch_march_c(const MarchArgs &a, cudaStream_t st) {
  switch (a.dtype) {
    case MVP_F32: return launch_march_m<MVP_F32, COUNT>(a, st);
    case MVP_BF16: return launch_march_m<MVP_BF16, COUNT>(a, st);
    case MVP_F16: return launch_march_m<MVP_F16, COUNT>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_march(const MarchArgs &a, cudaStream_t st) {
  return a.n_eval ? launch_march_c<true>(a, st) : launch_march_c<false>(a, st);
}

cudaError_t launch_hits(const HitArgs &a, int64_t *counts, cudaStream_t st) {
  int64_t blocks = (a.geom.n_warp_tiles + TILE_WARPS - 1) / TILE_WARPS;
  size_t smem = sizeof(TileShared<1>) * TILE_WARPS;
  if (blocks > 0) {
    HitArgs c = a;
    c.counts = counts;
    k_hits<false><<<(unsigned)blocks, TILE_WARPS * 32, smem, st>>>(c);
  }
  k_offsets<<<1, 1024, 0, st>>>(counts, a.geom.n_rays, a.offs);
  return cudaGetLastError();
}

cudaError_t launch_hits_fill(const HitArgs &a, cudaStream_t st) {
  int64_t blocks = (a.geom.n_warp_tiles + TILE_WARPS - 1) / TILE_WARPS;
  size_t smem = sizeof(TileShared<1>) * TILE_WARPS;
  if (blocks > 0) k_hits<true><<<(unsigned)blocks, TILE_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mvp
