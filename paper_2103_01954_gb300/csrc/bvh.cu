// bvh.cu -- per-frame LBVH over oriented primitives (Sec. 3.2.1: the paper rebuilds
// a data-parallel BVH every frame because the primitives move; it cites Karras'
// construction from sorted Morton codes).
//
// Steps, all on one stream without host synchronisation (for n <= BVH_SORT1_N steps
// 1-3 are k_prims_partial and the one-block k_sort_one instead, for n <= BVH_SORTC_N
// k_prims_partial and the one-cluster k_sort_cluster):
//   1. k_bounds   : min/max of the centres (one block; exact).
//   2. k_prims    : rotation, membership pose, march transform, oriented-box world
//                   bounds, 30-bit Morton code of the centre.
//   3. radix sort : stable LSD sort of the 30-bit codes with the primitive index as
//                   value (4 passes of 8 bits: count, scan, scatter).
//   4. k_hierarchy: leaves and internal nodes of the binary radix tree over the
//                   unique keys (morton << 32 | k), one thread per node.
//   5. refit      : each internal node's box as the union of the leaves in its sorted
//                   range (k_refit_ranges), from 32- and 1024-leaf chunk unions.
#include <cooperative_groups.h>

#include <mutex>
#include <unordered_map>

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

// 30-bit Morton code of centre k in the centres' bounds `scene`.
__device__ __forceinline__ uint32_t morton_code(const float *__restrict__ t, int k, const float scene[6]) {
  const uint32_t qx = quant10(t[3 * k], scene[0], scene[3]);
  const uint32_t qy = quant10(t[3 * k + 1], scene[1], scene[4]);
  const uint32_t qz = quant10(t[3 * k + 2], scene[2], scene[5]);
  return (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
}

// Pose, march transform and world box of primitive k. A pose that defines no box (a
// non-finite value, a zero quaternion, a scale <= 0) sets STATUS_POSE and gets a
// box no ray meets: an inverted world box (lo = +1e30 > hi = -1e30, neutral in the
// nodes' unions and refused by the traversal) and a unit box centred at 1e30 for the
// exact test, so the primitive is absent from every image and gradient.
__device__ __forceinline__ void prim_setup(const float *__restrict__ t, const float *__restrict__ q,
                                           const float *__restrict__ s, int k, int M, Pose *__restrict__ pose,
                                           Xform *__restrict__ xf, float4 *__restrict__ pbox, int *status) {
  float tx = t[3 * k], ty = t[3 * k + 1], tz = t[3 * k + 2];
  float sx = s[3 * k], sy = s[3 * k + 1], sz = s[3 * k + 2];
  const float qw = q[4 * k], qx = q[4 * k + 1], qy = q[4 * k + 2], qz = q[4 * k + 3];
  const float qn = qw * qw + qx * qx + qy * qy + qz * qz;
  const bool ok = isfinite(tx) && isfinite(ty) && isfinite(tz) && sx > 0.0f && sy > 0.0f && sz > 0.0f &&
                  isfinite(sx) && isfinite(sy) && isfinite(sz) && qn > 0.0f && isfinite(qn);
  if (!ok) {
    if (status) atomicOr(status, STATUS_POSE);
    const float far = 1.0e30f;
    Pose P;
    P.p0 = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    P.p1 = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    P.p2 = make_float4(1.0f, far, far, far);
    P.p3 = make_float4(1.0f, 1.0f, 1.0f, 0.0f);
    pose[k] = P;
    Xform X;
    X.r0 = X.r1 = X.r2 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    xf[k] = X;
    pbox[2 * k] = make_float4(far, far, far, 0.0f);
    pbox[2 * k + 1] = make_float4(-far, -far, -far, 0.0f);
    return;
  }
  float R[9];
  rot_spec(qw, qx, qy, qz, R);
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
}

__global__ void k_prims(const float *__restrict__ t, const float *__restrict__ q, const float *__restrict__ s,
                        int n, int M, const float *__restrict__ scene, Pose *__restrict__ pose,
                        Xform *__restrict__ xf, float4 *__restrict__ pbox, uint32_t *__restrict__ keys,
                        int *__restrict__ vals, int *status) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float sc[6] = {scene[0], scene[1], scene[2], scene[3], scene[4], scene[5]};
  prim_setup(t, q, s, k, M, pose, xf, pbox, status);
  keys[k] = morton_code(t, k, sc);
  vals[k] = k;
}

// Pose, march transform and world box of each primitive, and per block the bounds of
// its centres (partial[block] = {lo xyz, hi xyz}) for the one-block sort to reduce.
__global__ void __launch_bounds__(256) k_prims_partial(const float *__restrict__ t, const float *__restrict__ q,
                                                       const float *__restrict__ s, int n, int M,
                                                       Pose *__restrict__ pose, Xform *__restrict__ xf,
                                                       float4 *__restrict__ pbox, float *__restrict__ partial,
                                                       int *status) {
  __shared__ float sb[8][6];
  pdl_trigger();  // the one-block sort may be scheduled now; it waits for this grid
  const int k = blockIdx.x * 256 + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  if (k < n) {
    prim_setup(t, q, s, k, M, pose, xf, pbox, status);
#pragma unroll
    for (int j = 0; j < 3; ++j) b[j] = b[3 + j] = t[3 * k + j];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    b[j] = warp_min(b[j]);
    b[3 + j] = warp_max(b[3 + j]);
  }
  if (lane == 0)
    for (int j = 0; j < 6; ++j) sb[warp][j] = b[j];
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = sb[0][threadIdx.x];
    for (int w = 1; w < 8; ++w) v = threadIdx.x < 3 ? fminf(v, sb[w][threadIdx.x]) : fmaxf(v, sb[w][threadIdx.x]);
    partial[6 * blockIdx.x + threadIdx.x] = v;
  }
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

// One-block sort for mid-sized n: reduces the per-block centre bounds, computes the
// Morton codes and sorts (code, primitive index) pairs: by buckets of the top code
// bits and an insertion sort per bucket, or, if some bucket is large (clustered
// centres), by a stable LSD radix (3 passes of 10 bits, ping-pong in global memory,
// tiles of 1024 keys in order). One launch instead of the multi-block sort's twelve;
// the result lands in (ka, va).
constexpr int SORT1_THREADS = 1024;
constexpr int SORT1_BITS = 10, SORT1_BINS = 1 << SORT1_BITS;
constexpr size_t SORT1_SMEM = sizeof(int) * (size_t)(SORT1_THREADS / 32) * SORT1_BINS;
constexpr int SORT1_BUCKET_BITS = 13, SORT1_BUCKETS = 1 << SORT1_BUCKET_BITS;
constexpr int SORT1_BUCKET_MAX = 64;  // largest bucket the insertion sort takes
static_assert((2 * SORT1_BUCKETS + 2 * BVH_SORT1_N) * sizeof(int) <= SORT1_SMEM,
              "bucket arrays and the staged keys live in the digit-count area");
static_assert(SORT1_BUCKETS % SORT1_THREADS == 0, "whole buckets per thread");
static_assert(BVH_SORT1_N % SORT1_THREADS == 0, "whole keys per thread");

__global__ void __launch_bounds__(SORT1_THREADS) k_sort_one(const float *__restrict__ t, int n,
                                                            const float *__restrict__ partial, int n_partial,
                                                            float *__restrict__ scene_out, uint32_t *ka, int *va,
                                                            uint32_t *kb, int *vb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int(*wcnt)[SORT1_BINS] = reinterpret_cast<int(*)[SORT1_BINS]>(smem_raw);  // [32][1024] per-warp digit counts
  __shared__ int base[SORT1_BINS + 1];
  __shared__ int tile_total[SORT1_BINS];
  __shared__ float sscene[6];
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  // centre bounds from the partials, then the codes: held in registers (key k =
  // tid + j * 1024 in code[j]), written to kb/vb only for the radix fallback (whose odd
  // pass count ends in ka/va)
  if (warp < 6) {  // warp j reduces component j, its lanes striding over the blocks
    float v = warp < 3 ? INFINITY : -INFINITY;
    for (int b = lane; b < n_partial; b += 32)
      v = warp < 3 ? fminf(v, partial[6 * b + warp]) : fmaxf(v, partial[6 * b + warp]);
    v = warp < 3 ? warp_min(v) : warp_max(v);
    if (lane == 0) {
      sscene[warp] = v;
      scene_out[warp] = v;
    }
  }
  __syncthreads();
  const float sc[6] = {sscene[0], sscene[1], sscene[2], sscene[3], sscene[4], sscene[5]};
  constexpr int KPT = BVH_SORT1_N / SORT1_THREADS;  // keys per thread
  uint32_t code[KPT];
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int k = tid + j * SORT1_THREADS;
    code[j] = k < n ? morton_code(t, k, sc) : 0u;
  }

  // Usual case: bucket by the top 13 code bits (atomic scatter), then sort each bucket
  // by (code, index) with insertion. The keys are unique, so this is the radix order.
  {
    int *cnt = reinterpret_cast<int *>(smem_raw);  // [8192] counts, then bucket starts
    int *cur = cnt + SORT1_BUCKETS;                // [8192] scatter cursors
    uint32_t *sk = reinterpret_cast<uint32_t *>(cur + SORT1_BUCKETS);  // [n] keys, bucketed, then sorted
    int *sv = reinterpret_cast<int *>(sk + BVH_SORT1_N);                // [n] their primitive indices
    for (int b = tid; b < SORT1_BUCKETS; b += SORT1_THREADS) cnt[b] = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < KPT; ++j)
      if (tid + j * SORT1_THREADS < n) atomicAdd(&cnt[code[j] >> (30 - SORT1_BUCKET_BITS)], 1);
    __syncthreads();
    // largest bucket, and this thread's 8 consecutive buckets' total
    constexpr int PER = SORT1_BUCKETS / SORT1_THREADS;
    int mx = 0, own = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int c = cnt[PER * tid + j];
      mx = max(mx, c);
      own += c;
    }
    mx = __reduce_max_sync(FULL, mx);
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) {
      tile_total[warp] = incl;
      base[warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
      const int w = tile_total[lane];
      int iw = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, iw, o);
        if (lane >= o) iw += u;
      }
      tile_total[lane] = iw - w;
      const int m = __reduce_max_sync(FULL, base[lane]);
      if (lane == 0) base[32] = m;
    }
    __syncthreads();
    const int bmax = base[32];
    if (bmax <= SORT1_BUCKET_MAX) {
      int run = tile_total[warp] + incl - own;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int c = cnt[PER * tid + j];
        cnt[PER * tid + j] = run;
        cur[PER * tid + j] = run;
        run += c;
      }
      __syncthreads();
      // scatter into shared memory, sort each bucket there, then write out coalesced
#pragma unroll
      for (int j = 0; j < KPT; ++j) {
        const int k = tid + j * SORT1_THREADS;
        if (k >= n) continue;
        const int pos = atomicAdd(&cur[code[j] >> (30 - SORT1_BUCKET_BITS)], 1);
        sk[pos] = code[j];
        sv[pos] = k;
      }
      __syncthreads();
      for (int b = tid; b < SORT1_BUCKETS; b += SORT1_THREADS) {
        const int s0 = cnt[b], e0 = b + 1 < SORT1_BUCKETS ? cnt[b + 1] : n;
        for (int x = s0 + 1; x < e0; ++x) {
          const uint32_t kx = sk[x];
          const int vx = sv[x];
          const uint64_t cx = ((uint64_t)kx << 32) | (uint32_t)vx;
          int y = x - 1;
          while (y >= s0 && (((uint64_t)sk[y] << 32) | (uint32_t)sv[y]) > cx) {
            sk[y + 1] = sk[y];
            sv[y + 1] = sv[y];
            --y;
          }
          sk[y + 1] = kx;
          sv[y + 1] = vx;
        }
      }
      __syncthreads();
      for (int k = tid; k < n; k += SORT1_THREADS) {
        ka[k] = sk[k];
        va[k] = sv[k];
      }
      return;
    }
    __syncthreads();  // a bucket holds more than SORT1_BUCKET_MAX keys: stable radix below
  }
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int k = tid + j * SORT1_THREADS;
    if (k < n) {
      kb[k] = code[j];
      vb[k] = k;
    }
  }
  __syncthreads();

  const uint32_t *kin = kb;
  const int *vin = vb;
  uint32_t *kout = ka;
  int *vout = va;
  for (int pass = 0; pass < 3; ++pass) {
    const int shift = SORT1_BITS * pass;
    // digit histogram and its exclusive scan
    base[tid] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += SORT1_THREADS) atomicAdd(&base[(kin[i] >> shift) & (SORT1_BINS - 1)], 1);
    __syncthreads();
    {
      const int v = base[tid];
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += u;
      }
      if (lane == 31) tile_total[warp] = incl;  // per-warp sums (reused below)
      __syncthreads();
      if (warp == 0) {
        const int w = tile_total[lane];
        int iw = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(FULL, iw, o);
          if (lane >= o) iw += u;
        }
        tile_total[lane] = iw - w;
      }
      __syncthreads();
      base[tid] = tile_total[warp] + incl - v;
      __syncthreads();
    }
    // stable scatter, one tile of 1024 keys at a time, in order
    for (int t0 = 0; t0 < n; t0 += SORT1_THREADS) {
      const int i = t0 + tid;
      const bool valid = i < n;
      const uint32_t key = valid ? kin[i] : 0u;
      const int val = valid ? vin[i] : 0;
      const int d = valid ? (int)((key >> shift) & (SORT1_BINS - 1)) : SORT1_BINS + lane;
#pragma unroll 4
      for (int w = 0; w < 32; ++w) wcnt[w][tid] = 0;
      __syncthreads();
      const unsigned peers = __match_any_sync(FULL, d);
      const int rank = __popc(peers & lt);
      if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
      __syncthreads();
      int sum = 0;
      for (int w = 0; w < 32; ++w) {
        const int c = wcnt[w][tid];
        wcnt[w][tid] = sum;
        sum += c;
      }
      tile_total[tid] = sum;
      __syncthreads();
      if (valid) {
        const int pos = base[d] + wcnt[warp][d] + rank;
        kout[pos] = key;
        vout[pos] = val;
      }
      __syncthreads();
      base[tid] += tile_total[tid];
      __syncthreads();
    }
    // every block thread wrote its keys; make them visible to the next pass's reads
    __threadfence_block();
    const uint32_t *tk = kout;
    const int *tv = vout;
    kout = const_cast<uint32_t *>(kin);
    vout = const_cast<int *>(vin);
    kin = tk;
    vin = tv;
  }
}

// One-cluster sort for BVH_SORT1_N < n <= BVH_SORTC_N: the eight CTAs of a thread-block
// cluster each hold a slice of 4096 (code, index) pairs in shared memory and run a stable
// LSD radix sort together (4 passes of 8 bits). Per pass a CTA ranks its whole slice at
// once (four keys per thread; per round and warp, the count of each digit), reads the
// other CTAs' digit counts through distributed shared memory to place its keys after every
// lower digit and after the same digit in lower slices, stages its slice in digit order,
// and stores each run of one digit into the slices that own those positions. Cluster
// barriers separate the steps. Two launches (k_prims_partial and this) instead of the
// multi-block sort's fourteen.
constexpr int SORTC_CTAS = 8;  // CTAs per cluster (the portable maximum)
constexpr int SORTC_THREADS = 1024;
constexpr int SORTC_SLICE = BVH_SORTC_N / SORTC_CTAS;        // keys per CTA
constexpr int SORTC_ROUNDS = SORTC_SLICE / SORTC_THREADS;    // keys per thread
constexpr int SORTC_BITS = 8, SORTC_BINS = 1 << SORTC_BITS, SORTC_PASSES = 4;  // 30-bit codes
constexpr int SORTC_WARPS = SORTC_THREADS / 32;
// keys and values twice (this pass, next pass), digit counts per round and warp, and per
// digit the slice's count, first position, first staged place and each round's first rank
constexpr size_t SORTC_SMEM = sizeof(int) * ((size_t)4 * SORTC_SLICE + (size_t)SORTC_ROUNDS * SORTC_WARPS * SORTC_BINS +
                                             (size_t)(3 + SORTC_ROUNDS) * SORTC_BINS);
static_assert(SORTC_ROUNDS * SORTC_WARPS * SORTC_BINS >= 2 * SORTC_SLICE, "the staged slice fits over the counts");
static_assert(SORTC_SLICE == SORTC_ROUNDS * SORTC_THREADS && SORTC_ROUNDS * SORTC_BINS == SORTC_THREADS,
              "one (round, digit) pair per thread in the count scan");
static_assert(SORTC_BITS * SORTC_PASSES >= 30, "the passes cover the Morton code");

__global__ void __launch_bounds__(SORTC_THREADS) k_sort_cluster(const float *__restrict__ t, int n,
                                                                const float *__restrict__ partial, int n_partial,
                                                                float *__restrict__ scene_out,
                                                                uint32_t *__restrict__ ka, int *__restrict__ va,
                                                                int *status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *key0 = reinterpret_cast<uint32_t *>(smem_raw);
  int *val0 = reinterpret_cast<int *>(key0 + SORTC_SLICE);
  uint32_t *key1 = reinterpret_cast<uint32_t *>(val0 + SORTC_SLICE);
  int *val1 = reinterpret_cast<int *>(key1 + SORTC_SLICE);
  // wcnt[j][w][d]: keys of digit d in round j, warp w (then their first rank in the round)
  int(*wcnt)[SORTC_WARPS][SORTC_BINS] = reinterpret_cast<int(*)[SORTC_WARPS][SORTC_BINS]>(val1 + SORTC_SLICE);
  int(*rbase)[SORTC_BINS] = reinterpret_cast<int(*)[SORTC_BINS]>(&wcnt[SORTC_ROUNDS][0][0]);  // [round][digit]
  int *hist = &rbase[SORTC_ROUNDS][0];  // the slice's digit counts (the other CTAs read them)
  int *base = hist + SORTC_BINS;        // each digit's first position for this slice's keys
  int *lstart = base + SORTC_BINS;      // each digit's first place in the slice's staged order
  __shared__ int wsum[SORTC_BINS / 32], lsum[SORTC_BINS / 32];
  __shared__ float sscene[6];
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int r = (int)cluster.block_rank();
  const int p0 = r * SORTC_SLICE;                    // the slice's first position
  const int cnt = max(0, min(n - p0, SORTC_SLICE));  // keys in it
  // centre bounds from the partials (each CTA reduces them), then the slice's codes
  if (warp < 6) {  // warp j reduces component j, its lanes striding over the blocks
    float v = warp < 3 ? INFINITY : -INFINITY;
    for (int b = lane; b < n_partial; b += 32)
      v = warp < 3 ? fminf(v, partial[6 * b + warp]) : fmaxf(v, partial[6 * b + warp]);
    v = warp < 3 ? warp_min(v) : warp_max(v);
    if (lane == 0) {
      sscene[warp] = v;
      if (r == 0) scene_out[warp] = v;
    }
  }
  __syncthreads();
  const float sc[6] = {sscene[0], sscene[1], sscene[2], sscene[3], sscene[4], sscene[5]};
  for (int i = tid; i < cnt; i += SORTC_THREADS) {
    key0[i] = morton_code(t, p0 + i, sc);
    val0[i] = p0 + i;
  }
  __syncthreads();
  uint32_t *kin = key0, *kout = key1;
  int *vin = val0, *vout = val1;
  for (int pass = 0; pass < SORTC_PASSES; ++pass) {
    const int shift = SORTC_BITS * pass;
    for (int x = tid; x < SORTC_ROUNDS * SORTC_WARPS * SORTC_BINS; x += SORTC_THREADS) (&wcnt[0][0][0])[x] = 0;
    __syncthreads();
    // round j holds positions j*1024 + tid, so (round, warp, lane) is the slice's order
    uint32_t key[SORTC_ROUNDS];
    int val[SORTC_ROUNDS], dig[SORTC_ROUNDS], rank[SORTC_ROUNDS];
#pragma unroll
    for (int j = 0; j < SORTC_ROUNDS; ++j) {
      const int i = j * SORTC_THREADS + tid;
      const bool valid = i < cnt;
      key[j] = valid ? kin[i] : 0u;
      val[j] = valid ? vin[i] : 0;
      dig[j] = valid ? (int)((key[j] >> shift) & (SORTC_BINS - 1)) : -1 - lane;  // invalid: unique, no count
      const unsigned peers = __match_any_sync(FULL, dig[j]);
      rank[j] = __popc(peers & lt);
      if (valid && rank[j] == 0) wcnt[j][warp][dig[j]] = __popc(peers);
    }
    __syncthreads();
    {  // (round jr, digit dr): counts over the round's warps -> first rank per warp
      const int jr = tid / SORTC_BINS, dr = tid % SORTC_BINS;
      int sum = 0;
      for (int w = 0; w < SORTC_WARPS; ++w) {
        const int c = wcnt[jr][w][dr];
        wcnt[jr][w][dr] = sum;
        sum += c;
      }
      rbase[jr][dr] = sum;  // the round's count, turned into its first rank below
    }
    __syncthreads();
    if (tid < SORTC_BINS) {
      int run = 0;
#pragma unroll
      for (int j = 0; j < SORTC_ROUNDS; ++j) {
        const int c = rbase[j][tid];
        rbase[j][tid] = run;
        run += c;
      }
      hist[tid] = run;
    }
    cluster.sync();  // every slice's counts are complete
    if (tid < SORTC_BINS) {
      // digit tid: its count over all slices, and in the slices before this one
      int tot = 0, below = 0;
#pragma unroll
      for (int q = 0; q < SORTC_CTAS; ++q) {
        const int h = cluster.map_shared_rank(hist, q)[tid];
        tot += h;
        below += q < r ? h : 0;
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += u;
      }
      if (lane == 31) wsum[warp] = incl;
      base[tid] = incl - tot + below;  // plus the lower warps' totals, below
      const int own = hist[tid];
      int lincl = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, lincl, o);
        if (lane >= o) lincl += u;
      }
      if (lane == 31) lsum[warp] = lincl;
      lstart[tid] = lincl - own;
    }
    __syncthreads();
    if (tid < SORTC_BINS) {
      int off = 0, loff = 0;
      for (int w = 0; w < warp; ++w) {
        off += wsum[w];
        loff += lsum[w];
      }
      base[tid] += off;
      lstart[tid] += loff;
    }
    __syncthreads();
    // The keys in digit order within the slice (staged over the counts, which are read
    // first), then each to the slice that owns its position: runs of one digit go to
    // consecutive positions, so a warp's stores to another CTA's slice coalesce.
    int lpos[SORTC_ROUNDS];
#pragma unroll
    for (int j = 0; j < SORTC_ROUNDS; ++j)
      lpos[j] = dig[j] < 0 ? -1 : lstart[dig[j]] + rbase[j][dig[j]] + wcnt[j][warp][dig[j]] + rank[j];
    __syncthreads();
    uint32_t *stage_k = reinterpret_cast<uint32_t *>(&wcnt[0][0][0]);
    int *stage_v = reinterpret_cast<int *>(stage_k + SORTC_SLICE);
#pragma unroll
    for (int j = 0; j < SORTC_ROUNDS; ++j) {
      if ((unsigned)lpos[j] < (unsigned)cnt) {
        stage_k[lpos[j]] = key[j];
        stage_v[lpos[j]] = val[j];
      } else if (dig[j] >= 0 && status) {
        atomicOr(status, STATUS_DEVICE);  // a position outside the slice: never expected
      }
    }
    __syncthreads();
    for (int i = tid; i < cnt; i += SORTC_THREADS) {
      const uint32_t k = stage_k[i];
      const int d = (int)((k >> shift) & (SORTC_BINS - 1));
      const int pos = base[d] + i - lstart[d];
      if ((unsigned)pos < (unsigned)n) {
        const int q = pos / SORTC_SLICE, li = pos - q * SORTC_SLICE;
        cluster.map_shared_rank(kout, q)[li] = k;
        cluster.map_shared_rank(vout, q)[li] = stage_v[i];
      } else if (status) {
        atomicOr(status, STATUS_DEVICE);  // a position outside [0, n): never expected
      }
    }
    cluster.sync();  // every key of the pass is in its slice; the counts may be reused
    uint32_t *tk = kin;
    kin = kout;
    kout = tk;
    int *tv = vin;
    vin = vout;
    vout = tv;
  }
  for (int i = tid; i < cnt; i += SORTC_THREADS) {
    ka[p0 + i] = kin[i];
    va[p0 + i] = vin[i];
  }
}

// ------------------------------------------------------------------ 4. hierarchy
// Children of internal node i of the binary radix tree over n sorted unique 64-bit
// keys (key(i) = morton << 32 | primitive): the direction of its range, its other
// end j, and the split (Karras). Children >= n-1 are leaves (n-1 + sorted index).
// prefix(a, b) = the number of leading bits keys a and b share, for 0 <= a, b < n.
template <class Prefix>
__device__ __forceinline__ void internal_children(const Prefix &prefix, int n, int i, int &lc, int &rc, int &j_end) {
  auto delta = [&](int a, int b) -> int {
    if (b < 0 || b >= n) return -1;
    return prefix(a, b);
  };
  int d = (delta(i, i + 1) - delta(i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(i, i - d);
  int lmax = 2;
  while (delta(i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int step = lmax >> 1; step >= 1; step >>= 1)
    if (delta(i, i + (l + step) * d) > dmin) l += step;
  int j = i + l * d;
  int dnode = delta(i, j);
  int sgap = 0;
  for (int div = 2;; div <<= 1) {
    int step = (l + div - 1) / div;
    if (delta(i, i + (sgap + step) * d) > dnode) sgap += step;
    if (step == 1) break;
  }
  int g = i + sgap * d + min(d, 0);
  lc = (min(i, j) == g) ? (n - 1 + g) : g;
  rc = (max(i, j) == g + 1) ? (n - 1 + g + 1) : g + 1;
  j_end = j;
}

__device__ __forceinline__ void write_leaf(Node *__restrict__ nodes, int n, int i, int k,
                                           const float4 *__restrict__ pbox) {
  float4 lo = pbox[2 * k], hi = pbox[2 * k + 1];
  Node L;
  L.lox = lo.x; L.loy = lo.y; L.loz = lo.z; L.left = -1 - k;
  L.hix = hi.x; L.hiy = hi.y; L.hiz = hi.z; L.right = 0;
  nodes[n - 1 + i] = L;
}

__device__ __forceinline__ void write_internal(Node *__restrict__ nodes, int i, int lc, int rc) {
  Node N;
  N.lox = N.loy = N.loz = 0.0f;
  N.hix = N.hiy = N.hiz = 0.0f;
  N.left = lc;
  N.right = rc;
  nodes[i] = N;
}

// One thread per node: leaf i (node n-1+i), the leaf position of its primitive
// (rank), and internal node i with the sorted leaf range [first, last] it covers
// (range[i]). Blocks of 1024 also union their leaves'
// boxes in chunks of 32 (chunk1, one per warp) and 1024 (chunk2, one per block) for
// the range refit.
// STAGE 1 (n <= HIER_STAGE_N): every block first copies the sorted codes and primitive
// indices into shared memory, so the searches of the hierarchy read shared memory
// instead of L2. STAGE 2 (n <= BVH_SORTC_N): the codes alone (128 KB at most); the
// indices, which only break ties between equal codes, are read from global memory.
constexpr int HIER_THREADS = 1024;
constexpr int HIER_STAGE_N = 8192;  // keys staged per block: 8 bytes each, 64 KB at most
template <int STAGE>
__global__ void __launch_bounds__(HIER_THREADS) k_hierarchy(const uint32_t *__restrict__ km,
                                                            const int *__restrict__ kv, int n,
                                                            const float4 *__restrict__ pbox, Node *__restrict__ nodes,
                                                            int2 *__restrict__ range, float4 *__restrict__ chunk1,
                                                            float4 *__restrict__ chunk2, int *__restrict__ rank) {
  __shared__ float sc[32][6];
  extern __shared__ __align__(16) unsigned char hier_smem[];
  uint32_t *skm = reinterpret_cast<uint32_t *>(hier_smem);
  int *skv = reinterpret_cast<int *>(hier_smem + sizeof(uint32_t) * (STAGE > 0 ? n : 0));
  pdl_wait();
  pdl_trigger();
  if (STAGE > 0) {
    for (int a = threadIdx.x; a < n; a += HIER_THREADS) {
      skm[a] = km[a];
      if (STAGE == 1) skv[a] = kv[a];
    }
    __syncthreads();
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = blockIdx.x * HIER_THREADS + tid;
  float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  if (i < n) {
    const int k = kv[i];
    write_leaf(nodes, n, i, k, pbox);  // leaf i: node n-1+i
    rank[k] = i;
    const float4 lo = pbox[2 * k], hi = pbox[2 * k + 1];
    b[0] = lo.x; b[1] = lo.y; b[2] = lo.z; b[3] = hi.x; b[4] = hi.y; b[5] = hi.z;
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    b[j] = warp_min(b[j]);
    b[3 + j] = warp_max(b[3 + j]);
  }
  if (lane == 0) {
    if (i < n) {
      chunk1[2 * (i >> 5)] = make_float4(b[0], b[1], b[2], 0.0f);
      chunk1[2 * (i >> 5) + 1] = make_float4(b[3], b[4], b[5], 0.0f);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) sc[warp][j] = b[j];
  }
  __syncthreads();
  if (warp == 0) {
    float c[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c[j] = warp_min(sc[lane][j]);
      c[3 + j] = warp_max(sc[lane][3 + j]);
    }
    if (lane == 0) {
      chunk2[2 * blockIdx.x] = make_float4(c[0], c[1], c[2], 0.0f);
      chunk2[2 * blockIdx.x + 1] = make_float4(c[3], c[4], c[5], 0.0f);
    }
  }
  if (i == 0) {  // the traversal's starting cut until the refit widens it: the root alone
    int *cut = reinterpret_cast<int *>(nodes + 2 * n - 1);
    cut[0] = 1;
    cut[1] = 0;
  }
  if (i >= n - 1) return;
  auto prefix = [&](int a, int b) -> int {
    if (STAGE == 2) {  // codes first; equal codes share 32 bits and then those of the indices
      const uint32_t ca = skm[a], cb = skm[b];
      return ca != cb ? __clz((int)(ca ^ cb)) : 32 + __clz((int)((uint32_t)kv[a] ^ (uint32_t)kv[b]));
    }
    const uint64_t ka = STAGE == 1 ? ((uint64_t)skm[a] << 32) | (uint32_t)skv[a]
                                   : ((uint64_t)km[a] << 32) | (uint32_t)kv[a];
    const uint64_t kb = STAGE == 1 ? ((uint64_t)skm[b] << 32) | (uint32_t)skv[b]
                                   : ((uint64_t)km[b] << 32) | (uint32_t)kv[b];
    return __clzll(ka ^ kb);
  };
  int lc, rc, j;
  internal_children(prefix, n, i, lc, rc, j);
  write_internal(nodes, i, lc, rc);
  range[i] = make_int2(min(i, j), max(i, j));
}

// ------------------------------------------------------------------ 5. refit
// Box of every internal node as the union of the leaves in its sorted range (the
// same min/max as a bottom-up union of children, so the same bits): one warp per
// node covers the range with whole 1024-leaf and 32-leaf chunks where it can and
// single leaves at its ends, a few coalesced loads per lane. No node waits for
// another.
constexpr int REFIT_WARPS = 8;

// The traversal's starting cut (one warp): the tree expanded level by level from the root
// while the nodes still fit 32, so a traversal tests the top levels in one step instead
// of one step per level. Written as {count, nodes...} (nodes cover every leaf once).
__device__ void build_cut(const Node *__restrict__ nodes, int n, int *buf, int *cut) {
  const int lane = threadIdx.x & 31;
  int node = lane == 0 ? 0 : -1;
  int cnt = 1;
  while (true) {
    const bool inner = node >= 0 && node < n - 1;
    const int ni = __popc(__ballot_sync(FULL, inner));
    if (ni == 0 || cnt + ni > 32) break;
    int l = -1, r = -1;
    if (inner) {
      l = nodes[node].left;
      r = nodes[node].right;
    }
    const int k = node < 0 ? 0 : (inner ? 2 : 1);  // entries this lane's node becomes
    int pre = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, pre, o);
      if (lane >= o) pre += v;
    }
    pre -= k;
    if (k == 1) buf[pre] = node;
    if (k == 2) {
      buf[pre] = l;
      buf[pre + 1] = r;
    }
    __syncwarp();
    cnt += ni;
    node = lane < cnt ? buf[lane] : -1;
    __syncwarp();
  }
  if (lane == 0) cut[0] = cnt;
  if (lane < cnt) cut[1 + lane] = node;
}

__global__ void __launch_bounds__(REFIT_WARPS * 32) k_refit_ranges(Node *__restrict__ nodes,
                                                                   const int2 *__restrict__ range,
                                                                   const float4 *__restrict__ chunk1,
                                                                   const float4 *__restrict__ chunk2, int n) {
  pdl_wait();
  pdl_trigger();  // the march may be scheduled now; it waits for this grid
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == gridDim.x - 1) {  // the extra block: the traversal's starting cut
    __shared__ int buf[32];
    if (threadIdx.x < 32) build_cut(nodes, n, buf, reinterpret_cast<int *>(nodes + 2 * n - 1));
    return;
  }
  const int i = blockIdx.x * REFIT_WARPS + (threadIdx.x >> 5);
  if (i >= n - 1) return;
  const int2 r = range[i];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  // union of boxes [s, e) of an array of {lo, hi} float4 pairs
  auto add = [&](const float4 *box, int s, int e) {
    for (int a = s + lane; a < e; a += 32) {
      const float4 b0 = __ldg(box + 2 * a), b1 = __ldg(box + 2 * a + 1);
      lo[0] = fminf(lo[0], b0.x);
      lo[1] = fminf(lo[1], b0.y);
      lo[2] = fminf(lo[2], b0.z);
      hi[0] = fmaxf(hi[0], b1.x);
      hi[1] = fmaxf(hi[1], b1.y);
      hi[2] = fmaxf(hi[2], b1.z);
    }
  };
  const float4 *leaf = reinterpret_cast<const float4 *>(nodes + (n - 1));
  const int a = r.x, e = r.y + 1;
  if (e - a <= 64) {
    add(leaf, a, e);
  } else {
    const int ca = (a + 31) >> 5, cb = e >> 5;  // whole 32-leaf chunks [ca, cb)
    add(leaf, a, ca * 32);
    add(leaf, cb * 32, e);
    if (cb - ca <= 64) {
      add(chunk1, ca, cb);
    } else {
      const int da = (ca + 31) >> 5, db = cb >> 5;  // whole 1024-leaf chunks [da, db)
      add(chunk1, ca, da * 32);
      add(chunk1, db * 32, cb);
      add(chunk2, da, db);
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lo[j] = warp_min(lo[j]);
    hi[j] = warp_max(hi[j]);
  }
  if (lane == 0) {
    Node &N = nodes[i];
    N.lox = lo[0];
    N.loy = lo[1];
    N.loz = lo[2];
    N.hix = hi[0];
    N.hiy = hi[1];
    N.hiz = hi[2];
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
  size_t o_nodes = off; off = align_up(off + (size_t)(2 * cap + CUT_NODES) * sizeof(Node));
  size_t o_par = off; off = align_up(off + (size_t)(2 * cap) * sizeof(int));
  size_t o_gmc = off; off = align_up(off + (size_t)cap * 12 * sizeof(float));
  size_t o_rank = off; off = align_up(off + (size_t)cap * sizeof(int));
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
  b.gmc = reinterpret_cast<float *>(p + o_gmc);
  b.rank = reinterpret_cast<int *>(p + o_rank);
  return cudaSuccess;
}

void bvh_release(BvhBuffers &b) {
  if (b.base) cudaFree(b.base);
  b = BvhBuffers();
}

// Whether the one-cluster sort can run in the current context: its dynamic shared memory
// is opted in and the GPU can hold a cluster of eight such CTAs. Asked once per context
// (allow_dynamic_smem remembers its opt-in per context; the answer is cached beside it).
static bool cluster_sort_ready() {
  if (allow_dynamic_smem(reinterpret_cast<const void *>(k_sort_cluster), SORTC_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  static std::mutex mu;
  static std::unordered_map<unsigned long long, bool> ready;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(mu);
  auto it = ready.find(ctx);
  if (it != ready.end()) return it->second;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(SORTC_CTAS);
  cfg.blockDim = dim3(SORTC_THREADS);
  cfg.dynamicSmemBytes = SORTC_SMEM;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = SORTC_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&clusters, k_sort_cluster, &cfg) == cudaSuccess && clusters >= 1;
  if (!ok) cudaGetLastError();
  ready[ctx] = ok;
  return ok;
}

cudaError_t bvh_build(BvhBuffers &b, const float *t, const float *q, const float *s, int n, int M,
                      cudaStream_t st, int *status) {
  b.n = n;
  b.M = M;
  if (n == 0) return cudaGetLastError();
  const int G = (n + SORT_TILE - 1) / SORT_TILE;
  const int n_partial = (n + 255) / 256;
  if (n <= BVH_SORT1_N && (size_t)6 * n_partial <= (size_t)256 * G) {
    // mid-sized n: primitives with per-block bounds, then one block sorts
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(k_sort_one), SORT1_SMEM);
    if (e != cudaSuccess) return e;
    float *partial = reinterpret_cast<float *>(b.counts);  // 6 floats per 256 primitives
    k_prims_partial<<<n_partial, 256, 0, st>>>(t, q, s, n, M, b.pose, b.xf, b.pbox, partial, status);
    // the rest of the chain is scheduled while its predecessor finishes (each kernel
    // waits for it before touching memory)
    e = pdl_launch(k_sort_one, dim3(1), dim3(SORT1_THREADS), SORT1_SMEM, st, t, n, (const float *)partial,
                   n_partial, b.scene, b.keys_a, b.vals_a, b.keys_b, b.vals_b);
    if (e != cudaSuccess) return e;
  } else if (n <= BVH_SORTC_N && (size_t)6 * n_partial <= (size_t)256 * G && cluster_sort_ready()) {
    // up to 32768: primitives with per-block bounds, then one cluster of eight CTAs sorts
    float *partial = reinterpret_cast<float *>(b.counts);
    k_prims_partial<<<n_partial, 256, 0, st>>>(t, q, s, n, M, b.pose, b.xf, b.pbox, partial, status);
    cudaError_t e = cluster_launch(k_sort_cluster, dim3(SORTC_CTAS), dim3(SORTC_THREADS), SORTC_CTAS, SORTC_SMEM, st,
                                   t, n, (const float *)partial, n_partial, b.scene, b.keys_a, b.vals_a, status);
    if (e != cudaSuccess) return e;
  } else {
    k_bounds<<<1, 1024, 0, st>>>(t, n, b.scene);
    k_prims<<<(n + 255) / 256, 256, 0, st>>>(t, q, s, n, M, b.scene, b.pose, b.xf, b.pbox, b.keys_a, b.vals_a,
                                             status);
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
  }
  // scratch after the sort: ranges in the parent buffer (2n ints), chunk boxes in the
  // second key and value buffers (n/32 and n/1024 boxes of 32 bytes fit in 4n bytes)
  int2 *range = reinterpret_cast<int2 *>(b.parent);
  float4 *chunk1 = reinterpret_cast<float4 *>(b.keys_b), *chunk2 = reinterpret_cast<float4 *>(b.vals_b);
  const int stage = n <= HIER_STAGE_N ? 1 : (n <= BVH_SORTC_N ? 2 : 0);
  const size_t hsmem = stage == 1 ? (size_t)n * 8 : (stage == 2 ? (size_t)n * 4 : 0);
  const dim3 hgrid((n + HIER_THREADS - 1) / HIER_THREADS), hblock(HIER_THREADS);
  cudaError_t e = cudaSuccess;
  if (stage == 1) {
    e = allow_dynamic_smem(reinterpret_cast<const void *>(k_hierarchy<1>), hsmem);
    if (e == cudaSuccess)
      e = pdl_launch(k_hierarchy<1>, hgrid, hblock, hsmem, st, (const uint32_t *)b.keys_a, (const int *)b.vals_a, n,
                     (const float4 *)b.pbox, b.nodes, range, chunk1, chunk2, b.rank);
  } else if (stage == 2) {
    e = allow_dynamic_smem(reinterpret_cast<const void *>(k_hierarchy<2>), hsmem);
    if (e == cudaSuccess)
      e = pdl_launch(k_hierarchy<2>, hgrid, hblock, hsmem, st, (const uint32_t *)b.keys_a, (const int *)b.vals_a, n,
                     (const float4 *)b.pbox, b.nodes, range, chunk1, chunk2, b.rank);
  } else {
    e = pdl_launch(k_hierarchy<0>, hgrid, hblock, 0, st, (const uint32_t *)b.keys_a, (const int *)b.vals_a, n,
                   (const float4 *)b.pbox, b.nodes, range, chunk1, chunk2, b.rank);
  }
  if (e == cudaSuccess && n > 1)
    e = pdl_launch(k_refit_ranges, dim3((n - 1 + REFIT_WARPS - 1) / REFIT_WARPS + 1), dim3(REFIT_WARPS * 32), 0, st,
                   b.nodes, (const int2 *)range, (const float4 *)chunk1, (const float4 *)chunk2, n);
  return e != cudaSuccess ? e : cudaGetLastError();
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
