// backward.cu -- adjoint of the ray march (Sec. 3.2.2: the additive accumulation
// lets the backward pass replay samples instead of storing the per-sample graph).
//
// With S the clamped sample of a ray (if any), rho = c_S/a_S and beta = (1-T_S)/a_S
// saved by the forward, and gI = dL/dI~, gA = dL/dA - gI.bg:
//   no clamp : dL/da_i = gA,              dL/dc_i = gI        (i <= i_last)
//   i < S    : dL/da_i = -gI.rho,         dL/dc_i = gI
//   i = S    : dL/da_S = -(gI.rho) beta,  dL/dc_S = gI beta
// These do not depend on the other samples, so the replay can run primitive by
// primitive: for each window entry (warp-uniform) and each of its samples, the
// lanes inside recompute the trilinear RGBA, scatter
//   dL/dalpha = dt (dL/da + dL/dc . rgb), dL/drgb = dt alpha dL/dc
// to the 8 cell voxels (float4 atomics), and accumulate dL/du (u = voxel
// coordinate) times p = x - t_k and dL/du itself in registers; one warp reduction
// per entry adds those 12 sums to the primitive's accumulator. A per-primitive
// kernel then maps them to dL/dt, dL/dq, dL/ds through u = diag(h/s) R^T p + h.
#include <algorithm>

#include "march.cuh"

namespace mvp {

// The adjoint of one warp tile whose lane ray is L (SEQ: the forward blended the
// saturating samples in BVH order; RANGED: only the primitives at the BVH positions
// of lr, the rest of the tile's work being another call's).
template <int DT, int CAP, int MT, bool SEQ, bool RANGED = false>
__device__ __forceinline__ void backward_tile(TileShared<CAP> &sh, const BwdArgs &b, const LaneRay &L,
                                              LeafRange lr = LeafRange{nullptr, 0, 0}) {
  const MarchArgs &a = b.m;
  const int lane = threadIdx.x & 31;
  const bool valid = L.r >= 0;

  // per-ray adjoint constants
  int i_last = -1, i_clamp = -1, rank_clamp = -1;
  float ga_pre = 0.0f, gcr = 0.0f, gcg = 0.0f, gcb = 0.0f;
  float ga_s = 0.0f, gsr = 0.0f, gsg = 0.0f, gsb = 0.0f;
  if (valid) {
    const Saved S = b.saved[L.r];
    const float4 g = reinterpret_cast<const float4 *>(b.grad)[L.r];
    i_last = S.i_last;
    i_clamp = S.i_clamp;
    if (SEQ) rank_clamp = S.rank_clamp;
    gcr = g.x;
    gcg = g.y;
    gcb = g.z;
    if (i_clamp < 0) {
      ga_pre = g.w - (g.x * a.bg[0] + g.y * a.bg[1] + g.z * a.bg[2]);
    } else {
      const float grho = g.x * S.rho_r + g.y * S.rho_g + g.z * S.rho_b;
      ga_pre = -grho;
      ga_s = -grho * S.beta;
      gsr = g.x * S.beta;
      gsg = g.y * S.beta;
      gsb = g.z * S.beta;
    }
  }
  if (a.n_prims <= 0 || a.n_steps <= 0) return;
  make_packet(sh.pk, valid, L.o, L.d, a.t_far);
  const int M = MT > 0 ? MT : a.M, M2 = M * M;
  const float Mm1 = (float)(M - 1);
  constexpr int VB = DT == MVP_F32 ? 16 : 8;
  const int64_t prim_bytes = (int64_t)M2 * M * VB;
  const int max_last = __reduce_max_sync(FULL, i_last);

  int w0 = 0, wlen = a.n_steps, skip = 0;
  while (w0 <= max_last) {
    int w1 = min(a.n_steps, w0 + wlen);
    int ne = build_window<CAP, RANGED>(sh, a.nodes, a.pose, a.xf, reinterpret_cast<const char *>(a.payload),
                                       prim_bytes, a.n_prims, L, valid ? i_last : -1, a.t_near, a.t_far, a.dt,
                                       a.n_steps, w0, w1, skip, a.status, lr);
    if (ne == WINDOW_STACK) {
      if (lane == 0) atomicOr(a.status, STATUS_CAPACITY);
      return;
    }
    if (ne == WINDOW_FULL && w1 - w0 > 1) {  // split the depth range
      wlen = (w1 - w0 + 1) >> 1;
      continue;
    }
    // A one-sample window with more than CAP primitives is replayed in batches of
    // CAP (entries are independent here): the next pass skips the ones done.
    const int cnt = ne >= 0 ? ne : CAP;
    for (int e = 0; e < cnt; ++e) {
      const int k = sh.ek[e];
      const Xform X = sh.exf[e];
      const void *pbase = sh.eptr[e];
      int lo, hi;
      lane_range(sh, e, lane, lo, hi);
      const float4 tk = __ldg(reinterpret_cast<const float4 *>(a.pose + k) + 2);  // {R22, t0, t1, t2}
      const int rk = SEQ ? __ldg(a.rank + k) : 0;  // this primitive's leaf rank
      float2 acc[6];  // the 12 pose accumulators as packed pairs
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] = make_float2(0.0f, 0.0f);
      // Each lane walks its own samples of the primitive from its own first one (the
      // samples are independent here), so the warp loops max(count) times rather
      // than over the union of the lanes' ranges.
      const int cnt = max(hi - lo + 1, 0);
      const int max_cnt = __reduce_max_sync(FULL, cnt);
      const int64_t kbase = (int64_t)k * M2 * M;
      int held = -1;  // voxel (within the primitive) whose cell corners are held
      float4 c000, c001, c010, c011, c100, c101, c110, c111;
      // the held cell's 8 corner shares of dL/d(rgba), summed over the lane's consecutive
      // samples in that cell and reduced into g_payload once the lane leaves it
      float4 s000, s001, s010, s011, s100, s101, s110, s111;
      const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      s000 = s001 = s010 = s011 = s100 = s101 = s110 = s111 = zero4;
      float4 *G = b.g_payload ? reinterpret_cast<float4 *>(b.g_payload) + kbase : nullptr;
#define MVP_FLUSH(vox)                                                                                 \
  {                                                                                                    \
    float4 *g_ = G + (vox);                                                                            \
    atomicAdd(g_, s000), atomicAdd(g_ + 1, s001), atomicAdd(g_ + M, s010), atomicAdd(g_ + M + 1, s011); \
    atomicAdd(g_ + M2, s100), atomicAdd(g_ + M2 + 1, s101), atomicAdd(g_ + M2 + M, s110);             \
    atomicAdd(g_ + M2 + M + 1, s111);                                                                  \
    s000 = s001 = s010 = s011 = s100 = s101 = s110 = s111 = zero4;                                     \
  }
      for (int it = 0; it < max_cnt; ++it) {
        const int i = lo + it;
        const bool in = it < cnt;
        if (!in) continue;
        // sequential rule at the clamped sample: the primitive before the clamped one in
        // BVH order is differentiated like a sample before it (role 1), the clamped one
        // contributes w_J c_J (role 2), those after it nothing (role 3)
        const int role = (i == i_clamp && rank_clamp >= 0) ? (rk < rank_clamp ? 1 : (rk == rank_clamp ? 2 : 3)) : 0;
        if (role == 3) continue;
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
        float4 gv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int vo = -1;
        {
          const float ti = sample_t(a.t_near, a.dt, i);
          const float x0 = fmaf(ti, L.d[0], L.o[0]);
          const float x1 = fmaf(ti, L.d[1], L.o[1]);
          const float x2 = fmaf(ti, L.d[2], L.o[2]);
          const float ux = fmaf(X.r0.x, x0, fmaf(X.r0.y, x1, fmaf(X.r0.z, x2, X.r0.w)));
          const float uy = fmaf(X.r1.x, x0, fmaf(X.r1.y, x1, fmaf(X.r1.z, x2, X.r1.w)));
          const float uz = fmaf(X.r2.x, x0, fmaf(X.r2.y, x1, fmaf(X.r2.z, x2, X.r2.w)));
          const bool kx = ux >= 0.0f && ux <= Mm1, ky = uy >= 0.0f && uy <= Mm1, kz = uz >= 0.0f && uz <= Mm1;
          const int ix = voxel_cell(ux, M - 2, fx), iy = voxel_cell(uy, M - 2, fy), iz = voxel_cell(uz, M - 2, fz);
          vo = iz * M2 + iy * M + ix;  // voxel within the primitive
          if (!MVP_IN_BOUNDS(vo >= 0 && vo + M2 + M + 1 < M2 * M, a.status)) continue;
          if (vo != held) {            // consecutive samples often stay in one cell
            if (G && held >= 0) MVP_FLUSH(held);
            c000 = Voxel<DT>::load(pbase, vo);
            c001 = Voxel<DT>::load(pbase, vo + 1);
            c010 = Voxel<DT>::load(pbase, vo + M);
            c011 = Voxel<DT>::load(pbase, vo + M + 1);
            c100 = Voxel<DT>::load(pbase, vo + M2);
            c101 = Voxel<DT>::load(pbase, vo + M2 + 1);
            c110 = Voxel<DT>::load(pbase, vo + M2 + M);
            c111 = Voxel<DT>::load(pbase, vo + M2 + M + 1);
            held = vo;
          }
          // the forward march's interpolation, rounding for rounding
          const float2 wx = splat2(fx), nwx = splat2(-fx), wy = splat2(fy), nwy = splat2(-fy);
          const float4 c00 = lerp4x2(c000, c001, wx, nwx), c01 = lerp4x2(c010, c011, wx, nwx);
          const float4 c10 = lerp4x2(c100, c101, wx, nwx), c11 = lerp4x2(c110, c111, wx, nwx);
          const float4 c0 = lerp4x2(c00, c01, wy, nwy), c1 = lerp4x2(c10, c11, wy, nwy);
          const float4 val = lerp4x2(c0, c1, splat2(fz), splat2(-fz));
          const bool at_clamp = i == i_clamp && role == 0;
          const float ga = at_clamp ? ga_s : ga_pre;
          const float gr = at_clamp ? gsr : gcr, gg = at_clamp ? gsg : gcg, gb = at_clamp ? gsb : gcb;
          // dL/d(rgba) of this primitive's sample
          gv = role == 2 ? make_float4(gsr, gsg, gsb, 0.0f)  // w_J dL/dI
                         : make_float4(a.dt * val.w * gr, a.dt * val.w * gg, a.dt * val.w * gb,
                                       a.dt * (ga + gr * val.x + gg * val.y + gb * val.z));
          if (b.gmc) {
            // dval/du along each axis (zero along an axis where u was clamped), on packed pairs
            const float2 wz = splat2(fz), nwz = splat2(-fz);
            const float4 dx0 = lerp4x2(sub4x2(c001, c000), sub4x2(c011, c010), wy, nwy);
            const float4 dx1 = lerp4x2(sub4x2(c101, c100), sub4x2(c111, c110), wy, nwy);
            const float4 dvx = lerp4x2(dx0, dx1, wz, nwz);
            const float4 dvy = lerp4x2(sub4x2(c01, c00), sub4x2(c11, c10), wz, nwz);
            const float4 dvz = sub4x2(c1, c0);
            const float gux = kx ? dot4x2(gv, dvx) : 0.0f;
            const float guy = ky ? dot4x2(gv, dvy) : 0.0f;
            const float guz = kz ? dot4x2(gv, dvz) : 0.0f;
            const float p0 = x0 - tk.y, p1 = x1 - tk.z, p2 = x2 - tk.w;
            // acc = (gux p, guy p, guz p, gux, guy, guz) as 6 packed pairs
            acc[0] = __ffma2_rn(splat2(gux), make_float2(p0, p1), acc[0]);
            acc[1] = __ffma2_rn(make_float2(gux, guy), make_float2(p2, p0), acc[1]);
            acc[2] = __ffma2_rn(splat2(guy), make_float2(p1, p2), acc[2]);
            acc[3] = __ffma2_rn(splat2(guz), make_float2(p0, p1), acc[3]);
            acc[4] = __ffma2_rn(make_float2(guz, gux), make_float2(p2, 1.0f), acc[4]);
            acc[5] = __ffma2_rn(make_float2(guy, guz), make_float2(1.0f, 1.0f), acc[5]);
          }
        }
        if (G) {
          // this sample's trilinear-weighted shares of gv, added to the held cell's
          const float wx0 = 1.0f - fx, wy0 = 1.0f - fy, wz0 = 1.0f - fz;
          const float w00 = wy0 * wz0, w01 = fy * wz0, w10 = wy0 * fz, w11 = fy * fz;
          const float2 glo = lo2(gv), ghi = hi2(gv);
#define MVP_SHARE(S, WGT)                                                                \
  {                                                                                      \
    const float2 wg = splat2(WGT);                                                       \
    const float2 l_ = __ffma2_rn(wg, glo, lo2(S)), h_ = __ffma2_rn(wg, ghi, hi2(S));     \
    S = make_float4(l_.x, l_.y, h_.x, h_.y);                                             \
  }
          MVP_SHARE(s000, wx0 * w00);
          MVP_SHARE(s001, fx * w00);
          MVP_SHARE(s010, wx0 * w01);
          MVP_SHARE(s011, fx * w01);
          MVP_SHARE(s100, wx0 * w10);
          MVP_SHARE(s101, fx * w10);
          MVP_SHARE(s110, wx0 * w11);
          MVP_SHARE(s111, fx * w11);
#undef MVP_SHARE
        }
      }
      if (G && held >= 0) MVP_FLUSH(held);
#undef MVP_FLUSH
      if (b.gmc) {
        float sums[12];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          sums[2 * c] = warp_sum(acc[c].x);
          sums[2 * c + 1] = warp_sum(acc[c].y);
        }
        if (lane < 12) {
          float mine = sums[0];
#pragma unroll
          for (int c = 1; c < 12; ++c)
            if (lane == c) mine = sums[c];
          if (mine != 0.0f) atomicAdd(b.gmc + 12 * (int64_t)k + lane, mine);
        }
      }
    }
    if (ne == WINDOW_FULL) {
      skip += CAP;
      continue;
    }
    skip = 0;
    w0 = w1;
    wlen = min(a.n_steps, wlen * 2);
  }
}

// The tile schedule as in the frame kernel (its own cost record: the adjoint's
// expensive tiles are not quite the forward's).
#ifndef MVP_BWD_MINB
#define MVP_BWD_MINB 3  // resident blocks per SM the adjoint is compiled for
#endif

template <int DT, int CAP, int MT, bool SEQ>
__global__ void __launch_bounds__(TILE_WARPS * 32, MVP_BWD_MINB) k_backward(BwdArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MarchArgs &a = b.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<CAP> &sh = reinterpret_cast<TileShared<CAP> *>(smem_raw)[warp];
  const int64_t slot = (int64_t)blockIdx.x * TILE_WARPS + warp;
  if (slot >= a.geom.n_warp_tiles) return;
  int64_t wt = slot;
  if (a.order) {
    const int o = __ldg(a.order + slot);
    if (o >= 0 && o < a.geom.n_warp_tiles) wt = o;
  }
  LaneRay L;
  load_lane_ray(L, a.o, a.d, tile_ray(a.geom, wt, lane));
  if (__ballot_sync(FULL, L.r >= 0) == 0) return;
  if (lane == 0) sh.clk = (unsigned int)clock();
  backward_tile<DT, CAP, MT, SEQ>(sh, b, L);
  if (a.cost) {
    __syncwarp();
    if (lane == 0) {
      int64_t t = slot;
      if (a.order) {
        const int o = __ldg(a.order + slot);
        if (o >= 0 && o < a.geom.n_warp_tiles) t = o;
      }
      a.cost[t] = (unsigned int)clock() - sh.clk;
    }
  }
}

// ------------------------------------------------------------------ primitive groups
// When the payload and its gradient outgrow L2, the four cameras' tiles of the
// differentiation workload would each sweep them from DRAM. The grouped adjoint
// instead cuts the primitives into groups of consecutive BVH positions (spatially
// compact, each sized to stay in L2 with its gradient) and replays every tile once per
// group it meets, group after group, so a group's payload and g_payload lines are
// read and written back about once.

// Shared memory of the group-mask pass: the traversal's buffers only.
struct TraverseShared {
  Packet pk;
  int stack[STACK];
  int cand[CBUF];
};

// mask[t] = the groups (bit g: BVH positions [g gsize, (g+1) gsize)) whose primitives
// tile t's rays may meet up to their last live sample: one traversal of the tile's
// packet, each candidate kept if its oriented box passes the packet test. A tile whose
// traversal overflows the stack gets every group, so its replay reports the overflow.
__global__ void __launch_bounds__(TILE_WARPS * 32) k_bwd_groups(BwdArgs b, int gsize, int n_groups,
                                                                unsigned long long *__restrict__ mask) {
  __shared__ TraverseShared shm[TILE_WARPS];
  const MarchArgs &a = b.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TraverseShared &sh = shm[warp];
  const int64_t slot = (int64_t)blockIdx.x * TILE_WARPS + warp;
  if (slot >= a.geom.n_warp_tiles) return;
  LaneRay L;
  load_lane_ray(L, a.o, a.d, tile_ray(a.geom, slot, lane));
  const bool valid = L.r >= 0;
  const int i_last = valid ? b.saved[L.r].i_last : -1;
  const int max_last = __reduce_max_sync(FULL, i_last);
  unsigned long long m = 0;
  if (max_last >= 0 && a.n_prims > 0 && a.n_steps > 0) {
    make_packet(sh.pk, valid, L.o, L.d, a.t_far);
    const float ta = sample_t(a.t_near, a.dt, 0), tb = sample_t(a.t_near, a.dt, min(max_last, a.n_steps - 1));
    const float slack = 1.0e-5f * (fabsf(ta) + fabsf(tb)) + 1.0e-30f;
    auto emit = [&](int nc) -> bool {
      for (int c = lane; c < nc; c += 32) {
        const int k = sh.cand[c];
        const float4 *qa = reinterpret_cast<const float4 *>(a.pose + k);
        Pose Pk;
        Pk.p0 = __ldg(qa);
        Pk.p1 = __ldg(qa + 1);
        Pk.p2 = __ldg(qa + 2);
        Pk.p3 = __ldg(qa + 3);
        if (packet_hits_obb(sh.pk, Pk, ta - slack, tb + slack)) {
          const int g = __ldg(a.rank + k) / gsize;
          if (MVP_IN_BOUNDS(g >= 0 && g < n_groups, a.status)) m |= 1ull << g;
        }
      }
      __syncwarp();
      return true;
    };
    if (!traverse_tile(sh, a.nodes, a.n_prims, ta - slack, tb + slack, emit, a.status))
      m = n_groups >= 64 ? ~0ull : (1ull << n_groups) - 1ull;
  }
  const unsigned lo = __reduce_or_sync(FULL, (unsigned)m), hi = __reduce_or_sync(FULL, (unsigned)(m >> 32));
  if (lane == 0) mask[slot] = ((unsigned long long)hi << 32) | lo;
}

// The work list, group by group: items[goff[g] .. goff[g+1]) are the tiles of group g
// (goff[G] = the total). Also clears the grouped adjoint's work counter. One block.
constexpr int ITEMS_THREADS = 1024;
__global__ void __launch_bounds__(ITEMS_THREADS) k_bwd_items(const unsigned long long *__restrict__ mask,
                                                             int64_t n_tiles, int n_groups, int *__restrict__ items,
                                                             int *__restrict__ goff, int *__restrict__ work) {
  __shared__ int cnt[64], cur[64];
  const int tid = threadIdx.x;
  if (tid < 64) cnt[tid] = 0;
  __syncthreads();
  for (int64_t t = tid; t < n_tiles; t += ITEMS_THREADS) {
    unsigned long long m = mask[t];
    while (m) {
      atomicAdd(&cnt[__ffsll((long long)m) - 1], 1);
      m &= m - 1;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int g = 0; g < n_groups; ++g) {
      goff[g] = run;
      cur[g] = run;
      run += cnt[g];
    }
    goff[n_groups] = run;
    *work = 0;
  }
  __syncthreads();
  for (int64_t t = tid; t < n_tiles; t += ITEMS_THREADS) {
    unsigned long long m = mask[t];
    while (m) {
      items[atomicAdd(&cur[__ffsll((long long)m) - 1], 1)] = (int)t;
      m &= m - 1;
    }
  }
}

// The grouped adjoint: persistent warps take (tile, group) items in list order (a
// work counter), so the groups are replayed one after another across the GPU; each
// item replays its tile against its group's primitives only.
template <int DT, int CAP, int MT, bool SEQ>
__global__ void __launch_bounds__(TILE_WARPS * 32, MVP_BWD_MINB)
    k_backward_grouped(BwdArgs b, const int *__restrict__ items, const int *__restrict__ goff, int n_groups,
                       int gsize, int *__restrict__ work, const int2 *__restrict__ range) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MarchArgs &a = b.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<CAP> &sh = reinterpret_cast<TileShared<CAP> *>(smem_raw)[warp];
  const int total = goff[n_groups];
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(work, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    // the group of the item: the last g with goff[g] <= item (goff ascends, goff[0] = 0)
    const unsigned m0 = __ballot_sync(FULL, lane < n_groups && goff[lane] <= item);
    const unsigned m1 = __ballot_sync(FULL, lane + 32 < n_groups && goff[lane + 32] <= item);
    const int g = __popc(m0) + __popc(m1) - 1;
    const int tile = items[item];
    if (!MVP_IN_BOUNDS(tile >= 0 && tile < a.geom.n_warp_tiles && g >= 0, a.status)) continue;
    LaneRay L;
    load_lane_ray(L, a.o, a.d, tile_ray(a.geom, tile, lane));
    if (__ballot_sync(FULL, L.r >= 0) == 0) continue;
    const LeafRange lr{range, g * gsize, min(a.n_prims, (g + 1) * gsize)};
    backward_tile<DT, CAP, MT, SEQ, true>(sh, b, L, lr);
    __syncwarp();
  }
}

// Map the 12 accumulators of each primitive to pose gradients (+=):
// u = Mx p + h with Mx_jm = h R_mj / s_j and p = x - t, A_jm = sum dL/du_j p_m,
// g_j = sum dL/du_j:  dL/dt_m = -sum_j Mx_jm g_j;  dL/dR_mj = A_jm h / s_j;
// dL/ds_j = -sum_m A_jm Mx_jm / s_j;  dL/dq through R(q/|q|).
__global__ void k_pose_grads(const float *__restrict__ gmc, const Xform *__restrict__ xf,
                             const float *__restrict__ sv, const float *__restrict__ q, int n, int M,
                             float *__restrict__ g_t, float *__restrict__ g_q, float *__restrict__ g_s) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float *A = gmc + 12 * (int64_t)k;
  const Xform X = xf[k];
  const float Mx[3][3] = {{X.r0.x, X.r0.y, X.r0.z}, {X.r1.x, X.r1.y, X.r1.z}, {X.r2.x, X.r2.y, X.r2.z}};
  const float s[3] = {sv[3 * k], sv[3 * k + 1], sv[3 * k + 2]};
  const float h = 0.5f * (float)(M - 1);
  float G[9];  // dL/dR, row-major
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    float gt = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) gt -= Mx[j][m] * A[9 + j];
    g_t[3 * k + m] += gt;
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float gs = 0.0f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      G[3 * m + j] = A[3 * j + m] * h / s[j];
      gs -= A[3 * j + m] * Mx[j][m];
    }
    g_s[3 * k + j] += gs / s[j];
  }
  float w = q[4 * k], x = q[4 * k + 1], y = q[4 * k + 2], z = q[4 * k + 3];
  const float nrm = sqrtf(w * w + x * x + y * y + z * z);
  w /= nrm; x /= nrm; y /= nrm; z /= nrm;
  const float gw = G[1] * (-2 * z) + G[2] * (2 * y) + G[3] * (2 * z) + G[5] * (-2 * x) + G[6] * (-2 * y) + G[7] * (2 * x);
  const float gx = G[1] * (2 * y) + G[2] * (2 * z) + G[3] * (2 * y) + G[4] * (-4 * x) + G[5] * (-2 * w) +
                   G[6] * (2 * z) + G[7] * (2 * w) + G[8] * (-4 * x);
  const float gy = G[0] * (-4 * y) + G[1] * (2 * x) + G[2] * (2 * w) + G[3] * (2 * x) + G[5] * (2 * z) +
                   G[6] * (-2 * w) + G[7] * (2 * z) + G[8] * (-4 * y);
  const float gz = G[0] * (-4 * z) + G[1] * (-2 * w) + G[2] * (2 * x) + G[3] * (2 * w) + G[4] * (-4 * z) +
                   G[5] * (2 * y) + G[6] * (2 * x) + G[7] * (2 * y);
  const float dot = w * gw + x * gx + y * gy + z * gz;
  g_q[4 * k] += (gw - w * dot) / nrm;
  g_q[4 * k + 1] += (gx - x * dot) / nrm;
  g_q[4 * k + 2] += (gy - y * dot) / nrm;
  g_q[4 * k + 3] += (gz - z * dot) / nrm;
}

template <int DT, int CAP, int MT, bool SEQ = false>
static cudaError_t launch_bwd_t(const BwdArgs &b, cudaStream_t st) {
  size_t smem = sizeof(TileShared<CAP>) * TILE_WARPS;
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(k_backward<DT, CAP, MT, SEQ>), smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (b.m.geom.n_warp_tiles + TILE_WARPS - 1) / TILE_WARPS;
  if (blocks > 0) k_backward<DT, CAP, MT, SEQ><<<(unsigned)blocks, TILE_WARPS * 32, smem, st>>>(b);
  return cudaGetLastError();
}

template <int DT, int CAP, int MT, bool SEQ = false>
static cudaError_t launch_bwd_grouped_t(const BwdArgs &b, const BwdGroups &gr, cudaStream_t st) {
  const void *k = reinterpret_cast<const void *>(k_backward_grouped<DT, CAP, MT, SEQ>);
  const size_t smem = sizeof(TileShared<CAP>) * TILE_WARPS;
  cudaError_t e = allow_dynamic_smem(k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_grouped<DT, CAP, MT, SEQ>,
                                                         TILE_WARPS * 32, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) per_sm = 1;
  // one block per resident slot, no more blocks than items could use
  const int64_t need = (b.m.geom.n_warp_tiles * gr.n_groups + TILE_WARPS - 1) / TILE_WARPS;
  const int64_t blocks = std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(need, 1));
  k_backward_grouped<DT, CAP, MT, SEQ><<<(unsigned)blocks, TILE_WARPS * 32, smem, st>>>(
      b, gr.items, gr.goff, gr.n_groups, gr.gsize, gr.work, gr.range);
  return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_bwd_m(const BwdArgs &b, const BwdGroups *gr, cudaStream_t st) {
  // the sequential rule's adjoint: one generic-M kernel per payload type
  if (gr) {
    if (b.m.sequential) return launch_bwd_grouped_t<DT, MARCH_CAP, 0, true>(b, *gr, st);
    switch (b.m.M) {
      case 8: return launch_bwd_grouped_t<DT, MARCH_CAP, 8>(b, *gr, st);
      case 16: return launch_bwd_grouped_t<DT, MARCH_CAP, 16>(b, *gr, st);
      case 32: return launch_bwd_grouped_t<DT, MARCH_CAP, 32>(b, *gr, st);
      default: return launch_bwd_grouped_t<DT, MARCH_CAP, 0>(b, *gr, st);
    }
  }
  if (b.m.sequential) return launch_bwd_t<DT, MARCH_CAP, 0, true>(b, st);
  switch (b.m.M) {
    case 8: return launch_bwd_t<DT, MARCH_CAP, 8>(b, st);
    case 16: return launch_bwd_t<DT, MARCH_CAP, 16>(b, st);
    case 32: return launch_bwd_t<DT, MARCH_CAP, 32>(b, st);
    default: return launch_bwd_t<DT, MARCH_CAP, 0>(b, st);
  }
}

cudaError_t launch_backward(const BwdArgs &b, const float *t, const float *q, const float *s, float *g_t,
                            float *g_q, float *g_s, cudaStream_t st, const BwdGroups *gr) {
  (void)t;
  if (b.gmc) cudaMemsetAsync(b.gmc, 0, sizeof(float) * 12 * (size_t)b.m.n_prims, st);
  cudaError_t e = cudaSuccess;
  if (gr) {
    const int64_t nt = b.m.geom.n_warp_tiles;
    k_bwd_groups<<<(unsigned)((nt + TILE_WARPS - 1) / TILE_WARPS), TILE_WARPS * 32, 0, st>>>(b, gr->gsize, gr->n_groups,
                                                                                         gr->mask);
    k_bwd_items<<<1, ITEMS_THREADS, 0, st>>>(gr->mask, nt, gr->n_groups, gr->items, gr->goff, gr->work);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  switch (b.m.dtype) {
    case MVP_F32: e = launch_bwd_m<MVP_F32>(b, gr, st); break;
    case MVP_BF16: e = launch_bwd_m<MVP_BF16>(b, gr, st); break;
    case MVP_F16: e = launch_bwd_m<MVP_F16>(b, gr, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (b.gmc && b.m.n_prims > 0)
    k_pose_grads<<<(b.m.n_prims + 255) / 256, 256, 0, st>>>(b.gmc, b.m.xf, s, q, b.m.n_prims, b.m.M, g_t, g_q,
                                                             g_s);
  return cudaGetLastError();
}

}  // namespace mvp
