// march_tile.cuh -- the per-warp-tile forward march (Sec. 3.2.1-3.2.2), shared by the
// frame kernel (k_march) and the serving kernel (k_serve).
//
// One warp marches a tile of 32 neighbouring rays in lock step over the sample
// index i (all rays share t_near and dt, so sample depths align). At each sample
// the warp loops over the primitives active in the tile at that depth (the window
// list built by build_window); each lane tests its own inclusive sample range for
// the primitive and, if inside, gathers the 8 voxels of the cell, interpolates
// RGBA and accumulates a = sum alpha, c = sum alpha*rgb. Then every lane applies
// the clamped update w = min(a*dt, 1 - T). A tile stops when all its rays are done
// (T >= 1 - eps_early). Empty depth ranges between primitives are skipped.
#pragma once

#include "march.cuh"

#ifndef MVP_MARCH_CHUNK
#define MVP_MARCH_CHUNK 4
#endif

namespace mvp {

constexpr int MARCH_CHUNK = MVP_MARCH_CHUNK;  // samples per chunk of the march loop

// Voxel bytes per payload dtype.
template <int DT>
struct VoxelBytes {
  static constexpr int value = DT == MVP_F32 ? 16 : 8;
};

// Trilinear RGBA of one primitive (march transform X, payload at pbase) at world
// point x: the arithmetic of the chunked loop in march_tile, rounding for rounding.
template <int DT, int MT>
__device__ __forceinline__ float4 sample_rgba(const Xform &X, const char *pbase, const float x[3], int Mr,
                                              float Mm1, int *status = nullptr) {
  const int M = MT > 0 ? MT : Mr;
  float ux = fmaf(X.r0.x, x[0], fmaf(X.r0.y, x[1], fmaf(X.r0.z, x[2], X.r0.w)));
  float uy = fmaf(X.r1.x, x[0], fmaf(X.r1.y, x[1], fmaf(X.r1.z, x[2], X.r1.w)));
  float uz = fmaf(X.r2.x, x[0], fmaf(X.r2.y, x[1], fmaf(X.r2.z, x[2], X.r2.w)));
  float fx, fy, fz;
  const int ix = voxel_cell(ux, M - 2, fx), iy = voxel_cell(uy, M - 2, fy), iz = voxel_cell(uz, M - 2, fz);
  const int v = (iz * M + iy) * M + ix;
  if (!MVP_IN_BOUNDS(v >= 0 && v + M * M + M + 1 < M * M * M, status)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const void *p = pbase;
  const float4 c000 = Voxel<DT>::load(p, v), c001 = Voxel<DT>::load(p, v + 1);
  const float4 c010 = Voxel<DT>::load(p, v + M), c011 = Voxel<DT>::load(p, v + M + 1);
  const float4 c100 = Voxel<DT>::load(p, v + M * M), c101 = Voxel<DT>::load(p, v + M * M + 1);
  const float4 c110 = Voxel<DT>::load(p, v + M * M + M), c111 = Voxel<DT>::load(p, v + M * M + M + 1);
  const float2 wx = splat2(fx), nwx = splat2(-fx), wy = splat2(fy), nwy = splat2(-fy);
  const float4 c00 = lerp4x2(c000, c001, wx, nwx), c01 = lerp4x2(c010, c011, wx, nwx);
  const float4 c10 = lerp4x2(c100, c101, wx, nwx), c11 = lerp4x2(c110, c111, wx, nwx);
  const float4 q0 = lerp4x2(c00, c01, wy, nwy), q1 = lerp4x2(c10, c11, wy, nwy);
  return lerp4x2(q0, q1, splat2(fz), splat2(-fz));
}

// Sample w0 of every live lane against all primitives that contain it, evaluated
// as one traversal of the tile finds them (no window list, so no limit on their
// number): per lane the sums (alpha*r, alpha*g), (alpha*b, alpha) and the number
// of evaluations. Membership is the window list's: the lane's exact sample range
// of the primitive holds w0. Used when more than a window list's worth of
// primitives meet one sample. Returns false on a traversal stack overflow.
template <int DT, int MT, class SH>
__device__ __forceinline__ bool sample_all(SH &sh, const MarchArgs &a, const LaneRay &L, bool live, int w0,
                                           int M, float Mm1, int64_t prim_bytes, float2 &rg, float2 &ba,
                                           int &nec) {
  const float ti = sample_t(a.t_near, a.dt, w0);
  const float inv_dt = 1.0f / a.dt;
  const float xs[3] = {fmaf(ti, L.d[0], L.o[0]), fmaf(ti, L.d[1], L.o[1]), fmaf(ti, L.d[2], L.o[2])};
  const char *payload = reinterpret_cast<const char *>(a.payload);
  rg = ba = make_float2(0.0f, 0.0f);
  nec = 0;
  auto emit = [&](int nc) -> bool {
    for (int c = 0; c < nc; ++c) {
      const int k = sh.cand[c];
      const float4 *q = reinterpret_cast<const float4 *>(a.pose + k);
      Pose P;
      P.p0 = __ldg(q);
      P.p1 = __ldg(q + 1);
      P.p2 = __ldg(q + 2);
      P.p3 = __ldg(q + 3);
      float tin, tout;
      bool in = live && slab_spec(P, L.o[0], L.o[1], L.o[2], L.d[0], L.d[1], L.d[2], a.t_near, a.t_far, tin, tout);
      if (in)
        in = first_sample_geq(tin, a.t_near, a.dt, inv_dt, a.n_steps) <= w0 &&
             w0 < first_sample_gt(tout, a.t_near, a.dt, inv_dt, a.n_steps);
      if (!in) continue;
      const float4 *xp = reinterpret_cast<const float4 *>(a.xf + k);
      Xform X;
      X.r0 = __ldg(xp);
      X.r1 = __ldg(xp + 1);
      X.r2 = __ldg(xp + 2);
      const float4 val = sample_rgba<DT, MT>(X, payload + (int64_t)k * prim_bytes, xs, M, Mm1, a.status);
      rg = __ffma2_rn(splat2(val.w), lo2(val), rg);
      ba = __ffma2_rn(make_float2(val.w, 1.0f), hi2(val), ba);
      ++nec;
    }
    return true;
  };
  const float slack = 2.0e-5f * fabsf(ti) + 1.0e-30f;
  const bool ok = traverse_tile(sh, a.nodes, a.n_prims, ti - slack, ti + slack, emit, a.status);
  __syncwarp();
  return ok;
}

// BVH order of a window list: sh.cand[p] = the entry of the p-th lowest leaf rank
// (ranks are unique). The traversal buffers are free once the list is built; ranks go
// to sh.stack, then each lane places the entries it holds by counting lower ranks.
template <int CAP>
__device__ __forceinline__ void order_window(TileShared<CAP> &sh, int ne, const int *__restrict__ rank) {
  const int lane = threadIdx.x & 31;
  static_assert(CAP <= 64 && CAP <= CBUF && CAP <= STACK, "window order buffers");
  __syncwarp();
  for (int e = lane; e < ne; e += 32) sh.stack[e] = __ldg(rank + sh.ek[e]);
  __syncwarp();
  for (int e = lane; e < ne; e += 32) {
    const int rk = sh.stack[e];
    int pos = 0;
    for (int f = 0; f < ne; ++f) pos += sh.stack[f] < rk;
    sh.cand[pos] = e;
  }
  __syncwarp();
}

// A lane's saturating sample ii (its summed opacity exceeds 1 - T) blended the
// paper's way: the window's primitives that contain it, one by one in BVH order
// (sh.cand, from order_window), each adding w = min(alpha dt, 1 - T) of its colour,
// until T = 1. x is the sample's world position. The adjoint's state: the colour,
// weight and leaf rank of the primitive whose weight reached what was left (w >= 1 -
// T; if rounding leaves every weight below it, the last primitive that contributed).
template <int DT, int MT, int CAP>
__device__ __forceinline__ void blend_sequential(const TileShared<CAP> &sh, int ne, const MarchArgs &a,
                                                 const float x[3], int ii, int M, float Mm1, float &T, float &Ir,
                                                 float &Ig, float &Ib, Saved &S) {
  const int lane = threadIdx.x & 31;
  float rem = 1.0f - T;
  S = {0.0f, 0.0f, 0.0f, 0.0f, ii, ii, 0x7fffffff, 0};
  int last = -1;  // the last contributing entry while none has been clamped
  float4 vlast = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float wlast = 0.0f;
  for (int p = 0; p < ne && rem > 0.0f; ++p) {
    const int e = sh.cand[p];
    int rlo, rhi;
    lane_range(sh, e, lane, rlo, rhi);
    if (rlo > ii || rhi < ii) continue;
    const float4 v = sample_rgba<DT, MT>(sh.exf[e], sh.eptr[e], x, M, Mm1, a.status);
    float w = v.w * a.dt;
    if (w >= rem) {  // this primitive's weight is clamped to what is left
      w = rem;
      S.rho_r = v.x;
      S.rho_g = v.y;
      S.rho_b = v.z;
      S.beta = w;
      S.rank_clamp = __ldg(a.rank + sh.ek[e]);
      last = -2;
    } else if (w > 0.0f) {
      last = e;
      vlast = v;
      wlast = w;
    }
    Ir = fmaf(v.x, w, Ir);
    Ig = fmaf(v.y, w, Ig);
    Ib = fmaf(v.z, w, Ib);
    rem -= w;
  }
  if (last >= 0) {
    S.rho_r = vlast.x;
    S.rho_g = vlast.y;
    S.rho_b = vlast.z;
    S.beta = wlast;
    S.rank_clamp = __ldg(a.rank + sh.ek[last]);
  }
  T = 1.0f;
}

// March one warp tile whose lane ray is L (L.r < 0: no ray). Writes the output
// (and the adjoint state / evaluation count) of each lane's ray. A traversal stack
// overflow sets STATUS_CAPACITY in a.status; any number of primitives may overlap.
// SEQ blends each ray's saturating sample in BVH order (within a window list; a
// sample met by more primitives than a list holds keeps the summed rule).
template <int DT, int CAP, bool COUNT, int MT, bool SEQ = false>
__device__ __forceinline__ void march_tile(TileShared<CAP> &sh, const MarchArgs &a, const LaneRay &L) {
  const int lane = threadIdx.x & 31;
  const bool valid = L.r >= 0;
  float T = 0.0f, Ir = 0.0f, Ig = 0.0f, Ib = 0.0f;
  int n_eval = 0;
  bool alive = valid && a.n_steps > 0 && a.n_prims > 0;
  bool saved_done = false;

  make_packet(sh.pk, valid, L.o, L.d, a.t_far);
  const int M = MT > 0 ? MT : a.M;
  const float Mm1 = (float)(M - 1);
  const int64_t prim_bytes = (int64_t)M * M * M * VoxelBytes<DT>::value;

  // Clamped additive accumulation of sample ii of a live lane with sums
  // (sum alpha*r, sum alpha*g) and (sum alpha*b, sum alpha): w = min(a, 1 - T),
  // I += c w / a, T += w.
  auto composite = [&](float2 rg, float2 ba, int ii) {
    const float aa = ba.y * a.dt;
    const float cr = rg.x * a.dt, cg = rg.y * a.dt, cb = ba.x * a.dt;
    const float rem = 1.0f - T;
    if (aa <= rem) {
      Ir += cr;
      Ig += cg;
      Ib += cb;
      T = fminf(T + aa, 1.0f);
      if (T >= a.stop_T) {
        alive = false;
        if (!COUNT && a.saved) {
          Saved S = {0.0f, 0.0f, 0.0f, 0.0f, ii, -1, -1, 0};
          a.saved[L.r] = S;
        }
        saved_done = true;
      }
    } else {
      const float bt = rem / aa;
      Ir = fmaf(cr, bt, Ir);
      Ig = fmaf(cg, bt, Ig);
      Ib = fmaf(cb, bt, Ib);
      T = 1.0f;
      alive = false;  // T = 1 >= 1 - eps_early
      if (!COUNT && a.saved) {
        Saved S = {cr / aa, cg / aa, cb / aa, bt, ii, ii, -1, 0};
        a.saved[L.r] = S;
      }
      saved_done = true;
    }
  };

  int w0 = 0, wlen = a.n_steps;
  bool stack_full = false;
  while (w0 < a.n_steps && __any_sync(FULL, alive)) {
    int w1 = min(a.n_steps, w0 + wlen);
    int lane_last = alive ? a.n_steps - 1 : -1;
    int ne = build_window<CAP>(sh, a.nodes, a.pose, a.xf, reinterpret_cast<const char *>(a.payload), prim_bytes,
                               a.n_prims, L, lane_last, a.t_near, a.t_far, a.dt, a.n_steps, w0, w1, 0, a.status);
    if (ne == WINDOW_STACK) {
      stack_full = true;
      break;
    }
    if (SEQ && ne > 0) order_window<CAP>(sh, ne, a.rank);
    if (ne == WINDOW_FULL && w1 - w0 > 1) {  // split the depth range
      wlen = (w1 - w0 + 1) >> 1;
      continue;
    }
    if (ne == WINDOW_FULL) {
      // more than CAP primitives meet this one sample in the tile: evaluate them as
      // one traversal finds them, then composite
      float2 rg, ba;
      int nec;
      if (!sample_all<DT, MT>(sh, a, L, alive, w0, M, Mm1, prim_bytes, rg, ba, nec)) {
        stack_full = true;
        break;
      }
      if (alive) {
        if (COUNT) n_eval += nec;
        composite(rg, ba, w0);
      }
      w0 = w1;
      wlen = 2;
      continue;
    }
    // Samples go in chunks of MARCH_CHUNK: each window entry's transform is read from
    // shared memory once per chunk, the chunk's samples give independent gathers, and
    // a lane whose next sample stays in the same voxel cell of the same primitive
    // reuses the 8 corners it already holds. Per sample, primitives are summed in
    // entry order, as before; the composite then runs sample by sample.
    int i = w0;
    while (i < w1) {
      if (!__any_sync(FULL, alive)) break;
      const int ie = min(i + MARCH_CHUNK, w1);
      uint32_t m0, m1;
      const int nxt = active_chunk<CAP>(sh, ne, i, ie, w1, m0, m1);
      if ((m0 | m1) == 0) {
        i = max(nxt, ie);
        continue;
      }
      float xs[MARCH_CHUNK][3];
#pragma unroll
      for (int c = 0; c < MARCH_CHUNK; ++c) {
        const float ti = sample_t(a.t_near, a.dt, i + c);
        xs[c][0] = fmaf(ti, L.d[0], L.o[0]);
        xs[c][1] = fmaf(ti, L.d[1], L.o[1]);
        xs[c][2] = fmaf(ti, L.d[2], L.o[2]);
      }
      // per sample: (sum alpha*r, sum alpha*g) and (sum alpha*b, sum alpha), packed pairs
      float2 srg[MARCH_CHUNK], sba[MARCH_CHUNK];
      int ne_c[MARCH_CHUNK];  // evaluations per sample (count variant)
#pragma unroll
      for (int c = 0; c < MARCH_CHUNK; ++c) {
        srg[c] = sba[c] = make_float2(0.0f, 0.0f);
        ne_c[c] = 0;
      }
      uint32_t b0 = m0, b1 = m1;
      while (b0 | b1) {
        int e;
        if (b0) { e = __ffs(b0) - 1; b0 &= b0 - 1; }
        else { e = 32 + __ffs(b1) - 1; b1 &= b1 - 1; }
        int lo, hi;
        lane_range(sh, e, lane, lo, hi);
        lo = max(lo, i);
        hi = min(hi, ie - 1);
        if (!alive || lo > hi) continue;
        const Xform X = sh.exf[e];
        const char *pbase = sh.eptr[e];
        int held = -1;  // voxel (within the primitive) of the corners held
        float4 c000, c001, c010, c011, c100, c101, c110, c111;
#pragma unroll
        for (int c = 0; c < MARCH_CHUNK; ++c) {
          const int ii = i + c;
          if (ii < lo || ii > hi) continue;
          // voxel coordinate u = Mx x + c (FP32, the cell decision of the oracle's
          // FP32 mode), clamped into the box
          const float ux = fmaf(X.r0.x, xs[c][0], fmaf(X.r0.y, xs[c][1], fmaf(X.r0.z, xs[c][2], X.r0.w)));
          const float uy = fmaf(X.r1.x, xs[c][0], fmaf(X.r1.y, xs[c][1], fmaf(X.r1.z, xs[c][2], X.r1.w)));
          const float uz = fmaf(X.r2.x, xs[c][0], fmaf(X.r2.y, xs[c][1], fmaf(X.r2.z, xs[c][2], X.r2.w)));
          float fx, fy, fz;
          const int ix = voxel_cell(ux, M - 2, fx), iy = voxel_cell(uy, M - 2, fy), iz = voxel_cell(uz, M - 2, fz);
          const int v = (iz * M + iy) * M + ix;
          if (!MVP_IN_BOUNDS(v >= 0 && v + M * M + M + 1 < M * M * M, a.status)) continue;
          if (v != held) {
            const void *p = pbase;
            c000 = Voxel<DT>::load(p, v);
            c001 = Voxel<DT>::load(p, v + 1);
            c010 = Voxel<DT>::load(p, v + M);
            c011 = Voxel<DT>::load(p, v + M + 1);
            c100 = Voxel<DT>::load(p, v + M * M);
            c101 = Voxel<DT>::load(p, v + M * M + 1);
            c110 = Voxel<DT>::load(p, v + M * M + M);
            c111 = Voxel<DT>::load(p, v + M * M + M + 1);
            held = v;
          }
          const float2 wx = splat2(fx), nwx = splat2(-fx), wy = splat2(fy), nwy = splat2(-fy);
          const float2 wz = splat2(fz), nwz = splat2(-fz);
          const float4 c00 = lerp4x2(c000, c001, wx, nwx), c01 = lerp4x2(c010, c011, wx, nwx);
          const float4 c10 = lerp4x2(c100, c101, wx, nwx), c11 = lerp4x2(c110, c111, wx, nwx);
          const float4 q0 = lerp4x2(c00, c01, wy, nwy), q1 = lerp4x2(c10, c11, wy, nwy);
          const float4 val = lerp4x2(q0, q1, wz, nwz);
          srg[c] = __ffma2_rn(splat2(val.w), lo2(val), srg[c]);
          sba[c] = __ffma2_rn(make_float2(val.w, 1.0f), hi2(val), sba[c]);
          if (COUNT) ++ne_c[c];
        }
      }
      int seq_ii = -1;  // SEQ: the lane's saturating sample in this chunk
#pragma unroll
      for (int c = 0; c < MARCH_CHUNK; ++c) {
        const int ii = i + c;
        if (!alive || ii >= ie) continue;
        if (COUNT) n_eval += ne_c[c];  // samples past a ray's termination are not counted
        if (SEQ && sba[c].y * a.dt > 1.0f - T) {
          seq_ii = ii;
          alive = false;
          continue;
        }
        composite(srg[c], sba[c], ii);
      }
      if (SEQ && seq_ii >= 0) {  // blend the saturating sample in BVH order
        const float ti = sample_t(a.t_near, a.dt, seq_ii);
        const float xq[3] = {fmaf(ti, L.d[0], L.o[0]), fmaf(ti, L.d[1], L.o[1]), fmaf(ti, L.d[2], L.o[2])};
        Saved S;
        blend_sequential<DT, MT, CAP>(sh, ne, a, xq, seq_ii, M, Mm1, T, Ir, Ig, Ib, S);
        if (a.saved) a.saved[L.r] = S;
        saved_done = true;
      }
      i = ie;
    }
    w0 = w1;
    wlen = min(a.n_steps, wlen * 2);
  }
  if (stack_full && lane == 0) atomicOr(a.status, STATUS_CAPACITY);
  if (!valid) return;
  if (COUNT) {
    a.n_eval[L.r] = n_eval;
    return;
  }
  const float bgw = 1.0f - T;
  if (a.literal) {  // the composite read with I not yet weighted by A
    Ir *= T;
    Ig *= T;
    Ib *= T;
  }
  float4 out = make_float4(fmaf(bgw, a.bg[0], Ir), fmaf(bgw, a.bg[1], Ig), fmaf(bgw, a.bg[2], Ib), T);
  reinterpret_cast<float4 *>(a.out)[L.r] = out;
  if (a.saved && !saved_done) {
    Saved S = {0.0f, 0.0f, 0.0f, 0.0f, a.n_steps - 1, -1, -1, 0};
    a.saved[L.r] = S;
  }
}

}  // namespace mvp
