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

namespace mvp {

// Voxel bytes per payload dtype.
template <int DT>
struct VoxelBytes {
  static constexpr int value = DT == MVP_F32 ? 16 : 8;
};

// Gather the 8 voxels of the cell at (ix, iy, iz) of one primitive's payload and
// interpolate RGBA. MT > 0 makes the payload edge a compile-time constant, so the
// eight addresses are immediate offsets from one base.
template <int DT, int MT>
__device__ __forceinline__ float4 trilinear(const char *base, int Mr, int ix, int iy, int iz, float fx, float fy,
                                            float fz) {
  const int M = MT > 0 ? MT : Mr;
  const int o = (iz * M + iy) * M + ix;
  const void *p = base;
  const float4 c000 = Voxel<DT>::load(p, o);
  const float4 c001 = Voxel<DT>::load(p, o + 1);
  const float4 c010 = Voxel<DT>::load(p, o + M);
  const float4 c011 = Voxel<DT>::load(p, o + M + 1);
  const float4 c100 = Voxel<DT>::load(p, o + M * M);
  const float4 c101 = Voxel<DT>::load(p, o + M * M + 1);
  const float4 c110 = Voxel<DT>::load(p, o + M * M + M);
  const float4 c111 = Voxel<DT>::load(p, o + M * M + M + 1);
  const float4 c00 = lerp4(c000, c001, fx), c01 = lerp4(c010, c011, fx);
  const float4 c10 = lerp4(c100, c101, fx), c11 = lerp4(c110, c111, fx);
  const float4 c0 = lerp4(c00, c01, fy), c1 = lerp4(c10, c11, fy);
  return lerp4(c0, c1, fz);
}

// March one warp tile whose lane ray is L (L.r < 0: no ray). Writes the output
// (and the adjoint state / evaluation count) of each lane's ray. A single sample
// overlapped by more than CAP primitives sets STATUS_CAPACITY in a.status.
template <int DT, int CAP, bool COUNT, int MT>
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

  int w0 = 0, wlen = a.n_steps;
  while (w0 < a.n_steps && __any_sync(FULL, alive)) {
    int w1 = min(a.n_steps, w0 + wlen);
    int lane_last = alive ? a.n_steps - 1 : -1;
    int ne = build_window<CAP>(sh, a.nodes, a.pose, a.xf, reinterpret_cast<const char *>(a.payload), prim_bytes,
                               a.n_prims, L, lane_last, a.t_near, a.t_far, a.dt, a.n_steps, w0, w1);
    if (ne < 0) {
      if (w1 - w0 == 1) {  // one sample overlapped by more than CAP primitives
        if (lane == 0) atomicOr(a.status, STATUS_CAPACITY);
        alive = false;
        break;
      }
      wlen = (w1 - w0 + 1) >> 1;
      continue;
    }
    int i = w0;
    while (i < w1) {
      if (!__any_sync(FULL, alive)) break;
      uint32_t m0, m1;
      int nxt = active_set<CAP>(sh, ne, i, w1, m0, m1);
      if ((m0 | m1) == 0) {
        i = nxt;
        continue;
      }
      for (; i < nxt; ++i) {
        if (!__any_sync(FULL, alive)) break;
        const float ti = sample_t(a.t_near, a.dt, i);
        const float x0 = fmaf(ti, L.d[0], L.o[0]);
        const float x1 = fmaf(ti, L.d[1], L.o[1]);
        const float x2 = fmaf(ti, L.d[2], L.o[2]);
        float sa = 0.0f, sr = 0.0f, sg = 0.0f, sb = 0.0f;
        uint32_t b0 = m0, b1 = m1;
        while (b0 | b1) {
          int e;
          if (b0) { e = __ffs(b0) - 1; b0 &= b0 - 1; }
          else { e = 32 + __ffs(b1) - 1; b1 &= b1 - 1; }
          const uint32_t rg = sh.erng[e][lane];
          const bool in = alive && i >= (int)(rg & 0xffffu) && i <= (int)(rg >> 16);
          if (in) {
            const Xform X = sh.exf[e];
            // voxel coordinate u = Mx x + c (FP32, the cell decision of the oracle's
            // FP32 mode), clamped into the box
            float ux = fmaf(X.r0.x, x0, fmaf(X.r0.y, x1, fmaf(X.r0.z, x2, X.r0.w)));
            float uy = fmaf(X.r1.x, x0, fmaf(X.r1.y, x1, fmaf(X.r1.z, x2, X.r1.w)));
            float uz = fmaf(X.r2.x, x0, fmaf(X.r2.y, x1, fmaf(X.r2.z, x2, X.r2.w)));
            ux = fminf(fmaxf(ux, 0.0f), Mm1);
            uy = fminf(fmaxf(uy, 0.0f), Mm1);
            uz = fminf(fmaxf(uz, 0.0f), Mm1);
            const int ix = min((int)ux, M - 2), iy = min((int)uy, M - 2), iz = min((int)uz, M - 2);
            const float4 val = trilinear<DT, MT>(sh.eptr[e], M, ix, iy, iz, ux - (float)ix, uy - (float)iy,
                                                 uz - (float)iz);
            sa += val.w;
            sr = fmaf(val.w, val.x, sr);
            sg = fmaf(val.w, val.y, sg);
            sb = fmaf(val.w, val.z, sb);
            if (COUNT) ++n_eval;
          }
        }
        if (alive) {
          // clamped additive accumulation: w = min(a, 1 - T), I += c w / a, T += w
          const float aa = sa * a.dt;
          const float cr = sr * a.dt, cg = sg * a.dt, cb = sb * a.dt;
          const float rem = 1.0f - T;
          if (aa <= rem) {
            Ir += cr;
            Ig += cg;
            Ib += cb;
            T = fminf(T + aa, 1.0f);
            if (T >= a.stop_T) {
              alive = false;
              if (!COUNT && a.saved) {
                Saved S = {0.0f, 0.0f, 0.0f, 0.0f, i, -1};
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
              Saved S = {cr / aa, cg / aa, cb / aa, bt, i, i};
              a.saved[L.r] = S;
            }
            saved_done = true;
          }
        }
      }
    }
    w0 = w1;
    wlen = min(a.n_steps, wlen * 2);
  }
  if (!valid) return;
  if (COUNT) {
    a.n_eval[L.r] = n_eval;
    return;
  }
  const float bgw = 1.0f - T;
  float4 out = make_float4(fmaf(bgw, a.bg[0], Ir), fmaf(bgw, a.bg[1], Ig), fmaf(bgw, a.bg[2], Ib), T);
  reinterpret_cast<float4 *>(a.out)[L.r] = out;
  if (a.saved && !saved_done) {
    Saved S = {0.0f, 0.0f, 0.0f, 0.0f, a.n_steps - 1, -1};
    a.saved[L.r] = S;
  }
}

}  // namespace mvp
