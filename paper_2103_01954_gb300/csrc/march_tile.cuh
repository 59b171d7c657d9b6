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
        const uint32_t rg = sh.erng[e][lane];
        const int lo = max((int)(rg & 0xffffu), i), hi = min((int)(rg >> 16), ie - 1);
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
          float ux = fmaf(X.r0.x, xs[c][0], fmaf(X.r0.y, xs[c][1], fmaf(X.r0.z, xs[c][2], X.r0.w)));
          float uy = fmaf(X.r1.x, xs[c][0], fmaf(X.r1.y, xs[c][1], fmaf(X.r1.z, xs[c][2], X.r1.w)));
          float uz = fmaf(X.r2.x, xs[c][0], fmaf(X.r2.y, xs[c][1], fmaf(X.r2.z, xs[c][2], X.r2.w)));
          ux = fminf(fmaxf(ux, 0.0f), Mm1);
          uy = fminf(fmaxf(uy, 0.0f), Mm1);
          uz = fminf(fmaxf(uz, 0.0f), Mm1);
          const int ix = min((int)ux, M - 2), iy = min((int)uy, M - 2), iz = min((int)uz, M - 2);
          const int v = (iz * M + iy) * M + ix;
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
          const float fx = ux - (float)ix, fy = uy - (float)iy, fz = uz - (float)iz;
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
#pragma unroll
      for (int c = 0; c < MARCH_CHUNK; ++c) {
        const int ii = i + c;
        if (!alive || ii >= ie) continue;
        if (COUNT) n_eval += ne_c[c];  // samples past a ray's termination are not counted
        // clamped additive accumulation: w = min(a, 1 - T), I += c w / a, T += w
        const float aa = sba[c].y * a.dt;
        const float cr = srg[c].x * a.dt, cg = srg[c].y * a.dt, cb = sba[c].x * a.dt;
        const float rem = 1.0f - T;
        if (aa <= rem) {
          Ir += cr;
          Ig += cg;
          Ib += cb;
          T = fminf(T + aa, 1.0f);
          if (T >= a.stop_T) {
            alive = false;
            if (!COUNT && a.saved) {
              Saved S = {0.0f, 0.0f, 0.0f, 0.0f, ii, -1};
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
            Saved S = {cr / aa, cg / aa, cb / aa, bt, ii, ii};
            a.saved[L.r] = S;
          }
          saved_done = true;
        }
      }
      i = ie;
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
