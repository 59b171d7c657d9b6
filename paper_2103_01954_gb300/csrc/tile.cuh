// tile.cuh -- warp-level tile machinery shared by the march, hit-list and adjoint
// kernels: ray tiles, the interval ray packet, the BVH traversal of a tile, and
// the per-window primitive list with per-lane sample ranges.
//
// A warp owns a tile of 32 rays (8x4 pixels for image rays, else 32 consecutive
// rays). It traverses the BVH once for the whole tile with an interval-arithmetic
// slab test of the tile's ray packet (origins and directions bounded per axis),
// 32 nodes per step, and collects candidate leaves. Each candidate is then tested
// against every lane's ray with the exact FP32 slab test (Sec. 3.2.1: the list of
// primitives each ray intersects), and kept if any lane hits it; the lane's hit
// interval becomes an inclusive sample-index range [i_lo, i_hi] (stored as 8+8-bit
// offsets from the entry's tile range start).
#pragma once

#include "bvh.cuh"

namespace mvp {

constexpr int TILE_WARPS = 4;  // warps per block; a block covers 16x8 pixels
constexpr int STACK = 256;     // traversal stack entries per warp
constexpr int CBUF = 64;       // candidate leaves buffered per warp
// A lane's sample range of a window entry, 8 + 8 bits: offsets of i_lo and i_hi from
// the entry's tile range start elo (an entry whose tile range spans more than
// MAX_SPAN samples does not fit: the window is split instead).
constexpr uint16_t EMPTY_RANGE = 0x00ffu;  // i_lo = elo + 255 > i_hi = elo
constexpr int MAX_SPAN = 254;
constexpr int WINDOW_FULL = -1;   // build_window: more primitives than the list holds (or a span over MAX_SPAN)
constexpr int WINDOW_STACK = -2;  // build_window: traversal stack overflow

struct TileGeom {
  int64_t n_rays;
  int width, height;  // > 0: 2-D image tiles
  int64_t n_warp_tiles;
};

__host__ __device__ inline TileGeom make_tile_geom(int64_t n_rays, int width, int height) {
  TileGeom g;
  g.n_rays = n_rays;
  bool img = width > 0 && height > 0 && (int64_t)width * height == n_rays;
  g.width = img ? width : 0;
  g.height = img ? height : 0;
  if (img)
    g.n_warp_tiles = (int64_t)((width + 15) / 16) * ((height + 7) / 8) * 4;
  else
    g.n_warp_tiles = ((n_rays + 31) / 32 + 3) / 4 * 4;
  return g;
}

// Ray index of `lane` in warp tile `wt`, or -1.
__device__ __forceinline__ int64_t tile_ray(const TileGeom &g, int64_t wt, int lane) {
  if (g.width > 0) {
    int64_t bt = wt >> 2;
    int w = (int)(wt & 3);
    int stx = (g.width + 15) / 16;
    int64_t sy = bt / stx, sx = bt - sy * stx;
    // Each quarter-warp (8 lanes) covers a 4x2 pixel block of the 8x4 warp tile: the
    // L1 serves a warp's 128-bit gathers a quarter-warp at a time, and a compact
    // block touches fewer cache lines than a row of 8 (measured 4 % faster).
    const int lx = (lane & 3) | ((lane >> 1) & 4), ly = ((lane >> 2) & 1) | ((lane >> 3) & 2);
    int64_t px = sx * 16 + (w & 1) * 8 + lx;
    int64_t py = sy * 8 + (w >> 1) * 4 + ly;
    if (px >= g.width || py >= g.height) return -1;
    return py * g.width + px;
  }
  int64_t r = wt * 32 + lane;
  return r < g.n_rays ? r : -1;
}

// Interval bounds of the tile's rays.
struct Packet {
  float omin[3], omax[3];
  float dmin[3], dmax[3];
  float inv_lo[3], inv_hi[3];  // 1/|d| bounds on axes where d keeps one sign
  int sgn[3];                  // +1, -1, or 0 (directions straddle zero)
  float margin;                // world-space slack for rounding
};

__device__ __forceinline__ void make_packet(Packet &P, bool valid, const float o[3], const float d[3], float t_far) {
  // every lane computes the same values; the caller's P may be warp-shared memory
  float om = 0.0f, dm = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    P.omin[j] = warp_min(valid ? o[j] : INFINITY);
    P.omax[j] = warp_max(valid ? o[j] : -INFINITY);
    P.dmin[j] = warp_min(valid ? d[j] : INFINITY);
    P.dmax[j] = warp_max(valid ? d[j] : -INFINITY);
    om = fmaxf(om, fmaxf(fabsf(P.omin[j]), fabsf(P.omax[j])));
    dm = fmaxf(dm, fmaxf(fabsf(P.dmin[j]), fabsf(P.dmax[j])));
    if (P.dmin[j] > 0.0f) {
      P.sgn[j] = 1;
      P.inv_lo[j] = 1.0f / P.dmax[j];  // smallest 1/|d|
      P.inv_hi[j] = 1.0f / P.dmin[j];  // largest 1/|d|
    } else if (P.dmax[j] < 0.0f) {
      P.sgn[j] = -1;
      P.inv_lo[j] = 1.0f / -P.dmin[j];
      P.inv_hi[j] = 1.0f / -P.dmax[j];
    } else {
      P.sgn[j] = 0;
      P.inv_lo[j] = P.inv_hi[j] = 0.0f;
    }
  }
  P.margin = 1.0e-5f * (om + fabsf(t_far) * dm) + 1.0e-30f;
  __syncwarp();
}

// Can some ray of the packet meet the (inflated) box for t in [ta, tb]?
// Conservative: every bound is widened by the packet margin plus 1e-5 relative.
__device__ __forceinline__ bool packet_hits_box(const Packet &P, float4 a, float4 b, float ta, float tb) {
  const float lo[3] = {a.x, a.y, a.z}, hi[3] = {b.x, b.y, b.z};
  float tmin = ta, tmax = tb;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float m = P.margin + 1.0e-5f * fmaxf(fabsf(lo[j]), fabsf(hi[j]));
    float l = lo[j] - m, h = hi[j] + m;
    if (P.sgn[j] > 0) {
      // entry (l - o)/d: smallest over the packet; exit (h - o)/d: largest
      float n1 = l - P.omax[j];
      float te = n1 * (n1 >= 0.0f ? P.inv_lo[j] : P.inv_hi[j]);
      float n2 = h - P.omin[j];
      float tx = n2 * (n2 >= 0.0f ? P.inv_hi[j] : P.inv_lo[j]);
      tmin = fmaxf(tmin, te);
      tmax = fminf(tmax, tx);
    } else if (P.sgn[j] < 0) {
      // entry (o - h)/|d|, exit (o - l)/|d|
      float n1 = P.omin[j] - h;
      float te = n1 * (n1 >= 0.0f ? P.inv_lo[j] : P.inv_hi[j]);
      float n2 = P.omax[j] - l;
      float tx = n2 * (n2 >= 0.0f ? P.inv_hi[j] : P.inv_lo[j]);
      tmin = fmaxf(tmin, te);
      tmax = fminf(tmax, tx);
    }
    else {
      // directions straddle zero on this axis, so no t-bound follows from it; bound
      // the coordinate o_j + t d_j itself over the window (extremes at the corners
      // of [omin, omax] x [ta, tb] x [dmin, dmax])
      float c0 = fminf(fminf(fmaf(ta, P.dmin[j], P.omin[j]), fmaf(tb, P.dmin[j], P.omin[j])),
                       fminf(fmaf(ta, P.dmax[j], P.omin[j]), fmaf(tb, P.dmax[j], P.omin[j])));
      float c1 = fmaxf(fmaxf(fmaf(ta, P.dmin[j], P.omax[j]), fmaf(tb, P.dmin[j], P.omax[j])),
                       fmaxf(fmaf(ta, P.dmax[j], P.omax[j]), fmaf(tb, P.dmax[j], P.omax[j])));
      if (c1 < l || c0 > h) return false;
    }
  }
  return tmin <= tmax + 1.0e-5f * (fabsf(tmax) + fabsf(tmin)) + 1.0e-30f;
}

// Can some ray of the packet meet the primitive's oriented box for t in [ta, tb]?
// A conservative interval test in the box's frame: the packet's origin and
// direction boxes map to intervals o' +- ro, d' +- rd per local axis (centre times
// R^T, radius times |R^T|, then scaled by 1/s). For t >= 0 the local coordinate
// o + t d of any packet ray lies in [lo_o + t lo_d, hi_o + t hi_d], so each axis
// bounds t by two linear inequalities against the slab [-1, 1]. Radii are widened
// by 1e-5 of the magnitudes involved and the slab by 1e-4, far above FP32 rounding,
// so a primitive that the exact FP32 slab test of any packet ray accepts passes.
__device__ __forceinline__ bool packet_hits_obb(const Packet &P, const Pose &K, float ta, float tb) {
  if (!(ta >= 0.0f)) return true;  // the interval form below assumes t >= 0
  const float R[9] = {K.p0.x, K.p0.y, K.p0.z, K.p0.w, K.p1.x, K.p1.y, K.p1.z, K.p1.w, K.p2.x};
  const float tk[3] = {K.p2.y, K.p2.z, K.p2.w};
  const float is[3] = {K.p3.x, K.p3.y, K.p3.z};
  float pc[3], pr[3], pm[3], dc[3], dr[3], dm[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    pc[i] = 0.5f * (P.omin[i] + P.omax[i]) - tk[i];
    pr[i] = 0.5f * (P.omax[i] - P.omin[i]);
    pm[i] = fabsf(P.omin[i]) + fabsf(P.omax[i]) + fabsf(tk[i]);
    dc[i] = 0.5f * (P.dmin[i] + P.dmax[i]);
    dr[i] = 0.5f * (P.dmax[i] - P.dmin[i]);
    dm[i] = fabsf(P.dmin[i]) + fabsf(P.dmax[i]);
  }
  constexpr float B = 1.0f + 1.0e-4f;
  float tmin = ta, tmax = tb;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float a0 = R[j], a1 = R[3 + j], a2 = R[6 + j];
    const float b0 = fabsf(a0), b1 = fabsf(a1), b2 = fabsf(a2);
    const float oc = is[j] * fmaf(a2, pc[2], fmaf(a1, pc[1], a0 * pc[0]));
    const float ro = is[j] * (fmaf(b2, pr[2], fmaf(b1, pr[1], b0 * pr[0])) +
                              1.0e-5f * fmaf(b2, pm[2], fmaf(b1, pm[1], b0 * pm[0])));
    const float ddc = is[j] * fmaf(a2, dc[2], fmaf(a1, dc[1], a0 * dc[0]));
    const float rd = is[j] * (fmaf(b2, dr[2], fmaf(b1, dr[1], b0 * dr[0])) +
                              1.0e-5f * fmaf(b2, dm[2], fmaf(b1, dm[1], b0 * dm[0])));
    const float lo_o = oc - ro, hi_o = oc + ro, lo_d = ddc - rd, hi_d = ddc + rd;
    // lo_o + t lo_d <= B
    if (lo_d > 0.0f) tmax = fminf(tmax, (B - lo_o) / lo_d);
    else if (lo_d < 0.0f) tmin = fmaxf(tmin, (B - lo_o) / lo_d);
    else if (lo_o > B) return false;
    // hi_o + t hi_d >= -B
    if (hi_d < 0.0f) tmax = fminf(tmax, (-B - hi_o) / hi_d);
    else if (hi_d > 0.0f) tmin = fmaxf(tmin, (-B - hi_o) / hi_d);
    else if (hi_o < -B) return false;
  }
  return tmin <= tmax + 1.0e-5f * (fabsf(tmin) + fabsf(tmax)) + 1.0e-30f;
}

// Warp-private shared memory of a tile. The packet bounds are warp-uniform, so
// they live here rather than in every lane's registers.
template <int CAP>
struct TileShared {
  Packet pk;
  int stack[STACK];
  int cand[CBUF];
  Xform exf[CAP];
  const char *eptr[CAP];  // payload of the entry's primitive
  int ek[CAP];
  int elo[CAP], ehi[CAP];
  uint16_t erng[CAP][32];  // per lane: (i_lo - elo) | (i_hi - elo) << 8
  unsigned int clk;  // the frame kernel's tile start (clock), for its tile schedule
};

// Leaves of a contiguous range of BVH positions [r0, r1): the adjoint's primitive
// groups. range[i] is internal node i's sorted leaf range [first, last]; leaf node
// n-1+j holds the primitive at position j.
struct LeafRange {
  const int2 *range;
  int r0, r1;
};

// A lane's inclusive sample range [lo, hi] of window entry e (lo > hi: none).
template <class SH>
__device__ __forceinline__ void lane_range(const SH &sh, int e, int lane, int &lo, int &hi) {
  const int base = sh.elo[e];
  const uint32_t r = sh.erng[e][lane];
  lo = base + (int)(r & 0xffu);
  hi = base + (int)(r >> 8);
}

// Traverse the BVH for the packet over [ta, tb]. Candidate leaves (primitive ids)
// are passed to `emit(nc)` in batches of up to CBUF via sh.cand; emit returns false
// to abort. Returns false on stack overflow or an aborted emit. RANGED: only nodes
// whose leaves meet the LeafRange are visited.
template <bool RANGED = false, class SH, class Emit>
__device__ __forceinline__ bool traverse_tile(SH &sh, const Node *__restrict__ nodes, int n_prims, float ta,
                                              float tb, Emit &&emit, int *status = nullptr,
                                              LeafRange lr = LeafRange{nullptr, 0, 0}) {
  const Packet &P = sh.pk;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (n_prims <= 0) return true;
  // start from the cut the BVH build leaves after the last node: up to 32 nodes covering
  // every leaf (the root alone for one primitive), all tested in the first step
  const int *cut = reinterpret_cast<const int *>(nodes + 2 * n_prims - 1);
  const int ncut = min(max(__ldg(cut), 1), 32);
  if (lane < ncut) sh.stack[lane] = __ldg(cut + 1 + lane);
  __syncwarp();
  int sp = ncut, nc = 0;
  while (true) {
    if (sp > 0 && nc < 32) {
      int take = sp < 32 ? sp : 32;
      sp -= take;
      int node = lane < take ? sh.stack[sp + lane] : -1;
      __syncwarp();
      if (node >= 0 && !MVP_IN_BOUNDS(node < 2 * n_prims - 1, status)) node = -1;
      if (RANGED && node >= 0) {
        const int2 span = node >= n_prims - 1 ? make_int2(node - (n_prims - 1), node - (n_prims - 1))
                                              : __ldg(lr.range + node);
        if (span.x >= lr.r1 || span.y < lr.r0) node = -1;
      }
      bool pass = false, leaf = false;
      int l = 0, r = 0;
      if (node >= 0) {
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        float4 a = __ldg(np), b = __ldg(np + 1);
        l = __float_as_int(a.w);
        r = __float_as_int(b.w);
        leaf = l < 0;
        // an inverted box holds no primitive that any ray can meet
        pass = a.x <= b.x && packet_hits_box(P, a, b, ta, tb);
      }
      unsigned mleaf = __ballot_sync(FULL, pass && leaf);
      unsigned minner = __ballot_sync(FULL, pass && !leaf);
      int nl = __popc(mleaf), ni = __popc(minner);
      if (sp + 2 * ni > STACK) return false;
      if (pass && leaf)
        sh.cand[nc + __popc(mleaf & lt)] = MVP_IN_BOUNDS(-1 - l >= 0 && -1 - l < n_prims, status) ? -1 - l : 0;
      if (pass && !leaf) {
        int pos = sp + 2 * __popc(minner & lt);
        sh.stack[pos] = r;
        sh.stack[pos + 1] = l;
      }
      sp += 2 * ni;
      nc += nl;
      __syncwarp();
    } else {
      if (nc == 0) break;
      if (!emit(nc)) return false;
      nc = 0;
      __syncwarp();
    }
  }
  return true;
}

// Per-lane ray data of a tile.
struct LaneRay {
  int64_t r;  // ray index or -1
  float o[3], d[3];
};

__device__ __forceinline__ void load_lane_ray(LaneRay &L, const float *__restrict__ o, const float *__restrict__ d,
                                              int64_t r) {
  L.r = r;
  if (r >= 0) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      L.o[j] = o[3 * r + j];
      L.d[j] = d[3 * r + j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) L.o[j] = L.d[j] = 0.0f;
  }
}

// Build the window's primitive list for samples [w0, w1): every traversal
// candidate (RANGED: in the LeafRange) that some lane's exact slab interval meets at
// a sample of the window with index <= lane_last (the lane's last live sample). The
// first `skip` such primitives (in the fixed traversal order) are passed over.
// Returns the number of entries; WINDOW_FULL if more than CAP remain after the
// skipped ones (the list then holds the first CAP of them, ready to use) or if an
// entry's tile range spans more than MAX_SPAN samples (a window of at most MAX_SPAN + 1
// samples never does); WINDOW_STACK if the traversal stack overflowed.
template <int CAP, bool RANGED = false>
__device__ __forceinline__ int build_window(TileShared<CAP> &sh, const Node *__restrict__ nodes,
                                            const Pose *__restrict__ pose, const Xform *__restrict__ xf,
                                            const char *payload, int64_t prim_bytes, int n_prims,
                                            const LaneRay &L, int lane_last, float t_near, float t_far, float dt,
                                            int n_steps, int w0, int w1, int skip = 0, int *status = nullptr,
                                            LeafRange lr = LeafRange{nullptr, 0, 0}) {
  const int lane = threadIdx.x & 31;
  float ta = sample_t(t_near, dt, w0);
  float tb = sample_t(t_near, dt, w1 - 1);
  int ne = 0, seen = 0;
  bool full = false;
  bool live = L.r >= 0 && lane_last >= w0;
  int hi_cap = min(w1 - 1, lane_last);
  const float inv_dt = 1.0f / dt;
  // the packet tests use the window's time range with a small slack
  const float slack = 1.0e-5f * (fabsf(ta) + fabsf(tb)) + 1.0e-30f;
  auto emit = [&](int nc) -> bool {
    // drop candidates whose oriented box no packet ray can meet in the window (one
    // candidate per lane), keeping the survivors in traversal order
    {
      int kept = 0;
      for (int c0 = 0; c0 < nc; c0 += 32) {
        const int c = c0 + lane;
        int k = -1;
        bool keep = false;
        if (c < nc) {
          k = sh.cand[c];
          const float4 *qa = reinterpret_cast<const float4 *>(pose + k);
          Pose Pk;
          Pk.p0 = __ldg(qa);
          Pk.p1 = __ldg(qa + 1);
          Pk.p2 = __ldg(qa + 2);
          Pk.p3 = __ldg(qa + 3);
          keep = packet_hits_obb(sh.pk, Pk, ta - slack, tb + slack);
        }
        const unsigned m = __ballot_sync(FULL, keep);
        __syncwarp();  // every lane has read its candidate before any is overwritten
        if (keep) sh.cand[kept + __popc(m & ((1u << lane) - 1u))] = k;
        kept += __popc(m);
        __syncwarp();
      }
      nc = kept;
    }
    // the exact per-lane test, two candidates at a time so that their dependency
    // chains overlap; entries are appended in candidate order
    auto append = [&](int k, int ilo, int ihi) -> bool {
      const bool has = ilo <= ihi;
      if (__ballot_sync(FULL, has) == 0) return true;
      if (seen++ < skip) return true;
      if (ne >= CAP) {
        full = true;
        return false;
      }
      const int lo_min = __reduce_min_sync(FULL, has ? ilo : 0x7fffffff);
      const int hi_max = __reduce_max_sync(FULL, has ? ihi : -1);
      if (hi_max - lo_min > MAX_SPAN) {  // the lanes' offsets would not fit 8 bits: split the window
        full = true;
        return false;
      }
      sh.erng[ne][lane] = has ? (uint16_t)((ilo - lo_min) | ((ihi - lo_min) << 8)) : EMPTY_RANGE;
      if (lane == 0) {
        sh.ek[ne] = k;
        sh.elo[ne] = lo_min;
        sh.ehi[ne] = hi_max;
      }
      ++ne;
      return true;
    };
    for (int c = 0; c < nc; c += 2) {
      const bool two = c + 1 < nc;
      const int k0 = sh.cand[c], k1 = sh.cand[two ? c + 1 : c];
      const float4 *q0 = reinterpret_cast<const float4 *>(pose + k0);
      const float4 *q1 = reinterpret_cast<const float4 *>(pose + k1);
      Pose P0, P1;
      P0.p0 = __ldg(q0);
      P1.p0 = __ldg(q1);
      P0.p1 = __ldg(q0 + 1);
      P1.p1 = __ldg(q1 + 1);
      P0.p2 = __ldg(q0 + 2);
      P1.p2 = __ldg(q1 + 2);
      P0.p3 = __ldg(q0 + 3);
      P1.p3 = __ldg(q1 + 3);
      float tin0, tout0, tin1, tout1;
      const bool h0 = slab_spec(P0, L.o[0], L.o[1], L.o[2], L.d[0], L.d[1], L.d[2], t_near, t_far, tin0, tout0) && live;
      const bool h1 = slab_spec(P1, L.o[0], L.o[1], L.o[2], L.d[0], L.d[1], L.d[2], t_near, t_far, tin1, tout1) && live;
      // lanes that miss search from t_near (a cheap, exact case) and discard the result
      const float u0 = h0 ? tin0 : t_near, v0 = h0 ? tout0 : t_near;
      const float u1 = h1 ? tin1 : t_near, v1 = h1 ? tout1 : t_near;
      const int a0 = first_sample_geq(u0, t_near, dt, inv_dt, n_steps);
      const int a1 = first_sample_geq(u1, t_near, dt, inv_dt, n_steps);
      const int b0 = first_sample_gt(v0, t_near, dt, inv_dt, n_steps);
      const int b1 = first_sample_gt(v1, t_near, dt, inv_dt, n_steps);
      if (!append(k0, h0 ? max(a0, w0) : 1, h0 ? min(b0 - 1, hi_cap) : 0)) return false;
      if (two && !append(k1, h1 ? max(a1, w0) : 1, h1 ? min(b1 - 1, hi_cap) : 0)) return false;
    }
    return true;
  };
  bool ok = traverse_tile<RANGED>(sh, nodes, n_prims, ta - slack, tb + slack, emit, status, lr);
  __syncwarp();
  if (!ok && !full) return WINDOW_STACK;
  // the entries' march transforms and payload pointers, loaded in parallel
  for (int e = lane; e < ne; e += 32) {
    const int k = sh.ek[e];
    const float4 *xp = reinterpret_cast<const float4 *>(xf + k);
    sh.exf[e].r0 = __ldg(xp);
    sh.exf[e].r1 = __ldg(xp + 1);
    sh.exf[e].r2 = __ldg(xp + 2);
    sh.eptr[e] = payload + (int64_t)k * prim_bytes;
  }
  __syncwarp();
  return ok ? ne : WINDOW_FULL;
}

// Active entries at sample i (two 32-bit masks) and the next sample at which the
// active set changes (capped at w1).
template <int CAP>
__device__ __forceinline__ int active_set(const TileShared<CAP> &sh, int ne, int i, int w1, uint32_t &m0,
                                          uint32_t &m1) {
  const int lane = threadIdx.x & 31;
  int nxt = 0x7fffffff;
  bool a0 = false, a1 = false;
  if (lane < ne) {
    int lo = sh.elo[lane], hi = sh.ehi[lane];
    a0 = lo <= i && i <= hi;
    nxt = lo > i ? lo : (hi >= i ? hi + 1 : 0x7fffffff);
  }
  if (CAP > 32 && lane + 32 < ne) {
    int lo = sh.elo[lane + 32], hi = sh.ehi[lane + 32];
    a1 = lo <= i && i <= hi;
    int v = lo > i ? lo : (hi >= i ? hi + 1 : 0x7fffffff);
    nxt = min(nxt, v);
  }
  m0 = __ballot_sync(FULL, a0);
  m1 = __ballot_sync(FULL, a1);
  nxt = __reduce_min_sync(FULL, nxt);
  return min(nxt, w1);
}

// Entries whose tile sample range meets the chunk [i, ie) (two 32-bit masks), and
// the first sample at or after ie where some entry starts (w1 if none): where the
// chunk is empty the march jumps there.
template <int CAP>
__device__ __forceinline__ int active_chunk(const TileShared<CAP> &sh, int ne, int i, int ie, int w1, uint32_t &m0,
                                            uint32_t &m1) {
  const int lane = threadIdx.x & 31;
  int nxt = 0x7fffffff;
  bool a0 = false, a1 = false;
  if (lane < ne) {
    const int lo = sh.elo[lane], hi = sh.ehi[lane];
    a0 = lo < ie && hi >= i;
    if (lo >= ie) nxt = lo;
  }
  if (CAP > 32 && lane + 32 < ne) {
    const int lo = sh.elo[lane + 32], hi = sh.ehi[lane + 32];
    a1 = lo < ie && hi >= i;
    if (lo >= ie) nxt = min(nxt, lo);
  }
  m0 = __ballot_sync(FULL, a0);
  m1 = __ballot_sync(FULL, a1);
  nxt = __reduce_min_sync(FULL, nxt);
  return min(nxt, w1);
}

}  // namespace mvp
