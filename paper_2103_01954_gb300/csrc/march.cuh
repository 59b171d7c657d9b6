// march.cuh -- launch arguments of the march, hit-list and adjoint kernels.
#pragma once

#include "tile.cuh"

namespace mvp {

#ifndef MVP_MARCH_CAP
#define MVP_MARCH_CAP 48
#endif
constexpr int MARCH_CAP = MVP_MARCH_CAP;  // primitives a warp tile holds per depth window

// Window capacity of the forward kernels by payload edge (MT: the edge fixed at compile
// time; 0 = any edge; -1 = any edge up to 12, the serving kernels' small grids): the
// smallest voxel grids come with the most primitives per ray, where a longer list saves
// more re-traversals than the L1 it takes costs (measured: 32768 primitives of 8^3, 64
// entries 6 % faster than 48; at 16^3 and 32^3, 48 is best).
template <int MT>
__host__ __device__ constexpr int march_cap() { return MT == 8 || MT == -1 ? 64 : MARCH_CAP; }

#ifndef MVP_MARCH_MINB
#define MVP_MARCH_MINB 5  // resident blocks per SM the march kernels are compiled for
#endif

struct MarchArgs {
  // primitives and their BVH
  int n_prims, M, dtype;
  const void *payload;
  const Node *nodes;
  const Pose *pose;
  const Xform *xf;
  const int *rank;  // leaf position of each primitive (BVH order)
  int sequential;   // blend a ray's saturating sample in BVH order (MVP_BLEND_SEQUENTIAL)
  int literal;      // composite A I + (1 - A) B (MVP_COMPOSITE_LITERAL) instead of I + (1 - A) B
  // rays
  TileGeom geom;
  const float *o, *d;
  float t_near, t_far, dt, stop_T;
  float bg[3];
  int n_steps;
  // outputs
  float *out;
  Saved *saved;
  int32_t *n_eval;  // count variant when non-null
  int *status;
  // tile schedule (frame kernel only): warp slot s marches tile order[s] (a
  // permutation of the warp tiles) when order is set; cost[t] receives the clock
  // cycles tile t took when cost is set
  const int *order;
  unsigned int *cost;
};

struct HitArgs {
  int n_prims;
  const Node *nodes;
  const Pose *pose;
  TileGeom geom;
  const float *o, *d;
  float t_near, t_far;
  int64_t *counts;       // count pass
  const int64_t *offs_in;
  int64_t *offs;
  int32_t *ids;
  float *tin, *tout;
  int64_t cap;
  int *status;
};

struct BwdArgs {
  MarchArgs m;             // geometry, rays, payload (out/saved/n_eval unused)
  const Saved *saved;
  const float *grad;       // [n][4]
  float *g_payload;        // [n][M^3][4] or null
  float *gmc;              // [n][12] accumulators or null
};

// The grouped adjoint's primitive groups (consecutive BVH positions, gsize each) and
// its scratch: per warp tile the groups it meets (mask), the (tile, group) work list
// (items, goff[n_groups + 1]) and the work counter. range = the BVH's internal-node
// leaf ranges.
struct BwdGroups {
  int gsize = 0, n_groups = 0;  // n_groups <= 64
  unsigned long long *mask = nullptr;  // [n_warp_tiles]
  int *items = nullptr;                // [n_warp_tiles * n_groups]
  int *goff = nullptr;                 // [n_groups + 1]
  int *work = nullptr;                 // [1]
  const int2 *range = nullptr;         // [n_prims - 1]
};

cudaError_t launch_march(const MarchArgs &a, cudaStream_t st);
// order = the n warp tiles by descending cost bucket (a permutation of 0..n-1,
// whatever cost holds): the next frame's schedule, heaviest tiles first.
cudaError_t launch_tile_order(const unsigned int *cost, int64_t n, int *order, cudaStream_t st);
void record_error(const char *msg);
int ctx_device(const mvp_ctx *ctx);
cudaError_t launch_hits(const HitArgs &a, int64_t *counts, cudaStream_t st);
cudaError_t launch_hits_fill(const HitArgs &a, cudaStream_t st);
// gr (nullable): replay the tiles group by group (the BwdGroups scratch is the caller's)
cudaError_t launch_backward(const BwdArgs &a, const float *t, const float *q, const float *s, float *g_t,
                            float *g_q, float *g_s, cudaStream_t st, const BwdGroups *gr = nullptr);

}  // namespace mvp
