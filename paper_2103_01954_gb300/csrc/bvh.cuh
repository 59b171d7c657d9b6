// bvh.cuh -- device buffers of a per-frame LBVH and the build entry points.
#pragma once

#include "common.cuh"

namespace mvp {

constexpr int BVH_SORT_TILE = 2048;  // keys per radix-sort block (sizes BvhBuffers::counts)
constexpr int BVH_SORT1_N = 8192;    // primitives up to which one block sorts the keys
constexpr int BVH_SORTC_N = 32768;   // primitives up to which one thread-block cluster sorts them
// The traversal's starting cut: up to 32 nodes that together cover every leaf, stored as
// {count, node...} right after the last node; node arrays hold CUT_NODES extra nodes for it.
constexpr int CUT_INTS = 33;
constexpr int CUT_NODES = (CUT_INTS * 4 + 31) / 32;

struct BvhBuffers {
  char *base = nullptr;
  size_t bytes = 0;
  int cap = 0;  // primitives the buffers hold
  int n = 0;    // primitives of the last build
  int M = 0;    // payload edge of the last build (the march transform depends on it)
  float *scene = nullptr;  // [6] centre bounds
  Pose *pose = nullptr;    // [n]
  Xform *xf = nullptr;     // [n]
  float4 *pbox = nullptr;  // [n][2] world boxes per primitive
  uint32_t *keys_a = nullptr, *keys_b = nullptr;  // Morton codes (sorted result in keys_a)
  int *vals_a = nullptr, *vals_b = nullptr;       // primitive ids (sorted result in vals_a)
  int *counts = nullptr;   // radix digit counts [256][blocks]
  Node *nodes = nullptr;   // [2n-1], then the traversal's starting cut (CUT_INTS ints at nodes + 2n-1)
  int *parent = nullptr;   // [2n]: the internal nodes' sorted leaf ranges (int2) during the build
  int *rank = nullptr;     // [n] each primitive's leaf position (its place in BVH order)
  float *gmc = nullptr;    // [n][12] adjoint accumulators of the march transform
};

cudaError_t bvh_reserve(BvhBuffers &b, int n);
void bvh_release(BvhBuffers &b);
// status (device, nullable): STATUS_POSE is or-ed in for a primitive whose pose
// defines no box (non-finite, zero quaternion, scale <= 0).
cudaError_t bvh_build(BvhBuffers &b, const float *t, const float *q, const float *s, int n, int M, cudaStream_t st,
                      int *status);
cudaError_t bvh_export(const BvhBuffers &b, uint64_t *keys, int32_t *children, float *bounds, float *scene,
                       cudaStream_t st);

}  // namespace mvp
