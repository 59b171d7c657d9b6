// common.cuh -- shared device definitions of the MVP ray-march library.
//
// Discrete decisions (Morton codes, ray/box membership, the voxel cell of a sample)
// use explicit round-to-nearest intrinsics (__fmul_rn, __fadd_rn, __fmaf_rn,
// __frcp_rn, __fdiv_rn, __fsqrt_rn), which the compiler never contracts or
// reassociates, so their results are fixed bit for bit by the operation order
// written here. Everything else may use FMA.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/mvp.h"

namespace mvp {

constexpr unsigned FULL = 0xffffffffu;

// Device status word bits.
constexpr int STATUS_CAPACITY = 1;
constexpr int STATUS_DEVICE = 2;
constexpr int STATUS_POSE = 4;  // a primitive's t, q or s is not finite, |q| = 0 or s <= 0
constexpr int STATUS_BOUNDS = 8;  // checked builds: an index fell outside its array (access skipped)

// Programmatic dependent launch: a kernel started with pdl_launch may be scheduled
// while the kernel before it in the stream is still running; it calls pdl_wait()
// before its first global-memory access (afterwards everything earlier work wrote is
// visible), so only its launch overlaps. pdl_trigger() lets the next such kernel be
// scheduled early. Both are no-ops for kernels launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A launch of `kernel` in thread-block clusters of `cluster_x` CTAs along x, which may
// also be scheduled while the kernel before it runs (as pdl_launch).
template <typename... KArgs, typename... Args>
inline cudaError_t cluster_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, unsigned cluster_x, size_t smem,
                                  cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster_x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Host side (api.cu). Identity of the calling thread's current CUDA context: unique
// for the life of the process (a context re-created after cudaDeviceReset gets a new
// one); 0 when the thread has no current context.
unsigned long long current_context_id();

// Host side (api.cu). Lets `kernel` launch with `bytes` of dynamic shared memory in
// the current context. The opt-in (cudaFuncAttributeMaxDynamicSharedMemorySize)
// belongs to the kernel in one context, so it is remembered per (kernel, context)
// under a mutex: each device a process drives, and a context re-created after a
// reset, is opted in on its first launch there.
cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes);

// Checked builds (-DMVP_CHECK_BOUNDS, the stand-in for a memory checker): an index
// outside its array sets STATUS_BOUNDS and the access is skipped. Elsewhere the
// check compiles to nothing.
#ifdef MVP_CHECK_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, int *status) {
  if (!ok && status) atomicOr(status, STATUS_BOUNDS);
  return ok;
}
#define MVP_IN_BOUNDS(cond, status) ::mvp::in_bounds((cond), (status))
#else
#define MVP_IN_BOUNDS(cond, status) true
#endif

// Per-primitive pose as used by the membership test: R (row-major, R[3*i+j]),
// t, 1/s (each correctly rounded). 64 bytes: p0 = {R00,R01,R02,R10},
// p1 = {R11,R12,R20,R21}, p2 = {R22,t0,t1,t2}, p3 = {1/s0,1/s1,1/s2,0}.
struct __align__(16) Pose {
  float4 p0, p1, p2, p3;
};

// March transform of a primitive: voxel coordinate u = Mx * x + c, i.e. rows
// {M_j0, M_j1, M_j2, c_j} with M = diag(h/s) R^T, c = h - M t, h = (M-1)/2.
struct __align__(16) Xform {
  float4 r0, r1, r2;
};

// BVH node: box plus children. Internal nodes 0..n-2, leaves n-1..2n-2.
// Leaf: left = -1 - primitive id. Internal: left/right = child node indices.
struct __align__(16) Node {
  float lox, loy, loz;
  int left;
  float hix, hiy, hiz;
  int right;
};

// Per-ray state saved by the forward for the adjoint (32 bytes). Under the
// sequential rule a clamped ray keeps, instead of c/a and (1 - T)/a, the colour and
// the weight of the primitive whose weight was clamped and that primitive's leaf rank
// (rank_clamp = 0x7fffffff: none was; -1: the summed rule applied).
struct __align__(16) Saved {
  float rho_r, rho_g, rho_b;  // c/a at the clamped sample
  float beta;                 // (1 - T)/a at the clamped sample
  int i_last;                 // last processed sample (-1: none)
  int i_clamp;                // clamped sample or -1
  int rank_clamp;             // see above
  int pad;
};

// ---------------------------------------------------------------- spec math
// Rotation from q/|q| with a fixed operation order (Sec. 3.1.2).
__device__ __forceinline__ void rot_spec(float q0, float q1, float q2, float q3, float R[9]) {
  float n2 = __fmul_rn(q0, q0);
  n2 = __fadd_rn(n2, __fmul_rn(q1, q1));
  n2 = __fadd_rn(n2, __fmul_rn(q2, q2));
  n2 = __fadd_rn(n2, __fmul_rn(q3, q3));
  float nrm = __fsqrt_rn(n2);
  float w = __fdiv_rn(q0, nrm), x = __fdiv_rn(q1, nrm), y = __fdiv_rn(q2, nrm), z = __fdiv_rn(q3, nrm);
  float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  R[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  R[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  R[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  R[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  R[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  R[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
}

// Slab interval of ray (o, d) against the box of a pose in its local frame
// ([-1,1]^3), clipped to [t_near, t_far]. Fixed operation order, every step
// correctly rounded: p = o - t; per axis j the local origin and direction
// ol = fma(R2j, p2, fma(R1j, p1, R0j*p0)) * (1/s_j), dl likewise with d; if dl == 0
// the ray is inside the slab iff |ol| <= 1, else r = 1/dl, t1 = (-1 - ol)*r,
// t2 = (1 - ol)*r. Returns whether [max(t_near, lows), min(t_far, highs)] is nonempty.
__device__ __forceinline__ bool slab_spec(const Pose &P, float ox, float oy, float oz, float dx, float dy,
                                          float dz, float t_near, float t_far, float &tin, float &tout) {
  const float R[9] = {P.p0.x, P.p0.y, P.p0.z, P.p0.w, P.p1.x, P.p1.y, P.p1.z, P.p1.w, P.p2.x};
  const float is[3] = {P.p3.x, P.p3.y, P.p3.z};
  float p0 = __fsub_rn(ox, P.p2.y), p1 = __fsub_rn(oy, P.p2.z), p2 = __fsub_rn(oz, P.p2.w);
  float lo = t_near, hi = t_far;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float on = __fmaf_rn(R[2 * 3 + j], p2, __fmaf_rn(R[1 * 3 + j], p1, __fmul_rn(R[0 * 3 + j], p0)));
    float dn = __fmaf_rn(R[2 * 3 + j], dz, __fmaf_rn(R[1 * 3 + j], dy, __fmul_rn(R[0 * 3 + j], dx)));
    float ol = __fmul_rn(on, is[j]);
    float dl = __fmul_rn(dn, is[j]);
    if (dl == 0.0f) {
      if (ol < -1.0f || ol > 1.0f) ok = false;
    } else {
      float r = __frcp_rn(dl);
      float t1 = __fmul_rn(__fsub_rn(-1.0f, ol), r);
      float t2 = __fmul_rn(__fsub_rn(1.0f, ol), r);
      lo = fmaxf(lo, fminf(t1, t2));
      hi = fminf(hi, fmaxf(t1, t2));
    }
  }
  tin = lo;
  tout = hi;
  return ok && lo <= hi;
}

// Sample time t_i = t_near + i*dt (product rounded, then the sum).
__device__ __forceinline__ float sample_t(float t_near, float dt, int i) {
  return __fadd_rn(t_near, __fmul_rn((float)i, dt));
}

// Smallest i in [0, n] with t_i >= v (n if none). t_i is non-decreasing in i. The
// estimate (v - t_near) * (1/dt) is only a starting point. The four sample times
// around it settle, without branches, every case where it is off by at most one
// (t_{i-1} >= v moves down, t_i < v moves up); anything else takes the exact walk.
static __device__ __noinline__ int first_sample_walk(float v, float t_near, float dt, int n, int i, bool strict) {
  // strict: smallest i with t_i > v; else with t_i >= v
  auto after = [&](int j) { const float tj = sample_t(t_near, dt, j); return strict ? tj > v : tj >= v; };
  int it = 0;
  while (i > 0 && after(i - 1) && it < 64) { --i; ++it; }
  while (i < n && !after(i) && it < 128) { ++i; ++it; }
  if (it >= 64) {  // estimate far off (huge t_near relative to dt): bisect
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (after(mid)) hi = mid; else lo = mid + 1;
    }
    i = lo;
  }
  return i;
}

__device__ __forceinline__ int first_sample_settle(float v, float t_near, float dt, int n, int i, bool strict) {
  const float sm2 = sample_t(t_near, dt, max(i - 2, 0)), sm1 = sample_t(t_near, dt, max(i - 1, 0));
  const float s0 = sample_t(t_near, dt, min(i, n)), sp1 = sample_t(t_near, dt, min(i + 1, n));
  const bool m1 = i > 0 && (strict ? sm1 > v : sm1 >= v);       // answer <= i - 1
  const bool m2 = i > 1 && (strict ? sm2 > v : sm2 >= v);       // answer <= i - 2
  const bool p0 = i < n && !(strict ? s0 > v : s0 >= v);        // answer >= i + 1
  const bool p1 = i + 1 < n && !(strict ? sp1 > v : sp1 >= v);  // answer >= i + 2
  if (!m2 && !p1) return m1 ? i - 1 : (p0 ? i + 1 : i);
  return first_sample_walk(v, t_near, dt, n, i, strict);
}

__device__ __forceinline__ int first_sample_geq(float v, float t_near, float dt, float inv_dt, int n) {
  const float x = (v - t_near) * inv_dt;
  const int i = !(x > 0.0f) ? 0 : (x >= (float)n ? n : (int)ceilf(x));
  return first_sample_settle(v, t_near, dt, n, i, false);
}

// Smallest i in [0, n] with t_i > v (n if none).
__device__ __forceinline__ int first_sample_gt(float v, float t_near, float dt, float inv_dt, int n) {
  const float x = (v - t_near) * inv_dt;
  const int i = x < 0.0f ? 0 : (x >= (float)n ? n : (int)floorf(x) + 1);
  return first_sample_settle(v, t_near, dt, n, i, true);
}

// ---------------------------------------------------------------- payload loads
template <int DT>
struct Voxel;

template <>
struct Voxel<MVP_F32> {
  using T = float4;
  __device__ __forceinline__ static float4 load(const void *base, int64_t v) {
    return __ldg(reinterpret_cast<const float4 *>(base) + v);
  }
};

template <>
struct Voxel<MVP_BF16> {
  __device__ __forceinline__ static float4 load(const void *base, int64_t v) {
    uint2 r = __ldg(reinterpret_cast<const uint2 *>(base) + v);
    float4 o;
    o.x = __uint_as_float(r.x << 16);
    o.y = __uint_as_float(r.x & 0xffff0000u);
    o.z = __uint_as_float(r.y << 16);
    o.w = __uint_as_float(r.y & 0xffff0000u);
    return o;
  }
};

template <>
struct Voxel<MVP_F16> {
  __device__ __forceinline__ static float4 load(const void *base, int64_t v) {
    uint2 r = __ldg(reinterpret_cast<const uint2 *>(base) + v);
    __half2 a = *reinterpret_cast<__half2 *>(&r.x);
    __half2 b = *reinterpret_cast<__half2 *>(&r.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
};

// Cell and in-cell fraction along one axis of the voxel coordinate u (grid edge M,
// Mm2 = M - 2): the values that clamping u into [0, M-1], truncating, capping the cell
// at M - 2 and subtracting give, bit for bit, in four instructions instead of six. The
// unsigned conversion sends u < 0 and NaN to cell 0; the saturated difference is then
// 0 below the box (and for NaN) and 1 above it, as the clamped coordinate's would be.
__device__ __forceinline__ int voxel_cell(float u, unsigned Mm2, float &f) {
  const unsigned c = min(__float2uint_rz(u), Mm2);
  asm("sub.rn.sat.f32 %0, %1, %2;" : "=f"(f) : "f"(u), "f"((float)c));
  return (int)c;
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float w) {
  return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                     fmaf(w, b.w - a.w, a.w));
}

// Packed FP32x2 arithmetic (two FP32 FMAs per instruction on sm_100 and later).
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// (1 - w) a + w b per component as fma(w, b, fma(-w, a, a)) on packed pairs; exact at
// w = 0 and w = 1. w2 = (w, w), nw2 = (-w, -w).
__device__ __forceinline__ float4 lerp4x2(float4 a, float4 b, float2 w2, float2 nw2) {
  const float2 l = __ffma2_rn(w2, lo2(b), __ffma2_rn(nw2, lo2(a), lo2(a)));
  const float2 h = __ffma2_rn(w2, hi2(b), __ffma2_rn(nw2, hi2(a), hi2(a)));
  return make_float4(l.x, l.y, h.x, h.y);
}

// b - a per component on packed pairs (fma(a, -1, b): the correctly rounded difference).
__device__ __forceinline__ float4 sub4x2(float4 b, float4 a) {
  const float2 m = make_float2(-1.0f, -1.0f);
  const float2 l = __ffma2_rn(lo2(a), m, lo2(b)), h = __ffma2_rn(hi2(a), m, hi2(b));
  return make_float4(l.x, l.y, h.x, h.y);
}

// a . b over 4 components on packed pairs.
__device__ __forceinline__ float dot4x2(float4 a, float4 b) {
  const float2 t = __ffma2_rn(hi2(a), hi2(b), __fmul2_rn(lo2(a), lo2(b)));
  return t.x + t.y;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

}  // namespace mvp
