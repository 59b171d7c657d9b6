// noalloc.cu -- a render entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plug-in inside a host application that
// owns every device allocation (a game engine or VR compositor hands out no
// allocator), a real-time frame loop that must never stall on the implicit device
// synchronisation of cudaMalloc/cudaFree, or a component with a fixed memory budget
// set at start-up. mvp_raymarch_fwd_static serves them: it rebuilds the BVH and
// marches the rays exactly as mvp_build_bvh + mvp_raymarch_fwd do, but keeps the
// BVH and the status word in the file-scope device array below, so it allocates
// nothing and needs no context or handle.
//
// The array is sized for MVP_STATIC_MAX_PRIMS primitives (about 4 MB) and is held
// by every GPU that loads the library until the process exits. All calls share it
// and it keeps the last call's contents; the refit counters and the status word are
// cleared on every call. Calls whose work overlaps on the GPU (other streams, other
// host threads) race on the array and must be serialised by the caller.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "march.cuh"

namespace {

constexpr int kMaxPrims = MVP_STATIC_MAX_PRIMS;
constexpr int kMaxSortBlocks = (kMaxPrims + mvp::BVH_SORT_TILE - 1) / mvp::BVH_SORT_TILE;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of the array (each region 256-byte aligned).
constexpr size_t kOffStatus = 0;
constexpr size_t kOffScene = align256(kOffStatus + sizeof(int));
constexpr size_t kOffPose = align256(kOffScene + 6 * sizeof(float));
constexpr size_t kOffXf = align256(kOffPose + (size_t)kMaxPrims * sizeof(mvp::Pose));
constexpr size_t kOffPbox = align256(kOffXf + (size_t)kMaxPrims * sizeof(mvp::Xform));
constexpr size_t kOffKeysA = align256(kOffPbox + (size_t)kMaxPrims * 2 * sizeof(float4));
constexpr size_t kOffKeysB = align256(kOffKeysA + (size_t)kMaxPrims * sizeof(uint32_t));
constexpr size_t kOffValsA = align256(kOffKeysB + (size_t)kMaxPrims * sizeof(uint32_t));
constexpr size_t kOffValsB = align256(kOffValsA + (size_t)kMaxPrims * sizeof(int));
constexpr size_t kOffCounts = align256(kOffValsB + (size_t)kMaxPrims * sizeof(int));
constexpr size_t kOffNodes = align256(kOffCounts + (size_t)256 * kMaxSortBlocks * sizeof(int));
constexpr size_t kOffParent = align256(kOffNodes + (size_t)(2 * kMaxPrims + mvp::CUT_NODES) * sizeof(mvp::Node));
constexpr size_t kOffRank = align256(kOffParent + (size_t)2 * kMaxPrims * sizeof(int));
constexpr size_t kBytes = align256(kOffRank + (size_t)kMaxPrims * sizeof(int));

static __device__ __align__(256) unsigned char g_static_scratch[kBytes];

// Device address of the array, looked up once per device with that device current,
// and again when the device's context is not the one the address was taken in (the
// old address dies with its context, e.g. after cudaDeviceReset).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};

mvp_status reject(mvp_status s, const char *msg) {
  mvp::record_error(msg);  // reported by mvp_last_error()
  return s;
}

}  // namespace

extern "C" mvp_status mvp_raymarch_fwd_static(const mvp_prims *prims, const mvp_rays *rays, float *out_rgba,
                                              int32_t *status_out, mvp_stream stream) {
  if (!prims || !rays) return reject(MVP_ERR_INVALID_ARG, "prims and rays are required");
  if (prims->n < 0 || prims->n > kMaxPrims)
    return reject(MVP_ERR_INVALID_ARG, "prims.n exceeds MVP_STATIC_MAX_PRIMS (use mvp_raymarch_fwd)");
  if (prims->M < 2 || prims->M > MVP_MAX_M || prims->reserved != 0 ||
      (prims->dtype != MVP_F32 && prims->dtype != MVP_BF16 && prims->dtype != MVP_F16))
    return reject(MVP_ERR_INVALID_ARG, "bad prims.M, prims.dtype or prims.reserved");
  if (prims->n > 0 && (!prims->t || !prims->q || !prims->s || !prims->payload))
    return reject(MVP_ERR_INVALID_ARG, "prims has a NULL array");
  if (prims->n > 0 && reinterpret_cast<uintptr_t>(prims->payload) % (prims->dtype == MVP_F32 ? 16 : 8))
    return reject(MVP_ERR_INVALID_ARG, "payload is misaligned");
  if (rays->n < 0 || (rays->n > 0 && (!rays->o || !rays->d || !out_rgba)))
    return reject(MVP_ERR_INVALID_ARG, "rays.n < 0 or a NULL ray/output array");
  if (reinterpret_cast<uintptr_t>(out_rgba) % 16) return reject(MVP_ERR_INVALID_ARG, "out_rgba is misaligned");
  if (!(rays->dt > 0.0f) || !(rays->t_far > rays->t_near) || !(rays->eps_early >= 0.0f && rays->eps_early < 1.0f) ||
      !isfinite(rays->t_near) || !isfinite(rays->t_far) || !isfinite(rays->dt) || rays->width < 0 || rays->height < 0 ||
      (rays->flags & ~(MVP_BLEND_SEQUENTIAL | MVP_COMPOSITE_LITERAL)))
    return reject(MVP_ERR_INVALID_ARG, "bad ray parameters");
  const int64_t ns = mvp_num_steps(rays->t_near, rays->t_far, rays->dt);
  if (ns > MVP_MAX_STEPS) return reject(MVP_ERR_INVALID_ARG, "n_steps exceeds MVP_MAX_STEPS");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return reject(MVP_ERR_CUDA, "no current CUDA device");
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = mvp::current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);  // creates the context if there is none yet
      if (e != cudaSuccess || !p) return reject(MVP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_addr[dev] = static_cast<unsigned char *>(p);
      g_ctx[dev] = mvp::current_context_id();
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  (void)cudaGetLastError();
  int *d_status = reinterpret_cast<int *>(base + kOffStatus);
  if (cudaMemsetAsync(d_status, 0, sizeof(int), st) != cudaSuccess) return reject(MVP_ERR_CUDA, "status reset");

  mvp::BvhBuffers b;  // views into the array; nothing here is allocated or freed
  b.base = nullptr;
  b.cap = kMaxPrims;
  b.scene = reinterpret_cast<float *>(base + kOffScene);
  b.pose = reinterpret_cast<mvp::Pose *>(base + kOffPose);
  b.xf = reinterpret_cast<mvp::Xform *>(base + kOffXf);
  b.pbox = reinterpret_cast<float4 *>(base + kOffPbox);
  b.keys_a = reinterpret_cast<uint32_t *>(base + kOffKeysA);
  b.keys_b = reinterpret_cast<uint32_t *>(base + kOffKeysB);
  b.vals_a = reinterpret_cast<int *>(base + kOffValsA);
  b.vals_b = reinterpret_cast<int *>(base + kOffValsB);
  b.counts = reinterpret_cast<int *>(base + kOffCounts);
  b.nodes = reinterpret_cast<mvp::Node *>(base + kOffNodes);
  b.parent = reinterpret_cast<int *>(base + kOffParent);
  b.rank = reinterpret_cast<int *>(base + kOffRank);
  cudaError_t e = mvp::bvh_build(b, prims->t, prims->q, prims->s, prims->n, prims->M, st, d_status);
  if (e != cudaSuccess) return reject(MVP_ERR_CUDA, "BVH build launch failed");

  if (rays->n > 0) {
    mvp::MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.n_prims = prims->n;
    a.M = prims->M;
    a.dtype = prims->dtype;
    a.payload = prims->payload;
    a.nodes = b.nodes;
    a.pose = b.pose;
    a.xf = b.xf;
    a.rank = b.rank;
    a.sequential = (rays->flags & MVP_BLEND_SEQUENTIAL) ? 1 : 0;
    a.literal = (rays->flags & MVP_COMPOSITE_LITERAL) ? 1 : 0;
    a.geom = mvp::make_tile_geom(rays->n, rays->width, rays->height);
    a.o = rays->o;
    a.d = rays->d;
    a.t_near = rays->t_near;
    a.t_far = rays->t_far;
    a.dt = rays->dt;
    a.stop_T = (float)(1.0 - (double)rays->eps_early);
    a.bg[0] = rays->bg[0];
    a.bg[1] = rays->bg[1];
    a.bg[2] = rays->bg[2];
    a.n_steps = (int)ns;
    a.out = out_rgba;
    a.status = d_status;
    e = mvp::launch_march(a, st);
    if (e != cudaSuccess) return reject(MVP_ERR_CUDA, "march launch failed");
  }
  if (status_out && cudaMemcpyAsync(status_out, d_status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return reject(MVP_ERR_CUDA, "status copy failed");
  return MVP_OK;
}
