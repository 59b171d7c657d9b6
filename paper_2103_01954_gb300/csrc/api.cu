// api.cu -- the C ABI declared in include/mvp.h: argument validation, handles and
// dispatch to the kernels. Nothing here computes on the host beyond sizes.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "march.cuh"
#include "pack.cuh"

// The frame kernel's tile schedule: the warp tiles of the last frame sorted by the
// cycles each took, so that the next frame of the same size starts its heaviest
// tiles first (a tile started late on a busy GPU can otherwise outlast the rest of
// the frame). Only one call at a time may touch the buffers: a call uses them if
// the last call that did has finished or ran on the same stream, else it marches in
// the plain tile order and leaves them alone. The schedule never changes a result:
// each tile is still marched once, by one warp, in the same way.
struct TileSched {
  std::mutex mu;
  bool enabled = true;
  unsigned int *cost = nullptr;  // [cap] cycles per warp tile of the last frame
  int *order = nullptr;          // [cap] the schedule derived from them
  int64_t cap = 0;
  int64_t tiles = -1;            // warp tiles `order` was made for (-1: none)
  cudaEvent_t done = nullptr;    // after the last call's schedule kernel (on `side`)
  cudaEvent_t marched = nullptr; // after that call's march (on its stream)
  cudaStream_t side = nullptr;   // the schedule kernel runs here, beside the caller's next work
  cudaStream_t stream = nullptr; // the stream of the last call that touched the buffers
  bool pending = false;
};

struct mvp_ctx {
  int device = 0;
  int *d_status = nullptr;  // device status word (STATUS_* bits)
  TileSched sched;          // the frame kernel's
  TileSched sched_bwd;      // the adjoint's
  std::atomic<int64_t> bwd_group_bytes{0};  // mvp_ctx_set_bwd_group_bytes
};

struct mvp_bvh {
  int device = 0;  // copied from the context: the handle may outlive it
  mvp::BvhBuffers b;
};

namespace {

thread_local std::string g_err;

mvp_status fail(mvp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

mvp_status cuda_fail(cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(MVP_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
  return fail(MVP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

mvp_status ok() { return MVP_OK; }

bool finite(float v) { return isfinite(v); }

mvp_status check_prims(const mvp_prims *p) {
  if (!p) return fail(MVP_ERR_INVALID_ARG, "prims is NULL");
  if (p->n < 0 || p->n > MVP_MAX_PRIMS) return fail(MVP_ERR_INVALID_ARG, "prims.n = %d out of range", p->n);
  if (p->M < 2 || p->M > MVP_MAX_M) return fail(MVP_ERR_INVALID_ARG, "prims.M = %d out of [2, %d]", p->M, MVP_MAX_M);
  if (p->dtype != MVP_F32 && p->dtype != MVP_BF16 && p->dtype != MVP_F16)
    return fail(MVP_ERR_INVALID_ARG, "prims.dtype = %d unknown", p->dtype);
  if (p->reserved != 0) return fail(MVP_ERR_INVALID_ARG, "prims.reserved must be 0");
  if ((int64_t)p->n * p->M * p->M * p->M >= ((int64_t)1 << 40))
    return fail(MVP_ERR_INVALID_ARG, "payload too large");
  if (p->n > 0) {
    if (!p->t || !p->q || !p->s || !p->payload) return fail(MVP_ERR_INVALID_ARG, "prims has a NULL array");
    size_t align = p->dtype == MVP_F32 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(p->payload) % align)
      return fail(MVP_ERR_INVALID_ARG, "payload must be %zu-byte aligned", align);
  }
  return ok();
}

mvp_status check_rays(const mvp_rays *r, int64_t *n_steps) {
  if (!r) return fail(MVP_ERR_INVALID_ARG, "rays is NULL");
  if (r->n < 0) return fail(MVP_ERR_INVALID_ARG, "rays.n < 0");
  if (r->n > 0 && (!r->o || !r->d)) return fail(MVP_ERR_INVALID_ARG, "rays has a NULL array");
  if (!finite(r->t_near) || !finite(r->t_far) || !finite(r->dt) || !finite(r->eps_early))
    return fail(MVP_ERR_INVALID_ARG, "rays parameters must be finite");
  if (!(r->dt > 0.0f)) return fail(MVP_ERR_INVALID_ARG, "rays.dt must be > 0");
  if (!(r->t_far > r->t_near)) return fail(MVP_ERR_INVALID_ARG, "rays.t_far must be > t_near");
  if (!(r->eps_early >= 0.0f && r->eps_early < 1.0f)) return fail(MVP_ERR_INVALID_ARG, "rays.eps_early not in [0, 1)");
  if (r->width < 0 || r->height < 0) return fail(MVP_ERR_INVALID_ARG, "rays.width/height < 0");
  if (r->flags & ~(MVP_BLEND_SEQUENTIAL | MVP_COMPOSITE_LITERAL))
    return fail(MVP_ERR_INVALID_ARG, "rays.flags has unknown bits");
  for (int c = 0; c < 3; ++c)
    if (!finite(r->bg[c])) return fail(MVP_ERR_INVALID_ARG, "rays.bg must be finite");
  int64_t ns = mvp_num_steps(r->t_near, r->t_far, r->dt);
  if (ns > MVP_MAX_STEPS) return fail(MVP_ERR_INVALID_ARG, "n_steps = %lld exceeds %d", (long long)ns, MVP_MAX_STEPS);
  *n_steps = ns;
  return ok();
}

mvp_status check_bvh(const mvp_bvh *bvh, const mvp_prims *p) {
  if (!bvh) return fail(MVP_ERR_INVALID_ARG, "bvh is NULL");
  if (bvh->b.n != p->n || (p->n > 0 && bvh->b.M != p->M))
    return fail(MVP_ERR_INVALID_ARG, "bvh was built for n=%d M=%d, prims have n=%d M=%d", bvh->b.n, bvh->b.M, p->n,
                p->M);
  return ok();
}

// Tile schedule of one kernel launch (the caller holds S.mu): sched_begin decides
// whether this call may use the buffers (the last call that touched them has
// finished or ran on this stream), grows them if needed, points the launch at them
// and makes the stream wait for the last schedule kernel; sched_end queues the
// schedule kernel for the next call on the side stream. The plain tile order is the
// fallback whenever something is unavailable.
bool sched_begin(TileSched &S, mvp::MarchArgs &a, cudaStream_t st, cudaError_t &e) {
  e = cudaSuccess;
  const int64_t nt = a.geom.n_warp_tiles;
  bool use = S.enabled && nt <= 0x7fffffff;
  if (use && S.pending && S.stream != st) {
    const cudaError_t q = cudaEventQuery(S.done);
    if (q == cudaErrorNotReady) cudaGetLastError();  // not an error: the last scheduled call still runs
    use = q == cudaSuccess;
  }
  if (use && nt > S.cap) {  // grow (cudaFree waits for work that may still use the old buffers)
    if (S.cost) cudaFree(S.cost);
    if (S.order) cudaFree(S.order);
    S.cost = nullptr;
    S.order = nullptr;
    S.cap = 0;
    S.tiles = -1;
    if (cudaMalloc(&S.cost, (size_t)nt * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&S.order, (size_t)nt * sizeof(int)) != cudaSuccess ||
        cudaMemset(S.cost, 0, (size_t)nt * sizeof(unsigned int)) != cudaSuccess ||
        (!S.done && cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess) ||
        (!S.marched && cudaEventCreateWithFlags(&S.marched, cudaEventDisableTiming) != cudaSuccess) ||
        (!S.side && cudaStreamCreateWithFlags(&S.side, cudaStreamNonBlocking) != cudaSuccess)) {
      cudaGetLastError();
      if (S.cost) cudaFree(S.cost);
      if (S.order) cudaFree(S.order);
      S.cost = nullptr;
      S.order = nullptr;
      use = false;
    } else {
      S.cap = nt;
    }
  }
  if (use) {
    a.order = S.tiles == nt ? S.order : nullptr;
    a.cost = S.cost;
    if (S.pending) e = cudaStreamWaitEvent(st, S.done, 0);  // the last schedule kernel is done with them
  }
  return use;
}

cudaError_t sched_end(TileSched &S, int64_t nt, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(S.marched, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(S.side, S.marched, 0);
  if (e == cudaSuccess) e = mvp::launch_tile_order(S.cost, nt, S.order, S.side);
  if (e == cudaSuccess) e = cudaEventRecord(S.done, S.side);
  if (e == cudaSuccess) {
    S.tiles = nt;
    S.stream = st;
    S.pending = true;
  }
  return e;
}

void sched_free(TileSched &S) {
  if (S.cost) cudaFree(S.cost);
  if (S.order) cudaFree(S.order);
  if (S.done) cudaEventDestroy(S.done);
  if (S.marched) cudaEventDestroy(S.marched);
  if (S.side) cudaStreamDestroy(S.side);
}

mvp::MarchArgs march_args(mvp_ctx *ctx, const mvp_prims *p, const mvp_bvh *bvh, const mvp_rays *r, int64_t ns) {
  mvp::MarchArgs a;
  memset(&a, 0, sizeof(a));
  a.n_prims = p->n;
  a.M = p->M;
  a.dtype = p->dtype;
  a.payload = p->payload;
  a.nodes = bvh->b.nodes;
  a.pose = bvh->b.pose;
  a.xf = bvh->b.xf;
  a.rank = bvh->b.rank;
  a.sequential = (r->flags & MVP_BLEND_SEQUENTIAL) ? 1 : 0;
  a.literal = (r->flags & MVP_COMPOSITE_LITERAL) ? 1 : 0;
  a.geom = mvp::make_tile_geom(r->n, r->width, r->height);
  a.o = r->o;
  a.d = r->d;
  a.t_near = r->t_near;
  a.t_far = r->t_far;
  a.dt = r->dt;
  a.stop_T = (float)(1.0 - (double)r->eps_early);
  a.bg[0] = r->bg[0];
  a.bg[1] = r->bg[1];
  a.bg[2] = r->bg[2];
  a.n_steps = (int)ns;
  a.status = ctx->d_status;
  return a;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    (void)cudaGetLastError();  // a pending error of other code is not this call's
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace mvp {
// Lets other translation units of the library set the message mvp_last_error() returns.
void record_error(const char *msg) { g_err = msg; }

unsigned long long current_context_id() {
  // cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
  // library links no driver library of its own); looked up once per process
  using GetCurrent = int (*)(void **);  // CUresult is an int-sized enum; 0 = success
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return 0;
  void *c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
  return id;
}

cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void *, unsigned long long>, size_t>> done;
  const unsigned long long ctx = current_context_id();
  if (ctx != 0) {
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
      if (d.first.first == kernel && d.first.second == ctx && d.second >= bytes) return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  const unsigned long long now = ctx ? ctx : current_context_id();  // the set-up may have created it
  if (now != 0) {
    std::lock_guard<std::mutex> lk(mu);
    done.push_back({{kernel, now}, bytes});
  }
  return cudaSuccess;
}
int ctx_device(const mvp_ctx *ctx) { return ctx->device; }
}  // namespace mvp

extern "C" {

const char *mvp_version(void) { return "mvp-gb300 1.0 (abi 1, sm_103a)"; }

const char *mvp_status_string(int s) {
  switch (s) {
    case MVP_OK: return "MVP_OK";
    case MVP_NOT_READY: return "MVP_NOT_READY";
    case MVP_ERR_INVALID_ARG: return "MVP_ERR_INVALID_ARG";
    case MVP_ERR_CUDA: return "MVP_ERR_CUDA";
    case MVP_ERR_OOM: return "MVP_ERR_OOM";
    case MVP_ERR_CAPACITY: return "MVP_ERR_CAPACITY";
    case MVP_ERR_TIMEOUT: return "MVP_ERR_TIMEOUT";
    case MVP_ERR_DEVICE: return "MVP_ERR_DEVICE";
  }
  return "MVP_UNKNOWN_STATUS";
}

const char *mvp_last_error(void) { return g_err.c_str(); }

int64_t mvp_num_steps(float t_near, float t_far, float dt) {
  if (!(dt > 0.0f) || !(t_far > t_near)) return 0;
  double x = ((double)t_far - (double)t_near) / (double)dt;
  double c = ceil(x - 1e-4);
  return c > 0 ? (int64_t)c : 0;
}

mvp_status mvp_ctx_create(int device, mvp_ctx **out) {
  if (!out) return fail(MVP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(MVP_ERR_INVALID_ARG, "device %d of %d", device, count);
  DeviceGuard g(device);
  mvp_ctx *c = new (std::nothrow) mvp_ctx();
  if (!c) return fail(MVP_ERR_OOM, "host allocation");
  c->device = device;
  e = cudaMalloc(&c->d_status, sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(status)");
  }
  e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(c->d_status);
    delete c;
    return cuda_fail(e, "cudaMemset(status)");
  }
  *out = c;
  return ok();
}

void mvp_ctx_destroy(mvp_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaFree(ctx->d_status);
  sched_free(ctx->sched);
  sched_free(ctx->sched_bwd);
  delete ctx;
}

mvp_status mvp_ctx_set_bwd_group_bytes(mvp_ctx *ctx, int64_t bytes) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  ctx->bwd_group_bytes.store(bytes);
  return ok();
}

mvp_status mvp_ctx_set_tile_schedule(mvp_ctx *ctx, int32_t enable) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  for (TileSched *S : {&ctx->sched, &ctx->sched_bwd}) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->enabled = enable != 0;
    S->tiles = -1;  // start from the plain order
  }
  return ok();
}

int32_t mvp_bounds_checked(void) {
#ifdef MVP_CHECK_BOUNDS
  return 1;
#else
  return 0;
#endif
}

mvp_status mvp_ctx_sync(mvp_ctx *ctx, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  if (st) {
    cudaMemset(ctx->d_status, 0, sizeof(int));
    if (st & mvp::STATUS_CAPACITY)
      return fail(MVP_ERR_CAPACITY, "a kernel exceeded a capacity limit (a tile's BVH traversal stack of %d "
                                    "entries overflowed)",
                  mvp::STACK);
    if (st & mvp::STATUS_BOUNDS)
      return fail(MVP_ERR_DEVICE, "an index fell outside its array (checked build; the access was skipped)");
    if (st & mvp::STATUS_POSE)
      return fail(MVP_ERR_INVALID_ARG, "a primitive's pose defines no box (t, q or s not finite, q = 0 or s <= 0)");
    return fail(MVP_ERR_DEVICE, "device status word 0x%x", st);
  }
  return ok();
}

mvp_status mvp_bvh_create(mvp_ctx *ctx, mvp_bvh **out) {
  if (!ctx || !out) return fail(MVP_ERR_INVALID_ARG, "NULL argument");
  mvp_bvh *b = new (std::nothrow) mvp_bvh();
  if (!b) return fail(MVP_ERR_OOM, "host allocation");
  b->device = ctx->device;
  *out = b;
  return ok();
}

void mvp_bvh_destroy(mvp_bvh *bvh) {
  if (!bvh) return;
  DeviceGuard g(bvh->device);
  mvp::bvh_release(bvh->b);
  delete bvh;
}

int32_t mvp_bvh_size(const mvp_bvh *bvh) { return bvh ? bvh->b.n : -1; }

mvp_status mvp_build_bvh(mvp_ctx *ctx, const mvp_prims *prims, mvp_bvh *bvh, mvp_stream stream) {
  if (!ctx || !bvh) return fail(MVP_ERR_INVALID_ARG, "NULL argument");
  mvp_status s = check_prims(prims);
  if (s) return s;
  DeviceGuard g(ctx->device);
  if (prims->n > bvh->b.cap) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sync before BVH growth");
    e = mvp::bvh_reserve(bvh->b, prims->n);
    if (e != cudaSuccess) return cuda_fail(e, "BVH allocation");
  }
  cudaError_t e = mvp::bvh_build(bvh->b, prims->t, prims->q, prims->s, prims->n, prims->M, (cudaStream_t)stream,
                                 ctx->d_status);
  if (e != cudaSuccess) return cuda_fail(e, "BVH build launch");
  return ok();
}

mvp_status mvp_bvh_export(mvp_ctx *ctx, const mvp_bvh *bvh, uint64_t *keys, int32_t *children, float *bounds,
                          float *scene, mvp_stream stream) {
  if (!ctx || !bvh) return fail(MVP_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::bvh_export(bvh->b, keys, children, bounds, scene, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "BVH export");
  return ok();
}

size_t mvp_saved_bytes(int64_t n_rays) { return n_rays > 0 ? (size_t)n_rays * sizeof(mvp::Saved) : 0; }

mvp_status mvp_raymarch_fwd(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh, const mvp_rays *rays,
                            float *out_rgba, void *saved, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  int64_t ns = 0;
  mvp_status s;
  if ((s = check_prims(prims)) || (s = check_rays(rays, &ns)) || (s = check_bvh(bvh, prims))) return s;
  if (rays->n > 0 && !out_rgba) return fail(MVP_ERR_INVALID_ARG, "out_rgba is NULL");
  if (reinterpret_cast<uintptr_t>(out_rgba) % 16) return fail(MVP_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(saved) % 8) return fail(MVP_ERR_INVALID_ARG, "saved must be 8-byte aligned");
  if (rays->n == 0) return ok();
  DeviceGuard g(ctx->device);
  mvp::MarchArgs a = march_args(ctx, prims, bvh, rays, ns);
  a.out = out_rgba;
  a.saved = reinterpret_cast<mvp::Saved *>(saved);
  TileSched &S = ctx->sched;
  std::lock_guard<std::mutex> lk(S.mu);
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  const bool use = sched_begin(S, a, st, e);
  if (e != cudaSuccess) return cuda_fail(e, "tile schedule wait");
  e = mvp::launch_march(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "march launch");
  if (use && (e = sched_end(S, a.geom.n_warp_tiles, st)) != cudaSuccess) return cuda_fail(e, "tile schedule");
  return ok();
}

mvp_status mvp_raymarch_count(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh, const mvp_rays *rays,
                              int32_t *n_eval, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  int64_t ns = 0;
  mvp_status s;
  if ((s = check_prims(prims)) || (s = check_rays(rays, &ns)) || (s = check_bvh(bvh, prims))) return s;
  if (rays->n > 0 && !n_eval) return fail(MVP_ERR_INVALID_ARG, "n_eval is NULL");
  if (rays->n == 0) return ok();
  DeviceGuard g(ctx->device);
  mvp::MarchArgs a = march_args(ctx, prims, bvh, rays, ns);
  a.n_eval = n_eval;
  cudaError_t e = mvp::launch_march(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "count launch");
  return ok();
}

mvp_status mvp_raymarch_bwd(mvp_ctx *ctx, const mvp_prims *prims, mvp_bvh *bvh, const mvp_rays *rays,
                            const void *saved, const float *grad_rgba, float *g_payload, float *g_t, float *g_q,
                            float *g_s, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  int64_t ns = 0;
  mvp_status s;
  if ((s = check_prims(prims)) || (s = check_rays(rays, &ns)) || (s = check_bvh(bvh, prims))) return s;
  bool pose = g_t || g_q || g_s;
  if (pose && !(g_t && g_q && g_s)) return fail(MVP_ERR_INVALID_ARG, "g_t, g_q and g_s go together");
  if (rays->n > 0 && (!saved || !grad_rgba)) return fail(MVP_ERR_INVALID_ARG, "saved and grad_rgba are required");
  if (rays->flags & MVP_COMPOSITE_LITERAL)
    return fail(MVP_ERR_INVALID_ARG, "the adjoint supports the premultiplied composite only");
  if (reinterpret_cast<uintptr_t>(g_payload) % 16 || reinterpret_cast<uintptr_t>(grad_rgba) % 16 ||
      reinterpret_cast<uintptr_t>(saved) % 8)
    return fail(MVP_ERR_INVALID_ARG, "g_payload and grad_rgba must be 16-byte aligned, saved 8-byte aligned");
  if (rays->n == 0 || prims->n == 0) return ok();
  DeviceGuard g(ctx->device);
  mvp::BwdArgs b;
  b.m = march_args(ctx, prims, bvh, rays, ns);
  b.saved = reinterpret_cast<const mvp::Saved *>(saved);
  b.grad = grad_rgba;
  b.g_payload = g_payload;
  b.gmc = pose ? bvh->b.gmc : nullptr;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // Group the primitives when the payload and its gradient exceed twice the group budget.
  const int64_t vox = (int64_t)prims->M * prims->M * prims->M;
  const int64_t per_prim = vox * (prims->dtype == MVP_F32 ? 16 : 8) + (g_payload ? vox * 16 : 0);
  int64_t budget = ctx->bwd_group_bytes.load();
  if (budget == 0) {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess) cudaGetLastError();
    budget = l2 > 0 ? l2 / 3 : 0;
  }
  const int n = prims->n;
  mvp::BwdGroups gr;
  char *scratch = nullptr;
  const int64_t nt = b.m.geom.n_warp_tiles;
  if (budget > 0 && n > 1 && per_prim * n > 2 * budget && nt <= 0x7fffffff / 64) {
    gr.gsize = (int)std::max<int64_t>(1, std::min<int64_t>(n, budget / per_prim));
    if ((n + gr.gsize - 1) / gr.gsize > 64) gr.gsize = (n + 63) / 64;
    gr.n_groups = (n + gr.gsize - 1) / gr.gsize;
    gr.range = reinterpret_cast<const int2 *>(bvh->b.parent);
    // stream-ordered scratch: mask, work list, group offsets, work counter
    const size_t bytes = (size_t)nt * 8 + (size_t)nt * gr.n_groups * 4 + (size_t)(gr.n_groups + 2) * 4;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
      cudaGetLastError();  // no room for the work list: replay in one pass below (same gradients)
      scratch = nullptr;
    }
  }
  if (scratch) {
    gr.mask = reinterpret_cast<unsigned long long *>(scratch);
    gr.items = reinterpret_cast<int *>(scratch + (size_t)nt * 8);
    gr.goff = gr.items + (size_t)nt * gr.n_groups;
    gr.work = gr.goff + gr.n_groups + 1;
    e = mvp::launch_backward(b, prims->t, prims->q, prims->s, g_t, g_q, g_s, st, &gr);
    const cudaError_t f = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped backward launch");
    if (f != cudaSuccess) return cuda_fail(f, "adjoint group scratch");
    return ok();
  }
  TileSched &S = ctx->sched_bwd;
  std::lock_guard<std::mutex> lk(S.mu);
  const bool use = sched_begin(S, b.m, st, e);
  if (e != cudaSuccess) return cuda_fail(e, "tile schedule wait");
  e = mvp::launch_backward(b, prims->t, prims->q, prims->s, g_t, g_q, g_s, st);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  if (use && (e = sched_end(S, b.m.geom.n_warp_tiles, st)) != cudaSuccess) return cuda_fail(e, "tile schedule");
  return ok();
}

mvp_status mvp_hitlists(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh, const mvp_rays *rays,
                        int64_t *offs, int32_t *ids, float *tin, float *tout, int64_t cap, int64_t *n_hits,
                        mvp_stream stream) {
  if (!ctx || !n_hits) return fail(MVP_ERR_INVALID_ARG, "NULL argument");
  int64_t ns = 0;
  mvp_status s;
  if ((s = check_prims(prims)) || (s = check_rays(rays, &ns)) || (s = check_bvh(bvh, prims))) return s;
  if (!offs) return fail(MVP_ERR_INVALID_ARG, "offs is NULL");
  if (cap > 0 && (!ids || !tin || !tout)) return fail(MVP_ERR_INVALID_ARG, "ids/tin/tout are NULL");
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  mvp::HitArgs a;
  memset(&a, 0, sizeof(a));
  a.n_prims = prims->n;
  a.nodes = bvh->b.nodes;
  a.pose = bvh->b.pose;
  a.geom = mvp::make_tile_geom(rays->n, rays->width, rays->height);
  a.o = rays->o;
  a.d = rays->d;
  a.t_near = rays->t_near;
  a.t_far = rays->t_far;
  a.offs = offs;
  a.ids = ids;
  a.tin = tin;
  a.tout = tout;
  a.cap = cap;
  a.status = ctx->d_status;
  int64_t *counts = nullptr;
  cudaError_t e = cudaMallocAsync(&counts, sizeof(int64_t) * (size_t)(rays->n > 0 ? rays->n : 1), st);
  if (e != cudaSuccess) return cuda_fail(e, "hit-list scratch");
  cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)(rays->n > 0 ? rays->n : 1), st);
  e = mvp::launch_hits(a, counts, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n_hits, offs + rays->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFreeAsync(counts, st);
    return cuda_fail(e, "hit-list count");
  }
  if (cap > 0) {
    e = mvp::launch_hits_fill(a, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(counts, st);
  if (e != cudaSuccess) return cuda_fail(e, "hit-list fill");
  if ((s = mvp_ctx_sync(ctx, stream))) return s;
  if (*n_hits > cap) return fail(MVP_ERR_CAPACITY, "%lld hits exceed cap %lld", (long long)*n_hits, (long long)cap);
  return ok();
}

mvp_status mvp_pack_payload(mvp_ctx *ctx, const float *src, void *dst, int64_t n_values, int32_t dtype,
                            mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n_values < 0) return fail(MVP_ERR_INVALID_ARG, "n_values < 0");
  if (dtype != MVP_F32 && dtype != MVP_BF16 && dtype != MVP_F16) return fail(MVP_ERR_INVALID_ARG, "dtype unknown");
  if (n_values > 0 && (!src || !dst)) return fail(MVP_ERR_INVALID_ARG, "NULL buffer");
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_pack(src, dst, n_values, dtype, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pack launch");
  return ok();
}

mvp_status mvp_camera_rays(mvp_ctx *ctx, const float *c2w, float focal, int32_t width, int32_t height, float *o,
                           float *d, mvp_stream stream) {
  if (!ctx || !c2w) return fail(MVP_ERR_INVALID_ARG, "NULL argument");
  if (width < 0 || height < 0 || !(focal > 0.0f) || !finite(focal))
    return fail(MVP_ERR_INVALID_ARG, "bad camera size or focal");
  if ((int64_t)width * height > 0 && (!o || !d)) return fail(MVP_ERR_INVALID_ARG, "NULL ray buffer");
  mvp::Cam c;
  for (int i = 0; i < 12; ++i) {
    if (!finite(c2w[i])) return fail(MVP_ERR_INVALID_ARG, "c2w must be finite");
    c.m[i] = c2w[i];
  }
  c.focal = focal;
  c.width = width;
  c.height = height;
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_camera(c, o, d, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "camera launch");
  return ok();
}

// ---------------------------------------------------------------- decode-side epilogues
mvp_status mvp_fade_payload(mvp_ctx *ctx, const float *src, void *dst, int64_t n_prims, int32_t M, int32_t dtype,
                            float alpha, int32_t beta, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n_prims < 0 || n_prims > MVP_MAX_PRIMS) return fail(MVP_ERR_INVALID_ARG, "n_prims out of range");
  if (M < 2 || M > MVP_MAX_M) return fail(MVP_ERR_INVALID_ARG, "M out of [2, %d]", MVP_MAX_M);
  if (dtype != MVP_F32 && dtype != MVP_BF16 && dtype != MVP_F16) return fail(MVP_ERR_INVALID_ARG, "dtype unknown");
  if (!finite(alpha) || beta < 0 || beta > 64) return fail(MVP_ERR_INVALID_ARG, "alpha not finite or beta out of [0, 64]");
  if (n_prims > 0 && (!src || !dst)) return fail(MVP_ERR_INVALID_ARG, "NULL buffer");
  const size_t nv = (size_t)n_prims * M * M * M;
  if (reinterpret_cast<uintptr_t>(src) % 16 || reinterpret_cast<uintptr_t>(dst) % (dtype == MVP_F32 ? 16 : 8))
    return fail(MVP_ERR_INVALID_ARG, "misaligned buffer");
  if (dtype != MVP_F32 && n_prims > 0) {
    const char *a = reinterpret_cast<const char *>(src), *b = reinterpret_cast<const char *>(dst);
    if (a < b + nv * 8 && b < a + nv * 16) return fail(MVP_ERR_INVALID_ARG, "src and dst overlap (only FP32 may be in place)");
  }
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_fade(src, dst, n_prims, M, dtype, alpha, beta, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "fade launch");
  return ok();
}

mvp_status mvp_assemble_payload(mvp_ctx *ctx, const float *rgb, const float *opacity, void *dst, int64_t n_prims,
                                int32_t M, int32_t dtype, float alpha, int32_t beta, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n_prims < 0 || n_prims > MVP_MAX_PRIMS) return fail(MVP_ERR_INVALID_ARG, "n_prims out of range");
  if (M < 2 || M > MVP_MAX_M) return fail(MVP_ERR_INVALID_ARG, "M out of [2, %d]", MVP_MAX_M);
  if (dtype != MVP_F32 && dtype != MVP_BF16 && dtype != MVP_F16) return fail(MVP_ERR_INVALID_ARG, "dtype unknown");
  if (!finite(alpha) || beta < 0 || beta > 64) return fail(MVP_ERR_INVALID_ARG, "alpha not finite or beta out of [0, 64]");
  if (n_prims > 0 && (!rgb || !opacity || !dst)) return fail(MVP_ERR_INVALID_ARG, "NULL buffer");
  if (reinterpret_cast<uintptr_t>(rgb) % 4 || reinterpret_cast<uintptr_t>(opacity) % 4 ||
      reinterpret_cast<uintptr_t>(dst) % (dtype == MVP_F32 ? 16 : 8))
    return fail(MVP_ERR_INVALID_ARG, "misaligned buffer");
  if (n_prims > 0) {
    const size_t nv = (size_t)n_prims * M * M * M;
    const char *o = reinterpret_cast<const char *>(dst);
    const size_t ob = nv * (dtype == MVP_F32 ? 16 : 8);
    const char *c = reinterpret_cast<const char *>(rgb), *a = reinterpret_cast<const char *>(opacity);
    if ((c < o + ob && o < c + nv * 12) || (a < o + ob && o < a + nv * 4))
      return fail(MVP_ERR_INVALID_ARG, "dst overlaps an input");
  }
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_assemble(rgb, opacity, dst, n_prims, M, dtype, alpha, beta, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "assemble launch");
  return ok();
}

mvp_status mvp_axis_angle_to_quat(mvp_ctx *ctx, const float *r, int32_t n, float *q, mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0) return fail(MVP_ERR_INVALID_ARG, "n < 0");
  if (n > 0 && (!r || !q)) return fail(MVP_ERR_INVALID_ARG, "NULL buffer");
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_aa_to_quat(r, n, q, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "axis-angle launch");
  return ok();
}

mvp_status mvp_axis_angle_backward(mvp_ctx *ctx, const float *r, const float *g_q, int32_t n, float *g_r,
                                   mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0) return fail(MVP_ERR_INVALID_ARG, "n < 0");
  if (n > 0 && (!r || !g_q || !g_r)) return fail(MVP_ERR_INVALID_ARG, "NULL buffer");
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_aa_vjp(r, g_q, n, g_r, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "axis-angle gradient launch");
  return ok();
}

mvp_status mvp_volume_prior(mvp_ctx *ctx, const float *s, int32_t n, float lambda, float *loss, float *g_s,
                            mvp_stream stream) {
  if (!ctx) return fail(MVP_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0) return fail(MVP_ERR_INVALID_ARG, "n < 0");
  if (!finite(lambda)) return fail(MVP_ERR_INVALID_ARG, "lambda not finite");
  if (n > 0 && !s) return fail(MVP_ERR_INVALID_ARG, "s is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = mvp::launch_volume_prior(s, n, lambda, loss, g_s, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "volume prior launch");
  return ok();
}

}  // extern "C"
