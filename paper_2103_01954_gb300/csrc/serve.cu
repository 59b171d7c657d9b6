// serve.cu -- continuous batching of render requests (different avatars, cameras
// and resolutions), each batch in one persistent kernel launch.
//
// Device side. A batch is a list of admitted requests; each request is cut into
// warp tiles of 8x4 pixels numbered consecutively across the batch. The batch's
// grid (one CTA set per SM) has every warp claim tile numbers from the batch's own
// counter, find the owning request (its descriptor is copied once into shared
// memory), generate the tile's pinhole rays and march it with the same code as
// mvp_raymarch_fwd (march_tile). A warp past the batch's last tile returns: nothing
// on the device ever waits. The warp that finishes a request's last tile publishes
// its completion to mapped host memory (system-scope release), so a small request
// completes without waiting for the rest of its batch.
//
// Host side. Admission: a request needs a free slot and its image (W*H*16 bytes)
// must fit the HBM budget (resident avatars + images in flight) and the server's
// image arena; otherwise it waits in a FIFO and is admitted by a later submit or
// poll as slots and memory free up. Admitted requests are launched as a batch on
// one of several streams as soon as one is idle; requests that arrive while batches
// run form the next batch on another stream, whose blocks start as SMs free up, so
// requests overlap on the device. A request larger than the budget is refused
// (MVP_ERR_CAPACITY).
#include <math.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "camera.cuh"
#include "march_tile.cuh"

namespace mvp {

constexpr int SERVE_CAP = MARCH_CAP;
constexpr int SERVE_STREAMS = 4;  // batches that may run at once

// One request of a batch (device memory, copied in before the batch's launch).
struct BatchReq {
  unsigned long long seq;  // request sequence number
  int slot;                // completion record index
  int tile_begin;          // first tile of the request within the batch
  int n_tiles;
  int n_prims, M, dtype, n_steps, width, height;
  const void *payload;
  const Node *nodes;
  const Pose *pose;
  const Xform *xf;
  float *out;
  float c2w[12];
  float focal, t_near, t_far, dt, stop_T;
  float bg[3];
  int pad;
};

// Completion record of a slot (mapped host memory): written by the device.
struct ReqDone {
  unsigned long long seq_done;  // 1 + sequence number of the request completed in this slot (0: none)
  unsigned long long t_start_ns, t_end_ns;
  unsigned long long pad;
};

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

struct BatchArgs {
  const BatchReq *reqs;     // device, n_req entries
  int n_req;
  int total_tiles;
  unsigned int *claimed;    // device, zeroed before the launch
  unsigned int *tiles_done; // device, n_req entries, zeroed before the launch
  ReqDone *done;            // mapped host memory, indexed by slot
  int *status;
};

template <int DT>
__device__ __noinline__ void serve_tile(TileShared<SERVE_CAP> &sh, const MarchArgs &a, const LaneRay &L) {
  march_tile<DT, SERVE_CAP, false, 0>(sh, a, L);
}

__global__ void __launch_bounds__(TILE_WARPS * 32, 4) k_serve(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<SERVE_CAP> &sh = reinterpret_cast<TileShared<SERVE_CAP> *>(smem_raw)[warp];
  BatchReq &D = reinterpret_cast<BatchReq *>(smem_raw + sizeof(TileShared<SERVE_CAP>) * TILE_WARPS)[warp];
  int cur = -1, c_begin = 0, c_n = 0;
  while (true) {
    unsigned int tl = 0;
    if (lane == 0) tl = atomicAdd(A.claimed, 1u);
    const int t = (int)__shfl_sync(FULL, tl, 0);
    if (t >= A.total_tiles) return;
    if (cur < 0 || t < c_begin || t >= c_begin + c_n) {
      // owning request: the last one whose first tile is <= t (requests are in tile order)
      int lo = 0, hi = A.n_req - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&A.reqs[mid].tile_begin) <= t) lo = mid; else hi = mid - 1;
      }
      cur = lo;
      constexpr int W = (int)(sizeof(BatchReq) / 4);
      static_assert(sizeof(BatchReq) % 4 == 0 && W <= 64, "descriptor copy");
      const unsigned int *src = reinterpret_cast<const unsigned int *>(&A.reqs[cur]);
      unsigned int *dst = reinterpret_cast<unsigned int *>(&D);
      __syncwarp();
      for (int w = lane; w < W; w += 32) dst[w] = __ldg(src + w);
      __syncwarp();
      c_begin = D.tile_begin;
      c_n = D.n_tiles;
    }
    if (lane == 0 && t == c_begin) A.done[D.slot].t_start_ns = globaltimer();
    MarchArgs a;
    a.n_prims = D.n_prims;
    a.M = D.M;
    a.dtype = D.dtype;
    a.payload = D.payload;
    a.nodes = D.nodes;
    a.pose = D.pose;
    a.xf = D.xf;
    const int width = D.width, height = D.height;
    a.geom.n_rays = (int64_t)width * height;
    a.geom.width = width;
    a.geom.height = height;
    a.geom.n_warp_tiles = D.n_tiles;
    a.o = a.d = nullptr;
    a.t_near = D.t_near;
    a.t_far = D.t_far;
    a.dt = D.dt;
    a.stop_T = D.stop_T;
    a.bg[0] = D.bg[0];
    a.bg[1] = D.bg[1];
    a.bg[2] = D.bg[2];
    a.n_steps = D.n_steps;
    a.out = D.out;
    a.saved = nullptr;
    a.n_eval = nullptr;
    a.status = A.status;
    LaneRay L;
    const int64_t r = tile_ray(a.geom, (int64_t)(t - c_begin), lane);
    L.r = r;
    if (r >= 0) {
      const int row = (int)(r / width), col = (int)(r - (int64_t)row * width);
      camera_ray(D.c2w, D.focal, width, height, row, col, L.o, L.d);
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) L.o[j] = L.d[j] = 0.0f;
    }
    if (__ballot_sync(FULL, r >= 0) != 0) {
      switch (a.dtype) {
        case MVP_F32: serve_tile<MVP_F32>(sh, a, L); break;
        case MVP_BF16: serve_tile<MVP_BF16>(sh, a, L); break;
        default: serve_tile<MVP_F16>(sh, a, L); break;
      }
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();  // this tile's pixels are visible before it is counted
      const unsigned int fin = atomicAdd(&A.tiles_done[cur], 1u);
      if (fin + 1 == (unsigned int)c_n) {
        __threadfence();
        A.done[D.slot].t_end_ns = globaltimer();
        __threadfence_system();
        st_release_sys(&A.done[D.slot].seq_done, D.seq + 1);
      }
    }
    __syncwarp();
  }
}

}  // namespace mvp

// ============================================================================ host
namespace {

using clock_type = std::chrono::steady_clock;

struct Avatar {
  mvp_prims prims;
  mvp::BvhBuffers bvh;
  size_t bytes = 0;
};

struct Pending {
  uint64_t ticket;
  mvp_request req;
  clock_type::time_point submit;
};

struct InFlight {
  uint64_t seq = 0;
  int slot = -1;
  size_t off = 0, bytes = 0;
  mvp_request req;
  clock_type::time_point submit;
  bool launched = false;
};

// First-fit allocator over the image arena (host bookkeeping only).
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t n) {
    size = n;
    free_.clear();
    if (n) free_[0] = n;
  }
  bool alloc(size_t n, size_t &off) {
    n = (n + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        off = it->first;
        size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~size_t(255);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Per-stream batch buffers: the batch table is staged in pinned memory and copied to
// the device on the stream before the launch; the stream is reused only after its
// previous batch (and that copy) finished.
struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  mvp::BatchReq *h_reqs = nullptr;  // pinned staging
  mvp::BatchReq *d_reqs = nullptr;
  unsigned int *d_counters = nullptr;  // [0] claimed, [1..] tiles done per request
};

}  // namespace

struct mvp_server {
  int device = 0;
  size_t budget = 0;
  int slots = 0;
  std::mutex mu;
  std::vector<Avatar> avatars;
  size_t resident = 0;
  size_t inflight_bytes = 0;
  Arena arena;
  char *arena_base = nullptr;
  mvp::ReqDone *h_done = nullptr, *d_done = nullptr;  // mapped
  int *d_status = nullptr;
  Lane lanes[mvp::SERVE_STREAMS];
  cudaStream_t copy = nullptr;
  int grid = 0;
  size_t smem = 0;
  uint64_t next_seq = 0, next_ticket = 1;
  std::vector<bool> slot_busy;
  std::deque<Pending> pending;
  std::map<uint64_t, InFlight> inflight;  // ticket -> request (admitted)
  size_t max_inflight_seen = 0;
  uint64_t completed = 0, batches = 0;
};

namespace {

mvp_status serve_fail(mvp_status s, const char *msg) {
  mvp::record_error(msg);
  return s;
}

size_t image_bytes(const mvp_request &r) { return (size_t)r.width * (size_t)r.height * 4 * sizeof(float); }

int warp_tiles(int w, int h) { return ((w + 15) / 16) * ((h + 7) / 8) * 4; }

// Admit pending requests in FIFO order while a slot, budget and arena space allow,
// then launch the admitted, not yet launched requests as one batch on an idle
// stream. Called with S->mu held.
mvp_status pump(mvp_server *S) {
  while (!S->pending.empty()) {
    Pending &p = S->pending.front();
    const size_t bytes = image_bytes(p.req);
    int slot = -1;
    for (int i = 0; i < S->slots; ++i)
      if (!S->slot_busy[i]) {
        slot = i;
        break;
      }
    if (slot < 0) break;
    if (S->resident + S->inflight_bytes + bytes > S->budget) break;
    size_t off = 0;
    if (!S->arena.alloc(bytes, off)) break;
    InFlight f;
    f.seq = S->next_seq++;
    f.slot = slot;
    f.off = off;
    f.bytes = bytes;
    f.req = p.req;
    f.submit = p.submit;
    __atomic_store_n(&S->h_done[slot].seq_done, 0ull, __ATOMIC_RELEASE);
    S->slot_busy[slot] = true;
    S->inflight[p.ticket] = f;
    S->inflight_bytes += bytes;
    if (S->inflight.size() > S->max_inflight_seen) S->max_inflight_seen = S->inflight.size();
    S->pending.pop_front();
  }
  // anything admitted but not launched?
  bool any = false;
  for (auto &kv : S->inflight)
    if (!kv.second.launched) {
      any = true;
      break;
    }
  if (!any) return MVP_OK;
  // an idle stream (its previous batch finished)
  Lane *L = nullptr;
  for (int i = 0; i < mvp::SERVE_STREAMS; ++i) {
    Lane &c = S->lanes[i];
    if (c.busy && cudaEventQuery(c.done) == cudaSuccess) c.busy = false;
    if (!c.busy && !L) L = &c;
  }
  if (!L) return MVP_OK;  // launched when a stream frees up (next submit or poll)
  int n = 0, tiles = 0;
  for (auto &kv : S->inflight) {
    InFlight &f = kv.second;
    if (f.launched) continue;
    const mvp_request &q = f.req;
    const Avatar &A = S->avatars[q.avatar];
    mvp::BatchReq &B = L->h_reqs[n++];
    memset(&B, 0, sizeof(B));
    B.seq = f.seq;
    B.slot = f.slot;
    B.tile_begin = tiles;
    B.n_tiles = warp_tiles(q.width, q.height);
    B.n_prims = A.prims.n;
    B.M = A.prims.M;
    B.dtype = A.prims.dtype;
    B.n_steps = (int)mvp_num_steps(q.t_near, q.t_far, q.dt);
    B.width = q.width;
    B.height = q.height;
    B.payload = A.prims.payload;
    B.nodes = A.bvh.nodes;
    B.pose = A.bvh.pose;
    B.xf = A.bvh.xf;
    B.out = reinterpret_cast<float *>(S->arena_base + f.off);
    memcpy(B.c2w, q.c2w, sizeof(B.c2w));
    B.focal = q.focal;
    B.t_near = q.t_near;
    B.t_far = q.t_far;
    B.dt = q.dt;
    B.stop_T = (float)(1.0 - (double)q.eps_early);
    memcpy(B.bg, q.bg, sizeof(B.bg));
    tiles += B.n_tiles;
    f.launched = true;
  }
  cudaError_t e = cudaMemcpyAsync(L->d_reqs, L->h_reqs, sizeof(mvp::BatchReq) * n, cudaMemcpyHostToDevice, L->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L->d_counters, 0, sizeof(unsigned int) * (n + 1), L->stream);
  if (e != cudaSuccess) return serve_fail(MVP_ERR_CUDA, cudaGetErrorString(e));
  mvp::BatchArgs a;
  a.reqs = L->d_reqs;
  a.n_req = n;
  a.total_tiles = tiles;
  a.claimed = L->d_counters;
  a.tiles_done = L->d_counters + 1;
  a.done = S->d_done;
  a.status = S->d_status;
  int grid = S->grid;
  const int need = (tiles + mvp::TILE_WARPS - 1) / mvp::TILE_WARPS;
  if (need < grid) grid = need;
  mvp::k_serve<<<grid, mvp::TILE_WARPS * 32, S->smem, L->stream>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(L->done, L->stream);
  if (e != cudaSuccess) return serve_fail(MVP_ERR_CUDA, cudaGetErrorString(e));
  L->busy = true;
  S->batches++;
  return MVP_OK;
}

bool is_done(mvp_server *S, const InFlight &f) {
  return __atomic_load_n(&S->h_done[f.slot].seq_done, __ATOMIC_ACQUIRE) == f.seq + 1;
}

}  // namespace

extern "C" {

mvp_status mvp_serve_create(mvp_ctx *ctx, size_t hbm_budget, int32_t max_slots, size_t arena_bytes,
                            mvp_server **out) {
  if (!ctx || !out) return serve_fail(MVP_ERR_INVALID_ARG, "NULL argument");
  if (max_slots < 1 || max_slots > 65536) return serve_fail(MVP_ERR_INVALID_ARG, "max_slots out of [1, 65536]");
  if (hbm_budget == 0) return serve_fail(MVP_ERR_INVALID_ARG, "hbm_budget is 0");
  *out = nullptr;
  const int dev = mvp::ctx_device(ctx);
  cudaSetDevice(dev);
  mvp_server *S = new (std::nothrow) mvp_server();
  if (!S) return serve_fail(MVP_ERR_OOM, "host allocation");
  S->device = dev;
  S->budget = hbm_budget;
  S->slots = max_slots;
  S->slot_busy.assign(max_slots, false);
  size_t arena = arena_bytes ? arena_bytes : hbm_budget;
  if (arena > hbm_budget) arena = hbm_budget;
  cudaError_t e = cudaSuccess;
  auto bail = [&](const char *what) {
    mvp_serve_destroy(S);
    return serve_fail(e == cudaErrorMemoryAllocation ? MVP_ERR_OOM : MVP_ERR_CUDA, what);
  };
  if ((e = cudaMalloc(&S->arena_base, arena)) != cudaSuccess) return bail("image arena allocation");
  S->arena.init(arena);
  char *h = nullptr;
  if ((e = cudaHostAlloc(&h, sizeof(mvp::ReqDone) * max_slots, cudaHostAllocMapped)) != cudaSuccess)
    return bail("mapped host memory");
  memset(h, 0, sizeof(mvp::ReqDone) * max_slots);
  S->h_done = reinterpret_cast<mvp::ReqDone *>(h);
  char *d = nullptr;
  if ((e = cudaHostGetDevicePointer(&d, h, 0)) != cudaSuccess) return bail("mapped device pointer");
  S->d_done = reinterpret_cast<mvp::ReqDone *>(d);
  if ((e = cudaMalloc(&S->d_status, 256)) != cudaSuccess) return bail("status word");
  if ((e = cudaMemset(S->d_status, 0, 256)) != cudaSuccess) return bail("status reset");
  for (int i = 0; i < mvp::SERVE_STREAMS; ++i) {
    Lane &L = S->lanes[i];
    if ((e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream");
    if ((e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming)) != cudaSuccess) return bail("event");
    if ((e = cudaHostAlloc(&L.h_reqs, sizeof(mvp::BatchReq) * max_slots, cudaHostAllocDefault)) != cudaSuccess)
      return bail("batch staging");
    if ((e = cudaMalloc(&L.d_reqs, sizeof(mvp::BatchReq) * max_slots)) != cudaSuccess) return bail("batch table");
    if ((e = cudaMalloc(&L.d_counters, sizeof(unsigned int) * (max_slots + 1))) != cudaSuccess)
      return bail("batch counters");
  }
  if ((e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking)) != cudaSuccess) return bail("copy stream");
  S->smem = (sizeof(mvp::TileShared<mvp::SERVE_CAP>) + sizeof(mvp::BatchReq)) * mvp::TILE_WARPS;
  if ((e = cudaFuncSetAttribute(mvp::k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem)) !=
      cudaSuccess)
    return bail("kernel attribute");
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mvp::k_serve, mvp::TILE_WARPS * 32, S->smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  S->grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  *out = S;
  return MVP_OK;
}

void mvp_serve_destroy(mvp_server *S) {
  if (!S) return;
  cudaSetDevice(S->device);
  for (auto &L : S->lanes)
    if (L.stream) cudaStreamSynchronize(L.stream);
  if (S->copy) cudaStreamSynchronize(S->copy);
  for (auto &a : S->avatars) mvp::bvh_release(a.bvh);
  if (S->arena_base) cudaFree(S->arena_base);
  if (S->d_status) cudaFree(S->d_status);
  if (S->h_done) cudaFreeHost(S->h_done);
  for (auto &L : S->lanes) {
    if (L.h_reqs) cudaFreeHost(L.h_reqs);
    if (L.d_reqs) cudaFree(L.d_reqs);
    if (L.d_counters) cudaFree(L.d_counters);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  if (S->copy) cudaStreamDestroy(S->copy);
  delete S;
}

mvp_status mvp_serve_register_avatar(mvp_server *S, const mvp_prims *prims, int32_t *avatar_id) {
  if (!S || !prims || !avatar_id) return serve_fail(MVP_ERR_INVALID_ARG, "NULL argument");
  if (prims->n < 1 || prims->n > MVP_MAX_PRIMS || prims->M < 2 || prims->M > MVP_MAX_M || prims->reserved ||
      (prims->dtype != MVP_F32 && prims->dtype != MVP_BF16 && prims->dtype != MVP_F16) || !prims->t || !prims->q ||
      !prims->s || !prims->payload)
    return serve_fail(MVP_ERR_INVALID_ARG, "bad avatar primitives");
  std::lock_guard<std::mutex> lk(S->mu);
  cudaSetDevice(S->device);
  Avatar A;
  A.prims = *prims;
  cudaError_t e = mvp::bvh_reserve(A.bvh, prims->n);
  if (e != cudaSuccess) return serve_fail(MVP_ERR_OOM, "avatar BVH allocation");
  e = mvp::bvh_build(A.bvh, prims->t, prims->q, prims->s, prims->n, prims->M, S->copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->copy);
  if (e != cudaSuccess) {
    mvp::bvh_release(A.bvh);
    return serve_fail(MVP_ERR_CUDA, "avatar BVH build");
  }
  const size_t vb = prims->dtype == MVP_F32 ? 16 : 8;
  A.bytes = (size_t)prims->n * prims->M * prims->M * prims->M * vb + A.bvh.bytes;
  if (S->resident + A.bytes > S->budget) {
    mvp::bvh_release(A.bvh);
    return serve_fail(MVP_ERR_CAPACITY, "avatar does not fit the HBM budget");
  }
  S->resident += A.bytes;
  S->avatars.push_back(A);
  *avatar_id = (int32_t)S->avatars.size() - 1;
  return MVP_OK;
}

mvp_status mvp_serve_submit(mvp_server *S, const mvp_request *req, uint64_t *ticket) {
  if (!S || !req || !ticket) return serve_fail(MVP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (req->avatar < 0 || req->avatar >= (int32_t)S->avatars.size())
    return serve_fail(MVP_ERR_INVALID_ARG, "unknown avatar");
  if (req->width < 1 || req->height < 1 || (int64_t)req->width * req->height > (int64_t)1 << 30 ||
      !(req->focal > 0.0f) || !(req->dt > 0.0f) || !(req->t_far > req->t_near) ||
      !(req->eps_early >= 0.0f && req->eps_early < 1.0f) ||
      mvp_num_steps(req->t_near, req->t_far, req->dt) > MVP_MAX_STEPS)
    return serve_fail(MVP_ERR_INVALID_ARG, "bad request parameters");
  for (int i = 0; i < 12; ++i)
    if (!isfinite(req->c2w[i])) return serve_fail(MVP_ERR_INVALID_ARG, "camera must be finite");
  const size_t bytes = image_bytes(*req);
  if (S->resident + bytes > S->budget || ((bytes + 255) & ~size_t(255)) > S->arena.size)
    return serve_fail(MVP_ERR_CAPACITY, "request image exceeds the HBM budget");
  cudaSetDevice(S->device);
  Pending p;
  p.ticket = S->next_ticket++;
  p.req = *req;
  p.submit = clock_type::now();
  S->pending.push_back(p);
  *ticket = p.ticket;
  return pump(S);
}

mvp_status mvp_serve_poll(mvp_server *S, uint64_t ticket, float *out_rgba, double *latency_ms) {
  if (!S) return serve_fail(MVP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  cudaSetDevice(S->device);
  auto it = S->inflight.find(ticket);
  if (it == S->inflight.end()) {
    for (auto &p : S->pending)
      if (p.ticket == ticket) {
        mvp_status st = pump(S);
        return st ? st : MVP_NOT_READY;
      }
    return serve_fail(MVP_ERR_INVALID_ARG, "unknown ticket");
  }
  InFlight f = it->second;
  if (!f.launched || !is_done(S, f)) {
    mvp_status st = pump(S);
    return st ? st : MVP_NOT_READY;
  }
  const double ms = std::chrono::duration<double, std::milli>(clock_type::now() - f.submit).count();
  if (out_rgba) {
    cudaError_t e = cudaMemcpyAsync(out_rgba, S->arena_base + f.off, f.bytes, cudaMemcpyDefault, S->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->copy);
    if (e != cudaSuccess) return serve_fail(MVP_ERR_CUDA, "image copy");
  }
  if (latency_ms) *latency_ms = ms;
  S->arena.release(f.off, f.bytes);
  S->inflight_bytes -= f.bytes;
  S->slot_busy[f.slot] = false;
  S->inflight.erase(it);
  S->completed++;
  mvp_status st = pump(S);
  return st ? st : MVP_OK;
}

mvp_status mvp_serve_wait(mvp_server *S, uint64_t ticket, double timeout_ms, float *out_rgba, double *latency_ms) {
  const auto t0 = clock_type::now();
  while (true) {
    mvp_status st = mvp_serve_poll(S, ticket, out_rgba, latency_ms);
    if (st != MVP_NOT_READY) return st;
    const double el = std::chrono::duration<double, std::milli>(clock_type::now() - t0).count();
    if (el >= timeout_ms) return serve_fail(MVP_ERR_TIMEOUT, "request not finished before the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

mvp_status mvp_serve_stats(mvp_server *S, mvp_serve_info *info) {
  if (!S || !info) return serve_fail(MVP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  info->pending = (int64_t)S->pending.size();
  info->in_flight = (int64_t)S->inflight.size();
  info->max_in_flight = (int64_t)S->max_inflight_seen;
  info->completed = (int64_t)S->completed;
  info->resident_bytes = (int64_t)S->resident;
  info->in_flight_bytes = (int64_t)S->inflight_bytes;
  info->grid_blocks = S->grid;
  info->avatars = (int32_t)S->avatars.size();
  int st = 0;
  cudaSetDevice(S->device);
  cudaMemcpyAsync(&st, S->d_status, sizeof(int), cudaMemcpyDeviceToHost, S->copy);
  cudaStreamSynchronize(S->copy);
  info->device_status = st;
  info->batches = (int64_t)S->batches;
  return MVP_OK;
}

}  // extern "C"
