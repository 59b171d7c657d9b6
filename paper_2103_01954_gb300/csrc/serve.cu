// serve.cu -- continuous batching of render requests (different avatars, cameras
// and resolutions) through one persistent kernel.
//
// Device side. Every admitted request is cut into warp tiles of 8x4 pixels that are
// numbered consecutively in one global, ever-growing tile sequence: request j owns
// tiles [base_j, base_j + n_j). The host publishes a request by writing its
// descriptor into a ring slot and then raising `published` (release). Worker warps
// claim the next tile number from a device counter (never past `published`), find
// the request that owns it, generate the tile's camera rays and march the tile with
// the same code as mvp_raymarch_fwd (march_tile). A warp that finds no unclaimed
// published tile returns: nothing on the device ever waits. The warp that finishes
// a request's last tile resets the slot's tile counter and publishes the request's
// completion (release, system scope).
//
// Host side. Each submit launches one worker grid (one CTA set per SM) on the
// server's work stream after publishing; a grid that starts after earlier grids
// have drained the queue exits at once, and a request published while a grid runs
// is picked up by that grid's warps as they free up, so requests of different sizes
// overlap on the device. Admission: a request needs a free ring slot and its image
// (W*H*16 bytes) must fit both the HBM budget (resident avatars + images in flight)
// and the server's image arena; otherwise it waits in a FIFO and is admitted by a
// later submit or poll, as slots and memory free up. A request larger than the
// budget itself is refused with MVP_ERR_CAPACITY.
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

// Request descriptor, in mapped pinned host memory: written by the host, read by
// the device. `seq` is written last (release) and read first (acquire).
struct ReqDesc {
  unsigned long long seq;
  unsigned long long base;  // first tile of the request in the global sequence
  int n_tiles;
  int n_prims, M, dtype, n_steps, width, height, pad0;
  const void *payload;
  const Node *nodes;
  const Pose *pose;
  const Xform *xf;
  float *out;
  float c2w[12];
  float focal, t_near, t_far, dt, stop_T;
  float bg[3];
};

// Completion record, written by the device, read by the host.
struct ReqDone {
  unsigned long long seq_done;  // 1 + sequence number of the request completed in this slot (0: none)
  unsigned long long t_start_ns, t_end_ns;
  unsigned long long pad;
};

// Shared host/device state (mapped pinned memory).
struct ServeShared {
  unsigned long long published;  // tiles published so far
  unsigned long long oldest;     // no request before this sequence number is incomplete
  unsigned long long pad[6];
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

struct ServeArgs {
  ServeShared *shared;     // mapped
  ReqDesc *ring;           // mapped, ring_size entries
  ReqDone *done;           // mapped, ring_size entries
  unsigned long long *claimed;  // device: next tile number to hand out
  unsigned int *tiles_done;     // device: finished tiles per slot
  int ring_size;
  int total_warps;
  int *status;
};

// Next published, unclaimed tile number, or -1 if there is none (lane 0 decides).
__device__ __forceinline__ long long claim_tile(const ServeArgs &A) {
  long long t = -1;
  if ((threadIdx.x & 31) == 0) {
    for (int it = 0; it < (1 << 20); ++it) {
      const unsigned long long p = ld_acquire_sys(&A.shared->published);
      const unsigned long long c = *reinterpret_cast<volatile unsigned long long *>(A.claimed);
      if (c >= p) break;
      if (p - c > (unsigned long long)A.total_warps) {
        // more unclaimed tiles than warps: a plain increment cannot pass `published`
        t = (long long)atomicAdd(A.claimed, 1ull);
        break;
      }
      if (atomicCAS(A.claimed, c, c + 1) == c) {
        t = (long long)c;
        break;
      }
      if (it == (1 << 20) - 1) atomicOr(A.status, STATUS_DEVICE);
    }
  }
  return __shfl_sync(FULL, t, 0);
}

template <int DT>
__device__ __noinline__ void serve_tile(TileShared<SERVE_CAP> &sh, const MarchArgs &a, const LaneRay &L) {
  march_tile<DT, SERVE_CAP, false, 0>(sh, a, L);
}

__global__ void __launch_bounds__(TILE_WARPS * 32, 4) k_serve(ServeArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileShared<SERVE_CAP> &sh = reinterpret_cast<TileShared<SERVE_CAP> *>(smem_raw)[warp];
  unsigned long long cursor = 0;
  while (true) {
    const long long t = claim_tile(A);
    if (t < 0) return;
    // every request before `oldest` is complete, and the owner of t is not, so the
    // owner is at most (requests in flight) ahead of this bound
    const unsigned long long lb = ld_acquire_sys(&A.shared->oldest);
    if (cursor < lb) cursor = lb;
    // find the request owning tile t: scan forward from the cursor (tile numbers a
    // warp claims only grow, and every request before the owner is published)
    int slot = -1;
    unsigned long long base = 0;
    for (int it = 0; it < 4 * A.ring_size + 64; ++it) {
      const int s = (int)(cursor % (unsigned long long)A.ring_size);
      const unsigned long long seq = ld_acquire_sys(&A.ring[s].seq);
      if (seq != cursor) {  // recycled: request `cursor` completed, so it cannot own t
        ++cursor;
        continue;
      }
      const volatile ReqDesc *D = &A.ring[s];
      const unsigned long long b = D->base;
      const int n = D->n_tiles;
      if (ld_acquire_sys(&A.ring[s].seq) != cursor) {
        ++cursor;
        continue;
      }
      if ((unsigned long long)t < b + (unsigned long long)n) {
        slot = s;
        base = b;
        break;
      }
      ++cursor;
    }
    if (slot < 0) {  // inconsistent queue state: report and stop this warp
      if (lane == 0) atomicOr(A.status, STATUS_DEVICE);
      return;
    }
    const volatile ReqDesc *D = &A.ring[slot];
    if (lane == 0 && (unsigned long long)t == base) A.done[slot].t_start_ns = globaltimer();
    MarchArgs a;
    a.n_prims = D->n_prims;
    a.M = D->M;
    a.dtype = D->dtype;
    a.payload = D->payload;
    a.nodes = D->nodes;
    a.pose = D->pose;
    a.xf = D->xf;
    const int width = D->width, height = D->height;
    a.geom.n_rays = (int64_t)width * height;
    a.geom.width = width;
    a.geom.height = height;
    a.geom.n_warp_tiles = D->n_tiles;
    a.o = a.d = nullptr;
    a.t_near = D->t_near;
    a.t_far = D->t_far;
    a.dt = D->dt;
    a.stop_T = D->stop_T;
    a.bg[0] = D->bg[0];
    a.bg[1] = D->bg[1];
    a.bg[2] = D->bg[2];
    a.n_steps = D->n_steps;
    a.out = D->out;
    a.saved = nullptr;
    a.n_eval = nullptr;
    a.status = A.status;
    float m[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) m[i] = D->c2w[i];
    const float focal = D->focal;
    // the tile's rays
    LaneRay L;
    const int64_t r = tile_ray(a.geom, t - (long long)base, lane);
    L.r = r;
    if (r >= 0) {
      const int row = (int)(r / width), col = (int)(r - (int64_t)row * width);
      camera_ray(m, focal, width, height, row, col, L.o, L.d);
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
      const unsigned int fin = atomicAdd(&A.tiles_done[slot], 1u);
      if (fin + 1 == (unsigned int)D->n_tiles) {
        __threadfence();
        A.tiles_done[slot] = 0;  // the slot is idle until the host reuses it
        A.done[slot].t_end_ns = globaltimer();
        __threadfence_system();
        st_release_sys(&A.done[slot].seq_done, cursor + 1);
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
  clock_type::time_point submit;
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

}  // namespace

struct mvp_server {
  int device = 0;
  size_t budget = 0;
  int ring = 0;
  std::mutex mu;
  std::vector<Avatar> avatars;
  size_t resident = 0;
  size_t inflight_bytes = 0;
  Arena arena;
  char *arena_base = nullptr;
  mvp::ServeShared *h_shared = nullptr, *d_shared = nullptr;
  mvp::ReqDesc *h_ring = nullptr, *d_ring = nullptr;
  mvp::ReqDone *h_done = nullptr, *d_done = nullptr;
  unsigned long long *d_claimed = nullptr;
  unsigned int *d_tiles_done = nullptr;
  int *d_status = nullptr;
  cudaStream_t work = nullptr, copy = nullptr;
  int grid = 0;
  size_t smem = 0;
  uint64_t next_seq = 0, next_ticket = 1, published = 0;
  std::vector<bool> slot_busy;
  std::vector<uint64_t> slot_seq;
  std::deque<Pending> pending;
  std::map<uint64_t, InFlight> inflight;
  size_t max_inflight_seen = 0;
  uint64_t completed = 0;
};

namespace {

mvp_status serve_fail(mvp_status s, const char *msg) {
  mvp::record_error(msg);
  return s;
}

size_t image_bytes(const mvp_request &r) { return (size_t)r.width * (size_t)r.height * 4 * sizeof(float); }

int64_t warp_tiles(int w, int h) { return (int64_t)((w + 15) / 16) * ((h + 7) / 8) * 4; }

// Oldest incomplete request (lower bound for the device's scans).
uint64_t oldest_incomplete(mvp_server *S) {
  uint64_t o = S->next_seq;
  for (auto &kv : S->inflight) {
    const unsigned long long v = __atomic_load_n(&S->h_done[kv.second.slot].seq_done, __ATOMIC_ACQUIRE);
    if (v != kv.second.seq + 1) o = kv.second.seq < o ? kv.second.seq : o;
  }
  return o;
}

// Admit pending requests in FIFO order while a slot, budget and arena space allow;
// launch one worker grid if anything was published. Called with S->mu held.
mvp_status pump(mvp_server *S) {
  bool launched = false;
  while (!S->pending.empty()) {
    Pending &p = S->pending.front();
    const size_t bytes = image_bytes(p.req);
    const int slot = (int)(S->next_seq % (uint64_t)S->ring);
    if (S->slot_busy[slot]) break;
    if (S->resident + S->inflight_bytes + bytes > S->budget) break;
    size_t off = 0;
    if (!S->arena.alloc(bytes, off)) break;
    const Avatar &A = S->avatars[p.req.avatar];
    const mvp_request &q = p.req;
    mvp::ReqDesc &D = S->h_ring[slot];
    const uint64_t seq = S->next_seq++;
    const int64_t nt = warp_tiles(q.width, q.height);
    D.base = S->published;
    D.n_tiles = (int)nt;
    D.n_prims = A.prims.n;
    D.M = A.prims.M;
    D.dtype = A.prims.dtype;
    D.n_steps = (int)mvp_num_steps(q.t_near, q.t_far, q.dt);
    D.width = q.width;
    D.height = q.height;
    D.payload = A.prims.payload;
    D.nodes = A.bvh.nodes;
    D.pose = A.bvh.pose;
    D.xf = A.bvh.xf;
    D.out = reinterpret_cast<float *>(S->arena_base + off);
    memcpy(D.c2w, q.c2w, sizeof(D.c2w));
    D.focal = q.focal;
    D.t_near = q.t_near;
    D.t_far = q.t_far;
    D.dt = q.dt;
    D.stop_T = (float)(1.0 - (double)q.eps_early);
    memcpy(D.bg, q.bg, sizeof(D.bg));
    // the completion record holds seq + 1 once done (0: nothing completed yet)
    __atomic_store_n(&S->h_done[slot].seq_done, 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&D.seq, (unsigned long long)seq, __ATOMIC_RELEASE);
    S->published += (uint64_t)nt;
    S->slot_busy[slot] = true;
    S->slot_seq[slot] = seq;
    InFlight f;
    f.seq = seq;
    f.slot = slot;
    f.off = off;
    f.bytes = bytes;
    f.submit = p.submit;
    S->inflight[p.ticket] = f;
    // the scan bound first (it includes this request), then the tiles (release)
    __atomic_store_n(&S->h_shared->oldest, (unsigned long long)oldest_incomplete(S), __ATOMIC_RELEASE);
    __atomic_store_n(&S->h_shared->published, (unsigned long long)S->published, __ATOMIC_RELEASE);
    S->inflight_bytes += bytes;
    if (S->inflight.size() > S->max_inflight_seen) S->max_inflight_seen = S->inflight.size();
    S->pending.pop_front();
    launched = true;
  }
  if (launched) {
    mvp::ServeArgs a;
    a.shared = S->d_shared;
    a.ring = S->d_ring;
    a.done = S->d_done;
    a.claimed = S->d_claimed;
    a.tiles_done = S->d_tiles_done;
    a.ring_size = S->ring;
    a.total_warps = S->grid * mvp::TILE_WARPS;
    a.status = S->d_status;
    mvp::k_serve<<<S->grid, mvp::TILE_WARPS * 32, S->smem, S->work>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return serve_fail(MVP_ERR_CUDA, cudaGetErrorString(e));
  }
  return MVP_OK;
}

}  // namespace

// The completion record of the slot holds seq + 1 once the request is done.
static bool is_done(mvp_server *S, const InFlight &f) {
  unsigned long long v = __atomic_load_n(&S->h_done[f.slot].seq_done, __ATOMIC_ACQUIRE);
  return v == f.seq + 1;
}

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
  S->ring = max_slots;
  S->slot_busy.assign(max_slots, false);
  S->slot_seq.assign(max_slots, 0);
  size_t arena = arena_bytes ? arena_bytes : hbm_budget;
  if (arena > hbm_budget) arena = hbm_budget;
  cudaError_t e = cudaSuccess;
  auto bail = [&](const char *what) {
    mvp_serve_destroy(S);
    return serve_fail(e == cudaErrorMemoryAllocation ? MVP_ERR_OOM : MVP_ERR_CUDA, what);
  };
  if ((e = cudaMalloc(&S->arena_base, arena)) != cudaSuccess) return bail("image arena allocation");
  S->arena.init(arena);
  size_t host_bytes = sizeof(mvp::ServeShared) + sizeof(mvp::ReqDesc) * max_slots + sizeof(mvp::ReqDone) * max_slots;
  char *h = nullptr;
  if ((e = cudaHostAlloc(&h, host_bytes, cudaHostAllocMapped)) != cudaSuccess) return bail("mapped host memory");
  memset(h, 0, host_bytes);
  S->h_shared = reinterpret_cast<mvp::ServeShared *>(h);
  S->h_ring = reinterpret_cast<mvp::ReqDesc *>(h + sizeof(mvp::ServeShared));
  S->h_done = reinterpret_cast<mvp::ReqDone *>(h + sizeof(mvp::ServeShared) + sizeof(mvp::ReqDesc) * max_slots);
  for (int i = 0; i < max_slots; ++i) S->h_ring[i].seq = ~0ull;
  char *d = nullptr;
  if ((e = cudaHostGetDevicePointer(&d, h, 0)) != cudaSuccess) return bail("mapped device pointer");
  S->d_shared = reinterpret_cast<mvp::ServeShared *>(d);
  S->d_ring = reinterpret_cast<mvp::ReqDesc *>(d + sizeof(mvp::ServeShared));
  S->d_done = reinterpret_cast<mvp::ReqDone *>(d + sizeof(mvp::ServeShared) + sizeof(mvp::ReqDesc) * max_slots);
  char *dev_state = nullptr;
  size_t dev_bytes = 256 + sizeof(unsigned int) * max_slots + 256;
  if ((e = cudaMalloc(&dev_state, dev_bytes)) != cudaSuccess) return bail("device state");
  if ((e = cudaMemset(dev_state, 0, dev_bytes)) != cudaSuccess) return bail("device state reset");
  S->d_claimed = reinterpret_cast<unsigned long long *>(dev_state);
  S->d_status = reinterpret_cast<int *>(dev_state + 64);
  S->d_tiles_done = reinterpret_cast<unsigned int *>(dev_state + 256);
  if ((e = cudaStreamCreateWithFlags(&S->work, cudaStreamNonBlocking)) != cudaSuccess) return bail("work stream");
  if ((e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking)) != cudaSuccess) return bail("copy stream");
  S->smem = sizeof(mvp::TileShared<mvp::SERVE_CAP>) * mvp::TILE_WARPS;
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
  if (S->work) cudaStreamSynchronize(S->work);
  if (S->copy) cudaStreamSynchronize(S->copy);
  for (auto &a : S->avatars) mvp::bvh_release(a.bvh);
  if (S->arena_base) cudaFree(S->arena_base);
  if (S->d_claimed) cudaFree(S->d_claimed);
  if (S->h_shared) cudaFreeHost(S->h_shared);
  if (S->work) cudaStreamDestroy(S->work);
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
  if (req->width < 1 || req->height < 1 || !(req->focal > 0.0f) || !(req->dt > 0.0f) ||
      !(req->t_far > req->t_near) || !(req->eps_early >= 0.0f && req->eps_early < 1.0f) ||
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
  if (!is_done(S, f)) return MVP_NOT_READY;
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
  return MVP_OK;
}

}  // extern "C"
