// serve.cu -- continuous batching of render requests (different avatars, cameras
// and resolutions) on one GPU.
//
// Device side. Each admitted request is one launch of k_serve, its arguments in the
// kernel's parameter block, with one warp per 8x4-pixel tile of its image (of both
// images for a stereo pair, which share the avatar's BVH and one launch). A warp
// generates its tile's pinhole rays and marches them with the same code as
// mvp_raymarch_fwd (march_tile, specialised for M = 8, 16, 32 and for the payload
// type). Nothing on the device ever waits. The warp that counts a request's last
// tile publishes its completion to mapped host memory (system-scope release), so the
// host sees it without synchronising a stream.
//
// Host side. Admission: a request needs a free slot and its image (W*H*16 bytes)
// must fit the HBM budget (resident avatars + images in flight) and the server's
// image arena; otherwise it waits in a FIFO and is admitted by a later submit or
// poll as slots and memory free up. An admitted request is launched at once on the
// least loaded of several streams, so requests overlap on the device: a new
// request's blocks start as SMs free up from the ones before it. A request larger
// than the budget is refused (MVP_ERR_CAPACITY).
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

constexpr int SERVE_STREAMS = 8;  // requests that may run at once without queueing on a stream

// Completion record of a slot (mapped host memory): written by the device.
struct ReqDone {
  unsigned long long seq_done;  // 1 + sequence number of the request completed in this slot (0: none)
  unsigned long long t_start_ns, t_end_ns;
  unsigned long long pad;
};

// One request: the kernel's parameter block (constant bank), so the march reads its
// arguments exactly as mvp_raymarch_fwd's kernel does.
struct ServeReq {
  MarchArgs m;               // payload, BVH, sampling, output image (m.o, m.d unused)
  float c2w[12];
  float c2w2[12];            // second view (views = 2)
  int views;                 // 1 or 2; the image is [views][height][width][4]
  float focal;
  int slot;                  // completion record and tile counter index
  unsigned long long seq;    // request sequence number
  unsigned int *tiles_done;  // device, per slot; zero between requests
  ReqDone *done;             // mapped host memory, per slot
};

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// One warp per warp tile of the request's image, specialised by payload type and
// resolution class (MT = M for M = 8, 16, 32, else 0: any M). The warp that counts
// the last tile publishes the completion and resets the slot's counter for its next
// request (every other warp of this request has counted by then).
#ifndef MVP_SERVE_HALF_MINB
#define MVP_SERVE_HALF_MINB 4  // resident blocks per SM of the BF16/FP16 serving kernels
#endif

template <int DT, int MT>
__global__ void __launch_bounds__(TILE_WARPS * 32, DT == MVP_F32 ? MVP_MARCH_MINB : MVP_SERVE_HALF_MINB)
    k_serve(const __grid_constant__ ServeReq R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int CAP = march_cap<MT>();
  TileShared<CAP> &sh = reinterpret_cast<TileShared<CAP> *>(smem_raw)[warp];
  const int64_t wt = (int64_t)blockIdx.x * TILE_WARPS + warp;
  const int64_t n_view = R.m.geom.n_warp_tiles;  // tiles per view
  const int64_t n_tiles = n_view * R.views;
  if (wt >= n_tiles) return;
  if (lane == 0 && wt == 0) R.done[R.slot].t_start_ns = globaltimer();
  // a stereo request's tiles run through view 0, then view 1 (a tile never spans both)
  const int view = wt >= n_view ? 1 : 0;
  LaneRay L;
  const int64_t r = tile_ray(R.m.geom, wt - view * n_view, lane);
  L.r = r >= 0 ? r + view * R.m.geom.n_rays : -1;  // pixel of the [views][h][w] image
  if (r >= 0) {
    const int width = R.m.geom.width;
    const int row = (int)(r / width), col = (int)(r - (int64_t)row * width);
    camera_ray(view ? R.c2w2 : R.c2w, R.focal, width, R.m.geom.height, row, col, L.o, L.d);
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) L.o[j] = L.d[j] = 0.0f;
  }
  if (__ballot_sync(FULL, L.r >= 0) != 0) march_tile<DT, CAP, false, MT>(sh, R.m, L);
  __syncwarp();
  if (lane == 0) {
    __threadfence();  // this tile's pixels are visible before it is counted
    unsigned int *cnt = R.tiles_done + R.slot;
    const unsigned int fin = atomicAdd(cnt, 1u);
    if (fin + 1 == (unsigned int)n_tiles) {
      *cnt = 0u;
      __threadfence();
      R.done[R.slot].t_end_ns = globaltimer();
      __threadfence_system();
      st_release_sys(&R.done[R.slot].seq_done, R.seq + 1);
    }
  }
}

// Kernel of a payload: dtype x {M = 8, 16, 32, other}.
// kernel class of an avatar: payload type x grid edge (8, 16, 32, another edge up to 12,
// another edge)
inline int serve_class(int dtype, int M) {
  return dtype * 5 + (M == 8 ? 0 : M == 16 ? 1 : M == 32 ? 2 : M <= 12 ? 3 : 4);
}
constexpr int SERVE_CLASSES = 15;

using ServeKernel = void (*)(const ServeReq);
static const ServeKernel k_serve_table[SERVE_CLASSES] = {
    k_serve<MVP_F32, 8>,  k_serve<MVP_F32, 16>,  k_serve<MVP_F32, 32>,  k_serve<MVP_F32, -1>,  k_serve<MVP_F32, 0>,
    k_serve<MVP_BF16, 8>, k_serve<MVP_BF16, 16>, k_serve<MVP_BF16, 32>, k_serve<MVP_BF16, -1>, k_serve<MVP_BF16, 0>,
    k_serve<MVP_F16, 8>,  k_serve<MVP_F16, 16>,  k_serve<MVP_F16, 32>,  k_serve<MVP_F16, -1>,  k_serve<MVP_F16, 0>};
// dynamic shared memory of each class's kernel (its window capacity depends on M)
inline size_t serve_smem(int cls) {
  switch (cls % 5) {
    case 0: return sizeof(TileShared<march_cap<8>()>) * TILE_WARPS;
    case 1: return sizeof(TileShared<march_cap<16>()>) * TILE_WARPS;
    case 2: return sizeof(TileShared<march_cap<32>()>) * TILE_WARPS;
    case 3: return sizeof(TileShared<march_cap<-1>()>) * TILE_WARPS;
    default: return sizeof(TileShared<march_cap<0>()>) * TILE_WARPS;
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
  int stream = -1;  // index into mvp_server::streams
  size_t off = 0, bytes = 0;
  mvp_request req;
  clock_type::time_point submit;
  bool detached = false;  // cancelled while running: freed by the server once done
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
  int slots = 0;
  std::mutex mu;
  std::vector<Avatar> avatars;
  size_t resident = 0;
  size_t inflight_bytes = 0;
  Arena arena;
  char *arena_base = nullptr;
  mvp::ReqDone *h_done = nullptr, *d_done = nullptr;  // mapped
  int *d_status = nullptr;
  unsigned int *d_tiles_done = nullptr;  // per slot
  cudaStream_t streams[mvp::SERVE_STREAMS] = {};
  int outstanding[mvp::SERVE_STREAMS] = {};  // requests launched and not yet collected
  int next_stream = 0;
  cudaStream_t copy = nullptr;
  int grid = 0;
  size_t smem = 0;
  uint64_t next_seq = 0, next_ticket = 1;
  std::vector<bool> slot_busy;
  std::deque<Pending> pending;
  std::map<uint64_t, InFlight> inflight;  // ticket -> request (admitted)
  size_t max_inflight_seen = 0;
  uint64_t completed = 0, launches = 0, cancelled = 0;
};

namespace {

mvp_status serve_fail(mvp_status s, const char *msg) {
  mvp::record_error(msg);
  return s;
}

int request_views(const mvp_request &r) { return r.views == 2 ? 2 : 1; }

size_t image_bytes(const mvp_request &r) {
  return (size_t)request_views(r) * (size_t)r.width * (size_t)r.height * 4 * sizeof(float);
}

// Launch one admitted request on the stream with the fewest requests outstanding
// (round robin among ties): its image's warp tiles run as soon as SMs free up,
// beside the requests on the other streams.
mvp_status launch(mvp_server *S, InFlight &f) {
  const mvp_request &q = f.req;
  const Avatar &A = S->avatars[q.avatar];
  mvp::ServeReq R;
  memset(&R, 0, sizeof(R));
  mvp::MarchArgs &m = R.m;
  m.n_prims = A.prims.n;
  m.M = A.prims.M;
  m.dtype = A.prims.dtype;
  m.payload = q.payload ? q.payload : A.prims.payload;  // a request's own (view-dependent) payload
  m.nodes = A.bvh.nodes;
  m.pose = A.bvh.pose;
  m.xf = A.bvh.xf;
  m.geom = mvp::make_tile_geom((int64_t)q.width * q.height, q.width, q.height);
  m.t_near = q.t_near;
  m.t_far = q.t_far;
  m.dt = q.dt;
  m.stop_T = (float)(1.0 - (double)q.eps_early);
  memcpy(m.bg, q.bg, sizeof(m.bg));
  m.n_steps = (int)mvp_num_steps(q.t_near, q.t_far, q.dt);
  m.out = reinterpret_cast<float *>(S->arena_base + f.off);
  m.status = S->d_status;
  memcpy(R.c2w, q.c2w, sizeof(R.c2w));
  memcpy(R.c2w2, q.c2w_right, sizeof(R.c2w2));
  R.views = request_views(q);
  R.focal = q.focal;
  R.slot = f.slot;
  R.seq = f.seq;
  R.tiles_done = S->d_tiles_done;
  R.done = S->d_done;
  int best = -1;
  for (int k = 0; k < mvp::SERVE_STREAMS; ++k) {
    const int i = (S->next_stream + k) % mvp::SERVE_STREAMS;
    if (best < 0 || S->outstanding[i] < S->outstanding[best]) best = i;
  }
  S->next_stream = (best + 1) % mvp::SERVE_STREAMS;
  const unsigned blocks = (unsigned)(m.geom.n_warp_tiles * R.views / mvp::TILE_WARPS);
  const int cls = mvp::serve_class(m.dtype, m.M);
  mvp::k_serve_table[cls]<<<blocks, mvp::TILE_WARPS * 32, mvp::serve_smem(cls), S->streams[best]>>>(R);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return serve_fail(MVP_ERR_CUDA, cudaGetErrorString(e));
  f.stream = best;
  S->outstanding[best]++;
  S->launches++;
  return MVP_OK;
}

// Admit pending requests in FIFO order while a slot, budget and arena space allow,
// launching each as it is admitted. Called with S->mu held.
// Give an admitted request's slot, stream share and image memory back.
void retire(mvp_server *S, std::map<uint64_t, InFlight>::iterator it) {
  const InFlight &f = it->second;
  S->arena.release(f.off, f.bytes);
  S->inflight_bytes -= f.bytes;
  S->outstanding[f.stream]--;
  S->slot_busy[f.slot] = false;
  S->inflight.erase(it);
}

bool is_done(mvp_server *S, const InFlight &f);

mvp_status pump(mvp_server *S) {
  for (auto it = S->inflight.begin(); it != S->inflight.end();) {  // cancelled requests that finished
    auto nx = std::next(it);
    if (it->second.detached && is_done(S, it->second)) retire(S, it);
    it = nx;
  }
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
    const mvp_status st = launch(S, f);
    if (st != MVP_OK) {
      S->arena.release(off, bytes);
      return st;
    }
    S->slot_busy[slot] = true;
    S->inflight[p.ticket] = f;
    S->inflight_bytes += bytes;
    if (S->inflight.size() > S->max_inflight_seen) S->max_inflight_seen = S->inflight.size();
    S->pending.pop_front();
  }
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
  if ((e = cudaMalloc(&S->d_tiles_done, sizeof(unsigned int) * max_slots)) != cudaSuccess) return bail("tile counters");
  if ((e = cudaMemset(S->d_tiles_done, 0, sizeof(unsigned int) * max_slots)) != cudaSuccess)
    return bail("tile counter reset");
  for (cudaStream_t &st : S->streams)
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream");
  if ((e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking)) != cudaSuccess) return bail("copy stream");
  S->smem = mvp::serve_smem(1);  // the 16^3 class, for the grid size below
  for (int c = 0; c < mvp::SERVE_CLASSES; ++c)
    if ((e = cudaFuncSetAttribute(mvp::k_serve_table[c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)mvp::serve_smem(c))) != cudaSuccess)
      return bail("kernel attribute");
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mvp::k_serve_table[1], mvp::TILE_WARPS * 32, S->smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  S->grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  *out = S;
  return MVP_OK;
}

void mvp_serve_destroy(mvp_server *S) {
  if (!S) return;
  cudaSetDevice(S->device);
  for (cudaStream_t st : S->streams)
    if (st) cudaStreamSynchronize(st);
  if (S->copy) cudaStreamSynchronize(S->copy);
  for (auto &a : S->avatars) mvp::bvh_release(a.bvh);
  if (S->arena_base) cudaFree(S->arena_base);
  if (S->d_status) cudaFree(S->d_status);
  if (S->h_done) cudaFreeHost(S->h_done);
  if (S->d_tiles_done) cudaFree(S->d_tiles_done);
  for (cudaStream_t st : S->streams)
    if (st) cudaStreamDestroy(st);
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
  // the build's pose check goes to a word of its own (the first one collects the
  // running requests' status bits)
  int *pose_word = S->d_status + 1;
  int bad = 0;
  e = cudaMemsetAsync(pose_word, 0, sizeof(int), S->copy);
  if (e == cudaSuccess) e = mvp::bvh_build(A.bvh, prims->t, prims->q, prims->s, prims->n, prims->M, S->copy, pose_word);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, pose_word, sizeof(int), cudaMemcpyDeviceToHost, S->copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->copy);
  if (e != cudaSuccess) {
    mvp::bvh_release(A.bvh);
    return serve_fail(MVP_ERR_CUDA, "avatar BVH build");
  }
  if (bad) {
    mvp::bvh_release(A.bvh);
    return serve_fail(MVP_ERR_INVALID_ARG, "avatar pose defines no box (t, q or s not finite, q = 0 or s <= 0)");
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
  if (req->views < 0 || req->views > 2) return serve_fail(MVP_ERR_INVALID_ARG, "views must be 1 or 2");
  if (req->width < 1 || req->height < 1 || (int64_t)req->width * req->height > (int64_t)1 << 30 ||
      !(req->focal > 0.0f) || !(req->dt > 0.0f) || !(req->t_far > req->t_near) ||
      !(req->eps_early >= 0.0f && req->eps_early < 1.0f) ||
      mvp_num_steps(req->t_near, req->t_far, req->dt) > MVP_MAX_STEPS)
    return serve_fail(MVP_ERR_INVALID_ARG, "bad request parameters");
  for (int i = 0; i < 12; ++i)
    if (!isfinite(req->c2w[i]) || (req->views == 2 && !isfinite(req->c2w_right[i])))
      return serve_fail(MVP_ERR_INVALID_ARG, "camera must be finite");
  if (req->payload &&
      reinterpret_cast<uintptr_t>(req->payload) % (S->avatars[req->avatar].prims.dtype == MVP_F32 ? 16 : 8))
    return serve_fail(MVP_ERR_INVALID_ARG, "request payload misaligned");
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
  if (it != S->inflight.end() && it->second.detached) return serve_fail(MVP_ERR_INVALID_ARG, "cancelled ticket");
  if (it == S->inflight.end()) {
    for (auto &p : S->pending)
      if (p.ticket == ticket) {
        mvp_status st = pump(S);
        return st ? st : MVP_NOT_READY;
      }
    return serve_fail(MVP_ERR_INVALID_ARG, "unknown ticket");
  }
  InFlight f = it->second;
  if (!is_done(S, f)) {
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
  retire(S, it);
  S->completed++;
  mvp_status st = pump(S);
  return st ? st : MVP_OK;
}

mvp_status mvp_serve_cancel(mvp_server *S, uint64_t ticket) {
  if (!S) return serve_fail(MVP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  cudaSetDevice(S->device);
  for (auto p = S->pending.begin(); p != S->pending.end(); ++p)
    if (p->ticket == ticket) {  // never admitted: nothing ran
      S->pending.erase(p);
      S->cancelled++;
      return MVP_OK;
    }
  auto it = S->inflight.find(ticket);
  if (it == S->inflight.end() || it->second.detached) return serve_fail(MVP_ERR_INVALID_ARG, "unknown ticket");
  S->cancelled++;
  if (is_done(S, it->second)) {
    retire(S, it);
  } else {
    it->second.detached = true;  // its launch runs to completion; the memory is freed after
  }
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
  info->cancelled = (int64_t)S->cancelled;
  info->resident_bytes = (int64_t)S->resident;
  info->in_flight_bytes = (int64_t)S->inflight_bytes;
  info->grid_blocks = S->grid;
  info->avatars = (int32_t)S->avatars.size();
  int st = 0;
  cudaSetDevice(S->device);
  cudaMemcpyAsync(&st, S->d_status, sizeof(int), cudaMemcpyDeviceToHost, S->copy);
  cudaStreamSynchronize(S->copy);
  info->device_status = st;
  info->batches = (int64_t)S->launches;
  return MVP_OK;
}

}  // extern "C"
