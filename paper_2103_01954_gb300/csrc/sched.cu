// sched.cu -- the frame kernel's tile schedule: the warp tiles of the last frame,
// sorted by the clock cycles each took (recorded by k_march), heaviest first.
#include "march.cuh"

namespace mvp {

// A counting sort of the warp tiles by descending cost bucket (one bucket per octave
// of clock cycles, coarse enough that neighbouring tiles mostly share a bucket and
// keep their order, so the payload they share stays in cache), in one block. The
// buckets are staged in shared memory first; then warp w owns a contiguous range of
// tiles and a row of per-bucket counters, and lanes with equal buckets in a round are
// grouped with a match, so the counters need no atomics and the result is a
// deterministic permutation.
constexpr int ORDER_BUCKETS = 32;

__device__ __forceinline__ int cost_bucket(unsigned int c) { return c ? 31 - __clz(c) : 0; }

constexpr int64_t ORDER_SMEM_KEYS = 160 * 1024;  // tiles whose buckets are staged in shared memory

__global__ void __launch_bounds__(1024) k_tile_order(const unsigned int *__restrict__ cost, int64_t n,
                                                     int *__restrict__ order) {
  extern __shared__ unsigned char key_s[];  // [n] buckets when n <= ORDER_SMEM_KEYS
  __shared__ int cnt[32][ORDER_BUCKETS];
  __shared__ int start[ORDER_BUCKETS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const bool staged = n <= ORDER_SMEM_KEYS;
  for (int i = threadIdx.x; i < 32 * ORDER_BUCKETS; i += blockDim.x) (&cnt[0][0])[i] = 0;
  if (staged) {  // coalesced, independent loads: the costs arrive in a few round trips
#pragma unroll 4
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) key_s[t] = (unsigned char)cost_bucket(__ldg(cost + t));
  }
  __syncthreads();
  auto key_of = [&](int64_t t) -> int { return staged ? (int)key_s[t] : cost_bucket(__ldg(cost + t)); };
  const int64_t per = (n + 31) / 32, t0 = warp * per, t1 = min(n, t0 + per);
  for (int64_t b = t0; b < t1; b += 32) {
    const int64_t t = b + lane;
    const int key = t < t1 ? key_of(t) : -1;
    const unsigned peers = __match_any_sync(FULL, key);
    if (key >= 0 && (peers & lt) == 0) cnt[warp][key] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x < ORDER_BUCKETS) {
    int tot = 0;
    for (int w = 0; w < 32; ++w) tot += cnt[w][threadIdx.x];
    start[threadIdx.x] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan, heaviest bucket first
    int run = 0;
    for (int k = ORDER_BUCKETS - 1; k >= 0; --k) {
      const int c = start[k];
      start[k] = run;
      run += c;
    }
  }
  __syncthreads();
  if (threadIdx.x < ORDER_BUCKETS) {  // per-warp cursors within each bucket
    int run = start[threadIdx.x];
    for (int w = 0; w < 32; ++w) {
      const int c = cnt[w][threadIdx.x];
      cnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int64_t b = t0; b < t1; b += 32) {
    const int64_t t = b + lane;
    const int key = t < t1 ? key_of(t) : -1;
    const unsigned peers = __match_any_sync(FULL, key);
    const int base = key >= 0 ? cnt[warp][key] : 0;
    __syncwarp();
    if (key >= 0) {
      order[base + __popc(peers & lt)] = (int)t;
      if ((peers & lt) == 0) cnt[warp][key] = base + __popc(peers);
    }
    __syncwarp();
  }
}

cudaError_t launch_tile_order(const unsigned int *cost, int64_t n, int *order, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void *>(k_tile_order), ORDER_SMEM_KEYS);
  if (e != cudaSuccess) return e;
  const size_t smem = n <= ORDER_SMEM_KEYS ? (size_t)n : 0;
  k_tile_order<<<1, 1024, smem, st>>>(cost, n, order);
  return cudaGetLastError();
}

}  // namespace mvp
