// Plaintext meaning of the selection step (the paper evaluates it inside
// garbled circuits, which stay out of scope): the k smallest reconstructed
// distances dist = ((client share + server share) mod t) >> r of every query
// (r: the paper's truncation of distances before selection, r_c for cluster
// centres and r_p for points, Algorithm 4).
//   exact:        the k smallest (value, position) pairs (the order of
//                 Algorithm 1, NaiveTopk, which never lets a later equal value
//                 displace an earlier one)
//   approximate:  Algorithm 2, ApproxTopk: position x falls in bin
//                 floor(x l / n); the minimum of every bin (the earlier
//                 position on ties), then the k smallest of the l minima.
// A (value, position) pair is one 64-bit key, value << 32 | position, so
// every comparison is a plain integer comparison and the result is unique.
// Selection runs per segment: a query's whole share vector (uniform: segment
// b = positions [b n, (b + 1) n) of both shares), or one of B ragged lists at
// its own offsets into the client and server shares (the per-query lists of
// the clustering protocol).  A segment shorter than k leaves missing keys.
#include "internal.h"

namespace sanns {

namespace {

constexpr int kTopkMax = 32;     // register lists (k <= kTopkMax)
constexpr int kTopkThreads = 256;
constexpr uint64_t kNoKey = ~0ull;
constexpr int kSortKeys = 4096;   // keys a block sorts in shared memory (larger k)
constexpr int kSortThreads = 512;
static_assert(kTopkLarge * 4 <= kSortKeys, "a sort pass must shrink the keys at least 4x");

// Where segment b lies: uniform (len == NULL) or from device arrays.
struct Segs {
  const uint64_t* cli_off;
  const uint64_t* srv_off;
  const uint64_t* len;
  uint64_t n;
  const uint64_t* kseg;  // winners per segment (NULL: k for all)
  const uint64_t* lseg;  // bins per segment (NULL: l for all)
};

__device__ __forceinline__ void seg_of(const Segs& sg, uint64_t b, uint64_t& co, uint64_t& so,
                                       uint64_t& ln) {
  if (sg.len == nullptr) {
    co = so = b * sg.n;
    ln = sg.n;
  } else {
    co = sg.cli_off[b];
    so = sg.srv_off[b];
    ln = sg.len[b];
  }
}

__device__ __forceinline__ uint64_t key_of(const uint32_t* cs, const uint32_t* ss, uint64_t p, uint64_t t,
                                           uint32_t shift) {
  uint64_t v = (uint64_t)cs[p] + ss[p];
  v = (v >= t ? v - t : v) >> shift;
  return (v << 32) | p;
}

// A thread keeps its kTopkMax smallest keys, ascending (at least the k the
// block needs, k <= kTopkMax; static indices keep the list in registers).
// Insert key, only called when key < best[kTopkMax - 1].
__device__ __forceinline__ void topk_insert(uint64_t (&best)[kTopkMax], uint64_t key) {
#pragma unroll
  for (int j = kTopkMax - 1; j >= 1; --j) {
    const uint64_t prev = best[j - 1];
    if (prev > key) best[j] = prev;
    else if (best[j] > key) best[j] = key;
  }
  if (best[0] > key) best[0] = key;
}

// The block's k smallest keys from every thread's ascending list, in k
// rounds of a block-wide minimum; thread 0 writes them to out[0 .. k-1].
__device__ void topk_block_merge(uint64_t (&best)[kTopkMax], int k, uint64_t* out) {
  __shared__ uint64_t warp_min[kTopkThreads / 32];
  __shared__ uint64_t round_min;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < k; ++r) {
    uint64_t m = best[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, m, o);
      m = other < m ? other : m;
    }
    if (lane == 0) warp_min[warp] = m;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < blockDim.x / 32 ? warp_min[lane] : kNoKey;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, w, o);
        w = other < w ? other : w;
      }
      if (lane == 0) {
        round_min = w;
        out[r] = w;
      }
    }
    __syncthreads();
    // keys are unique: exactly one thread holds a real minimum and pops it
    if (best[0] == round_min && round_min != kNoKey) {
#pragma unroll
      for (int j = 0; j < kTopkMax - 1; ++j) best[j] = best[j + 1];
      best[kTopkMax - 1] = kNoKey;
    }
    __syncthreads();
  }
}

// Pass 1, from the shares: block (chunk c, segment b) keeps the k smallest
// keys of positions [c chunk, (c + 1) chunk) of the segment in
// part[b][c][0 .. k-1].
__global__ void __launch_bounds__(kTopkThreads) topk_shares_kernel(const uint32_t* __restrict__ cli,
                                                                   const uint32_t* __restrict__ srv,
                                                                   Segs sg, uint64_t t, int k,
                                                                   uint64_t chunk, uint32_t shift,
                                                                   uint64_t* part) {
  const uint64_t b = blockIdx.y, c = blockIdx.x;
  uint64_t co, so, n;
  seg_of(sg, b, co, so, n);
  uint64_t best[kTopkMax];
#pragma unroll
  for (int j = 0; j < kTopkMax; ++j) best[j] = kNoKey;
  const uint64_t p0 = c * chunk, p1 = p0 + chunk < n ? p0 + chunk : n;
  for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const uint64_t key = key_of(cli + co, srv + so, p, t, shift);
    if (key < best[kTopkMax - 1]) topk_insert(best, key);
  }
  topk_block_merge(best, k, part + (b * gridDim.x + c) * k);
}

// Bin minima for ApproxTopk: one warp per bin i of segment b, l_b =
// min(l, length) bins (l per segment where given), bin i = positions [ceil(i n / l_b), ceil((i + 1) n / l_b));
// mins[b][i] = the smallest key of the bin (missing for i >= l_b).  l_b = n
// puts every position in a bin of its own: the selection is then exact.
__global__ void __launch_bounds__(kTopkThreads) bin_min_kernel(const uint32_t* __restrict__ cli,
                                                               const uint32_t* __restrict__ srv,
                                                               Segs sg, uint64_t t, uint64_t l,
                                                               uint32_t shift, uint64_t* mins) {
  const uint64_t b = blockIdx.y;
  const uint64_t i = blockIdx.x * (uint64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  const uint32_t lane = threadIdx.x & 31;
  if (i >= l) return;
  uint64_t co, so, n;
  seg_of(sg, b, co, so, n);
  const uint64_t ls = sg.lseg ? sg.lseg[b] : l;
  const uint64_t lb = ls < n ? ls : n;
  uint64_t m = kNoKey;
  if (i < lb) {
    const uint64_t p0 = (i * n + lb - 1) / lb, p1 = ((i + 1) * n + lb - 1) / lb;
    for (uint64_t p = p0 + lane; p < p1; p += 32) {
      const uint64_t key = key_of(cli + co, srv + so, p, t, shift);
      m = key < m ? key : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, m, o);
    m = other < m ? other : m;
  }
  if (lane == 0) mins[b * l + i] = m;
}

// Pass over keys: block (chunk c, query b) keeps the k smallest of
// keys[b][c chunk .. (c + 1) chunk) (count per query m).
__global__ void __launch_bounds__(kTopkThreads) topk_keys_kernel(const uint64_t* __restrict__ keys,
                                                                 uint64_t m, int k, uint64_t chunk,
                                                                 uint64_t* part) {
  const uint64_t b = blockIdx.y, c = blockIdx.x;
  uint64_t best[kTopkMax];
#pragma unroll
  for (int j = 0; j < kTopkMax; ++j) best[j] = kNoKey;
  const uint64_t p0 = c * chunk, p1 = p0 + chunk < m ? p0 + chunk : m;
  const uint64_t* ks = keys + b * m;
  for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const uint64_t key = ks[p];
    if (key < best[kTopkMax - 1]) topk_insert(best, key);
  }
  topk_block_merge(best, k, part + (b * gridDim.x + c) * k);
}

// Larger k (kTopkMax < k <= kTopkLarge): block (chunk c, segment b) sorts
// kSortKeys keys in shared memory (bitonic network, ascending) and keeps the
// first k in part[b][c][0 .. k-1].  The keys come from the shares
// (kFromShares, positions [c kSortKeys, (c + 1) kSortKeys) of the segment)
// or from a key array of m keys per segment; missing keys sort last.
template <bool kFromShares>
__global__ void __launch_bounds__(kSortThreads) topk_sort_kernel(const uint64_t* __restrict__ keys,
                                                                 const uint32_t* __restrict__ cli,
                                                                 const uint32_t* __restrict__ srv,
                                                                 Segs sg, uint64_t m, uint64_t t,
                                                                 uint32_t shift, int k,
                                                                 uint64_t* part) {
  __shared__ uint64_t s[kSortKeys];
  const uint64_t b = blockIdx.y, c = blockIdx.x;
  const uint64_t p0 = c * kSortKeys;
  uint64_t co = 0, so = 0;
  if (kFromShares) seg_of(sg, b, co, so, m);
  for (int i = threadIdx.x; i < kSortKeys; i += kSortThreads) {
    const uint64_t p = p0 + i;
    uint64_t key = kNoKey;
    if (p < m) key = kFromShares ? key_of(cli + co, srv + so, p, t, shift) : keys[b * m + p];
    s[i] = key;
  }
  __syncthreads();
  for (int size = 2; size <= kSortKeys; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < kSortKeys / 2; i += kSortThreads) {
        const int lo = 2 * i - (i & (stride - 1));  // the pair (lo, lo + stride), lo's stride bit clear
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t x = s[lo], y = s[hi];
        if ((x > y) == up) {
          s[lo] = y;
          s[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < k; r += kSortThreads) part[(b * gridDim.x + c) * k + r] = s[r];
}

// Split the keys: dist[b][r] = key >> 32, pos[b][r] = key & (2^32 - 1); a
// missing key, or r past segment b's own k, gives dist 2^32 - 1, pos 2^64 - 1.
__global__ void topk_split_kernel(const uint64_t* __restrict__ keys, uint64_t count, uint32_t k, Segs sg,
                                  uint32_t* __restrict__ dist, uint64_t* __restrict__ pos) {
  const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  uint64_t key = keys[e];
  if (sg.kseg && e % k >= sg.kseg[e / k]) key = kNoKey;  // past the segment's own k
  dist[e] = (uint32_t)(key >> 32);
  pos[e] = key == kNoKey ? kNoKey : (key & 0xffffffffull);
}

// The same with the shared-memory sort passes (k > kTopkMax).
cudaError_t reduce_keys_sorted(const uint64_t* keys, uint32_t B, uint64_t m, int k, uint64_t* a,
                               uint64_t* b, const uint64_t** res, cudaStream_t st) {
  const uint64_t* src = keys;
  uint64_t* dst = a;
  while (true) {
    const uint64_t chunks = (m + kSortKeys - 1) / kSortKeys;
    topk_sort_kernel<false><<<dim3((unsigned)chunks, B), kSortThreads, 0, st>>>(
        src, nullptr, nullptr, Segs{}, m, 0, 0, k, dst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    m = chunks * (uint64_t)k;
    src = dst;
    dst = dst == a ? b : a;
    if (chunks == 1) break;
  }
  *res = src;
  return cudaSuccess;
}

// k smallest of m keys per query, B queries, through chunked passes into
// scratch (ping-pong between a and b); the result ends in *res.
cudaError_t reduce_keys(const uint64_t* keys, uint32_t B, uint64_t m, int k, uint64_t* a, uint64_t* b,
                        const uint64_t** res, cudaStream_t st) {
  const uint64_t chunk = 8192;
  const uint64_t* src = keys;
  uint64_t* dst = a;
  while (true) {
    const uint64_t chunks = (m + chunk - 1) / chunk;
    topk_keys_kernel<<<dim3((unsigned)chunks, B), kTopkThreads, 0, st>>>(src, m, k, chunk, dst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    m = chunks * (uint64_t)k;
    src = dst;
    dst = dst == a ? b : a;
    if (chunks == 1) break;
  }
  *res = src;
  return cudaSuccess;
}

}  // namespace

// Selection over B segments; n is the longest segment (uniform: every
// segment), sg tells where they lie (seg_host: host copy of [5][B]: client
// offsets, server offsets, lengths, winners, bins; staged into the scratch).
static cudaError_t run_topk(const uint32_t* cli, const uint32_t* srv, uint32_t B, uint64_t n, Segs sg,
                            const uint64_t* seg_host, uint64_t t, uint32_t k, uint64_t bins,
                            uint32_t shift, uint32_t* dist, uint64_t* pos, cudaStream_t st) {
  const bool large = k > (uint32_t)kTopkMax;
  const uint64_t chunk = large ? kSortKeys : 1 << 16;
  const uint64_t chunks = n ? (n + chunk - 1) / chunk : 1;
  const uint64_t first = bins ? bins : chunks * k;  // keys per segment after pass 1
  const uint64_t words = 2 * (uint64_t)B * (first + 64);
  const uint64_t seg_words = seg_host ? 5 * (uint64_t)B : 0;
  uint64_t* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, sizeof(uint64_t) * (words + seg_words), st);
  if (e != cudaSuccess) return e;
  uint64_t* a = scratch;
  uint64_t* b = scratch + words / 2;
  if (seg_host) {
    uint64_t* d_seg = scratch + words;
    e = cudaMemcpyAsync(d_seg, seg_host, sizeof(uint64_t) * seg_words, cudaMemcpyHostToDevice, st);
    sg.cli_off = d_seg;
    sg.srv_off = d_seg + B;
    sg.len = d_seg + 2 * (uint64_t)B;
    sg.kseg = d_seg + 3 * (uint64_t)B;
    sg.lseg = bins ? d_seg + 4 * (uint64_t)B : nullptr;
  }
  if (e == cudaSuccess) {
    if (bins) {
      const unsigned per_block = kTopkThreads / 32;
      bin_min_kernel<<<dim3((unsigned)((bins + per_block - 1) / per_block), B), kTopkThreads, 0, st>>>(
          cli, srv, sg, t, bins, shift, a);
    } else if (large) {
      topk_sort_kernel<true><<<dim3((unsigned)chunks, B), kSortThreads, 0, st>>>(nullptr, cli, srv, sg, 0,
                                                                                t, shift, (int)k, a);
    } else {
      topk_shares_kernel<<<dim3((unsigned)chunks, B), kTopkThreads, 0, st>>>(cli, srv, sg, t, (int)k,
                                                                            chunk, shift, a);
    }
    e = cudaGetLastError();
  }
  const uint64_t* res = nullptr;
  // the first pass's keys sit in a; later passes alternate b, a, ..
  if (e == cudaSuccess)
    e = large ? reduce_keys_sorted(a, B, first, (int)k, b, a, &res, st)
              : reduce_keys(a, B, first, (int)k, b, a, &res, st);
  if (e == cudaSuccess) {
    const uint64_t count = (uint64_t)B * k;
    topk_split_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(res, count, k, sg, dist, pos);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  return e != cudaSuccess ? e : e2;
}

cudaError_t launch_topk(const uint32_t* cli, const uint32_t* srv, uint32_t B, uint64_t n, uint64_t t,
                        uint32_t k, uint64_t bins, uint32_t shift, uint32_t* dist, uint64_t* pos,
                        cudaStream_t st) {
  Segs sg{nullptr, nullptr, nullptr, n, nullptr, nullptr};
  return run_topk(cli, srv, B, n, sg, nullptr, t, k, bins, shift, dist, pos, st);
}

cudaError_t launch_topk_segments(const uint32_t* cli, const uint32_t* srv, uint32_t B,
                                 const uint64_t* seg_host, uint64_t t, uint32_t k, uint64_t bins,
                                 uint32_t shift, uint32_t* dist, uint64_t* pos, cudaStream_t st) {
  uint64_t n = 0;
  for (uint32_t b = 0; b < B; ++b) n = seg_host[2 * (uint64_t)B + b] > n ? seg_host[2 * (uint64_t)B + b] : n;
  Segs sg{nullptr, nullptr, nullptr, 0, nullptr, nullptr};
  return run_topk(cli, srv, B, n, sg, seg_host, t, k, bins, shift, dist, pos, st);
}

}  // namespace sanns
