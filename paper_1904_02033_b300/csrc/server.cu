// Server-side kernels around the MAC: standalone NTT/INTT, the database
// encoding (Sec. 5.3: coordinate i of N consecutive permuted points becomes
// one plaintext polynomial, kept in NTT form), and the fused epilogue of the
// distance step (INTT back to coefficient form, + Delta (||p||^2 + r), the
// server's share t - r).
#include "internal.h"

namespace sanns {

namespace {

__host__ __device__ inline uint32_t ntt_threads(uint32_t N) { return N / 16 < 32 ? 32 : (N / 16 > 256 ? 256 : N / 16); }

// One block per polynomial: data [count][L][N], polynomial p uses prime p % L.
__global__ void __launch_bounds__(512) ntt_kernel(PrimeSet P, uint64_t* data, int inverse) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N;
  const uint64_t poly = blockIdx.x;
  const int j = (int)(poly % P.L);
  uint64_t* g = data + poly * N;
  load_poly(sa, g, N);
  __syncthreads();
  if (inverse) ntt_inverse_smem(sa, P, j);
  else ntt_forward_smem(sa, P, j);
  __syncthreads();
  store_poly(g, sa, N);
}

// Encoding: block (k, i) builds coordinate i of positions kN .. kN+N-1 and
// writes its NTT for every prime into pt[k][j][i][:].  Coefficient encoding
// puts point x's coordinate in coefficient x; slot encoding (slots != 0)
// puts it in CRT slot x mod t: the plaintext is the inverse negacyclic
// transform mod t of the coordinates (coefficients in [0, t)), whose NTT is
// then taken for every prime.
__global__ void __launch_bounds__(512) encode_kernel(PrimeSet P, PrimeSet PT, int slots,
                              const uint8_t* __restrict__ coords, uint64_t n_points,
                              const uint32_t* __restrict__ perm, uint64_t n, uint32_t d,
                              uint64_t* __restrict__ pt, int* bad) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N;
  const uint64_t k = blockIdx.x;
  const uint32_t i = blockIdx.y;
  for (uint32_t j = 0; j < P.L; ++j) {
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
      uint64_t pos = k * N + x;
      uint64_t v = 0;
      if (pos < n) {
        uint64_t id = perm ? perm[pos] : pos;
        if (id < n_points) v = coords[id * d + i];
        else if (j == 0) atomicExch(bad, 1);
      }
      sa[SP(x)] = v;
    }
    __syncthreads();
    if (slots) {
      ntt_inverse_smem(sa, PT, 0);
      __syncthreads();
    }
    ntt_forward_smem(sa, P, j);
    __syncthreads();
    uint64_t* dst = pt + ((k * P.L + j) * d + i) * N;
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) dst[x] = split30(sa[SP(x)]);
    __syncthreads();
  }
}

__global__ void norms_kernel(const uint8_t* __restrict__ coords, uint64_t n_points,
                             const uint32_t* __restrict__ perm, uint64_t n, uint32_t d,
                             uint64_t total, uint32_t* __restrict__ norms) {
  uint64_t pos = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (pos >= total) return;
  uint32_t s = 0;
  if (pos < n) {
    uint64_t id = perm ? perm[pos] : pos;
    if (id < n_points) {
      const uint8_t* p = coords + id * d;
      for (uint32_t i = 0; i < d; ++i) s += (uint32_t)p[i] * p[i];
    }
  }
  norms[pos] = s;
}

// Slot encoding of the norms, in place: block k's ||p||^2 values (zero at
// padding positions) become the coefficients of the plaintext whose slots
// they are, so the epilogue adds Delta (that plaintext + the mask polynomial).
__global__ void __launch_bounds__(512) norms_slot_kernel(PrimeSet PT, uint32_t* __restrict__ norms) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = PT.N;
  uint32_t* g = norms + blockIdx.x * (uint64_t)N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) sa[SP(x)] = g[x];
  __syncthreads();
  ntt_inverse_smem(sa, PT, 0);
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) g[x] = (uint32_t)sa[SP(x)];
}

// Slot encoding, the server's shares: the mask is a polynomial R (its
// coefficients drawn as in coefficient encoding, padding positions included),
// so the server's share of slot s is t - NTT_t(R)[s].  One block per (b, k);
// runs after the epilogue, which reads the coefficient shares t - R.
__global__ void __launch_bounds__(512) slot_share_kernel(PrimeSet P, PrimeSet PT, uint64_t K, uint64_t n,
                                                         uint64_t pos0, uint64_t mask_seed,
                                                         const uint64_t* __restrict__ qids,
                                                         uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N;
  const uint64_t bk = blockIdx.x, b = bk / K, k = bk % K;
  const uint64_t qid = qids[b];
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    const uint64_t g0 = pos0 + k * N + 4 * u;
    uint32_t blk[16];
    chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)(g0 / 4), blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      sa[SP(4 * u + v)] = mod_t128(lo, hi, P);
    }
  }
  __syncthreads();
  ntt_forward_smem(sa, PT, 0);
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
    const uint64_t pos = k * N + x;
    if (pos >= n) break;
    const uint64_t r = sa[SP(x)];
    srv_share[b * n + pos] = (uint32_t)(r == 0 ? 0 : P.t - r);
  }
}

// The server's mask, drawn once per position: r = uniform mod t from ChaCha20
// stream (mask_seed, 4, qid_b) at global position pos0 + pos; srv_share[b][pos]
// = (t - r) mod t for pos < n.  One thread per four positions (one ChaCha20
// block; pos0 is a multiple of N, hence of 4).
__global__ void mask_share_kernel(PrimeSet P, uint32_t B, uint64_t n, uint64_t pos0,
                                  uint64_t mask_seed, const uint64_t* __restrict__ qids,
                                  uint32_t* __restrict__ srv_share) {
  const uint64_t groups = (n + 3) / 4;
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (gid >= (uint64_t)B * groups) return;
  const uint64_t b = gid / groups, u = gid % groups;
  uint32_t blk[16];
  chacha20_block(mask_seed, kPurposeMask, qids[b], (uint32_t)(pos0 / 4 + u), blk);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint64_t pos = 4 * u + v;
    if (pos >= n) break;
    uint64_t lo, hi;
    draw_pair(blk, v, lo, hi);
    const uint64_t r = mod_t128(lo, hi, P);
    srv_share[b * n + pos] = (uint32_t)(r == 0 ? 0 : P.t - r);
  }
}

// r of a padding position (global position gpos >= the database size), drawn
// directly from the mask stream; kept out of line so that the unrolled
// epilogue keeps its registers.
__device__ __noinline__ uint64_t mask_draw(const PrimeSet P, uint64_t gpos, uint64_t mask_seed,
                                           uint64_t qid) {
  uint32_t blk[16];
  chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)(gpos / 4), blk);
  uint64_t lo, hi;
  draw_pair(blk, (int)(gpos & 3), lo, hi);
  return mod_t128(lo, hi, P);
}

// Epilogue of the distance step, one block per (b, k, c, j) polynomial of
// ct_out (in place): the inverse NTT back to coefficient form and, for c = 0,
// + Delta_j ((||p||^2 + r) mod t) per coefficient.  The first stage
// (distance 1) runs while the polynomial is loaded, N^-1 is folded into the
// last stage (psi^-brv(1) N^-1 on the difference side, one extra product on
// the sum side), and the last radix-16 pass adds the mask in registers and
// writes the result straight back to global memory.
__global__ void __launch_bounds__(256, 3) intt_mask_kernel(PrimeSet P, uint64_t* __restrict__ ct_out,
                                 const uint32_t* __restrict__ norms, uint64_t K, uint64_t n,
                                 uint64_t pos0g, uint64_t mask_seed, const uint64_t* __restrict__ qids,
                                 const uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L, logN = P.logN;
  const uint64_t poly = blockIdx.x;                 // ((b K + k) 2 + c) L + j
  const uint32_t j = (uint32_t)(poly % L);
  const uint32_t c = (uint32_t)((poly / L) % 2);
  const uint64_t bk = poly / (2 * L);
  const uint64_t kb = bk % K, b = bk / K;
  const uint64_t q = P.q[j], q2 = 2 * q, q4 = 4 * q;  // values stay below 4q
  const ulonglong2* itw = P.itw + (size_t)j * N;
  uint64_t* g = ct_out + poly * N;
  const uint32_t r2 = logN & 3;  // leading radix-2 stages
  if (c == 0 && threadIdx.x == 0) {
    // the mask inputs of this block are read only in the last pass: start
    // pulling them into L2 now (16-byte aligned interior of each range)
    auto prefetch = [](const void* p, uint64_t bytes) {
      const uintptr_t a0 = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
      const uintptr_t a1 = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
      for (uintptr_t a = a0; a + 16 <= a1; a += 32768) {
        const uint32_t len = (uint32_t)(a1 - a < 32768 ? a1 - a : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(len) : "memory");
      }
    };
    prefetch(norms + kb * N, 4ull * N);
    if (kb * N < n) prefetch(srv_share + b * n + kb * N, 4ull * ((kb + 1) * N <= n ? N : n - kb * N));
  }

  // load; for r2 >= 1 the distance-1 stage (pair i = (2i, 2i + 1), twiddle
  // N / 2 + i) on the fly, four pairs in flight per thread
  {
    const ulonglong2* g2 = reinterpret_cast<const ulonglong2*>(g);
    for (uint32_t i0 = 0; i0 < N / 2; i0 += 4 * blockDim.x) {
      ulonglong2 v[4], w[4];
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t i = i0 + z * blockDim.x + threadIdx.x;
        v[z] = i < N / 2 ? __ldg(g2 + i) : make_ulonglong2(0, 0);
        w[z] = (r2 && i < N / 2) ? __ldg(itw + N / 2 + i) : make_ulonglong2(0, 0);
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t i = i0 + z * blockDim.x + threadIdx.x;
        if (i >= N / 2) continue;
        uint64_t X = v[z].x, Y = v[z].y;
        if (r2) inv_bfly4(X, Y, w[z].x, w[z].y, q, q4);
        sa[SP(2 * i)] = X;
        sa[SP(2 * i + 1)] = Y;
      }
    }
  }
  __syncthreads();
  uint32_t lt = r2 ? 1 : 0;
  for (; lt < r2; ++lt) {
    inv_pass2<true>(sa, itw, N, logN, lt, q, q4);
    __syncthreads();
  }
  for (; lt + 4 < logN; lt += 4) {
    inv_pass16<true>(sa, itw, N, logN, lt, q, q4);
    __syncthreads();
  }
  // last radix-16 pass, lt = logN - 4: a thread owns x0 + k N/16, k = 0..15
  const uint32_t t16 = N / 16;
  const uint64_t ni = P.n_inv[j], nis = P.n_inv_shoup[j];
  const uint64_t wl = P.last_inv[j], wls = P.last_inv_shoup[j];
  const uint64_t dl = P.delta[j], dls = P.delta_shoup[j], t = P.t;
  const uint32_t* sh = srv_share + b * n;
  for (uint32_t x0 = threadIdx.x; x0 < t16; x0 += blockDim.x) {
    uint64_t v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = sa[SP(x0 + k * t16)];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int hk = 1 << s;
      const uint32_t base = 1u << (3 - s);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & hk) continue;
        const ulonglong2 w = __ldg(itw + base + (k >> (s + 1)));
        inv_bfly4(v[k], v[k + hk], w.x, w.y, q, q4);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint64_t S = csub(v[k] + v[k + 8], q4);
      const uint64_t D = v[k] - v[k + 8] + q4;
      v[k] = csub(csub(mul_shoup_lazy4(S, ni, nis, q), q2), q);
      v[k + 8] = csub(csub(mul_shoup_lazy4(D, wl, wls, q), q2), q);
    }
    if (c == 0 && (kb + 1) * N <= n) {
      // every position holds a server share
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint64_t pos = kb * N + x0 + k * t16;
        const uint32_t sv = sh[pos];
        const uint64_t r = sv == 0 ? 0 : t - sv;
        const uint64_t val = norm_plus_mask_mod_t(P, norms[pos], r);
        v[k] = add_mod(v[k], mul_shoup_u32((uint32_t)val, dl, dls, q), q);
      }
    } else if (c == 0) {
      // block with padding positions (the last one): element by element
      // through this thread's own shared-memory slots
#pragma unroll
      for (int k = 0; k < 16; ++k) sa[SP(x0 + k * t16)] = v[k];
      for (int k = 0; k < 16; ++k) {
        const uint32_t x = x0 + k * t16;
        const uint64_t pos = kb * N + x;
        uint64_t r;
        if (pos < n) {
          const uint32_t sv = sh[pos];
          r = sv == 0 ? 0 : t - sv;
        } else {
          r = mask_draw(P, pos0g + pos, mask_seed, qids[b]);
        }
        const uint64_t val = norm_plus_mask_mod_t(P, norms[pos], r);
        g[x] = add_mod(sa[SP(x)], mul_shoup_u32((uint32_t)val, dl, dls, q), q);
      }
      continue;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) g[x0 + k * t16] = v[k];
  }
}

// The same epilogue as separate shared-memory passes (INTT, then the mask,
// then the store), which finishes a polynomial sooner: used when the launch
// is at most a couple of waves, where the latency of each block decides.
// r is recovered from the server share written by mask_share_kernel; padding
// positions (pos >= n) draw it directly.
__global__ void __launch_bounds__(256, 3) intt_mask_short_kernel(PrimeSet P, uint64_t* __restrict__ ct_out,
                                 const uint32_t* __restrict__ norms, uint64_t K, uint64_t n,
                                 uint64_t pos0g, uint64_t mask_seed, const uint64_t* __restrict__ qids,
                                 const uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L;
  const uint64_t poly = blockIdx.x;                 // ((b K + k) 2 + c) L + j
  const uint32_t j = (uint32_t)(poly % L);
  const uint32_t c = (uint32_t)((poly / L) % 2);
  const uint64_t bk = poly / (2 * L);
  const uint64_t k = bk % K, b = bk / K;
  uint64_t* g = ct_out + poly * N;
  load_poly(sa, g, N);
  __syncthreads();
  ntt_inverse_smem(sa, P, j);
  __syncthreads();
  if (c == 0) {
    const uint64_t q = P.q[j], dl = P.delta[j], dls = P.delta_shoup[j], t = P.t;
    const uint32_t* sh = srv_share + b * n;
    // four positions per thread per round; all loads of a round are issued
    // before any is used
    for (uint32_t u0 = 0; u0 < N / 4; u0 += 4 * blockDim.x) {
      uint4 nv[4], sv[4];
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t u = u0 + z * blockDim.x + threadIdx.x;
        const uint64_t pos0 = k * N + 4 * u;
        nv[z] = u < N / 4 ? __ldg(reinterpret_cast<const uint4*>(norms + pos0)) : make_uint4(0, 0, 0, 0);
        // server shares exist only below n; n need not be a multiple of 4
        if (u < N / 4 && pos0 + 3 < n && (reinterpret_cast<uintptr_t>(sh + pos0) & 15) == 0)
          sv[z] = __ldg(reinterpret_cast<const uint4*>(sh + pos0));
        else if (u < N / 4 && pos0 + 3 < n)
          sv[z] = make_uint4(sh[pos0], sh[pos0 + 1], sh[pos0 + 2], sh[pos0 + 3]);
        else
          sv[z] = make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t u = u0 + z * blockDim.x + threadIdx.x;
        if (u >= N / 4) continue;
        const uint64_t pos0 = k * N + 4 * u;
        uint64_t r[4];
        if (pos0 + 3 < n) {
          const uint32_t svv[4] = {sv[z].x, sv[z].y, sv[z].z, sv[z].w};
#pragma unroll
          for (int v = 0; v < 4; ++v) r[v] = svv[v] == 0 ? 0 : t - svv[v];
        } else {
          uint32_t blk[16];
          chacha20_block(mask_seed, kPurposeMask, qids[b], (uint32_t)((pos0g + pos0) / 4), blk);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            uint64_t lo, hi;
            draw_pair(blk, v, lo, hi);
            r[v] = mod_t128(lo, hi, P);
          }
        }
        const uint32_t nvv[4] = {nv[z].x, nv[z].y, nv[z].z, nv[z].w};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint64_t val = norm_plus_mask_mod_t(P, nvv[v], r[v]);
          const uint32_t x = 4 * u + v;
          sa[SP(x)] = add_mod(sa[SP(x)], mul_shoup_u32((uint32_t)val, dl, dls, q), q);
        }
      }
    }
    __syncthreads();
  }
  store_poly(g, sa, N);
}

// ------------------------------------------------------------------------
// Few polynomials (one query over a small database): each polynomial's
// epilogue on a cluster of four CTAs, so that its transform spreads over four
// SMs instead of waiting on one.  With M = N / 4, CTA r holds quarter r
// (positions rM .. rM + M - 1) in shared memory and runs the stages of
// distance below M on it (radix-4 register passes, the global twiddle index
// of each pair group being r M / 2^(lt+1) + its local index).  The stages of
// distance M and N/2 mix the quarters: after a cluster barrier, CTA r reads
// the four quarters' values at its own offsets through distributed shared
// memory and computes its quarter of the output,
//   stage M:    X0' = X0 + X1, X1' = (X0 - X1) w[2], X2' = X2 + X3,
//               X3' = (X2 - X3) w[3];
//   stage N/2:  out0 = (X0' + X2') N^-1, out2 = (X0' - X2') psi^-brv(1) N^-1,
//               out1, out3 likewise from X1', X3';
// then, for c = 0, adds Delta ((||p||^2 + r) mod t) and writes the server
// share from the j = 0 polynomial.  The mask r is drawn in the kernel (one
// ChaCha20 block per four positions, as mask_share_kernel does) by warps of
// its own while the other warps run the local stages.  A second cluster
// barrier keeps every CTA's shared memory alive until the others have read
// it.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The same barrier without ordering of memory accesses: enough where it only
// has to hold a CTA until the others have consumed (used) what they loaded
// from its shared memory.
__device__ __forceinline__ void cl_sync_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\nbarrier.cluster.wait.aligned;" ::: "memory");
}

// Two consecutive 64-bit words (16-byte aligned) from CTA `rank`'s copy of
// the shared memory at `local`; issued after the cluster barrier that made
// them visible, so the compiler may schedule these loads freely.
__device__ __forceinline__ ulonglong2 ld_cluster2(const uint64_t* local, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  ulonglong2 v;
  asm("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(ra));
  return v;
}

// bar.sync on barrier 1 for the data warps alone (warps 0 .. 7)
__device__ __forceinline__ void data_warps_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

constexpr uint32_t kClusterIntt = 4;
// warps 0 .. 7 load the quarter and run its local stages while warps 8 .. 15
// draw the mask terms (c = 0); all sixteen run the cross-quarter stages
constexpr uint32_t kClusterThreads = 512, kClusterDataThreads = 256;

// the cluster kernel's padded quarter keeps even pairs 16-byte aligned (two
// spare words after every 16)
__host__ __device__ __forceinline__ uint32_t SPC(uint32_t x) { return x + 2 * (x >> 4); }

// shared-memory words of the cluster kernel for a ring of N: the padded
// quarter, the quarter's twiddle pairs of every local stage (M - 1 pairs), the
// mask term of each of its M positions and their 32-bit server shares
__host__ __device__ __forceinline__ uint32_t cluster_intt_smem_words(uint32_t N) {
  const uint32_t M = N / kClusterIntt;
  return M + M / 8 + 2 * (M - 1) + M + M / 2;
}

__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(kClusterThreads, 1)
    intt_mask_cluster_kernel(PrimeSet P, uint64_t* __restrict__ ct_out, const uint32_t* __restrict__ norms,
                             uint64_t K, uint64_t n, uint64_t pos0g, uint64_t mask_seed,
                             const uint64_t* __restrict__ qids, uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L, logN = P.logN;
  const uint32_t M = N / kClusterIntt, logM = logN - 2;
  ulonglong2* tws = reinterpret_cast<ulonglong2*>(sa + M + M / 8);   // 16-byte aligned: M + M/8 even
  uint64_t* mval = sa + M + M / 8 + 2 * (M - 1);
  uint32_t* shs = reinterpret_cast<uint32_t*>(mval + M);
  const uint32_t r = cl_rank();
  const uint64_t poly = blockIdx.x / kClusterIntt;  // ((b K + k) 2 + c) L + j
  const uint32_t j = (uint32_t)(poly % L);
  const uint32_t c = (uint32_t)((poly / L) % 2);
  const uint64_t bk = poly / (2 * L);
  const uint64_t k = bk % K, b = bk / K;
  const uint64_t q = P.q[j], q2 = 2 * q, q4 = 4 * q;  // values stay below 4q
  const ulonglong2* itw = P.itw + (size_t)j * N;
  uint64_t* g = ct_out + poly * N;
  const uint32_t tid = threadIdx.x;

  if (tid < kClusterDataThreads) {
    // the quarter and the twiddles of its local stages (stage lt uses the
    // M / 2^(lt+1) pairs from N / 2^(lt+1) + r M / 2^(lt+1), kept from pair
    // M - M / 2^lt of tws), two data pairs and four twiddle pairs per thread
    // requested before any is stored
    for (uint32_t base = 0; 2 * base < M / 2 || 4 * base + 1 < M; base += kClusterDataThreads) {
      ulonglong2 dv[2], tv[4];
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        const uint32_t x = 2 * (2 * base + tid + z * kClusterDataThreads);
        dv[z] = x < M ? __ldg(reinterpret_cast<const ulonglong2*>(g + (uint64_t)r * M + x)) : make_ulonglong2(0, 0);
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        // flat index f of the stage-major twiddle copy: stage lt holds pairs
        // [M - M / 2^lt, M - M / 2^(lt+1)), i.e. lt = log2 M - ceil(log2 (M - f))
        const uint32_t f = 4 * base + tid + z * kClusterDataThreads;
        if (f + 1 < M) {
          const uint32_t lt = logM - (32 - __clz(M - f - 1));
          const uint32_t cnt = M >> (lt + 1), e = f - (M - (M >> lt));
          tv[z] = __ldg(itw + (N >> (lt + 1)) + r * cnt + e);
        }
      }
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        const uint32_t x = 2 * (2 * base + tid + z * kClusterDataThreads);
        if (x < M) *reinterpret_cast<ulonglong2*>(sa + SPC(x)) = dv[z];
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t f = 4 * base + tid + z * kClusterDataThreads;
        if (f + 1 < M) tws[f] = tv[z];
      }
    }
    data_warps_sync();
    // stages of distance 2^lt < M on the quarter: radix-4 passes (stages lt
    // and lt + 1), a radix-2 stage when log2 M is odd
    uint32_t lt = 0;
    for (; lt + 2 <= logM; lt += 2) {
      const ulonglong2* t0 = tws + (M - (M >> lt));
      const ulonglong2* t1 = tws + (M - (M >> (lt + 1)));
      for (uint32_t th = tid; th < M / 4; th += kClusterDataThreads) {
        const uint32_t gl = th >> lt, bl = th & ((1u << lt) - 1);
        const uint32_t x0 = (gl << (lt + 2)) + bl;
        uint64_t v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = sa[SPC(x0 + (e << lt))];
        const ulonglong2 wa = t0[2 * gl], wb = t0[2 * gl + 1], wc = t1[gl];
        inv_bfly4(v[0], v[1], wa.x, wa.y, q, q4);
        inv_bfly4(v[2], v[3], wb.x, wb.y, q, q4);
        inv_bfly4(v[0], v[2], wc.x, wc.y, q, q4);
        inv_bfly4(v[1], v[3], wc.x, wc.y, q, q4);
#pragma unroll
        for (int e = 0; e < 4; ++e) sa[SPC(x0 + (e << lt))] = v[e];
      }
      data_warps_sync();
    }
    if (lt < logM) {
      const uint32_t t = 1u << lt;
      const ulonglong2* t0 = tws + (M - (M >> lt));
      for (uint32_t bf = tid; bf < M / 2; bf += kClusterDataThreads) {
        const uint32_t i = bf >> lt, x = (i << (lt + 1)) + (bf & (t - 1));
        uint64_t X = sa[SPC(x)], Y = sa[SPC(x + t)];
        const ulonglong2 w = t0[i];
        inv_bfly4(X, Y, w.x, w.y, q, q4);
        sa[SPC(x)] = X;
        sa[SPC(x + t)] = Y;
      }
    }
  } else if (c == 0) {
    // mask terms Delta ((||p||^2 + r) mod t) and the shares t - r of the
    // quarter's positions, four per ChaCha20 block, meanwhile
    const uint64_t dl = P.delta[j], dls = P.delta_shoup[j], t = P.t;
    const uint64_t qid = qids[b];
    for (uint32_t u0 = 4 * (tid - kClusterDataThreads); u0 < M; u0 += 4 * (kClusterThreads - kClusterDataThreads)) {
      const uint64_t pos = k * N + (uint64_t)r * M + u0;
      const uint4 nv = __ldg(reinterpret_cast<const uint4*>(norms + pos));
      uint32_t blk[16];
      chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)((pos0g + pos) / 4), blk);
      const uint32_t nvv[4] = {nv.x, nv.y, nv.z, nv.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        uint64_t lo, hi;
        draw_pair(blk, v, lo, hi);
        const uint64_t rv = mod_t128(lo, hi, P);
        mval[u0 + v] = mul_shoup_u32((uint32_t)norm_plus_mask_mod_t(P, nvv[v], rv), dl, dls, q);
        shs[u0 + v] = (uint32_t)(rv == 0 ? 0 : t - rv);
      }
    }
  }
  cl_sync();  // every quarter's local stages (and mask terms) done and visible to the cluster

  const ulonglong2 w2 = __ldg(itw + 2), w3 = __ldg(itw + 3);
  const uint64_t ni = P.n_inv[j], nis = P.n_inv_shoup[j];
  const uint64_t wl = P.last_inv[j], wls = P.last_inv_shoup[j];
  for (uint32_t u0 = 2 * tid; u0 < M; u0 += 2 * kClusterThreads) {
    ulonglong2 X[4];  // the four quarters' values at offsets u0, u0 + 1
#pragma unroll
    for (uint32_t qi = 0; qi < 4; ++qi) X[qi] = ld_cluster2(sa + SPC(u0), qi);
    uint64_t out[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const uint64_t x0 = v ? X[0].y : X[0].x, x1 = v ? X[1].y : X[1].x;
      const uint64_t x2 = v ? X[2].y : X[2].x, x3 = v ? X[3].y : X[3].x;
      uint64_t A, B;
      if ((r & 1) == 0) {  // sum sides of the stage of distance M
        A = csub(x0 + x1, q4);
        B = csub(x2 + x3, q4);
      } else {             // difference sides
        A = mul_shoup_lazy4(x0 - x1 + q4, w2.x, w2.y, q);
        B = mul_shoup_lazy4(x2 - x3 + q4, w3.x, w3.y, q);
      }
      const uint64_t y = r < 2 ? mul_shoup_lazy4(csub(A + B, q4), ni, nis, q)
                               : mul_shoup_lazy4(A - B + q4, wl, wls, q);
      out[v] = csub(csub(y, q2), q);
      if (c == 0) out[v] = add_mod(out[v], mval[u0 + v], q);
    }
    const uint32_t x = r * M + u0;
    *reinterpret_cast<ulonglong2*>(g + x) = make_ulonglong2(out[0], out[1]);
    if (c == 0 && j == 0) {
      const uint64_t pos = k * N + x;
      if (pos < n) srv_share[b * n + pos] = shs[u0];
      if (pos + 1 < n) srv_share[b * n + pos + 1] = shs[u0 + 1];
    }
  }
  cl_sync_relaxed();  // the other CTAs have finished reading this CTA's quarter
}

// NTT-form responses: the response is the NTT of the coefficient-form one.
// Since the transform is linear, c0 = acc0 + NTT(Delta_j v) with v = (||p||^2
// + r) mod t per position, and c1 = acc1: one forward transform per (b, k, j)
// instead of two inverse ones.  With circuit privacy (after the
// re-randomisation in the NTT domain) e1 joins c0's transform and c1 gets
// NTT(e2).  One block per (b, k, c, j), c < comps (1 without privacy, 2 with).
__global__ void __launch_bounds__(256, 3) mask_ntt_kernel(PrimeSet P, uint64_t* __restrict__ ct_out,
                                const uint32_t* __restrict__ norms, uint64_t K, uint64_t n,
                                uint64_t pos0g, uint64_t mask_seed, const uint64_t* __restrict__ qids,
                                const uint32_t* __restrict__ srv_share, uint32_t comps, int privacy,
                                uint32_t F, PrivacyConsts C) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L;
  const uint64_t idx = blockIdx.x;                  // ((b K + k) comps + c) L + j
  const uint32_t j = (uint32_t)(idx % L);
  const uint32_t c = (uint32_t)((idx / L) % comps);
  const uint64_t bk = idx / ((uint64_t)L * comps);
  const uint64_t k = bk % K, b = bk / K;
  const uint64_t q = P.q[j], t = P.t;
  const uint64_t qid = qids[b];
  const uint32_t* sh = srv_share + b * n;
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    const uint64_t p4 = k * N + 4 * u;             // first of four positions
    uint64_t val[4] = {0, 0, 0, 0};
    if (c == 0) {
      uint64_t r[4];
      if (p4 + 3 < n) {
#pragma unroll
        for (int v = 0; v < 4; ++v) r[v] = sh[p4 + v] == 0 ? 0 : t - sh[p4 + v];
      } else {
        uint32_t blk[16];
        chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)((pos0g + p4) / 4), blk);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          uint64_t lo, hi;
          draw_pair(blk, v, lo, hi);
          r[v] = mod_t128(lo, hi, P);
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint64_t m = norm_plus_mask_mod_t(P, norms[p4 + v], r[v]);
        val[v] = mul_shoup(m, P.delta[j], P.delta_shoup[j], q);
      }
    }
    if (privacy) {
      const uint32_t ctr = (uint32_t)((pos0g + p4) / 4);
      if (c == 0) {
        uint32_t ba[16], bb[16];
        chacha20_block(mask_seed, kPurposeFloodLo, qid, ctr, ba);
        chacha20_block(mask_seed, kPurposeFloodHi, qid, ctr, bb);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          uint64_t w[4];
          draw_pair(ba, v, w[0], w[1]);
          draw_pair(bb, v, w[2], w[3]);
          val[v] = add_mod(val[v], flood_e1(w, F, q, C.q_barrett[j], P.r64[j], P.r64_shoup[j], C.two_f[j]), q);
        }
      } else {
        uint32_t be[16];
        chacha20_block(mask_seed, kPurposeE2, qid, ctr, be);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          uint64_t lo, hi;
          draw_pair(be, v, lo, hi);
          const int e2 = cbd21_of(lo);
          val[v] = e2 < 0 ? q - (uint64_t)(-e2) : (uint64_t)e2;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) sa[SP(4 * u + v)] = val[v];
  }
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  uint64_t* g = ct_out + ((bk * 2 + c) * L + j) * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) g[x] = add_mod(g[x], sa[SP(x)], q);
}

// NTT-form responses without circuit privacy, fused: c0 = acc0 + NTT(Delta_j
// v) with v = (||p||^2 + r) mod t per position; c1 is acc1 untouched, so one
// block per (b, k, j) and c = 0 only.  The mask values are built straight
// into the first butterfly stage (distance N/2), values stay lazily below 4q
// between passes, and the last radix-16 pass (16 consecutive slots per
// thread) adds the canonical transform to acc0 in global memory: two
// shared-memory passes and two block barriers fewer than building, then
// transforming, then adding.
__global__ void __launch_bounds__(256, 3) mask_ntt_fused_kernel(PrimeSet P, uint64_t* __restrict__ ct_out,
                                      const uint32_t* __restrict__ norms, uint64_t K, uint64_t n,
                                      uint64_t pos0g, uint64_t mask_seed,
                                      const uint64_t* __restrict__ qids,
                                      const uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L, logN = P.logN;
  const uint64_t idx = blockIdx.x;                  // (b K + k) L + j
  const uint32_t j = (uint32_t)(idx % L);
  const uint64_t bk = idx / L;
  const uint64_t k = bk % K, b = bk / K;
  const uint64_t q = P.q[j], q2 = 2 * q, t = P.t;
  const uint64_t qid = qids[b];
  const uint32_t* sh = srv_share + b * n;
  const ulonglong2* tw = P.tw + (size_t)j * N;
  const uint64_t dl = P.delta[j], dls = P.delta_shoup[j];
  if (threadIdx.x == 0) {
    // the accumulator row is read only at the end: start pulling it into L2
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(ct_out + (bk * 2 * L + j) * N);
    for (uint32_t off = 0; off < N * 8u; off += 32768u) {
      const uint32_t len = N * 8u - off < 32768u ? N * 8u - off : 32768u;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0 + off), "r"(len) : "memory");
    }
  }
  // the value at slot x from its raw inputs (norm, share), which the loops
  // below load for several slots at once so that their latencies overlap
  auto value = [&](uint32_t x, uint32_t nv, uint32_t sv) -> uint32_t {   // (||p||^2 + r) mod t
    const uint64_t pos = k * N + x;
    uint64_t r;
    if (pos < n) r = sv == 0 ? 0 : t - sv;
    else r = mask_draw(P, pos0g + pos, mask_seed, qid);
    return (uint32_t)norm_plus_mask_mod_t(P, nv, r);
  };
  const uint64_t dw = P.delta_w1[j], dws = P.delta_w1_shoup[j];
  const uint32_t* nk = norms + k * N;
  const uint64_t valid = n > k * N ? n - k * N : 0;      // slots of this block with a share
  const uint32_t r2 = logN & 3;  // leading radix-2 stages
  if (r2) {
    // stage 0: distance N/2, twiddle psi^brv(1) for every pair, with Delta
    // folded in: X = Delta v_x + (Delta psi^brv(1)) v_{x+N/2}, two products
    // of 32-bit values per pair; four pairs (eight slots) in flight per thread
    for (uint32_t x0 = threadIdx.x; x0 < N / 2; x0 += 4 * blockDim.x) {
      uint32_t nv[8], sv[8];
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t x = x0 + z * blockDim.x;
        if (x < N / 2) {
          nv[z] = __ldg(nk + x);
          nv[z + 4] = __ldg(nk + x + N / 2);
          sv[z] = x < valid ? __ldg(sh + k * N + x) : 0;
          sv[z + 4] = x + N / 2 < valid ? __ldg(sh + k * N + x + N / 2) : 0;
        }
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t x = x0 + z * blockDim.x;
        if (x < N / 2) {
          const uint64_t X = mul_shoup_u32(value(x, nv[z], sv[z]), dl, dls, q);
          const uint64_t T = mul_shoup_u32_lazy(value(x + N / 2, nv[z + 4], sv[z + 4]), dw, dws, q);
          sa[SP(x)] = X + T;               // below 3q
          sa[SP(x + N / 2)] = X - T + q2;  // below 3q
        }
      }
    }
  } else {
    for (uint32_t x0 = threadIdx.x; x0 < N; x0 += 8 * blockDim.x) {
      uint32_t nv[8], sv[8];
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        const uint32_t x = x0 + z * blockDim.x;
        if (x < N) {
          nv[z] = __ldg(nk + x);
          sv[z] = x < valid ? __ldg(sh + k * N + x) : 0;
        }
      }
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        const uint32_t x = x0 + z * blockDim.x;
        if (x < N) sa[SP(x)] = mul_shoup_u32(value(x, nv[z], sv[z]), dl, dls, q);
      }
    }
  }
  __syncthreads();
  uint32_t lt = logN - 1 - (r2 ? 1 : 0);
  for (uint32_t st = 1; st < r2; ++st, --lt) {
    const uint32_t tt = 1u << lt, m = 1u << st;
    for (uint32_t bf = threadIdx.x; bf < N / 2; bf += blockDim.x) {
      const uint32_t i = bf >> lt, x = (i << (lt + 1)) + (bf & (tt - 1));
      uint64_t X = sa[SP(x)], Y = sa[SP(x + tt)];
      const ulonglong2 w = __ldg(tw + m + i);
      fwd_bfly(X, Y, w.x, w.y, q, q2);
      sa[SP(x)] = X;
      sa[SP(x + tt)] = Y;
    }
    __syncthreads();
  }
  // radix-16 passes but the last (stages t, t/2, t/4, t/8 with t = 2^lt)
  for (; lt > 3; lt -= 4) {
    const uint32_t ls = lt - 3, S = 1u << ls;
    const uint32_t m0 = 1u << (logN - 1 - lt);
    for (uint32_t th = threadIdx.x; th < N / 16; th += blockDim.x) {
      const uint32_t g = th >> ls, bb = th & (S - 1);
      const uint32_t x0 = (g << (lt + 1)) + bb;
      uint64_t v[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) v[kk] = sa[SP(x0 + (kk << ls))];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int hk = 8 >> s;
        const uint32_t base = (m0 << s) + (g << s);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          if (kk & hk) continue;
          const ulonglong2 w = __ldg(tw + base + (kk >> (4 - s)));
          fwd_bfly(v[kk], v[kk + hk], w.x, w.y, q, q2);
        }
      }
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) sa[SP(x0 + (kk << ls))] = v[kk];
    }
    __syncthreads();
  }
  // last pass, lt = 3: a thread owns the 16 consecutive slots x0 = 16 th ..,
  // written back canonical; then the add to acc0 with coalesced 16-byte
  // accesses (consecutive threads, consecutive slot pairs)
  const uint32_t m0 = 1u << (logN - 4);
  for (uint32_t th = threadIdx.x; th < N / 16; th += blockDim.x) {
    const uint32_t x0 = th << 4;
    uint64_t v[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) v[kk] = sa[SP(x0 + kk)];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int hk = 8 >> s;
      const uint32_t base = (m0 << s) + (th << s);
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        if (kk & hk) continue;
        const ulonglong2 w = __ldg(tw + base + (kk >> (4 - s)));
        fwd_bfly(v[kk], v[kk + hk], w.x, w.y, q, q2);
      }
    }
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) sa[SP(x0 + kk)] = csub(csub(v[kk], q2), q);
  }
  __syncthreads();
  ulonglong2* gv = reinterpret_cast<ulonglong2*>(ct_out + (bk * 2 * L + j) * N);   // component 0
  // four 16-byte words of the accumulator row in flight per thread
  for (uint32_t i0 = threadIdx.x; i0 < N / 2; i0 += 4 * blockDim.x) {
    ulonglong2 a[4];
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const uint32_t i = i0 + z * blockDim.x;
      if (i < N / 2) a[z] = gv[i];
    }
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const uint32_t i = i0 + z * blockDim.x;
      if (i < N / 2) {
        a[z].x = add_mod(a[z].x, sa[SP(2 * i)], q);
        a[z].y = add_mod(a[z].y, sa[SP(2 * i + 1)], q);
        gv[i] = a[z];
      }
    }
  }
}

// Imported norms reduced mod t in place, so that every stored norm is below t
// (the mask epilogues rely on it when the context's norms_below_t is set).
__global__ void norms_mod_t_kernel(PrimeSet P, uint32_t* __restrict__ norms, uint64_t count) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < count) norms[i] = (uint32_t)mod_t64(norms[i], P.t, P.t_barrett);
}

}  // namespace

cudaError_t launch_norms_mod_t(const PrimeSet& P, uint32_t* norms, uint64_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  norms_mod_t_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(P, norms, count);
  return cudaGetLastError();
}

cudaError_t launch_ntt(const PrimeSet& P, uint64_t* data, uint64_t count, bool inverse,
                       cudaStream_t st) {
  const uint64_t polys = count * P.L;
  if (polys == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(ntt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ntt_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(P, data, inverse ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_encode(const PrimeSet& P, const PrimeSet* PT, const uint8_t* coords, uint64_t n_points,
                          const uint32_t* perm, uint64_t n, uint32_t d, uint64_t K, uint64_t* pt,
                          uint32_t* norms, int* bad, cudaStream_t st) {
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(encode_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)K, d);
  encode_kernel<<<grid, ntt_threads(P.N), smem, st>>>(P, PT ? *PT : P, PT ? 1 : 0, coords, n_points, perm,
                                                      n, d, pt, bad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t total = K * P.N;
  norms_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(coords, n_points, perm, n, d,
                                                                 total, norms);
  e = cudaGetLastError();
  if (e != cudaSuccess || !PT) return e;
  e = cudaFuncSetAttribute(norms_slot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  norms_slot_kernel<<<(unsigned)K, ntt_threads(P.N), smem, st>>>(*PT, norms);
  return cudaGetLastError();
}

__global__ void join30_kernel(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst, uint64_t count) {
  const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e < count) dst[e] = join30(src[e]);
}

// Imported plaintexts, in place: canonical residues [K][L][d][N] -> the
// split30 storage format; a value >= q_j of its prime raises *bad.
__global__ void import_pt_kernel(PrimeSet P, uint64_t* __restrict__ pt, uint64_t count, uint32_t d,
                                 int* bad) {
  const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  const uint32_t j = (uint32_t)((e / ((uint64_t)d * P.N)) % P.L);
  const uint64_t v = pt[e];
  if (v >= P.q[j]) {
    atomicExch(bad, 1);
    pt[e] = 0;
  } else {
    pt[e] = split30(v);
  }
}

cudaError_t launch_import_pt(const PrimeSet& P, uint64_t* pt, uint64_t count, uint32_t d, int* bad,
                             cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  import_pt_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(P, pt, count, d, bad);
  return cudaGetLastError();
}

cudaError_t launch_join30(const uint64_t* src, uint64_t* dst, uint64_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  join30_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_norms_slot(const PrimeSet& PT, uint32_t* norms, uint64_t K, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(PT.N);
  cudaError_t e = ensure_smem_attr((const void*)norms_slot_kernel, smem);
  if (e != cudaSuccess) return e;
  norms_slot_kernel<<<(unsigned)K, ntt_threads(PT.N), smem, st>>>(PT, norms);
  return cudaGetLastError();
}

cudaError_t launch_slot_share(const PrimeSet& P, const PrimeSet& PT, uint32_t B, uint64_t K, uint64_t n,
                              uint64_t pos0, uint64_t mask_seed, const uint64_t* qids,
                              uint32_t* srv_share, cudaStream_t st) {
  if ((uint64_t)B * K == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(slot_share_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  slot_share_kernel<<<(unsigned)((uint64_t)B * K), ntt_threads(P.N), smem, st>>>(P, PT, K, n, pos0, mask_seed,
                                                                                  qids, srv_share);
  return cudaGetLastError();
}

cudaError_t launch_intt_mask(const PrimeSet& P, uint64_t* ct_out, const uint32_t* norms,
                             uint32_t B, uint64_t K, uint64_t n, uint64_t pos0, uint64_t mask_seed,
                             const uint64_t* qids, uint32_t* srv_share, int sms, cudaStream_t st) {
  const uint64_t polys = (uint64_t)B * K * 2 * P.L;
  if (polys == 0) return cudaSuccess;
  // few polynomials: four SMs per polynomial, the mask drawn in the same
  // kernel (all clusters resident at once)
  if (polys * kClusterIntt <= (uint64_t)(sms > 0 ? sms : 148) && P.N >= 1024 && P.N <= 16384) {
    const size_t csmem = sizeof(uint64_t) * cluster_intt_smem_words(P.N);
    cudaError_t e = ensure_smem_attr((const void*)intt_mask_cluster_kernel, csmem);
    if (e != cudaSuccess) return e;
    intt_mask_cluster_kernel<<<(unsigned)(polys * kClusterIntt), kClusterThreads, csmem, st>>>(
        P, ct_out, norms, K, n, pos0, mask_seed, qids, srv_share);
    return cudaGetLastError();
  }
  const uint64_t groups = (uint64_t)B * ((n + 3) / 4);
  mask_share_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(P, B, n, pos0, mask_seed,
                                                                     qids, srv_share);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  e = ensure_smem_attr((const void*)intt_mask_kernel, smem);
  if (e == cudaSuccess) e = ensure_smem_attr((const void*)intt_mask_short_kernel, smem);
  if (e != cudaSuccess) return e;
  // three blocks per SM; up to two waves the per-block latency decides, past
  // that the throughput of the fused kernel
  if (polys <= 2ull * 3 * (uint64_t)(sms > 0 ? sms : 148))
    intt_mask_short_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(
        P, ct_out, norms, K, n, pos0, mask_seed, qids, srv_share);
  else
    intt_mask_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(P, ct_out, norms, K, n, pos0,
                                                                      mask_seed, qids, srv_share);
  return cudaGetLastError();
}

cudaError_t launch_mask_ntt(const PrimeSet& P, uint64_t* ct_out, const uint32_t* norms, uint32_t B,
                            uint64_t K, uint64_t n, uint64_t pos0, uint64_t mask_seed, const uint64_t* qids,
                            uint32_t* srv_share, bool privacy, uint32_t F, const PrivacyConsts& C,
                            cudaStream_t st) {
  const uint32_t comps = privacy ? 2 : 1;
  const uint64_t polys = (uint64_t)B * K * comps * P.L;
  if (polys == 0) return cudaSuccess;
  const uint64_t groups = (uint64_t)B * ((n + 3) / 4);
  mask_share_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(P, B, n, pos0, mask_seed,
                                                                     qids, srv_share);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  if (!privacy) {
    e = ensure_smem_attr((const void*)mask_ntt_fused_kernel, smem);
    if (e != cudaSuccess) return e;
    mask_ntt_fused_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(P, ct_out, norms, K, n, pos0,
                                                                           mask_seed, qids, srv_share);
    return cudaGetLastError();
  }
  e = ensure_smem_attr((const void*)mask_ntt_kernel, smem);
  if (e != cudaSuccess) return e;
  mask_ntt_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(P, ct_out, norms, K, n, pos0, mask_seed,
                                                                   qids, srv_share, comps, privacy ? 1 : 0,
                                                                   F, C);
  return cudaGetLastError();
}

}  // namespace sanns
