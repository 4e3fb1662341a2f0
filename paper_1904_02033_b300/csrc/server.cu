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
// writes its NTT for every prime into pt[k][j][i][:].
__global__ void __launch_bounds__(512) encode_kernel(PrimeSet P, const uint8_t* __restrict__ coords, uint64_t n_points,
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
    ntt_forward_smem(sa, P, j);
    __syncthreads();
    uint64_t* dst = pt + ((k * P.L + j) * d + i) * N;
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) dst[x] = sa[SP(x)];
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

// Epilogue of the distance step, one block per (b, k, c, j) polynomial of
// ct_out (in place): INTT; for c = 0 add Delta_j ((||p||^2 + r) mod t) per
// coefficient.  r is recovered from the server share written by
// mask_share_kernel; padding positions (pos >= n) draw it directly.
__global__ void __launch_bounds__(256, 3) intt_mask_kernel(PrimeSet P, uint64_t* __restrict__ ct_out,
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
          const uint64_t val = mod_t64((uint64_t)nvv[v] + r[v], t, P.t_barrett);
          const uint32_t x = 4 * u + v;
          sa[SP(x)] = add_mod(sa[SP(x)], mul_shoup(val, dl, dls, q), q);
        }
      }
    }
    __syncthreads();
  }
  store_poly(g, sa, N);
}

}  // namespace

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

cudaError_t launch_encode(const PrimeSet& P, const uint8_t* coords, uint64_t n_points,
                          const uint32_t* perm, uint64_t n, uint32_t d, uint64_t K, uint64_t* pt,
                          uint32_t* norms, int* bad, cudaStream_t st) {
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(encode_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)K, d);
  encode_kernel<<<grid, ntt_threads(P.N), smem, st>>>(P, coords, n_points, perm, n, d, pt, bad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t total = K * P.N;
  norms_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(coords, n_points, perm, n, d,
                                                                 total, norms);
  return cudaGetLastError();
}

cudaError_t launch_intt_mask(const PrimeSet& P, uint64_t* ct_out, const uint32_t* norms,
                             uint32_t B, uint64_t K, uint64_t n, uint64_t pos0, uint64_t mask_seed,
                             const uint64_t* qids, uint32_t* srv_share, cudaStream_t st) {
  const uint64_t polys = (uint64_t)B * K * 2 * P.L;
  if (polys == 0) return cudaSuccess;
  const uint64_t groups = (uint64_t)B * ((n + 3) / 4);
  mask_share_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(P, B, n, pos0, mask_seed,
                                                                     qids, srv_share);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  static bool configured = false;
  if (!configured) {
    e = cudaFuncSetAttribute(intt_mask_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(uint64_t) * ntt_smem_words(kMaxN)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  intt_mask_kernel<<<(unsigned)polys, ntt_threads(P.N), smem, st>>>(P, ct_out, norms, K, n, pos0,
                                                                    mask_seed, qids, srv_share);
  return cudaGetLastError();
}

}  // namespace sanns
