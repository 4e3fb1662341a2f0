// K4: distances for the clustering protocol (Pi_cl steps 5-8 / Algorithm 4's
// "for p in C u S: d_p = ||q - p||^2" over the retrieved clusters).  Each
// query b probes P clusters; the points of those clusters, concatenated in
// probe order with members ascending, form the query's own gathered list of
// n_b points.  That list is treated exactly like a permuted database in the
// linear scan: blocks of N positions (zero padded), one plaintext polynomial
// per (block, dimension, prime), ct x pt MAC over the d dimensions, INTT,
// + Delta (||p||^2 + r), server share t - r.  The paper fetches the points as
// secret shares through DORAM; here the server holds them in the clear.
//
// Two launches:
//   pack        one thread per gathered position: finds the probe segment by
//               binary search, copies the point's d bytes into a
//               coordinate-major tile [item][i][x] and its ||p||^2;
//   persistent  three blocks per multiprocessor walk the units (work item,
//               prime j, slice of the dimensions) of every query -- uneven
//               per-query counts included: the slice's encodings (NTT of the
//               coordinate polynomials) times the query's c0 and c1, summed
//               mod q_j into the unit's partial-sum slab in global memory
//               (at most 32 slices per item and prime).  The block that completes
//               the last slice of an (item, prime) (a ticket counter after a
//               memory fence; nobody waits) sums the partials mod q_j (the
//               order does not matter, so the result is exact), runs the
//               INTT, adds Delta (||p||^2 + r) to c0, stores both components
//               and the server share t - r.  Slices are sized so that even a
//               single work item spreads over every multiprocessor.
// A work item is one block of N positions of one query's gathered list.
// Each query's list is treated as a database of its own (positions from 0),
// so with circuit privacy the finishing block adds pk * NTT(u) before the
// INTT and the flooding terms e1, e2 after it, drawn at the list positions;
// with slot encoding the coordinates and norms go through the inverse
// transform mod t first and a last pass writes the slot shares.
#include <cstring>
#include <vector>

#include "internal.h"

namespace sanns {

namespace {

__global__ void check_indices_kernel(const uint32_t* idx, uint64_t m, uint64_t bound, int* bad) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < m && idx[i] >= bound) atomicExch(bad, 1);
}

struct GatherItem {
  uint32_t b;       // query
  uint32_t kb;      // block within the query's gathered list
  uint64_t blk;     // output block index (query-major)
};

struct GatherQuery {
  uint64_t n;       // gathered points
  uint64_t pos_off; // offset of the query's positions in srv_share / ids
};

__global__ void pack_kernel(uint32_t N, uint32_t d, uint64_t W, const GatherItem* __restrict__ items,
                            const GatherQuery* __restrict__ qs, const uint64_t* __restrict__ seg,
                            const uint32_t* __restrict__ probes, uint32_t P,
                            const uint64_t* __restrict__ offsets, const uint32_t* __restrict__ members,
                            const uint8_t* __restrict__ coords, uint8_t* __restrict__ gco,
                            uint32_t* __restrict__ gnorm, uint32_t* __restrict__ ids) {
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (gid >= W * N) return;
  const uint64_t w = gid / N;
  const uint32_t x = (uint32_t)(gid % N);
  const GatherItem it = items[w];
  const uint64_t pos = (uint64_t)it.kb * N + x;
  const GatherQuery Q = qs[it.b];
  uint8_t* dst = gco + w * (uint64_t)d * N + x;
  if (pos >= Q.n) {
    for (uint32_t i = 0; i < d; ++i) dst[(uint64_t)i * N] = 0;
    gnorm[w * N + x] = 0;
    return;
  }
  // segment p with seg[p] <= pos < seg[p + 1] (seg has P + 1 entries per query)
  const uint64_t* sg = seg + (uint64_t)it.b * (P + 1);
  uint32_t lo = 0, hi = P;  // invariant: sg[lo] <= pos < sg[hi]
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (sg[mid] <= pos) lo = mid; else hi = mid;
  }
  const uint32_t c = probes[(uint64_t)it.b * P + lo];
  const uint32_t pt = members[offsets[c] + (pos - sg[lo])];
  const uint8_t* src = coords + (uint64_t)pt * d;
  uint32_t nrm = 0;
  for (uint32_t i = 0; i < d; ++i) {
    const uint32_t v = src[i];
    nrm += v * v;
    dst[(uint64_t)i * N] = (uint8_t)v;
  }
  gnorm[w * N + x] = nrm;
  if (ids) ids[Q.pos_off + pos] = pt;
}

// The same packing for d a multiple of 16 and N a multiple of 128 (the
// coordinates 16-byte aligned): a block takes 128 consecutive positions of
// one work item; each thread finds its point, reads the point's d bytes with
// 16-byte loads into a shared tile [dimension][position] and sums ||p||^2;
// the block then writes the tile's d rows of 128 positions with 16-byte
// stores, instead of one byte per thread and dimension.
__global__ void __launch_bounds__(128) pack_tile_kernel(uint32_t N, uint32_t d, const GatherItem* __restrict__ items,
                                                        const GatherQuery* __restrict__ qs,
                                                        const uint64_t* __restrict__ seg,
                                                        const uint32_t* __restrict__ probes, uint32_t P,
                                                        const uint64_t* __restrict__ offsets,
                                                        const uint32_t* __restrict__ members,
                                                        const uint8_t* __restrict__ coords, uint8_t* __restrict__ gco,
                                                        uint32_t* __restrict__ gnorm, uint32_t* __restrict__ ids) {
  __shared__ __align__(16) uint8_t tile[kMaxD][128];
  const uint32_t per_item = N / 128;
  const uint64_t w = blockIdx.x / per_item;
  const uint32_t x0 = (uint32_t)(blockIdx.x % per_item) * 128;
  const uint32_t x = x0 + threadIdx.x;
  const GatherItem it = items[w];
  const uint64_t pos = (uint64_t)it.kb * N + x;
  const GatherQuery Q = qs[it.b];
  uint32_t nrm = 0;
  if (pos < Q.n) {
    const uint64_t* sg = seg + (uint64_t)it.b * (P + 1);
    uint32_t lo = 0, hi = P;  // invariant: sg[lo] <= pos < sg[hi]
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (sg[mid] <= pos) lo = mid; else hi = mid;
    }
    const uint32_t c = probes[(uint64_t)it.b * P + lo];
    const uint32_t pt = members[offsets[c] + (pos - sg[lo])];
    const uint4* src = reinterpret_cast<const uint4*>(coords + (uint64_t)pt * d);
    for (uint32_t k = 0; k < d / 16; ++k) {
      const uint4 v = __ldg(src + k);
      const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const uint32_t b = (vw[m >> 2] >> (8 * (m & 3))) & 255u;
        nrm += b * b;
        tile[16 * k + m][threadIdx.x] = (uint8_t)b;
      }
    }
    if (ids) ids[Q.pos_off + pos] = pt;
  } else {
    for (uint32_t i = 0; i < d; ++i) tile[i][threadIdx.x] = 0;
  }
  gnorm[w * N + x] = nrm;
  __syncthreads();
  uint8_t* dst = gco + w * (uint64_t)d * N + x0;
  for (uint32_t e = threadIdx.x; e < d * 8; e += blockDim.x) {
    const uint32_t i = e >> 3, c16 = e & 7;
    *reinterpret_cast<uint4*>(dst + (uint64_t)i * N + 16 * c16) =
        *reinterpret_cast<const uint4*>(&tile[i][16 * c16]);
  }
}

// c * p mod q for c, p < q < 2^60 with p_mont = p 2^64 mod q: one Montgomery
// reduction of the 120-bit product gives a value below q + 2^56 < 2q.
__device__ __forceinline__ uint64_t mont_mul(uint64_t c, uint64_t p_mont, uint64_t q, uint64_t qn) {
  return csub(redc128((u128)c * p_mont, q, qn), q);
}

// Options of the gather: slot encoding (PT) and circuit privacy (pk and its
// Shoup companions in NTT form, flooding exponent F).
struct GatherOpts {
  PrimeSet PT;
  int slots;
  int ntt_form;  // responses in NTT form
  const uint64_t* pk;
  const uint64_t* pks;
  uint32_t F;
  PrivacyConsts C;
};

// One component of one (item, prime), its NTT-domain sum held in a (padded
// shared memory): back to coefficient form, mask (c = 0), flooding (with
// privacy), store.  For NTT-form responses the sum stays in the NTT domain:
// it is kept in save (global, owned by this block), the coefficient-domain
// terms are built in a, transformed and added.
__device__ void gather_finish(uint64_t* a, uint64_t* save, const PrimeSet& P, uint32_t j, uint32_t c,
                              uint64_t w, const GatherItem& it, const GatherQuery& Q,
                              const uint32_t* gnorm, uint64_t mask_seed, uint64_t qid, const GatherOpts& O,
                              uint64_t* ct_out, uint32_t* srv_share) {
  const uint32_t N = P.N, L = P.L;
  const uint64_t q = P.q[j];
  uint64_t* dst = ct_out + ((it.blk * 2 + c) * L + j) * N;
  __syncthreads();
  if (O.ntt_form) {
    if (c == 1 && !O.pk) {  // nothing to add to c1
      for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) dst[x] = a[SP(x)];
      return;
    }
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
      save[x] = a[SP(x)];
      a[SP(x)] = 0;
    }
    __syncthreads();
  } else {
    ntt_inverse_smem(a, P, (int)j);
    __syncthreads();
  }
  if (c == 0) {
    const uint64_t dl = P.delta[j], dls = P.delta_shoup[j];
    for (uint32_t t4 = threadIdx.x; t4 < N / 4; t4 += blockDim.x) {
      const uint64_t pos0 = (uint64_t)it.kb * N + 4 * t4;
      uint32_t blk[16];
      chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)(pos0 / 4), blk);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        uint64_t lo, hi;
        draw_pair(blk, v, lo, hi);
        const uint64_t rr = mod_t128(lo, hi, P);
        const uint32_t x = 4 * t4 + v;
        const uint64_t val = norm_plus_mask_mod_t(P, gnorm[w * N + x], rr);
        a[SP(x)] = add_mod(a[SP(x)], mul_shoup_u32((uint32_t)val, dl, dls, q), q);
        const uint64_t pos = pos0 + v;
        if (j == 0 && pos < Q.n) srv_share[Q.pos_off + pos] = (uint32_t)(rr == 0 ? 0 : P.t - rr);
      }
    }
    __syncthreads();
  }
  if (O.pk) {
    // flooding: e1 on c0 (uniform in [-2^F, 2^F)), e2 on c1 (CBD 21)
    for (uint32_t t4 = threadIdx.x; t4 < N / 4; t4 += blockDim.x) {
      const uint32_t ctr = (uint32_t)(((uint64_t)it.kb * N + 4 * t4) / 4);
      uint32_t ba[16], bb[16];
      if (c == 0) {
        chacha20_block(mask_seed, kPurposeFloodLo, qid, ctr, ba);
        chacha20_block(mask_seed, kPurposeFloodHi, qid, ctr, bb);
      } else {
        chacha20_block(mask_seed, kPurposeE2, qid, ctr, ba);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint32_t x = 4 * t4 + v;
        uint64_t e;
        if (c == 0) {
          uint64_t wv[4];
          draw_pair(ba, v, wv[0], wv[1]);
          draw_pair(bb, v, wv[2], wv[3]);
          e = flood_e1(wv, O.F, q, O.C.q_barrett[j], P.r64[j], P.r64_shoup[j], O.C.two_f[j]);
        } else {
          uint64_t lo, hi;
          draw_pair(ba, v, lo, hi);
          const int e2 = cbd21_of(lo);
          e = e2 < 0 ? q - (uint64_t)(-e2) : (uint64_t)e2;
        }
        a[SP(x)] = add_mod(a[SP(x)], e, q);
      }
    }
    __syncthreads();
  }
  if (O.ntt_form) {
    ntt_forward_smem(a, P, (int)j);
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) dst[x] = add_mod(save[x], a[SP(x)], q);
  } else {
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) dst[x] = a[SP(x)];
  }
}

// Persistent: block k takes units k, k + grid, ..; unit u = (w L + j) S + s.
// Shared memory holds only the polynomial being transformed; the unit's two
// accumulators (c0, c1) are its partial-sum slab part[u] in global memory
// (L2-resident), which each thread reads back and updates only at its own
// slots.  So three blocks fit on a multiprocessor.
__global__ void __launch_bounds__(256, 3)
gather_kernel(PrimeSet P, uint32_t d, uint64_t W, uint32_t S, uint32_t ds,
              const GatherItem* __restrict__ items, const GatherQuery* __restrict__ qs,
              const uint8_t* __restrict__ gco, const uint32_t* __restrict__ gnorm,
              const uint64_t* __restrict__ ct_in, uint64_t mask_seed, const uint64_t* __restrict__ qids,
              uint64_t* __restrict__ part, uint32_t* __restrict__ tickets, uint64_t* __restrict__ ct_out,
              uint32_t* __restrict__ srv_share, GatherOpts O) {
  extern __shared__ uint64_t smem[];
  __shared__ uint32_t ticket;
  const uint32_t N = P.N, L = P.L;
  uint64_t* poly = smem;
  const uint64_t units = W * L * S;
  for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const uint32_t sl = (uint32_t)(u % S);
    const uint64_t wj = u / S;
    const uint32_t j = (uint32_t)(wj % L);
    const uint64_t w = wj / L;
    const GatherItem it = items[w];
    const uint8_t* g = gco + w * (uint64_t)d * N;
    const uint64_t q = P.q[j], qn = P.q_neg_inv[j];
    const uint32_t i0 = sl * ds, i1 = i0 + ds < d ? i0 + ds : d;
    uint64_t* mine = part + u * 2 * N;  // this unit's accumulators: c0 at [0, N), c1 at [N, 2N)
    for (uint32_t i = i0; i < i1; ++i) {
      __syncthreads();
      const uint8_t* gi = g + (uint64_t)i * N;   // 16-byte aligned: item and row offsets are multiples of N
      // Coefficient encoding: each byte a enters as its Montgomery image
      // a 2^64 mod q (a table lookup), so by linearity the transform comes out
      // in Montgomery form, ready for the MAC's Montgomery products.
      const uint64_t* mb = P.mbyte + (size_t)j * 512;
      if (!O.slots && (P.logN & 3)) {
        // the coordinate bytes, 16 of each half per thread, go straight
        // through the first forward stage (distance N/2, twiddle psi^brv(1)):
        // X = aR + b psi^brv(1) R, Y = aR - b psi^brv(1) R, both from tables
        for (uint32_t gx = threadIdx.x; gx < N / 32; gx += blockDim.x) {
          const uint32_t x = gx * 16;
          const uint4 lo = __ldg(reinterpret_cast<const uint4*>(gi + x));
          const uint4 hi = __ldg(reinterpret_cast<const uint4*>(gi + x + N / 2));
          const uint32_t lw[4] = {lo.x, lo.y, lo.z, lo.w}, hw[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const uint64_t A = __ldg(mb + ((lw[k >> 2] >> (8 * (k & 3))) & 255u));
            const uint64_t T = __ldg(mb + 256 + ((hw[k >> 2] >> (8 * (k & 3))) & 255u));
            poly[SP(x + k)] = A + T;              // below 2q
            poly[SP(x + N / 2 + k)] = A - T + q;  // below 2q
          }
        }
        __syncthreads();
        ntt_forward_smem(poly, P, (int)j, 1);
      } else {
        for (uint32_t gx = threadIdx.x; gx < N / 16; gx += blockDim.x) {
          const uint32_t x = gx * 16;
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(gi + x));
          const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const uint32_t a = (vw[k >> 2] >> (8 * (k & 3))) & 255u;
            poly[SP(x + k)] = O.slots ? a : __ldg(mb + a);   // slot rows go mod t first
          }
        }
        __syncthreads();
        if (O.slots) {
          ntt_inverse_smem(poly, O.PT, 0);
          __syncthreads();
        }
        ntt_forward_smem(poly, P, (int)j);
      }
      __syncthreads();
      const uint64_t* c0 = ct_in + ((((uint64_t)it.b * d + i) * 2 + 0) * L + j) * N;
      const uint64_t* c1 = ct_in + ((((uint64_t)it.b * d + i) * 2 + 1) * L + j) * N;
      const bool first = i == i0;
      // four slots' ciphertext words and accumulators requested before any is used
      for (uint32_t x0 = threadIdx.x; x0 < N; x0 += 4 * blockDim.x) {
        uint64_t v0[4], v1[4], a0[4], a1[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const uint32_t x = x0 + r * blockDim.x;
          const bool in = x < N;
          v0[r] = in ? __ldg(c0 + x) : 0;
          v1[r] = in ? __ldg(c1 + x) : 0;
          a0[r] = in && !first ? __ldcg(mine + x) : 0;
          a1[r] = in && !first ? __ldcg(mine + N + x) : 0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const uint32_t x = x0 + r * blockDim.x;
          if (x >= N) break;
          // Montgomery form already, except for slot rows (transformed mod t)
          const uint64_t pm = O.slots ? mul_shoup(poly[SP(x)], P.r64[j], P.r64_shoup[j], q) : poly[SP(x)];
          mine[x] = add_mod(a0[r], mont_mul(v0[r], pm, q, qn), q);
          mine[N + x] = add_mod(a1[r], mont_mul(v1[r], pm, q, qn), q);
        }
      }
    }
    // publish the partial, then take a ticket; the last slice finishes
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(tickets + wj, 1u);
    __syncthreads();
    if (ticket != S - 1) continue;
    __threadfence();
    const GatherQuery Q = qs[it.b];
    const uint64_t qid = qids[it.b];
    uint64_t* all = part + wj * S * 2 * N;
    if (O.pk) {
      // re-randomisation: u ternary at the list positions, transformed, and
      // pk_c * u_hat added into slice 0's partial (which only this block reads)
      __syncthreads();
      for (uint32_t u4 = threadIdx.x; u4 < N / 4; u4 += blockDim.x) {
        uint32_t blk[16];
        chacha20_block(mask_seed, kPurposeU, qid, (uint32_t)(((uint64_t)it.kb * N) / 4 + u4), blk);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          uint64_t lo, hi;
          draw_pair(blk, v, lo, hi);
          const int uv = (int)(lo % 3) - 1;
          poly[SP(4 * u4 + v)] = uv < 0 ? q - 1 : (uint64_t)uv;
        }
      }
      __syncthreads();
      ntt_forward_smem(poly, P, (int)j);
      __syncthreads();
      for (uint32_t c = 0; c < 2; ++c) {
        const uint64_t* pkc = O.pk + ((size_t)c * L + j) * N;
        const uint64_t* pksc = O.pks + ((size_t)c * L + j) * N;
        for (uint32_t x = threadIdx.x; x < N; x += blockDim.x)
          all[(uint64_t)c * N + x] = add_mod(__ldcg(all + (uint64_t)c * N + x),
                                             mul_shoup(poly[SP(x)], pkc[x], pksc[x], q), q);
      }
    }
    for (uint32_t c = 0; c < 2; ++c) {
      __syncthreads();  // the polynomial buffer is free again
      for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
        // eight slices' partials requested before any is added
        uint64_t v = 0;
        uint32_t s2 = 0;
        for (; s2 + 8 <= S; s2 += 8) {
          uint64_t t8[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) t8[r] = __ldcg(all + ((uint64_t)(s2 + r) * 2 + c) * N + x);
#pragma unroll
          for (int r = 0; r < 8; ++r) v = add_mod(v, t8[r], q);
        }
        for (; s2 < S; ++s2) v = add_mod(v, __ldcg(all + ((uint64_t)s2 * 2 + c) * N + x), q);
        poly[SP(x)] = v;
      }
      gather_finish(poly, all + (uint64_t)c * N, P, j, c, w, it, Q, gnorm, mask_seed, qid, O, ct_out,
                    srv_share);
    }
  }
}

// Slot encoding: one block per work item; the mask polynomial R of the item
// (coefficient draws at the list positions, padding included) to slots,
// srv_share = t - NTT_t(R) at the query's positions.
__global__ void __launch_bounds__(512) gather_slot_share_kernel(PrimeSet P, PrimeSet PT,
                                                                const GatherItem* __restrict__ items,
                                                                const GatherQuery* __restrict__ qs,
                                                                uint64_t mask_seed, const uint64_t* __restrict__ qids,
                                                                uint32_t* __restrict__ srv_share) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N;
  const GatherItem it = items[blockIdx.x];
  const GatherQuery Q = qs[it.b];
  const uint64_t qid = qids[it.b];
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(mask_seed, kPurposeMask, qid, (uint32_t)(((uint64_t)it.kb * N) / 4 + u), blk);
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
    const uint64_t pos = (uint64_t)it.kb * N + x;
    if (pos >= Q.n) break;
    const uint64_t r = sa[SP(x)];
    srv_share[Q.pos_off + pos] = (uint32_t)(r == 0 ? 0 : P.t - r);
  }
}

}  // namespace

cudaError_t launch_check_indices(const uint32_t* idx, uint64_t m, uint64_t bound, int* bad,
                                 cudaStream_t st) {
  check_indices_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(idx, m, bound, bad);
  return cudaGetLastError();
}

int gather_threads(uint32_t N) { return N >= 512 ? 256 : (int)(N / 2); }

namespace {

// Host plan of one gather: items (query-major), per-query offsets and the
// probe segments of every query's list.
struct PlanHost {
  std::vector<GatherItem> items;
  std::vector<GatherQuery> qs;
  std::vector<uint64_t> seg;
};

void build_plan(uint32_t N, const sanns_clusters* cl, const uint32_t* probes_host, uint32_t B,
                uint32_t Pr, const uint64_t* n_b, PlanHost& H) {
  H.qs.assign(B, GatherQuery{0, 0});
  H.seg.assign((size_t)B * (Pr + 1), 0);
  uint64_t blk = 0, pos = 0;
  for (uint32_t b = 0; b < B; ++b) {
    uint64_t acc = 0;
    for (uint32_t p = 0; p < Pr; ++p) {
      H.seg[(size_t)b * (Pr + 1) + p] = acc;
      const uint32_t c = probes_host[(size_t)b * Pr + p];
      acc += cl->h_offsets[c + 1] - cl->h_offsets[c];
    }
    H.seg[(size_t)b * (Pr + 1) + Pr] = acc;
    H.qs[b].n = n_b[b];
    H.qs[b].pos_off = pos;
    const uint64_t Kb = (n_b[b] + N - 1) / N;
    for (uint64_t k = 0; k < Kb; ++k) H.items.push_back(GatherItem{b, (uint32_t)k, blk + k});
    blk += Kb;
    pos += n_b[b];
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets of the plan tables in one allocation; returns its size.
size_t plan_layout(uint64_t W, uint32_t B, uint32_t Pr, size_t& o_items, size_t& o_qs, size_t& o_seg,
                   size_t& o_pr) {
  o_items = 0;
  o_qs = up256(sizeof(GatherItem) * W);
  o_seg = o_qs + up256(sizeof(GatherQuery) * B);
  o_pr = o_seg + up256(sizeof(uint64_t) * (size_t)B * (Pr + 1));
  return o_pr + up256(sizeof(uint32_t) * (size_t)B * Pr);
}

cudaError_t upload_plan(uint8_t* tables, const PlanHost& H, const uint32_t* probes_host, uint32_t B,
                        uint32_t Pr, size_t o_items, size_t o_qs, size_t o_seg, size_t o_pr,
                        cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(tables + o_items, H.items.data(), sizeof(GatherItem) * H.items.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tables + o_qs, H.qs.data(), sizeof(GatherQuery) * B, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tables + o_seg, H.seg.data(), sizeof(uint64_t) * H.seg.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tables + o_pr, probes_host, sizeof(uint32_t) * (size_t)B * Pr, cudaMemcpyHostToDevice, st);
  // the host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// The launches of one gather over an uploaded plan: a stream-ordered scratch
// allocation (packed coordinates, norms, partial sums, tickets) and the
// kernels, nothing that waits on the host.
cudaError_t gather_kernels(const PrimeSet& P, uint32_t d, const sanns_clusters* cl, const uint8_t* tables,
                           size_t o_items, size_t o_qs, size_t o_seg, size_t o_pr, uint64_t W,
                           uint32_t Pr, const uint64_t* ct_in, uint64_t mask_seed, const uint64_t* qids,
                           uint64_t* ct_out, uint32_t* srv_share, uint32_t* ids, int sms, const PrimeSet* PT,
                           const uint64_t* pk, const uint64_t* pks, uint32_t F, const PrivacyConsts& C,
                           bool ntt_form, cudaStream_t st) {
  const uint32_t N = P.N;
  // dimension slices per (item, prime): about four units per multiprocessor
  // in all, at least one dimension per slice, and at most kMaxSlices: the
  // finishing block reads every slice's partial (2 N words each), so more
  // slices than that cost more in the finish than they save in the MAC
  constexpr uint64_t kMaxSlices = 32;
  const uint64_t nsm = (uint64_t)(sms > 0 ? sms : 148);
  uint64_t want = (4 * nsm + W * P.L - 1) / (W * P.L);
  if (want > kMaxSlices) want = kMaxSlices;
  const uint32_t S0 = (uint32_t)(want < d ? want : d);
  const uint32_t ds = (d + S0 - 1) / S0;
  const uint32_t S = (d + ds - 1) / ds;
  const size_t o_norm = 0, o_gco = up256(sizeof(uint32_t) * W * N);
  const size_t o_part = o_gco + up256((size_t)W * d * N);
  const size_t o_tick = o_part + up256(sizeof(uint64_t) * (size_t)W * P.L * S * 2 * N);
  const size_t total = o_tick + up256(sizeof(uint32_t) * (size_t)W * P.L);
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(N);
  cudaError_t e = ensure_smem_attr((const void*)gather_kernel, smem);
  if (e == cudaSuccess && PT) e = ensure_smem_attr((const void*)gather_slot_share_kernel, smem);
  if (e != cudaSuccess) return e;
  uint8_t* scratch = nullptr;
  e = cudaMallocAsync(&scratch, total, st);
  if (e != cudaSuccess) return e;
  const GatherItem* d_items = reinterpret_cast<const GatherItem*>(tables + o_items);
  const GatherQuery* d_qs = reinterpret_cast<const GatherQuery*>(tables + o_qs);
  if (d % 16 == 0 && N % 128 == 0 && (reinterpret_cast<uintptr_t>(cl->d_coords) & 15) == 0) {
    pack_tile_kernel<<<(unsigned)(W * (N / 128)), 128, 0, st>>>(
        N, d, d_items, d_qs, reinterpret_cast<const uint64_t*>(tables + o_seg),
        reinterpret_cast<const uint32_t*>(tables + o_pr), Pr, cl->d_offsets, cl->d_members,
        cl->d_coords, scratch + o_gco, reinterpret_cast<uint32_t*>(scratch + o_norm), ids);
    e = cudaGetLastError();
  } else {
    const uint64_t threads = W * N;
    pack_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        N, d, W, d_items, d_qs, reinterpret_cast<const uint64_t*>(tables + o_seg),
        reinterpret_cast<const uint32_t*>(tables + o_pr), Pr, cl->d_offsets, cl->d_members,
        cl->d_coords, scratch + o_gco, reinterpret_cast<uint32_t*>(scratch + o_norm), ids);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && PT) e = launch_norms_slot(*PT, reinterpret_cast<uint32_t*>(scratch + o_norm), W, st);
  GatherOpts O;
  memset(&O, 0, sizeof(O));
  if (PT) {
    O.PT = *PT;
    O.slots = 1;
  } else {
    O.PT = P;
  }
  O.ntt_form = ntt_form ? 1 : 0;
  O.pk = pk;
  O.pks = pks;
  O.F = F;
  O.C = C;
  uint64_t* part = reinterpret_cast<uint64_t*>(scratch + o_part);
  uint32_t* tickets = reinterpret_cast<uint32_t*>(scratch + o_tick);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, sizeof(uint32_t) * (size_t)W * P.L, st);
  if (e == cudaSuccess) {
    const int th = gather_threads(N);
    const uint64_t units = W * P.L * S;
    const uint64_t slots = 3 * nsm;  // three blocks per multiprocessor
    const unsigned grid = (unsigned)(units < slots ? units : slots);
    gather_kernel<<<grid, th, smem, st>>>(P, d, W, S, ds, d_items, d_qs, scratch + o_gco,
                                          reinterpret_cast<const uint32_t*>(scratch + o_norm), ct_in,
                                          mask_seed, qids, part, tickets, ct_out, srv_share, O);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && PT) {
    gather_slot_share_kernel<<<(unsigned)W, gather_threads(N), smem, st>>>(P, *PT, d_items, d_qs, mask_seed,
                                                                           qids, srv_share);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t launch_gather(const PrimeSet& P, uint32_t d, const sanns_clusters* cl,
                          const uint64_t* ct_in, uint32_t B, const uint32_t* probes_host,
                          uint32_t Pr, const uint64_t* n_b, uint64_t mask_seed,
                          const uint64_t* qids, uint64_t* ct_out, uint32_t* srv_share,
                          uint32_t* ids, int sms, const PrimeSet* PT, const uint64_t* pk,
                          const uint64_t* pks, uint32_t F, const PrivacyConsts& C, bool ntt_form,
                          cudaStream_t st) {
  PlanHost H;
  build_plan(P.N, cl, probes_host, B, Pr, n_b, H);
  const uint64_t W = H.items.size();
  if (W == 0) return cudaSuccess;
  size_t o_items, o_qs, o_seg, o_pr;
  const size_t bytes = plan_layout(W, B, Pr, o_items, o_qs, o_seg, o_pr);
  uint8_t* tables = nullptr;
  cudaError_t e = cudaMallocAsync(&tables, bytes, st);
  if (e != cudaSuccess) return e;
  e = upload_plan(tables, H, probes_host, B, Pr, o_items, o_qs, o_seg, o_pr, st);
  if (e == cudaSuccess)
    e = gather_kernels(P, d, cl, tables, o_items, o_qs, o_seg, o_pr, W, Pr, ct_in, mask_seed, qids, ct_out,
                       srv_share, ids, sms, PT, pk, pks, F, C, ntt_form, st);
  cudaError_t e2 = cudaFreeAsync(tables, st);
  return e != cudaSuccess ? e : e2;
}

cudaError_t gather_prepare(uint32_t N, const uint32_t* probes_host, sanns_gather_batch* gb) {
  PlanHost H;
  build_plan(N, gb->cl, probes_host, gb->B, gb->P, gb->n_b.data(), H);
  gb->W = H.items.size();
  gb->d_tables = nullptr;
  if (gb->W == 0) return cudaSuccess;
  const size_t bytes = plan_layout(gb->W, gb->B, gb->P, gb->o_items, gb->o_qs, gb->o_seg, gb->o_pr);
  cudaError_t e = cudaMalloc(&gb->d_tables, bytes);
  if (e != cudaSuccess) {
    gb->d_tables = nullptr;
    return e;
  }
  e = upload_plan(gb->d_tables, H, probes_host, gb->B, gb->P, gb->o_items, gb->o_qs, gb->o_seg, gb->o_pr,
                  nullptr);
  if (e != cudaSuccess) {
    cudaFree(gb->d_tables);
    gb->d_tables = nullptr;
  }
  return e;
}

cudaError_t launch_gather_prepared(const PrimeSet& P, uint32_t d, const sanns_gather_batch* gb,
                                   const uint64_t* ct_in, uint64_t mask_seed, const uint64_t* qids,
                                   uint64_t* ct_out, uint32_t* srv_share, uint32_t* ids, int sms,
                                   const PrimeSet* PT, const uint64_t* pk, const uint64_t* pks, uint32_t F,
                                   const PrivacyConsts& C, bool ntt_form, cudaStream_t st) {
  if (gb->W == 0) return cudaSuccess;
  return gather_kernels(P, d, gb->cl, gb->d_tables, gb->o_items, gb->o_qs, gb->o_seg, gb->o_pr, gb->W, gb->P,
                        ct_in, mask_seed, qids, ct_out, srv_share, ids, sms, PT, pk, pks, F, C, ntt_form, st);
}

}  // namespace sanns
