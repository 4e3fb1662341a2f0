// The extern "C" entry points of sanns.h: host-side validation, handle
// management and the launch sequences of the linear-scan protocol's steps
// 1-4 (Sec. 5.3), the clustering protocol's gathers (Algorithm 4) and the
// selections (Algorithms 1 and 2).
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"

namespace sanns {

namespace {
thread_local std::string g_last_error;
std::mutex g_attr_mu;
std::map<std::pair<const void*, int>, size_t> g_attr_done;
}

cudaError_t ensure_smem_attr(const void* kernel, size_t bytes) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  const auto key = std::make_pair(kernel, dev);
  auto it = g_attr_done.find(key);
  if (it != g_attr_done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g_attr_done[key] = bytes;
  return e;
}

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SANNS_ENOMEM : SANNS_ECUDA;
}

}  // namespace sanns

using namespace sanns;

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int check_device(const sanns_ctx* ctx) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != ctx->device) return fail(SANNS_EINVAL, "current device differs from the context's device");
  return SANNS_OK;
}

}  // namespace

extern "C" {

const char* sanns_last_error(void) { return g_last_error.c_str(); }

int sanns_device_sms(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

int sanns_ctx_create(const sanns_params* p, sanns_ctx** out) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(SANNS_EINVAL, "params is NULL");
  const uint32_t N = p->N;
  if (N < kMinN || N > kMaxN || (N & (N - 1)))
    return fail(SANNS_EINVAL, "N must be a power of two in [64, 16384]");
  if (p->L < 1 || p->L > (uint32_t)kMaxPrimes) return fail(SANNS_EINVAL, "L must be in [1, 4]");
  if (p->d < 1 || p->d > kMaxD) return fail(SANNS_EINVAL, "d must be in [1, 224]");
  if (p->t_rule == 1 && (p->b_c < 1 || p->b_c > 12)) return fail(SANNS_EINVAL, "b_c must be in [1, 12]");
  uint64_t q[kMaxPrimes], psi[kMaxPrimes], t = 0;
  int rc = derive_params(*p, q, psi, &t);
  if (rc) return rc;
  if (t >= (1ull << 31)) return fail(SANNS_EINVAL, "t must be below 2^31");

  sanns_ctx* c = new sanns_ctx();
  c->params = *p;
  memset(&c->P, 0, sizeof(c->P));
  c->P.N = N;
  uint32_t logN = 0;
  while ((1u << logN) < N) ++logN;
  c->P.logN = logN;
  fill_prime_constants(c->P, q, t, p->L);
  // every norm encode_db stores, d 255^2 at most, is below t: the mask
  // epilogues then reduce ||p||^2 + r mod t with one conditional subtraction
  // (imported norms are reduced mod t on import)
  c->P.norms_below_t = (uint64_t)p->d * 255u * 255u < t ? 1u : 0u;
  for (uint32_t j = 0; j < p->L; ++j) c->psi[j] = psi[j];
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDevice"); }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  {
    // stream-ordered scratch (decryption, gather, batched path) stays cached
    // in the device's default pool instead of going back to the driver at
    // every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  c->mac_variant = 0;
  c->mac_sms = 0;
  c->batched_tune[0] = 0;
  c->batched_tune[1] = 0;
  c->batched_tune[2] = 32;
  c->batched_tune[3] = 128;
  c->batched_tune[4] = 0;
  c->batched_tune[5] = 4096;
  c->batched_tune[6] = 7;

  const size_t per = (size_t)p->L * N;
  std::vector<uint64_t> fw(per), fws(per), iw(per), iws(per);
  for (uint32_t j = 0; j < p->L; ++j)
    fill_twiddles(N, q[j], psi[j], &fw[j * N], &fws[j * N], &iw[j * N], &iws[j * N]);
  for (uint32_t j = 0; j < p->L; ++j) {
    c->P.last_inv[j] = (uint64_t)(((unsigned __int128)iw[j * N + 1] * c->P.n_inv[j]) % q[j]);
    c->P.last_inv_shoup[j] = shoup_of(c->P.last_inv[j], q[j]);
    c->P.delta_w1[j] = (uint64_t)(((unsigned __int128)fw[j * N + 1] * c->P.delta[j]) % q[j]);
    c->P.delta_w1_shoup[j] = shoup_of(c->P.delta_w1[j], q[j]);
  }
  // interleave {w, w_shoup}: forward table then inverse table, [L][N] pairs
  // each; then the Montgomery byte tables, [L][2][256]
  const size_t mb = (size_t)p->L * 512;
  std::vector<uint64_t> host(4 * per + mb);
  for (size_t x = 0; x < per; ++x) {
    host[2 * x] = fw[x];
    host[2 * x + 1] = fws[x];
    host[2 * per + 2 * x] = iw[x];
    host[2 * per + 2 * x + 1] = iws[x];
  }
  for (uint32_t j = 0; j < p->L; ++j) {
    const u128 R = (((u128)1) << 64) % q[j];
    const u128 w1R = (u128)fw[(size_t)j * N + 1] * R % q[j];
    for (uint32_t a = 0; a < 256; ++a) {
      host[4 * per + (size_t)j * 512 + a] = (uint64_t)(a * R % q[j]);
      host[4 * per + (size_t)j * 512 + 256 + a] = (uint64_t)(a * w1R % q[j]);
    }
  }
  e = cudaMalloc(&c->d_tables, sizeof(uint64_t) * (4 * per + mb));
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(tables)"); }
  e = cudaMemcpy(c->d_tables, host.data(), sizeof(uint64_t) * (4 * per + mb), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(c->d_tables); delete c; return cuda_fail(e, "cudaMemcpy(tables)"); }
  c->P.tw = reinterpret_cast<const ulonglong2*>(c->d_tables);
  c->P.itw = reinterpret_cast<const ulonglong2*>(c->d_tables + 2 * per);
  c->P.mbyte = c->d_tables + 4 * per;
  // responses at every prime by default; the one-prime view (q_0 alone, its
  // tables the first rows of the full ones) decrypts switched responses
  c->response_primes = p->L;
  c->P1 = c->P;
  fill_prime_constants(c->P1, q, t, 1);
  c->P1.last_inv[0] = c->P.last_inv[0];
  c->P1.last_inv_shoup[0] = c->P.last_inv_shoup[0];
  c->P1.delta_w1[0] = (uint64_t)(((unsigned __int128)fw[1] * c->P1.delta[0]) % q[0]);
  c->P1.delta_w1_shoup[0] = shoup_of(c->P1.delta_w1[0], q[0]);
  make_mod_switch_consts(c->P, &c->MS);
  e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e != cudaSuccess) { cudaFree(c->d_tables); delete c; return cuda_fail(e, "cudaMalloc(err)"); }
  // slot encoding needs a primitive 2N-th root of unity mod t (t = 1 mod 2N)
  memset(&c->PT, 0, sizeof(c->PT));
  if (t % (2ull * N) == 1) {
    PrimeSet& T = c->PT;
    T.N = N;
    T.logN = logN;
    T.L = 1;
    T.t = t;
    T.q[0] = t;
    c->psi_t = smallest_psi(t, N);
    std::vector<uint64_t> tf(N), tfs(N), ti(N), tis(N);
    fill_twiddles(N, t, c->psi_t, tf.data(), tfs.data(), ti.data(), tis.data());
    // N^-1 mod t by Fermat (t prime)
    uint64_t ninv = 1, base = N % t, ex = t - 2;
    while (ex) {
      if (ex & 1) ninv = (uint64_t)((u128)ninv * base % t);
      base = (uint64_t)((u128)base * base % t);
      ex >>= 1;
    }
    T.n_inv[0] = ninv;
    T.n_inv_shoup[0] = shoup_of(ninv, t);
    // psi_t^-brv(1) N^-1: the last inverse stage with N^-1 folded in
    T.last_inv[0] = (uint64_t)((u128)ti[1] * ninv % t);
    T.last_inv_shoup[0] = shoup_of(T.last_inv[0], t);
    std::vector<uint64_t> th(4 * (size_t)N);
    for (uint32_t x = 0; x < N; ++x) {
      th[2 * x] = tf[x];
      th[2 * x + 1] = tfs[x];
      th[2 * N + 2 * x] = ti[x];
      th[2 * N + 2 * x + 1] = tis[x];
    }
    e = cudaMalloc(&c->d_tables_t, sizeof(uint64_t) * 4 * N);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_tables_t, th.data(), sizeof(uint64_t) * 4 * N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(c->d_tables_t);
      cudaFree(c->d_tables);
      cudaFree(c->d_err);
      delete c;
      return cuda_fail(e, "cudaMalloc(slot tables)");
    }
    T.tw = reinterpret_cast<const ulonglong2*>(c->d_tables_t);
    T.itw = reinterpret_cast<const ulonglong2*>(c->d_tables_t + 2 * N);
  }
  *out = c;
  return SANNS_OK;
}

int sanns_set_encoding(sanns_ctx* ctx, int slots) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (slots != 0 && slots != 1) return fail(SANNS_EINVAL, "encoding must be 0 (coefficients) or 1 (slots)");
  if (slots && !ctx->d_tables_t) return fail(SANNS_EINVAL, "slot encoding needs t = 1 mod 2N");
  ctx->slots = slots == 1;
  return SANNS_OK;
}

void sanns_ctx_free(sanns_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->d_pk);
  cudaFree(ctx->d_pk_shoup);
  cudaFree(ctx->d_tables);
  cudaFree(ctx->d_tables_t);
  cudaFree(ctx->d_err);
  delete ctx;
}

int sanns_ctx_query(const sanns_ctx* ctx, uint64_t* q, uint64_t* psi, uint64_t* t, uint64_t* delta) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  for (uint32_t j = 0; j < ctx->params.L; ++j) {
    if (q) q[j] = ctx->P.q[j];
    if (psi) psi[j] = ctx->psi[j];
    if (delta) delta[j] = ctx->P.delta[j];
  }
  if (t) *t = ctx->P.t;
  return SANNS_OK;
}

int sanns_ntt(sanns_ctx* ctx, uint64_t* data, uint64_t count, int inverse, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (count && !data) return fail(SANNS_EINVAL, "data is NULL");
  if (count * ctx->params.L > 0x7fffffffull) return fail(SANNS_EINVAL, "too many polynomials");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_ntt(ctx->P, data, count, inverse != 0, as_stream(stream)));
  return SANNS_OK;
}

int sanns_keygen(sanns_ctx* ctx, uint64_t seed, sanns_sk** out, void* stream) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  const uint32_t N = ctx->P.N, L = ctx->P.L;
  sanns_sk* sk = new sanns_sk();
  sk->ctx = ctx;
  cudaError_t e = cudaMalloc(&sk->d_s, N);
  if (e == cudaSuccess) e = cudaMalloc(&sk->d_s_hat, sizeof(uint64_t) * 2 * L * N);
  if (e != cudaSuccess) {
    cudaFree(sk->d_s);
    delete sk;
    return cuda_fail(e, "cudaMalloc(sk)");
  }
  sk->d_s_hat_shoup = sk->d_s_hat + (size_t)L * N;
  e = launch_keygen(ctx->P, seed, sk->d_s, sk->d_s_hat, sk->d_s_hat_shoup, as_stream(stream));
  if (e != cudaSuccess) {
    sanns_sk_free(sk);
    return cuda_fail(e, "keygen kernel");
  }
  *out = sk;
  return SANNS_OK;
}

void sanns_sk_free(sanns_sk* sk) {
  if (!sk) return;
  cudaFree(sk->d_s);
  cudaFree(sk->d_s_hat);
  delete sk;
}

int sanns_sk_export(const sanns_sk* sk, int8_t* s, uint64_t* s_hat, void* stream) {
  if (!sk) return fail(SANNS_EINVAL, "sk is NULL");
  const uint32_t N = sk->ctx->P.N, L = sk->ctx->P.L;
  cudaStream_t st = as_stream(stream);
  if (s) SANNS_CUDA(cudaMemcpyAsync(s, sk->d_s, N, cudaMemcpyDefault, st));
  if (s_hat) SANNS_CUDA(cudaMemcpyAsync(s_hat, sk->d_s_hat, sizeof(uint64_t) * L * N, cudaMemcpyDefault, st));
  SANNS_CUDA(cudaStreamSynchronize(st));
  return SANNS_OK;
}

int sanns_encode_db(sanns_ctx* ctx, const uint8_t* coords, uint64_t n_points, const uint32_t* perm,
                    uint64_t n, sanns_db** out, void* stream) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (n == 0) return fail(SANNS_EINVAL, "n must be positive");
  if (!coords) return fail(SANNS_EINVAL, "coords is NULL");
  if (!perm && n > n_points) return fail(SANNS_EINVAL, "n exceeds n_points without a permutation");
  int rc = check_device(ctx);
  if (rc) return rc;
  const uint32_t N = ctx->P.N, L = ctx->P.L, d = ctx->params.d;
  const uint64_t K = (n + N - 1) / N;
  if (K > 0x7fffffffull) return fail(SANNS_EINVAL, "too many blocks");
  cudaStream_t st = as_stream(stream);
  sanns_db* db = new sanns_db();
  db->ctx = ctx;
  db->n = n;
  db->K = K;
  db->slots = ctx->slots;
  int* d_bad = nullptr;
  cudaError_t e = cudaMalloc(&db->d_pt, sizeof(uint64_t) * K * L * d * N);
  if (e == cudaSuccess) e = cudaMalloc(&db->d_norms, sizeof(uint32_t) * K * N);
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_encode(ctx->P, db->slots ? &ctx->PT : nullptr, coords, n_points, perm, n, d, K, db->d_pt,
                      db->d_norms, d_bad, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_bad);
  if (e != cudaSuccess) {
    sanns_db_free(db);
    return cuda_fail(e, "encode_db");
  }
  if (bad) {
    sanns_db_free(db);
    return fail(SANNS_EINVAL, "perm holds an index >= n_points");
  }
  *out = db;
  return SANNS_OK;
}

int sanns_db_import(sanns_ctx* ctx, uint64_t n, const uint64_t* pt, const uint32_t* norms, sanns_db** out,
                    void* stream) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (n == 0) return fail(SANNS_EINVAL, "n must be positive");
  if (!pt || !norms) return fail(SANNS_EINVAL, "pt or norms is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  const uint32_t N = ctx->P.N, L = ctx->P.L, d = ctx->params.d;
  const uint64_t K = (n + N - 1) / N;
  if (K > 0x7fffffffull) return fail(SANNS_EINVAL, "too many blocks");
  cudaStream_t st = as_stream(stream);
  sanns_db* db = new sanns_db();
  db->ctx = ctx;
  db->n = n;
  db->K = K;
  db->slots = ctx->slots;
  const uint64_t count = K * L * d * N;
  int* d_bad = nullptr;
  cudaError_t e = cudaMalloc(&db->d_pt, sizeof(uint64_t) * count);
  if (e == cudaSuccess) e = cudaMalloc(&db->d_norms, sizeof(uint32_t) * K * N);
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(db->d_pt, pt, sizeof(uint64_t) * count, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(db->d_norms, norms, sizeof(uint32_t) * K * N, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = launch_import_pt(ctx->P, db->d_pt, count, d, d_bad, st);
  if (e == cudaSuccess) e = launch_norms_mod_t(ctx->P, db->d_norms, K * N, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_bad) cudaFree(d_bad);
  if (e != cudaSuccess) {
    sanns_db_free(db);
    return cuda_fail(e, "db import");
  }
  if (bad) {
    sanns_db_free(db);
    return fail(SANNS_EINVAL, "a plaintext residue is not below its prime");
  }
  *out = db;
  return SANNS_OK;
}

void sanns_db_free(sanns_db* db) {
  if (!db) return;
  cudaFree(db->d_plimb);
  cudaFree(db->d_pt);
  cudaFree(db->d_norms);
  delete db;
}

int sanns_db_set_position_base(sanns_db* db, uint64_t pos0) {
  if (!db) return fail(SANNS_EINVAL, "db is NULL");
  if (pos0 % db->ctx->P.N) return fail(SANNS_EINVAL, "the position base must be a multiple of N");
  if (pos0 + db->K * db->ctx->P.N > (1ull << 34)) return fail(SANNS_EINVAL, "positions beyond 2^34");
  db->pos0 = pos0;
  return SANNS_OK;
}

int sanns_db_info(const sanns_db* db, uint64_t* n, uint64_t* K) {
  if (!db) return fail(SANNS_EINVAL, "db is NULL");
  if (n) *n = db->n;
  if (K) *K = db->K;
  return SANNS_OK;
}

int sanns_db_export(const sanns_db* db, uint64_t k0, uint64_t k1, uint64_t* pt, uint32_t* norms,
                    void* stream) {
  if (!db) return fail(SANNS_EINVAL, "db is NULL");
  if (k0 > k1 || k1 > db->K) return fail(SANNS_EINVAL, "block range out of bounds");
  const sanns_ctx* ctx = db->ctx;
  const size_t per_block = (size_t)ctx->P.L * ctx->params.d * ctx->P.N;
  cudaStream_t st = as_stream(stream);
  if (pt && k1 > k0) {
    // canonical values from the split storage format, through a device copy
    const uint64_t count = (k1 - k0) * per_block;
    uint64_t* tmp = nullptr;
    SANNS_CUDA(cudaMallocAsync(&tmp, sizeof(uint64_t) * count, st));
    cudaError_t e = launch_join30(db->d_pt + k0 * per_block, tmp, count, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pt, tmp, sizeof(uint64_t) * count, cudaMemcpyDefault, st);
    cudaError_t e2 = cudaFreeAsync(tmp, st);
    if (e != cudaSuccess) return cuda_fail(e, "db export");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  }
  if (norms)
    SANNS_CUDA(cudaMemcpyAsync(norms, db->d_norms + k0 * ctx->P.N,
                               sizeof(uint32_t) * (k1 - k0) * ctx->P.N, cudaMemcpyDefault, st));
  SANNS_CUDA(cudaStreamSynchronize(st));
  return SANNS_OK;
}

int sanns_encrypt_query(sanns_ctx* ctx, const sanns_sk* sk, const uint8_t* qv, uint32_t B,
                        uint64_t seed, const uint64_t* qids, uint64_t* ct, void* stream) {
  if (!ctx || !sk) return fail(SANNS_EINVAL, "ctx or sk is NULL");
  if (sk->ctx != ctx) return fail(SANNS_EINVAL, "sk belongs to another context");
  if (B == 0) return SANNS_OK;
  if (!qv || !qids || !ct) return fail(SANNS_EINVAL, "NULL buffer");
  if (B > 65535) return fail(SANNS_EINVAL, "B must be <= 65535");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_encrypt(ctx->P, sk->d_s_hat, sk->d_s_hat_shoup, qv, B, ctx->params.d, seed, qids,
                            ct, as_stream(stream)));
  return SANNS_OK;
}

int sanns_expand_query(sanns_ctx* ctx, const uint64_t* c0, uint32_t B, uint64_t seed,
                       const uint64_t* qids, uint64_t* ct, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (B == 0) return SANNS_OK;
  if (!c0 || !qids || !ct) return fail(SANNS_EINVAL, "NULL buffer");
  if (B > 65535) return fail(SANNS_EINVAL, "B must be <= 65535");
  const uint64_t words = (uint64_t)B * ctx->params.d * ctx->P.L * ctx->P.N;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(c0), a1 = a0 + 8 * words;
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(ct), b1 = b0 + 16 * words;
  if (a0 < b1 && b0 < a1) return fail(SANNS_EINVAL, "c0 and ct_in overlap");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_seeded_query(ctx->P, c0, B, ctx->params.d, seed, qids, ct, as_stream(stream)));
  return SANNS_OK;
}

namespace {
int check_distance_args(sanns_ctx* ctx, const sanns_db* db, uint32_t B) {
  if (!ctx || !db) return fail(SANNS_EINVAL, "ctx or db is NULL");
  if (db->ctx != ctx) return fail(SANNS_EINVAL, "db belongs to another context");
  if ((uint64_t)B * db->K * 2 * ctx->P.L > 0x7fffffffull) return fail(SANNS_EINVAL, "batch too large");
  if (db->slots != ctx->slots)
    return fail(SANNS_EINVAL, "the database was encoded in the other encoding than the context's");
  return check_device(ctx);
}
}  // namespace

// SMs the MAC kernels' persistent grids spread over (sanns_set_mac_sms)
static int mac_grid_sms(const sanns_ctx* ctx) {
  return ctx->mac_sms > 0 && ctx->mac_sms < ctx->sms ? ctx->mac_sms : ctx->sms;
}

int sanns_distances_mac(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                        uint64_t* ct_out, void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0) return SANNS_OK;
  if (!ct_in || !ct_out) return fail(SANNS_EINVAL, "NULL buffer");
  if (!aligned16(ct_in) || !aligned16(ct_out)) return fail(SANNS_EINVAL, "ct buffers must be 16-byte aligned");
  const int sms = mac_grid_sms(ctx);
  SANNS_CUDA(launch_mac(ctx->P, ct_in, db->d_pt, B, ctx->params.d, db->K, ct_out, sms,
                        ctx->mac_variant, as_stream(stream)));
  return SANNS_OK;
}

int sanns_distances_finish(sanns_ctx* ctx, const sanns_db* db, uint32_t B, uint64_t mask_seed,
                           const uint64_t* qids, uint64_t* ct_out, uint32_t* srv_share, void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0) return SANNS_OK;
  if (!qids || !ct_out || !srv_share) return fail(SANNS_EINVAL, "NULL buffer");
  cudaStream_t st = as_stream(stream);
  if (ctx->d_pk)
    SANNS_CUDA(launch_rerandomize(ctx->P, ct_out, B, db->K, db->pos0, mask_seed, qids, ctx->d_pk,
                                  ctx->d_pk_shoup, st));
  if (ctx->ntt_responses) {
    SANNS_CUDA(launch_mask_ntt(ctx->P, ct_out, db->d_norms, B, db->K, db->n, db->pos0, mask_seed, qids,
                               srv_share, ctx->d_pk != nullptr, ctx->flood_bits, ctx->privacy, st));
    if (ctx->slots)
      SANNS_CUDA(launch_slot_share(ctx->P, ctx->PT, B, db->K, db->n, db->pos0, mask_seed, qids, srv_share, st));
    return SANNS_OK;
  }
  SANNS_CUDA(launch_intt_mask(ctx->P, ct_out, db->d_norms, B, db->K, db->n, db->pos0, mask_seed, qids,
                              srv_share, ctx->sms, st));
  if (ctx->d_pk)
    SANNS_CUDA(launch_flood(ctx->P, ct_out, B, db->K, db->pos0, mask_seed, qids, ctx->flood_bits,
                            ctx->privacy, st));
  if (ctx->slots)
    SANNS_CUDA(launch_slot_share(ctx->P, ctx->PT, B, db->K, db->n, db->pos0, mask_seed, qids, srv_share, st));
  if (ctx->response_primes == 1)
    SANNS_CUDA(launch_mod_switch(ctx->P, ctx->MS, ct_out, (uint64_t)B * db->K * 2, st));
  return SANNS_OK;
}

int sanns_set_response_form(sanns_ctx* ctx, int form) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (form != 0 && form != 1) return fail(SANNS_EINVAL, "form must be 0 (coefficients) or 1 (NTT)");
  if (form == 1 && ctx->response_primes != ctx->P.L)
    return fail(SANNS_EINVAL, "NTT-form responses cannot be modulus-switched (switching needs coefficients)");
  ctx->ntt_responses = form == 1;
  return SANNS_OK;
}

int sanns_set_response_primes(sanns_ctx* ctx, uint32_t primes) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (primes != 1 && primes != ctx->P.L)
    return fail(SANNS_EINVAL, "primes must be 1 (switch to q_0) or L (every prime)");
  if (primes != ctx->P.L && ctx->ntt_responses)
    return fail(SANNS_EINVAL, "NTT-form responses cannot be modulus-switched (switching needs coefficients)");
  // after the switch the phase noise is (q_0 / Q) e plus the rounding
  // (|eps_0 + eps_1 s| <= (N + 1) / 2); decryption mod q_0 needs it below
  // q_0 / (2t), with e up to the largest flooding, Q / (4t): q_0 > 2t (N + 5)
  if (primes == 1 && (u128)ctx->P.q[0] <= (u128)2 * ctx->P.t * (ctx->P.N + 5))
    return fail(SANNS_EINVAL, "q_0 too small to switch to: decryption needs q_0 > 2 t (N + 5)");
  ctx->response_primes = primes;
  return SANNS_OK;
}

int sanns_copy_responses(const sanns_ctx* ctx, const uint64_t* ct_out, uint32_t B, uint64_t K, uint64_t* dst,
                         void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (B == 0 || K == 0) return SANNS_OK;
  if (!ct_out || !dst) return fail(SANNS_EINVAL, "NULL buffer");
  const uint64_t N = ctx->P.N, L = ctx->P.L, rows = (uint64_t)B * K * 2;
  cudaStream_t st = as_stream(stream);
  if (ctx->response_primes == L)
    SANNS_CUDA(cudaMemcpyAsync(dst, ct_out, sizeof(uint64_t) * rows * L * N, cudaMemcpyDefault, st));
  else
    SANNS_CUDA(cudaMemcpy2DAsync(dst, sizeof(uint64_t) * N, ct_out, sizeof(uint64_t) * L * N,
                                 sizeof(uint64_t) * N, rows, cudaMemcpyDefault, st));
  return SANNS_OK;
}

int sanns_topk(sanns_ctx* ctx, const uint32_t* cli, const uint32_t* srv, uint32_t B, uint64_t n,
               uint32_t k, uint64_t bins, uint32_t shift, uint32_t* dist, uint64_t* pos, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (B == 0) return SANNS_OK;
  if (!cli || !srv || !dist || !pos) return fail(SANNS_EINVAL, "NULL buffer");
  if (k < 1 || k > kTopkLarge) return fail(SANNS_EINVAL, "k must be in [1, 1024]");
  if (B > 65535) return fail(SANNS_EINVAL, "B must be <= 65535");
  if (n < k || n >= (1ull << 32)) return fail(SANNS_EINVAL, "need k <= n < 2^32");
  if (bins && (bins < k || bins > n)) return fail(SANNS_EINVAL, "need k <= bins <= n");
  if (shift > 31) return fail(SANNS_EINVAL, "shift must be <= 31");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_topk(cli, srv, B, n, ctx->P.t, k, bins, shift, dist, pos, as_stream(stream)));
  return SANNS_OK;
}

int sanns_topk_segments(sanns_ctx* ctx, const uint32_t* cli, const uint32_t* srv, uint32_t B,
                        const uint64_t* cli_off, const uint64_t* srv_off, const uint64_t* len,
                        const uint32_t* k_seg, const uint64_t* bins_seg, uint32_t k, uint64_t bins,
                        uint32_t shift, uint32_t* dist, uint64_t* pos, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (B == 0) return SANNS_OK;
  if (!cli || !srv || !dist || !pos || !cli_off || !srv_off || !len)
    return fail(SANNS_EINVAL, "NULL buffer");
  if (k < 1 || k > kTopkLarge) return fail(SANNS_EINVAL, "k must be in [1, 1024]");
  if (B > 65535) return fail(SANNS_EINVAL, "B must be <= 65535");
  if (shift > 31) return fail(SANNS_EINVAL, "shift must be <= 31");
  if (bins && bins < k) return fail(SANNS_EINVAL, "need bins = 0 or bins >= k");
  std::vector<uint64_t> seg(5 * (size_t)B);
  for (uint32_t b = 0; b < B; ++b) {
    if (len[b] >= (1ull << 32)) return fail(SANNS_EINVAL, "segment longer than 2^32 - 1");
    const uint64_t kb = k_seg ? k_seg[b] : k;
    const uint64_t lb = bins_seg ? bins_seg[b] : bins;
    if (kb < 1 || kb > k) return fail(SANNS_EINVAL, "need 1 <= k_seg[b] <= k");
    if (bins && (lb < kb || lb > bins)) return fail(SANNS_EINVAL, "need k_seg[b] <= bins_seg[b] <= bins");
    seg[b] = cli_off[b];
    seg[B + b] = srv_off[b];
    seg[2 * (size_t)B + b] = len[b];
    seg[3 * (size_t)B + b] = kb;
    seg[4 * (size_t)B + b] = lb;
  }
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_topk_segments(cli, srv, B, seg.data(), ctx->P.t, k, bins, shift, dist, pos,
                                  as_stream(stream)));
  return SANNS_OK;
}

int sanns_public_key(sanns_ctx* ctx, const sanns_sk* sk, uint64_t seed, uint64_t* pk, void* stream) {
  if (!ctx || !sk || !pk) return fail(SANNS_EINVAL, "ctx, sk or pk is NULL");
  if (sk->ctx != ctx) return fail(SANNS_EINVAL, "key belongs to another context");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_public_key(ctx->P, sk->d_s_hat, sk->d_s_hat_shoup, seed, pk, as_stream(stream)));
  return SANNS_OK;
}

int sanns_circuit_privacy_max_flood_bits(const sanns_ctx* ctx) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  // Delta = floor(Q / t): Q = prod q_j in 64-bit limbs, long division by t
  uint64_t Q[kMaxPrimes + 1] = {1};
  for (uint32_t j = 0; j < ctx->params.L; ++j) {
    u128 carry = 0;
    for (uint32_t i = 0; i <= kMaxPrimes; ++i) {
      const u128 v = (u128)Q[i] * ctx->P.q[j] + carry;
      Q[i] = (uint64_t)v;
      carry = v >> 64;
    }
  }
  u128 rem = 0;
  int bits = 0;
  for (int i = kMaxPrimes; i >= 0; --i) {
    const u128 cur = (rem << 64) | Q[i];
    const uint64_t qd = (uint64_t)(cur / ctx->P.t);
    rem = cur % ctx->P.t;
    if (!bits && qd) bits = 64 * i + (64 - __builtin_clzll(qd));
  }
  // 2^F plus the structured noise stays below Delta / 2
  return bits - 3 > 255 ? 255 : bits - 3;
}

int sanns_set_circuit_privacy(sanns_ctx* ctx, const uint64_t* pk, uint32_t flood_bits, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if (!pk) {
    SANNS_CUDA(cudaStreamSynchronize(st));
    cudaFree(ctx->d_pk);
    cudaFree(ctx->d_pk_shoup);
    ctx->d_pk = ctx->d_pk_shoup = nullptr;
    return SANNS_OK;
  }
  const int fmax = sanns_circuit_privacy_max_flood_bits(ctx);
  if ((int)flood_bits > fmax)
    return fail(SANNS_EINVAL, "flood_bits above " + std::to_string(fmax) +
                                  " would break decryption (2^F must stay below Delta / 4)");
  const size_t words = 2ull * ctx->params.L * ctx->P.N;
  if (!ctx->d_pk) {
    SANNS_CUDA(cudaMalloc(&ctx->d_pk, sizeof(uint64_t) * words));
    SANNS_CUDA(cudaMalloc(&ctx->d_pk_shoup, sizeof(uint64_t) * words));
  }
  SANNS_CUDA(cudaMemcpyAsync(ctx->d_pk, pk, sizeof(uint64_t) * words, cudaMemcpyDefault, st));
  SANNS_CUDA(launch_key_shoup(ctx->P, ctx->d_pk, ctx->d_pk_shoup, st));
  SANNS_CUDA(cudaStreamSynchronize(st));
  ctx->flood_bits = flood_bits;
  for (uint32_t j = 0; j < ctx->params.L; ++j) {
    const uint64_t q = ctx->P.q[j];
    ctx->privacy.q_barrett[j] = (uint64_t)(((u128)1 << 64) / q);
    u128 v = 1 % q;
    for (uint32_t i = 0; i < flood_bits; ++i) v = (v * 2) % q;
    ctx->privacy.two_f[j] = (uint64_t)v;
  }
  return SANNS_OK;
}

int sanns_mac_variants(void) { return mac_num_variants(); }

const char* sanns_mac_variant_name(int v) { return mac_variant_name(v); }

int sanns_set_mac_sms(sanns_ctx* ctx, int sms) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (sms < 0) return fail(SANNS_EINVAL, "sms must be >= 0");
  ctx->mac_sms = sms;
  return SANNS_OK;
}

int sanns_set_mac_variant(sanns_ctx* ctx, int v) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (v < 0 || v >= mac_num_variants()) return fail(SANNS_EINVAL, "no such MAC variant");
  ctx->mac_variant = v;
  return SANNS_OK;
}

int sanns_autotune_mac(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                       uint64_t* ct_out, int reps, float* ms_out, void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0 || !ct_in || !ct_out) return fail(SANNS_EINVAL, "NULL buffer or empty batch");
  if (reps < 1) reps = 1;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  SANNS_CUDA(cudaEventCreate(&e0));
  SANNS_CUDA(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  for (int v = 0; v < mac_num_variants(); ++v) {
    cudaError_t e = launch_mac(ctx->P, ct_in, db->d_pt, B, ctx->params.d, db->K, ct_out, ctx->sms, v, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
      e = launch_mac(ctx->P, ct_in, db->d_pt, B, ctx->params.d, db->K, ct_out, ctx->sms, v, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(e, "autotune");
    }
    ms /= reps;
    if (ms_out) ms_out[v] = ms;
    if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->mac_variant = best;
  return best;
}

int sanns_distances(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                    uint64_t mask_seed, const uint64_t* qids, uint64_t* ct_out, uint32_t* srv_share,
                    void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0) return SANNS_OK;
  if (!ct_in || !qids || !ct_out || !srv_share) return fail(SANNS_EINVAL, "NULL buffer");
  rc = sanns_distances_mac(ctx, db, ct_in, B, ct_out, stream);
  if (rc) return rc;
  return sanns_distances_finish(ctx, db, B, mask_seed, qids, ct_out, srv_share, stream);
}

int sanns_clusters_create(sanns_ctx* ctx, const uint8_t* coords, uint64_t n,
                          const uint64_t* offsets_host, const uint32_t* members, uint32_t C,
                          sanns_clusters** out, void* stream) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (!coords || !offsets_host || !members || n == 0 || C == 0)
    return fail(SANNS_EINVAL, "NULL buffer or empty clustering");
  if (offsets_host[0] != 0) return fail(SANNS_EINVAL, "offsets[0] must be 0");
  for (uint32_t c = 0; c < C; ++c)
    if (offsets_host[c + 1] < offsets_host[c]) return fail(SANNS_EINVAL, "offsets must be non-decreasing");
  const uint64_t M = offsets_host[C];
  if (M > n) return fail(SANNS_EINVAL, "more members than points");
  int rc = check_device(ctx);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  const uint32_t d = ctx->params.d;
  sanns_clusters* cl = new sanns_clusters();
  cl->ctx = ctx;
  cl->n = n;
  cl->C = C;
  cl->h_offsets.assign(offsets_host, offsets_host + C + 1);
  int* d_bad = nullptr;
  cudaError_t e = cudaMalloc(&cl->d_coords, n * d);
  if (e == cudaSuccess) e = cudaMalloc(&cl->d_members, sizeof(uint32_t) * (M ? M : 1));
  if (e == cudaSuccess) e = cudaMalloc(&cl->d_offsets, sizeof(uint64_t) * (C + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(cl->d_coords, coords, n * d, cudaMemcpyDefault, st);
  if (e == cudaSuccess && M) e = cudaMemcpyAsync(cl->d_members, members, sizeof(uint32_t) * M, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cl->d_offsets, offsets_host, sizeof(uint64_t) * (C + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (e == cudaSuccess && M) e = launch_check_indices(cl->d_members, M, n, d_bad, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_bad);
  if (e != cudaSuccess) {
    sanns_clusters_free(cl);
    return cuda_fail(e, "clusters_create");
  }
  if (bad) {
    sanns_clusters_free(cl);
    return fail(SANNS_EINVAL, "members holds an index >= n");
  }
  *out = cl;
  return SANNS_OK;
}

void sanns_clusters_free(sanns_clusters* cl) {
  if (!cl) return;
  cudaFree(cl->d_coords);
  cudaFree(cl->d_members);
  cudaFree(cl->d_offsets);
  delete cl;
}

int sanns_gather_plan(const sanns_clusters* cl, const uint32_t* probes, uint32_t B, uint32_t P,
                      uint64_t* n_out, uint64_t* blocks_out) {
  if (!cl) return fail(SANNS_EINVAL, "clusters is NULL");
  if (B && (!probes || !n_out)) return fail(SANNS_EINVAL, "NULL buffer");
  if (B && P == 0) return fail(SANNS_EINVAL, "P must be positive");
  const uint32_t N = cl->ctx->P.N;
  for (uint32_t b = 0; b < B; ++b) {
    uint64_t acc = 0;
    for (uint32_t p = 0; p < P; ++p) {
      const uint32_t c = probes[(size_t)b * P + p];
      if (c >= cl->C) return fail(SANNS_EINVAL, "probe names a cluster id >= C");
      acc += cl->h_offsets[c + 1] - cl->h_offsets[c];
    }
    n_out[b] = acc;
    if (blocks_out) blocks_out[b] = (acc + N - 1) / N;
  }
  return SANNS_OK;
}

int sanns_distances_gather(sanns_ctx* ctx, const sanns_clusters* cl, const uint64_t* ct_in, uint32_t B,
                           const uint32_t* probes, uint32_t P, uint64_t mask_seed, const uint64_t* qids,
                           uint64_t* ct_out, uint32_t* srv_share, uint32_t* ids, void* stream) {
  if (!ctx || !cl) return fail(SANNS_EINVAL, "ctx or clusters is NULL");
  if (cl->ctx != ctx) return fail(SANNS_EINVAL, "clusters belong to another context");
  if (ctx->P.N > 8192) return fail(SANNS_EINVAL, "the gather path supports N <= 8192");
  if (B == 0) return SANNS_OK;
  if (!ct_in || !qids || !ct_out || !srv_share || !probes) return fail(SANNS_EINVAL, "NULL buffer");
  std::vector<uint64_t> nb(B), kb(B);
  int rc = sanns_gather_plan(cl, probes, B, P, nb.data(), kb.data());
  if (rc) return rc;
  uint64_t W = 0;
  for (uint32_t b = 0; b < B; ++b) W += kb[b];
  if (W * 2 * ctx->P.L > 0x7fffffffull || W * ctx->P.N > (1ull << 40)) return fail(SANNS_EINVAL, "batch too large");
  rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_gather(ctx->P, ctx->params.d, cl, ct_in, B, probes, P, nb.data(), mask_seed, qids,
                           ct_out, srv_share, ids, ctx->sms, ctx->slots ? &ctx->PT : nullptr, ctx->d_pk,
                           ctx->d_pk_shoup, ctx->flood_bits, ctx->privacy, ctx->ntt_responses,
                           as_stream(stream)));
  if (ctx->response_primes == 1)
    SANNS_CUDA(launch_mod_switch(ctx->P, ctx->MS, ct_out, W * 2, as_stream(stream)));
  return SANNS_OK;
}

int sanns_gather_prepare(sanns_ctx* ctx, const sanns_clusters* cl, const uint32_t* probes, uint32_t B,
                         uint32_t P, sanns_gather_batch** out) {
  if (!out) return fail(SANNS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx || !cl) return fail(SANNS_EINVAL, "ctx or clusters is NULL");
  if (cl->ctx != ctx) return fail(SANNS_EINVAL, "clusters belong to another context");
  if (ctx->P.N > 8192) return fail(SANNS_EINVAL, "the gather path supports N <= 8192");
  if (B == 0 || B > 65535) return fail(SANNS_EINVAL, "B must be in 1..65535");
  if (!probes) return fail(SANNS_EINVAL, "probes is NULL");
  sanns_gather_batch* gb = new sanns_gather_batch();
  gb->ctx = ctx;
  gb->cl = cl;
  gb->B = B;
  gb->P = P;
  gb->n_b.assign(B, 0);
  gb->k_b.assign(B, 0);
  int rc = sanns_gather_plan(cl, probes, B, P, gb->n_b.data(), gb->k_b.data());
  uint64_t W = 0;
  for (uint32_t b = 0; rc == 0 && b < B; ++b) W += gb->k_b[b];
  if (rc == 0 && (W * 2 * ctx->P.L > 0x7fffffffull || W * ctx->P.N > (1ull << 40)))
    rc = fail(SANNS_EINVAL, "batch too large");
  if (rc == 0) rc = check_device(ctx);
  if (rc == 0) {
    const cudaError_t e = gather_prepare(ctx->P.N, probes, gb);
    if (e != cudaSuccess) rc = cuda_fail(e, "upload the gather plan");
  }
  if (rc) {
    delete gb;
    return rc;
  }
  *out = gb;
  return SANNS_OK;
}

void sanns_gather_batch_free(sanns_gather_batch* gb) {
  if (!gb) return;
  if (gb->d_tables) cudaFree(gb->d_tables);
  delete gb;
}

int sanns_distances_gather_prepared(sanns_ctx* ctx, const sanns_gather_batch* gb, const uint64_t* ct_in,
                                    uint64_t mask_seed, const uint64_t* qids, uint64_t* ct_out,
                                    uint32_t* srv_share, uint32_t* ids, void* stream) {
  if (!ctx || !gb) return fail(SANNS_EINVAL, "ctx or batch is NULL");
  if (gb->ctx != ctx) return fail(SANNS_EINVAL, "the batch belongs to another context");
  if (!ct_in || !qids || !ct_out || !srv_share) return fail(SANNS_EINVAL, "NULL buffer");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_gather_prepared(ctx->P, ctx->params.d, gb, ct_in, mask_seed, qids, ct_out, srv_share, ids,
                                    ctx->sms, ctx->slots ? &ctx->PT : nullptr, ctx->d_pk, ctx->d_pk_shoup,
                                    ctx->flood_bits, ctx->privacy, ctx->ntt_responses, as_stream(stream)));
  if (ctx->response_primes == 1)
    SANNS_CUDA(launch_mod_switch(ctx->P, ctx->MS, ct_out, gb->W * 2, as_stream(stream)));
  return SANNS_OK;
}

int sanns_db_prepare_batched(sanns_ctx* ctx, sanns_db* db, void* stream) {
  if (!ctx || !db) return fail(SANNS_EINVAL, "ctx or db is NULL");
  if (db->ctx != ctx) return fail(SANNS_EINVAL, "db belongs to another context");
  if (ctx->params.d > 128) return fail(SANNS_EINVAL, "the batched path needs d <= 128 (exact fp32 sums)");
  if (ctx->P.N < 32) return fail(SANNS_EINVAL, "the batched path needs N >= 32");
  if (db->K > 0x7fffffffull) return fail(SANNS_EINVAL, "too many blocks");
  int rc = check_device(ctx);
  if (rc) return rc;
  if (db->d_plimb) return SANNS_OK;
  cudaStream_t st = as_stream(stream);
  const size_t bytes = batched_limb_bytes(ctx->P.L, ctx->P.N, db->K, ctx->params.d);
  uint16_t* pl = nullptr;
  SANNS_CUDA(cudaMalloc(&pl, bytes));
  cudaError_t e = launch_prepare_limbs(ctx->P, db->d_pt, db->K, ctx->params.d, pl, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { cudaFree(pl); return cuda_fail(e, "prepare batched digits"); }
  rc = make_limb_map(ctx->P, pl, db->K, ctx->params.d, db->limb_map);
  if (rc) { cudaFree(pl); return rc; }
  db->d_plimb = pl;
  return SANNS_OK;
}

int sanns_distances_batched_mac(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                                uint64_t* ct_out, void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0) return SANNS_OK;
  if (!db->d_plimb) return fail(SANNS_EINVAL, "call sanns_db_prepare_batched first");
  if (!ct_in || !ct_out) return fail(SANNS_EINVAL, "NULL buffer");
  if (B > 4096) return fail(SANNS_EINVAL, "B must be <= 4096");
  SANNS_CUDA(launch_batched_mac(ctx->P, db->limb_map, db->d_plimb, ct_in, B, ctx->params.d, db->K, ct_out, ctx->d_err,
                                mac_grid_sms(ctx), ctx->batched_tune, as_stream(stream)));
  return SANNS_OK;
}

int sanns_distances_batched(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                            uint64_t mask_seed, const uint64_t* qids, uint64_t* ct_out, uint32_t* srv_share,
                            void* stream) {
  int rc = sanns_distances_batched_mac(ctx, db, ct_in, B, ct_out, stream);
  if (rc) return rc;
  return sanns_distances_finish(ctx, db, B, mask_seed, qids, ct_out, srv_share, stream);
}

int sanns_distances_scratch_bytes(const sanns_ctx* ctx, uint32_t B, int batched, uint64_t* bytes) {
  if (!ctx || !bytes) return fail(SANNS_EINVAL, "ctx or bytes is NULL");
  *bytes = 0;
  if (B == 0 || !batched) return SANNS_OK;   // the per-query path allocates nothing
  if (B > 4096) return fail(SANNS_EINVAL, "B must be <= 4096");
  *bytes = batched_scratch_bytes(ctx->P, B, ctx->params.d, ctx->batched_tune);
  return SANNS_OK;
}

int sanns_batched_tune(sanns_ctx* ctx, uint32_t tma_ns, uint32_t mma_ns, uint32_t producer_ns,
                       uint32_t epilogue_ns, uint32_t prefetch_units, uint32_t scratch_mib,
                       uint32_t tile) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (tma_ns > 100000 || mma_ns > 100000 || producer_ns > 100000 || epilogue_ns > 100000)
    return fail(SANNS_EINVAL, "back-off above 100 us");
  if (prefetch_units > 8) return fail(SANNS_EINVAL, "prefetch distance above 8 units");
  if (scratch_mib < 1 || scratch_mib > (1u << 20)) return fail(SANNS_EINVAL, "scratch cap outside 1 MiB .. 1 TiB");
  if (tile > 8)
    return fail(SANNS_EINVAL,
                "tile must be 0..8 (0..3: bit 0 = 256 blocks on an SM pair, bit 1 = query digits by TMA; "
                "4, 5: TMA-fed, clusters of 2 or 4 sharing the query tile; 6, 7: TMA-fed, four slots per "
                "CTA with 32-byte stores, alone or in clusters of 2; 8: four slots per SM pair)");
  ctx->batched_tune[0] = tma_ns;
  ctx->batched_tune[1] = mma_ns;
  ctx->batched_tune[2] = producer_ns;
  ctx->batched_tune[3] = epilogue_ns;
  ctx->batched_tune[4] = prefetch_units;
  ctx->batched_tune[5] = scratch_mib;
  ctx->batched_tune[6] = tile;
  return SANNS_OK;
}

int sanns_autotune_batched(sanns_ctx* ctx, const sanns_db* db, const uint64_t* ct_in, uint32_t B,
                           uint64_t* ct_out, int reps, float* ms_out, void* stream) {
  int rc = check_distance_args(ctx, db, B);
  if (rc) return rc;
  if (B == 0 || !ct_in || !ct_out) return fail(SANNS_EINVAL, "NULL buffer or empty batch");
  if (!db->d_plimb) return fail(SANNS_EINVAL, "call sanns_db_prepare_batched first");
  if (B > 4096) return fail(SANNS_EINVAL, "B must be <= 4096");
  if (reps < 1) reps = 1;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  SANNS_CUDA(cudaEventCreate(&e0));
  SANNS_CUDA(cudaEventCreate(&e1));
  const uint32_t saved[2] = {ctx->batched_tune[4], ctx->batched_tune[6]};
  int best = -1;
  float best_ms = 0.f;
  for (int cfg = 0; cfg < kBatchedConfigs; ++cfg) {
    ctx->batched_tune[6] = (uint32_t)(cfg >> 1);   // tile shape
    ctx->batched_tune[4] = (uint32_t)(cfg & 1);    // L2 prefetch distance
    auto launch = [&]() {
      return launch_batched_mac(ctx->P, db->limb_map, db->d_plimb, ct_in, B, ctx->params.d, db->K, ct_out,
                                ctx->d_err, mac_grid_sms(ctx), ctx->batched_tune, st);
    };
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      ctx->batched_tune[4] = saved[0];
      ctx->batched_tune[6] = saved[1];
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(e, "batched autotune");
    }
    ms /= reps;
    if (ms_out) ms_out[cfg] = ms;
    if (best < 0 || ms < best_ms) { best = cfg; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->batched_tune[6] = (uint32_t)(best >> 1);
  ctx->batched_tune[4] = (uint32_t)(best & 1);
  return best;
}

int sanns_selftest_wait_timeout(sanns_ctx* ctx, uint32_t limit_ms, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  if (limit_ms < 1 || limit_ms > 1000) return fail(SANNS_EINVAL, "limit_ms must be in [1, 1000]");
  int rc = check_device(ctx);
  if (rc) return rc;
  SANNS_CUDA(launch_wait_selftest(ctx->d_err, limit_ms, ctx->device, as_stream(stream)));
  return SANNS_OK;
}

int sanns_measure_mma_rates(sanns_ctx* ctx, double* rates_host, void* stream) {
  if (!ctx || !rates_host) return fail(SANNS_EINVAL, "ctx or rates_host is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  double r[3] = {0, 0, 0};
  SANNS_CUDA(measure_mma_rates(ctx->sms, ctx->d_err, r, as_stream(stream)));
  rc = sanns_device_status(ctx, stream);
  if (rc) return rc;
  for (int i = 0; i < 3; ++i) rates_host[i] = r[i];
  return SANNS_OK;
}

int sanns_measure_int_rates(sanns_ctx* ctx, double* rates_host, void* stream) {
  if (!ctx || !rates_host) return fail(SANNS_EINVAL, "ctx or rates_host is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  double r[2] = {0, 0};
  SANNS_CUDA(measure_int_rates(ctx->P, ctx->sms, r, as_stream(stream)));
  rates_host[0] = r[0];
  rates_host[1] = r[1];
  return SANNS_OK;
}

int sanns_device_status(sanns_ctx* ctx, void* stream) {
  if (!ctx) return fail(SANNS_EINVAL, "ctx is NULL");
  int rc = check_device(ctx);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  int h = 0;
  SANNS_CUDA(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SANNS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    SANNS_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
    SANNS_CUDA(cudaStreamSynchronize(st));
    return fail(h, "a bounded device-side wait gave up");
  }
  return SANNS_OK;
}

int sanns_decrypt_shares(sanns_ctx* ctx, const sanns_sk* sk, const uint64_t* ct_out, uint32_t B,
                         uint64_t n, const uint8_t* qv, uint32_t* cli_share, void* stream) {
  if (!ctx || !sk) return fail(SANNS_EINVAL, "ctx or sk is NULL");
  if (sk->ctx != ctx) return fail(SANNS_EINVAL, "sk belongs to another context");
  if (B == 0 || n == 0) return SANNS_OK;
  if (!ct_out || !qv || !cli_share) return fail(SANNS_EINVAL, "NULL buffer");
  const uint64_t K = (n + ctx->P.N - 1) / ctx->P.N;
  // switched responses ([B][K][2][N], modulo q_0) decrypt in the one-prime view
  const PrimeSet& PD = ctx->response_primes == 1 ? ctx->P1 : ctx->P;
  if ((uint64_t)B * K * PD.L > 0x7fffffffull || (uint64_t)B * n > (1ull << 40))
    return fail(SANNS_EINVAL, "batch too large");
  int rc = check_device(ctx);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  uint64_t* scratch = nullptr;
  SANNS_CUDA(cudaMallocAsync(&scratch, sizeof(uint64_t) * B * K * PD.L * PD.N, st));
  cudaError_t e = launch_decrypt(PD, ct_out, sk->d_s, sk->d_s_hat, sk->d_s_hat_shoup, B, K, n, qv,
                                 ctx->params.d, scratch, cli_share, ctx->ntt_responses,
                                 ctx->slots ? &ctx->PT : nullptr, st);
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_fail(e, "decrypt kernels");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return SANNS_OK;
}

}  // extern "C"
