// Host-side structures behind the opaque handles of sanns.h.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

struct sanns_ctx {
  sanns_params params;
  sanns::PrimeSet P;        // device pointers inside
  uint64_t psi[sanns::kMaxPrimes];
  uint64_t* d_tables;       // one allocation for the four twiddle tables
  int device;
  int sms;
  int mac_variant;          // launch variant of the MAC kernel (autotuned)
  int mac_sms;              // SMs the MAC kernel's persistent grid uses (0: all)
  int* d_err;               // device error word raised by bounded waits
  uint32_t batched_tune[7]; // batched kernel: back-off ns (TMA, MMA, producers, epilogue), L2 prefetch
                            // units, scratch cap (MiB) of the query multiples, tile (0..3: bit 0 =
                            // 256 blocks on an SM pair instead of 128 on one SM, bit 1 = query
                            // digits by TMA from fp16 rows instead of producer warps; 4, 5: one
                            // SM, TMA-fed, clusters of 2 or 4 sharing the query tile by multicast)
  // circuit privacy: the client's public key (library copy, [2][L][N] NTT
  // form) and its Shoup companions, or NULL; flooding exponent F
  uint64_t* d_pk;
  uint64_t* d_pk_shoup;
  uint32_t flood_bits;
  sanns::PrivacyConsts privacy;
  bool ntt_responses;       // responses in NTT form (server finish and client decryption)
  // responses switched down to q_0 (1) or kept at every prime (L): the
  // one-prime view of the parameters that decrypts them, and the constants
  // of the switch
  uint32_t response_primes;
  sanns::PrimeSet P1;
  sanns::ModSwitchConsts MS;
  // slot encoding (t = 1 mod 2N): the negacyclic transform mod t as a
  // one-prime set (its tables in d_tables_t), and whether new databases and
  // decryptions use it
  sanns::PrimeSet PT;
  uint64_t psi_t;
  uint64_t* d_tables_t;
  bool slots;
};

struct sanns_sk {
  const sanns_ctx* ctx;
  int8_t* d_s;              // [N]
  uint64_t* d_s_hat;        // [L][N]
  uint64_t* d_s_hat_shoup;  // [L][N]
};

struct sanns_db {
  const sanns_ctx* ctx;
  uint64_t n, K;
  uint64_t pos0;            // global position of local position 0 (shards), multiple of N
  bool slots;               // encoded with slot encoding (points in the CRT slots mod t)
  uint64_t* d_pt;           // [K][L][d][N], NTT form in the split30 format (common.cuh)
  uint32_t* d_norms;        // [K N]
  uint16_t* d_plimb;        // [L][N][K][8 dpad] fp16 digits (batched path), or NULL
  alignas(64) unsigned char limb_map[128];  // TMA descriptor of d_plimb
};

struct sanns_clusters {
  const sanns_ctx* ctx;
  uint64_t n;               // points
  uint32_t C;               // clusters
  uint8_t* d_coords;        // [n][d], library-owned copy
  uint32_t* d_members;      // [offsets[C]]
  uint64_t* d_offsets;      // [C + 1]
  std::vector<uint64_t> h_offsets;
};

// A prepared gather batch: the plan of one sanns_distances_gather call (work
// items, per-query offsets, probe segments and the probes) uploaded once, so
// that the launches over it are kernels and stream-ordered scratch only.
struct sanns_gather_batch {
  const sanns_ctx* ctx;
  const sanns_clusters* cl;
  uint32_t B, P;
  uint64_t W;               // work items (blocks of the gathered lists)
  std::vector<uint64_t> n_b, k_b;  // gathered points and blocks per query
  uint8_t* d_tables;        // items | queries | segments | probes, or NULL when W = 0
  size_t o_items, o_qs, o_seg, o_pr;
};

namespace sanns {

// error reporting (thread-local message)
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SANNS_CUDA(call)                                  \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return sanns::cuda_fail(_e, #call); \
  } while (0)

// The dynamic shared-memory opt-in of a kernel, set once per (kernel, device)
// for at least `bytes` (thread-safe; a process may drive several devices).
cudaError_t ensure_smem_attr(const void* kernel, size_t bytes);

// parameter derivation (params.cpp)
int derive_params(const sanns_params& in, uint64_t q[], uint64_t psi[], uint64_t* t);
uint64_t smallest_psi(uint64_t q, uint64_t N);
void fill_prime_constants(PrimeSet& P, const uint64_t q[], uint64_t t, uint32_t L);
void fill_twiddles(uint32_t N, uint64_t q, uint64_t psi, uint64_t* tw, uint64_t* tws, uint64_t* itw,
                   uint64_t* itws);
uint64_t shoup_of(uint64_t w, uint64_t q);

cudaError_t launch_norms_mod_t(const PrimeSet& P, uint32_t* norms, uint64_t count, cudaStream_t st);

// modulus switching of the responses down to q_0 (modswitch.cu)
void make_mod_switch_consts(const PrimeSet& P, ModSwitchConsts* C);
cudaError_t launch_mod_switch(const PrimeSet& P, const ModSwitchConsts& C, uint64_t* buf, uint64_t tuples,
                              cudaStream_t st);

// kernel launchers (ntt.cu, mac.cu, client.cu)
cudaError_t launch_ntt(const PrimeSet& P, uint64_t* data, uint64_t count, bool inverse,
                       cudaStream_t st);
cudaError_t launch_public_key(const PrimeSet& P, const uint64_t* s_hat, const uint64_t* s_hat_shoup,
                              uint64_t seed, uint64_t* pk, cudaStream_t st);
cudaError_t launch_key_shoup(const PrimeSet& P, const uint64_t* pk, uint64_t* pks, cudaStream_t st);
cudaError_t launch_rerandomize(const PrimeSet& P, uint64_t* ct, uint32_t B, uint64_t K, uint64_t pos0,
                               uint64_t seed, const uint64_t* qids, const uint64_t* pk,
                               const uint64_t* pks, cudaStream_t st);
cudaError_t launch_flood(const PrimeSet& P, uint64_t* ct, uint32_t B, uint64_t K, uint64_t pos0,
                         uint64_t seed, const uint64_t* qids, uint32_t F, const PrivacyConsts& C,
                         cudaStream_t st);
cudaError_t launch_mask_ntt(const PrimeSet& P, uint64_t* ct_out, const uint32_t* norms, uint32_t B,
                            uint64_t K, uint64_t n, uint64_t pos0, uint64_t mask_seed, const uint64_t* qids,
                            uint32_t* srv_share, bool privacy, uint32_t F, const PrivacyConsts& C,
                            cudaStream_t st);
constexpr uint32_t kTopkLarge = 1024;  // largest k of a selection
cudaError_t launch_topk(const uint32_t* cli, const uint32_t* srv, uint32_t B, uint64_t n, uint64_t t,
                        uint32_t k, uint64_t bins, uint32_t shift, uint32_t* dist, uint64_t* pos,
                        cudaStream_t st);
cudaError_t launch_topk_segments(const uint32_t* cli, const uint32_t* srv, uint32_t B,
                                 const uint64_t* seg_host, uint64_t t, uint32_t k, uint64_t bins,
                                 uint32_t shift, uint32_t* dist, uint64_t* pos, cudaStream_t st);
cudaError_t launch_keygen(const PrimeSet& P, uint64_t seed, int8_t* s, uint64_t* s_hat,
                          uint64_t* s_hat_shoup, cudaStream_t st);
cudaError_t launch_encrypt(const PrimeSet& P, const uint64_t* s_hat, const uint64_t* s_hat_shoup,
                           const uint8_t* qv, uint32_t B, uint32_t d, uint64_t seed,
                           const uint64_t* qids, uint64_t* ct, cudaStream_t st);
cudaError_t launch_seeded_query(const PrimeSet& P, const uint64_t* c0, uint32_t B, uint32_t d,
                                uint64_t seed, const uint64_t* qids, uint64_t* ct, cudaStream_t st);
cudaError_t launch_encode(const PrimeSet& P, const PrimeSet* PT, const uint8_t* coords, uint64_t n_points,
                          const uint32_t* perm, uint64_t n, uint32_t d, uint64_t K, uint64_t* pt,
                          uint32_t* norms, int* bad, cudaStream_t st);
cudaError_t launch_slot_share(const PrimeSet& P, const PrimeSet& PT, uint32_t B, uint64_t K, uint64_t n,
                              uint64_t pos0, uint64_t mask_seed, const uint64_t* qids,
                              uint32_t* srv_share, cudaStream_t st);
int mac_num_variants();
const char* mac_variant_name(int v);
cudaError_t launch_mac(const PrimeSet& P, const uint64_t* ct, const uint64_t* pt, uint32_t B,
                       uint32_t d, uint64_t K, uint64_t* out, int sms, int variant,
                       cudaStream_t st);
cudaError_t launch_intt_mask(const PrimeSet& P, uint64_t* ct_out, const uint32_t* norms,
                             uint32_t B, uint64_t K, uint64_t n, uint64_t pos0, uint64_t mask_seed,
                             const uint64_t* qids, uint32_t* srv_share, int sms, cudaStream_t st);
int gather_threads(uint32_t N);
cudaError_t launch_check_indices(const uint32_t* idx, uint64_t m, uint64_t bound, int* bad,
                                 cudaStream_t st);
cudaError_t launch_gather(const PrimeSet& P, uint32_t d, const sanns_clusters* cl,
                          const uint64_t* ct_in, uint32_t B, const uint32_t* probes_host,
                          uint32_t Pr, const uint64_t* n_b, uint64_t mask_seed,
                          const uint64_t* qids, uint64_t* ct_out, uint32_t* srv_share,
                          uint32_t* ids, int sms, const PrimeSet* PT, const uint64_t* pk,
                          const uint64_t* pks, uint32_t F, const PrivacyConsts& C, bool ntt_form,
                          cudaStream_t st);
cudaError_t gather_prepare(uint32_t N, const uint32_t* probes_host, sanns_gather_batch* gb);
cudaError_t launch_gather_prepared(const PrimeSet& P, uint32_t d, const sanns_gather_batch* gb,
                                   const uint64_t* ct_in, uint64_t mask_seed, const uint64_t* qids,
                                   uint64_t* ct_out, uint32_t* srv_share, uint32_t* ids, int sms,
                                   const PrimeSet* PT, const uint64_t* pk, const uint64_t* pks, uint32_t F,
                                   const PrivacyConsts& C, bool ntt_form, cudaStream_t st);
cudaError_t launch_norms_slot(const PrimeSet& PT, uint32_t* norms, uint64_t K, cudaStream_t st);
cudaError_t launch_join30(const uint64_t* src, uint64_t* dst, uint64_t count, cudaStream_t st);
cudaError_t launch_import_pt(const PrimeSet& P, uint64_t* pt, uint64_t count, uint32_t d, int* bad,
                             cudaStream_t st);
size_t batched_limb_bytes(uint32_t L, uint32_t N, uint64_t K, uint32_t d);
void batched_slot_range(const PrimeSet& P, uint32_t B, uint32_t d, const uint32_t tune[7],
                        uint64_t* per_slot, uint64_t* slots);
size_t batched_scratch_bytes(const PrimeSet& P, uint32_t B, uint32_t d, const uint32_t tune[7]);
cudaError_t launch_wait_selftest(int* err, uint32_t limit_ms, int device, cudaStream_t st);
cudaError_t measure_mma_rates(int sms, int* d_err, double out[3], cudaStream_t st);
cudaError_t measure_int_rates(const PrimeSet& P, int sms, double out[2], cudaStream_t st);
cudaError_t launch_prepare_limbs(const PrimeSet& P, const uint64_t* pt, uint64_t K, uint32_t d,
                                 uint16_t* plimb, cudaStream_t st);
constexpr int kBatchedConfigs = 18;  // (tile shape 0..8, L2 prefetch 0/1) pairs timed by the autotuner
int make_limb_map(const PrimeSet& P, const uint16_t* plimb, uint64_t K, uint32_t d, void* map_out);
cudaError_t launch_batched_mac(const PrimeSet& P, const void* map, const uint16_t* plimb,
                               const uint64_t* ct, uint32_t B,
                               uint32_t d, uint64_t K, uint64_t* out, int* err, int sms,
                               const uint32_t tune[7], cudaStream_t st);
cudaError_t launch_decrypt(const PrimeSet& P, const uint64_t* ct_out, const int8_t* s,
                           const uint64_t* s_hat, const uint64_t* s_hat_shoup, uint32_t B,
                           uint64_t K, uint64_t n, const uint8_t* qv, uint32_t d,
                           uint64_t* scratch, uint32_t* cli_share, bool ntt_form, const PrimeSet* PT,
                           cudaStream_t st);

}  // namespace sanns
