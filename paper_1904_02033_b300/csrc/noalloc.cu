// sanns_decrypt_shares_noalloc: client decryption (the linear-scan protocol's
// step 4, Sec. 5.3; the paper has no allocation-free form) for callers that cannot
// allocate device memory at call time -- for instance code running inside a
// CUDA graph capture, a real-time loop that must not call cudaMalloc (it can
// synchronise the device and its latency is unbounded), or a host that runs
// under a fixed device-memory budget.  It runs the same kernels as
// sanns_decrypt_shares, but the intermediate residues live in a file-scope
// device array instead of a stream-ordered allocation.
#include <mutex>

#include "internal.h"

namespace {

// Scratch for B K L N residues of the decryption's first phase.  Every GPU
// that loads this library holds the array (32 MiB) until the process exits.
constexpr uint64_t kNoAllocWords = 1ull << 22;
__device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
uint64_t* g_scratch_addr[kMaxDevices] = {};

// The array's name is only a host-side stand-in; the device address comes
// from cudaGetSymbolAddress, looked up once per device with that device
// current.
int scratch_for_device(int dev, uint64_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return sanns::fail(SANNS_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return sanns::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return SANNS_OK;
}

}  // namespace

extern "C" uint64_t sanns_decrypt_noalloc_max_words(void) { return kNoAllocWords; }

extern "C" int sanns_decrypt_shares_noalloc(sanns_ctx* ctx, const sanns_sk* sk, const uint64_t* ct_out,
                                            uint32_t B, uint64_t n, const uint8_t* qv,
                                            uint32_t* cli_share, void* stream) {
  using namespace sanns;
  if (!ctx || !sk) return fail(SANNS_EINVAL, "ctx or sk is NULL");
  if (sk->ctx != ctx) return fail(SANNS_EINVAL, "sk belongs to another context");
  if (B == 0 || n == 0) return SANNS_OK;
  if (!ct_out || !qv || !cli_share) return fail(SANNS_EINVAL, "NULL buffer");
  const uint64_t K = (n + ctx->P.N - 1) / ctx->P.N;
  const PrimeSet& PD = ctx->response_primes == 1 ? ctx->P1 : ctx->P;   // switched responses: q_0 alone
  const uint64_t words = (uint64_t)B * K * PD.L * PD.N;
  if (words > kNoAllocWords)
    return fail(SANNS_EINVAL, "decryption needs " + std::to_string(words) +
                                  " scratch words; the static scratch holds " +
                                  std::to_string(kNoAllocWords) + " (B K L N must not exceed it)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != ctx->device) return fail(SANNS_EINVAL, "current device differs from the context's device");
  uint64_t* scratch = nullptr;
  int rc = scratch_for_device(dev, &scratch);
  if (rc) return rc;
  // every scratch word the second phase reads is written by the first phase
  // of the same call, so nothing needs clearing between calls
  e = launch_decrypt(PD, ct_out, sk->d_s, sk->d_s_hat, sk->d_s_hat_shoup, B, K, n, qv,
                     ctx->params.d, scratch, cli_share, ctx->ntt_responses,
                     ctx->slots ? &ctx->PT : nullptr, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "decrypt kernels");
  return SANNS_OK;
}
