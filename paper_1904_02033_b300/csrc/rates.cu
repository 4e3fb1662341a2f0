// Measured peak rates of the current GPU (no counterpart in the paper): the
// denominators of the rooflines.
//
// Tensor cores, for the batched path.  The batched MAC contracts exact small
// integers; the candidate instruction families are
//   - tcgen05.mma kind::f16 (fp16 operands, fp32 accumulation in TMEM), the
//     one the batched kernel uses;
//   - the legacy warp-level mma.sync with fp16 operands;
//   - the legacy warp-level mma.sync with s8 operands and s32 accumulation.
// tcgen05.mma kind::i8 (8-bit integer operands on the 5th-generation tensor
// cores) does not exist on sm_103a: ptxas rejects the instruction for that
// target, so the only INT8 tensor instruction left is the legacy mma.sync.
//
// Each probe keeps its operands in registers or in zeroed shared memory, so
// it measures issue-to-completion throughput only; the values are irrelevant.
#include "internal.h"

namespace sanns {
namespace {

constexpr uint32_t kRateThreadsSync = 256;

__global__ void __launch_bounds__(kRateThreadsSync) sync_f16_rate_kernel(uint32_t iters, float* out) {
  const uint32_t a = 0x3c003c00u, b = 0x3c003c00u;  // fp16 pairs (1.0, 1.0)
  float acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(acc[u][0]), "+f"(acc[u][1]), "+f"(acc[u][2]), "+f"(acc[u][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += acc[u][0] + acc[u][1] + acc[u][2] + acc[u][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRateThreadsSync) sync_s8_rate_kernel(uint32_t iters, float* out) {
  const uint32_t a = 0x01010101u, b = 0x01010101u;
  int acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+r"(acc[u][0]), "+r"(acc[u][1]), "+r"(acc[u][2]), "+r"(acc[u][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  int s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += acc[u][0] + acc[u][1] + acc[u][2] + acc[u][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// tcgen05 probe: A (128 x 64 fp16) and B (256 x 64 fp16) zeroed in shared
// memory in the 128-byte-swizzled K-major layout; one thread issues `iters`
// groups of four M128 N256 K16 MMAs into one TMEM accumulator, commits once
// and waits (bounded) for completion.  One CTA per SM (the shared-memory
// request leaves room for one).
constexpr uint32_t kTcA = 128 * 64 * 2, kTcB = 256 * 64 * 2;
constexpr uint32_t kTcSmem = 120 * 1024;
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__global__ void __launch_bounds__(128, 1) tc_f16_rate_kernel(uint32_t iters, int* err) {
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  uint8_t* base = dsmem + ((1024 - (smem_addr(dsmem) & 1023)) & 1023);
  for (uint32_t i = threadIdx.x; i < (kTcA + kTcB) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        smem_addr(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    const uint64_t ad = sw128_desc(smem_addr(base)), bd = sw128_desc(smem_addr(base + kTcA));
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(kTcIdesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(&bar))
                 : "memory");
    const unsigned long long t0 = clock64();
    for (;;) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_addr(&bar))
          : "memory");
      if (ok) break;
      if (clock64() - t0 > (8ull << 30)) {  // ~4 s; the work itself takes milliseconds
        atomicExch(err, SANNS_ETIMEOUT);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

// Integer-pipe probes: the radix-2 butterflies of the transforms (inverse:
// Gentleman-Sande with values below 4q and the three-product Shoup quotient,
// as in the fused INTT; forward: Cooley-Tukey with values below 4q and the
// exact Shoup quotient, as in the forward transforms) on 16 values per thread
// in registers, four stages per round like one radix-16 pass, twiddles read
// once from the context's table.  No memory traffic in the loop: the rate is
// the arithmetic ceiling of one butterfly.
constexpr uint32_t kIntThreads = 256;

__global__ void __launch_bounds__(kIntThreads) inv_bfly_rate_kernel(PrimeSet P, uint32_t iters, uint64_t* out) {
  const uint64_t q = P.q[0], q4 = 4 * q;
  ulonglong2 w[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) w[s] = P.itw[1 + ((threadIdx.x + s) & 31)];
  uint64_t v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = (threadIdx.x * 16ull + k + blockIdx.x) % q;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int hk = 1 << s;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & hk) continue;
        inv_bfly4(v[k], v[k + hk], w[s].x, w[s].y, q, q4);
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc ^= v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(kIntThreads) fwd_bfly_rate_kernel(PrimeSet P, uint32_t iters, uint64_t* out) {
  const uint64_t q = P.q[0], q2 = 2 * q;
  ulonglong2 w[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) w[s] = P.tw[1 + ((threadIdx.x + s) & 31)];
  uint64_t v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = (threadIdx.x * 16ull + k + blockIdx.x) % q;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int hk = 8 >> s;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & hk) continue;
        fwd_bfly(v[k], v[k + hk], w[s].x, w[s].y, q, q2);
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc ^= v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <typename F>
cudaError_t time_launch(cudaStream_t st, F launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  launch();  // warm-up
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) { launch(); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

cudaError_t measure_int_rates(const PrimeSet& P, int sms, double out[2], cudaStream_t st) {
  const uint32_t blocks = (uint32_t)sms * 8;   // 2048 threads per SM
  uint64_t* d_out = nullptr;
  cudaError_t e = cudaMallocAsync(&d_out, sizeof(uint64_t) * blocks * kIntThreads, st);
  if (e != cudaSuccess) return e;
  const uint32_t iters = 256;
  // 4 stages x 8 butterflies per round and thread
  const double bflies = (double)blocks * kIntThreads * iters * 32;
  float ms = 0.f;
  e = time_launch(st, [&] { inv_bfly_rate_kernel<<<blocks, kIntThreads, 0, st>>>(P, iters, d_out); }, &ms);
  if (e == cudaSuccess) out[0] = bflies / (ms * 1e-3);
  if (e == cudaSuccess)
    e = time_launch(st, [&] { fwd_bfly_rate_kernel<<<blocks, kIntThreads, 0, st>>>(P, iters, d_out); }, &ms);
  if (e == cudaSuccess) out[1] = bflies / (ms * 1e-3);
  cudaError_t e2 = cudaFreeAsync(d_out, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t measure_mma_rates(int sms, int* d_err, double out[3], cudaStream_t st) {
  const uint32_t blocks_sync = (uint32_t)sms * 4;
  float* d_out = nullptr;
  cudaError_t e = cudaMallocAsync(&d_out, sizeof(float) * blocks_sync * kRateThreadsSync, st);
  if (e != cudaSuccess) return e;
  float ms = 0.f;
  // tcgen05 kind::f16: 2 * 128 * 256 * 16 flops per MMA, 4 per iteration
  const uint32_t tc_iters = 4096;
  e = cudaFuncSetAttribute(tc_f16_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e == cudaSuccess)
    e = time_launch(st, [&] { tc_f16_rate_kernel<<<sms, 128, kTcSmem, st>>>(tc_iters, d_err); }, &ms);
  if (e == cudaSuccess) out[0] = (double)sms * tc_iters * 4 * (2.0 * 128 * 256 * 16) / (ms * 1e-3) / 1e12;
  // mma.sync f16: 2 * 16 * 8 * 16 flops per instruction and warp, 8 per iteration
  const uint32_t sync_iters = 4096;
  const double warps = (double)blocks_sync * (kRateThreadsSync / 32);
  if (e == cudaSuccess)
    e = time_launch(st, [&] { sync_f16_rate_kernel<<<blocks_sync, kRateThreadsSync, 0, st>>>(sync_iters, d_out); }, &ms);
  if (e == cudaSuccess) out[1] = warps * sync_iters * 8 * (2.0 * 16 * 8 * 16) / (ms * 1e-3) / 1e12;
  // mma.sync s8: 2 * 16 * 8 * 32 ops per instruction and warp
  if (e == cudaSuccess)
    e = time_launch(st, [&] { sync_s8_rate_kernel<<<blocks_sync, kRateThreadsSync, 0, st>>>(sync_iters, d_out); }, &ms);
  if (e == cudaSuccess) out[2] = warps * sync_iters * 8 * (2.0 * 16 * 8 * 32) / (ms * 1e-3) / 1e12;
  cudaError_t e2 = cudaFreeAsync(d_out, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace sanns
