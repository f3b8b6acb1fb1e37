// Measured arithmetic peaks of the device, the denominators of the bench's ALU
// roofline fractions (the paper has no counterpart).
//
//   FP32 CUDA cores: every thread runs 8 independent FMA chains.
//   TF32 tensor cores: one CTA per SM, one thread issuing back-to-back
//   tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8) from shared memory into one
//   TMEM accumulator; the operands are zero (the values do not change the rate).
//
// Both are timed with CUDA events around one launch after a warm-up launch.
// The tensor kernel waits for its MMAs on an mbarrier with a bounded wait
// (about one second); a wait that runs out is reported as
// CMCG_ERR_DEVICE_TIMEOUT.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cmcg.h"

namespace {

__global__ void fma_loop(float* out, int iters, float seed) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + float(threadIdx.x + k);
  const float b = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.0f) out[threadIdx.x] = s;  // keeps the chains live
}

constexpr int PK_N = 256;
constexpr int PK_K = 8;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__global__ void __launch_bounds__(128, 1) tf32_mma_loop(int iters, int* err) {
  __shared__ __align__(128) uint32_t sA[128 * PK_K];
  __shared__ __align__(128) uint32_t sB[PK_N * PK_K];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 128 * PK_K; i += blockDim.x) sA[i] = 0u;
  for (int i = tid; i < PK_N * PK_K; i += blockDim.x) sB[i] = 0u;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(s_addr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s_addr(&tbase)),
                 "r"(PK_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tbase;
  if (tid == 0) {
    // K-major, no swizzle: core matrices of 8 rows x 16 bytes, LBO 128 bytes (along K),
    // SBO 256 bytes (8 rows x 2 core matrices of K = 8).
    auto desc = [](uint32_t addr) {
      return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t(256 >> 4) << 32) |
             (uint64_t(1) << 46);
    };
    const uint64_t da = desc(s_addr(sA)), db = desc(s_addr(sB));
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(PK_N >> 3) << 17) | (uint32_t(128 >> 4) << 24);
    for (int i = 0; i < iters; ++i) {
      const uint32_t acc = i > 0 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(idesc), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(s_addr(&bar))
                 : "memory");
  }
  uint32_t done = 0;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (;;) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(s_addr(&bar))
        : "memory");
    if (done) break;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) break;
  }
  if (!done && tid == 0) atomicOr(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(PK_N));
  }
}

int fail(cudaError_t e) { return e == cudaErrorNoDevice ? CMCG_ERR_NO_DEVICE : CMCG_ERR_CUDA; }

}  // namespace

extern "C" int cmcg_measure_peaks(int device, double* fp32_tflops, double* tf32_tflops) {
  if (device < 0) return CMCG_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(e);
  int nsm = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return fail(e);
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreate(&b)) != cudaSuccess) return fail(e);
  float* sink = nullptr;
  int* err = nullptr;
  int rc = CMCG_OK;
  float ms = 0;
  if (cudaMalloc(&sink, 1024 * sizeof(float)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    rc = CMCG_ERR_OUT_OF_MEMORY;
    goto done;
  }
  cudaMemset(err, 0, sizeof(int));
  if (fp32_tflops) {
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    fma_loop<<<blocks, threads>>>(sink, iters / 8, 1.0f);
    cudaEventRecord(a);
    fma_loop<<<blocks, threads>>>(sink, iters, 1.0f);
    cudaEventRecord(b);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
      rc = fail(e);
      goto done;
    }
    cudaEventElapsedTime(&ms, a, b);
    *fp32_tflops = double(blocks) * threads * iters * 8 * 2 / (ms * 1e-3) / 1e12;
  }
  if (tf32_tflops) {
    const int iters = 20000;
    tf32_mma_loop<<<nsm, 128>>>(iters / 10, err);
    cudaEventRecord(a);
    tf32_mma_loop<<<nsm, 128>>>(iters, err);
    cudaEventRecord(b);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
      rc = fail(e);
      goto done;
    }
    int herr = 0;
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) {
      rc = CMCG_ERR_DEVICE_TIMEOUT;
      goto done;
    }
    cudaEventElapsedTime(&ms, a, b);
    *tf32_tflops = double(nsm) * iters * 2.0 * 128 * PK_N * PK_K / (ms * 1e-3) / 1e12;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) rc = fail(e);
done:
  cudaFree(sink);
  cudaFree(err);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}
