// probe.cu -- bandwidth of 1-D bulk copies from L2 into shared memory
// (diagnostic entry point pat_probe_l2_to_smem, include/pat_bp.h).
//
// The staged gather streams every stage's table block and integrand windows
// from L2 into shared memory with cp.async.bulk; the achievable aggregate rate
// of that stream is one of the rooflines of the batched gather.  This probe
// measures it: one CTA per SM streams 64 KB chunks of an L2-resident 64 MB
// buffer into a ring of three shared-memory slots (every thread reads its
// share of each chunk once, so the data really lands), for about 2 GB in all.
// Every wait is bounded; on expiry the CTA records a flag, drains its own
// copies in flight (bounded again) and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "handle.h"

using namespace patbp;

namespace {

constexpr int kChunk = 64 << 10;
constexpr int kSlots = 3;
constexpr size_t kBuffer = size_t(64) << 20;

__global__ void __launch_bounds__(512) l2_to_smem_kernel(const unsigned char* src, int reps,
                                                         uint64_t timeout_ns, int* flag, float* sink) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  unsigned char* ring = sm + 128;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kSlots; ++i) mbar_init(&bar[i], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const size_t n_chunks = kBuffer / kChunk;
  auto issue = [&](int k) {
    const size_t c = (size_t(blockIdx.x) * 131 + size_t(k) * gridDim.x) % n_chunks;
    mbar_arrive_expect_tx(&bar[k % kSlots], kChunk);
    bulk_g2s(ring + (k % kSlots) * kChunk, src + c * kChunk, kChunk, &bar[k % kSlots]);
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < kSlots && k < reps; ++k) issue(k);
  float acc = 0.0f;
  for (int k = 0; k < reps; ++k) {
    const bool got = mbar_wait_bounded(&bar[k % kSlots], uint32_t((k / kSlots) & 1), timeout_ns, nullptr);
    if (__syncthreads_or(!got)) {
      if (threadIdx.x == 0) {
        atomicOr(flag, 1);
        for (int j = k; j < reps && j < k + kSlots; ++j)
          mbar_wait_bounded(&bar[j % kSlots], uint32_t((j / kSlots) & 1), timeout_ns, nullptr);
      }
      return;
    }
    const float4* v = reinterpret_cast<const float4*>(ring + (k % kSlots) * kChunk);
    for (int i = threadIdx.x; i < kChunk / 16; i += blockDim.x) {
      const float4 q = v[i];
      acc += q.x + q.w;
    }
    __syncthreads();
    if (threadIdx.x == 0 && k + kSlots < reps) issue(k + kSlots);
  }
  if (acc == 1234.5f) sink[0] = acc;  // keeps the reads
}

}  // namespace

extern "C" pat_status pat_probe_l2_to_smem(double* gbps) {
  if (!gbps) return fail(PAT_ERR_INVALID, "gbps NULL");
  *gbps = 0.0;
  int dev = 0;
  PAT_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  PAT_CUDA(cudaGetDeviceProperties(&prop, dev));
  const size_t smem = 128 + size_t(kChunk) * kSlots;
  if (smem > size_t(prop.sharedMemPerBlockOptin))
    return fail(PAT_ERR_INVALID, "the probe's ring does not fit in shared memory");
  unsigned char* src = nullptr;
  int* flag = nullptr;
  float* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  pat_status st = PAT_OK;
  float ms = 0.0f;
  const int grid = prop.multiProcessorCount;
  const int reps = int((size_t(2) << 30) / (size_t(kChunk) * grid));
  cudaError_t e = cudaMalloc(&src, kBuffer);
  if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(src, 1, kBuffer);
  if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(l2_to_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    l2_to_smem_kernel<<<grid, 512, smem>>>(src, reps, 1000000000ull, flag, sink);  // warm-up: fills L2
    cudaEventRecord(a);
    l2_to_smem_kernel<<<grid, 512, smem>>>(src, reps, 1000000000ull, flag, sink);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  int fl = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = cuda_fail(e, "l2-to-shared probe");
  else if (fl) st = fail(PAT_ERR_TIMEOUT, "a probe wait ran out of time");
  else *gbps = double(kChunk) * reps * grid / (double(ms) * 1e6);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(src);
  cudaFree(flag);
  cudaFree(sink);
  return st;
}
