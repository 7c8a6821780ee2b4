// Measured integer speed of light of this GPU for the benchmark's roofline
// (nqs_probe_peaks).  The paper has no counterpart.
//
// Two kernels, each timed with CUDA events on the caller's stream at the
// LoopOverTerms search kernel's launch shape (one 1024-thread block per SM):
//
//   alu_mix_kernel  -- register-only integer work made of the operations of
//     one filter probe (XOR, AND, 32-bit funnel shift, shift-or): sixteen
//     independent chains per thread so that issue, not latency, limits it.
//     Counted as source-level lane operations.
//   probe_loop_kernel -- the search's filter loop itself: eight row hashes
//     per lane against a stream of pattern hashes, each probe reading one
//     word of a 128 KB shared-memory filter and testing three bits, with no
//     survivor handling.  Counted in probes.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr int kPeakThreads = 1024;
constexpr int kAluChains = 16;
constexpr int kAluOpsPerStep = 4;     // XOR, AND, funnel shift, OR per chain per step
constexpr int kProbeRows = 8;
constexpr int kPeakFilterWords = 32768;   // 128 KB, the search kernel's largest filter

__global__ void __launch_bounds__(kPeakThreads, 1) alu_mix_kernel(int iters, uint32_t seed, uint32_t* sink) {
  uint32_t v[kAluChains];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < kAluChains; ++c) v[c] = (t + 1u) * (2654435761u + 2u * c) ^ seed;
  uint32_t k = seed ^ t;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kAluChains; ++c) {
      const uint32_t x = v[c] ^ k;                 // hash XOR
      const uint32_t m = x & 0x7FFFCu;             // filter address mask
      const uint32_t f = __funnelshift_r(x, x, m); // bit select
      v[c] = (f << 1) | (m >> 2);                  // accumulate
    }
    k += 0x9E3779B9u;
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kAluChains; ++c) r ^= v[c];
  if (r == 0x12345678u) sink[t] = r;  // keeps the chains live; practically never stores
}

__global__ void __launch_bounds__(kPeakThreads, 1) probe_loop_kernel(const uint32_t* __restrict__ filt, int groups,
                                                                     uint32_t seed, uint32_t* sink) {
  extern __shared__ __align__(16) uint32_t bloom[];
  for (int i = threadIdx.x; i < kPeakFilterWords; i += blockDim.x) bloom[i] = __ldg(filt + i);
  __syncthreads();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t wmask4 = (uint32_t)(kPeakFilterWords - 1) << 2;
  const char* bytes = reinterpret_cast<const char*>(bloom);
  uint32_t hr4[kProbeRows];
#pragma unroll
  for (int r = 0; r < kProbeRows; ++r) hr4[r] = ((t * 8u + r + 1u) * 2246822519u ^ seed) << 2;
  uint32_t hk = seed * 3266489917u + t;
  uint32_t acc = 0;
  for (int g = 0; g < groups; ++g) {
    const uint32_t hk4 = hk << 2;
    uint32_t hm = 0;
#pragma unroll
    for (int r = 0; r < kProbeRows; ++r) {
      const uint32_t v4 = hr4[r] ^ hk4;
      const uint32_t w = *reinterpret_cast<const uint32_t*>(bytes + (v4 & wmask4));
      const uint32_t b = __funnelshift_r(w, w, v4 >> 17) & __funnelshift_r(w, w, v4 >> 22) &
                         __funnelshift_r(w, w, v4 >> 27);
      hm = __funnelshift_l(b, hm, 1);
    }
    acc += hm;
    hk = hk * 1664525u + 1013904223u;   // next pattern hash (stands in for the table load)
  }
  if (acc == 0x9E3779B9u) sink[t] = acc;
}

cudaError_t probe_peaks(double* out, cudaStream_t s) {
  const int sms = num_sms();
  cudaError_t e;
  uint32_t* filt = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  const size_t smem = sizeof(uint32_t) * kPeakFilterWords;
  const int alu_iters = 4096, groups = 4096;
  float ms_alu = 0.f, ms_probe = 0.f;
  if ((e = cudaMalloc(&filt, smem)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sink, sizeof(uint32_t) * (size_t)sms * kPeakThreads)) != cudaSuccess) goto done;
  // a filter with about a quarter of its bits set, as the staged filter of 1e5 samples
  if ((e = cudaMemsetAsync(filt, 0x11, smem, s)) != cudaSuccess) goto done;
  if ((e = cudaFuncSetAttribute(probe_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    goto done;
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) goto done;
  // warm-up launches, then one timed launch of each
  alu_mix_kernel<<<sms, kPeakThreads, 0, s>>>(64, 1u, sink);
  probe_loop_kernel<<<sms, kPeakThreads, smem, s>>>(filt, 64, 1u, sink);
  cudaEventRecord(ev[0], s);
  alu_mix_kernel<<<sms, kPeakThreads, 0, s>>>(alu_iters, 7u, sink);
  cudaEventRecord(ev[1], s);
  probe_loop_kernel<<<sms, kPeakThreads, smem, s>>>(filt, groups, 7u, sink);
  cudaEventRecord(ev[2], s);
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  if ((e = cudaEventSynchronize(ev[2])) != cudaSuccess) goto done;
  cudaEventElapsedTime(&ms_alu, ev[0], ev[1]);
  cudaEventElapsedTime(&ms_probe, ev[1], ev[2]);
  {
    const double threads = (double)sms * kPeakThreads;
    out[0] = threads * alu_iters * kAluChains * kAluOpsPerStep / (ms_alu * 1e-3);
    out[1] = threads * groups * kProbeRows / (ms_probe * 1e-3);
  }
done:
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  cudaFree(sink);
  cudaFree(filt);
  return e;
}

}  // namespace nqs
