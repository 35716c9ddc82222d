// probe.cu -- throughput probes for the roofline denominators (bchol_probe_rate).
//
// The factorization's FP64 roofline uses the nominal FP64 rate (152 SMs x 2
// FP64 FMA per clock x 2 flop x the SM clock).  These loops measure what the
// units deliver on the GPU at hand, with every SM busy and independent
// accumulators so that no dependent latency is timed:
//   kind 0  FP64 FMA (DFMA)                       8 chains per thread
//   kind 1  FP64 MMA (mma.sync m8n8k4 .f64)       4 chains per warp
//   kind 2  FP32 FMA (FFMA)                       8 chains per thread
//   kind 3  bf16 MMA on the tensor cores (tcgen05.mma kind::f16, M = 128,
//           N = 256, K = 16, FP32 accumulators in tensor memory), the
//           instruction family of the split updates
#include <algorithm>

#include "../../include/bchol.h"
#include "bchol_internal.h"
#include "split_update.cuh"

namespace bchol {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) probe_dfma(double* out, int iters, double seed) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed * (threadIdx.x + c);
  const double m = 1.0 + 1e-12 * seed, d = 1e-9 * seed;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, d);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the loop; never true for the seeds used
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma(float* out, int iters, float seed) {
  float a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed * (threadIdx.x + c);
  const float m = 1.0f + 1e-6f * seed, d = 1e-5f * seed;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], m, d);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dmma(double* out, int iters, double seed) {
  double acc[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double a = seed * (threadIdx.x & 7), b = seed * 0.5;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

// One CTA per SM: warp 0 holds 256 tensor-memory columns, thread 0 issues
// `iters` MMAs of 128 x 256 x 16 on zeroed bf16 operands, then waits for them.
__global__ void __launch_bounds__(kProbeThreads) probe_tc(int iters, int* status, uint64_t wait_ns) {
  __shared__ __align__(128) uint4 sa[128 * 16 / 8];  // A: 128 x 16 bf16
  __shared__ __align__(128) uint4 sb[256 * 16 / 8];  // B: 256 x 16 bf16
  __shared__ unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  for (int i = threadIdx.x; i < 128 * 2; i += kProbeThreads) sa[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < 256 * 2; i += kProbeThreads) sb[i] = make_uint4(0, 0, 0, 0);
  split::fence_async_smem();
  split::Ctx cx = split::ctx_begin<32>(&mbar, &tmem_slot);
  if (threadIdx.x == 0) {
    split::tc_fence_after();
    constexpr uint32_t idesc = split::idesc_bf16(128, 256);
    const uint64_t ad = split::smem_desc<16>(sa), bd = split::smem_desc<16>(sb);
    for (int i = 0; i < iters; ++i) split::mma_bf16(cx.tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
    split::mma_commit(cx.mbar);
    const uint64_t t0 = split::globaltimer_now();
    bool ok;
    while (!(ok = split::mbar_try_wait(cx.mbar, 0)) && split::globaltimer_now() - t0 < wait_ns) {
    }
    if (!ok) {
      atomicExch(status, kStatusTimeout);
      const uint64_t t1 = split::globaltimer_now();
      while (!split::mbar_try_wait(cx.mbar, 0) && split::globaltimer_now() - t1 < wait_ns) {
      }
    }
  }
  split::ctx_end<32>(cx);
}

cudaError_t probe_rate(int kind, int iters, double* tflops, int* status, uint64_t wait_ns, cudaStream_t stream) {
  const int sms = num_sms();
  double* dout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess && kind != 3) e = cudaMalloc(&dout, sizeof(double) * 4096);
  if (e != cudaSuccess) return e;
  double flops = 0.0;
  const int grid = sms * (kind == 3 ? 1 : 8);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first pass warms up
    cudaEventRecord(e0, stream);
    switch (kind) {
      case 0:
        probe_dfma<<<grid, kProbeThreads, 0, stream>>>(dout, iters, 1.0);
        flops = 2.0 * 8 * iters * (double)grid * kProbeThreads;
        break;
      case 1:
        probe_dmma<<<grid, kProbeThreads, 0, stream>>>(dout, iters, 1.0);
        flops = 2.0 * 256 * 4 * iters * (double)grid * (kProbeThreads / 32);
        break;
      case 2:
        probe_ffma<<<grid, kProbeThreads, 0, stream>>>(reinterpret_cast<float*>(dout), iters, 1.0f);
        flops = 2.0 * 8 * iters * (double)grid * kProbeThreads;
        break;
      default:
        probe_tc<<<grid, kProbeThreads, 0, stream>>>(iters, status, wait_ns);
        flops = 2.0 * 128 * 256 * 16 * (double)iters * grid;
        break;
    }
    cudaEventRecord(e1, stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  }
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *tflops = flops / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (dout) cudaFree(dout);
  return e;
}

}  // namespace bchol
