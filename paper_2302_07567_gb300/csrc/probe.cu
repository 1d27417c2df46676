// FP32 fused multiply-add throughput of the current device: the peak that the
// ALU-bound kernels of this library (P2P, M2L and their adjoints) are
// reported against.  Every thread runs kChains independent FMA chains for
// `iters` steps, in the scalar form (one FMA per lane per instruction) or the
// paired form (two per lane per instruction, __ffma2_rn, as the particle
// kernels issue their arithmetic); the chains end in a store to the caller's
// sink so that nothing is optimised away.  Not part of the method.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fma_scalar(float mul, float add, int iters, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], mul, add);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_paired(float mul, float add, int iters, float* __restrict__ sink) {
  float2 a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
  const float2 m2 = make_float2(mul, mul), a2 = make_float2(add, add);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m2, a2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" int fmm_fp32_fma_rate(void* sink, size_t sink_bytes, int paired, double* tflops, void* stream) {
  if (!sink || !tflops) return FMM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto kern = paired ? k_fma_paired : k_fma_scalar;
  int sms = 0, per_sm = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (int rc = blocks_per_sm(kern, kProbeThreads, 0, &per_sm)) return rc;
  if (per_sm < 1) return FMM_EINVAL;
  const int64_t blocks = (int64_t)sms * per_sm;
  if (sink_bytes < (size_t)blocks * kProbeThreads * sizeof(float)) return FMM_EINVAL;
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FMM_CUDA_TRY(cudaEventCreate(&e0));
  FMM_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 0.f;
  int rc = FMM_OK;
  for (int rep = 0; rep < 4 && rc == FMM_OK; ++rep) {  // the first launch warms up, the best of the rest counts
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      kern<<<(unsigned)blocks, kProbeThreads, 0, s>>>(1.0000001f, 1e-7f, iters, static_cast<float*>(sink));
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      set_last_cuda_error(e);
      rc = FMM_ECUDA;
    } else if (rep > 0 && (best_ms == 0.f || ms < best_ms)) {
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FMM_OK) return rc;
  const double fma = (double)blocks * kProbeThreads * iters * 8.0 * kChains * (paired ? 2.0 : 1.0);
  *tflops = 2.0 * fma / (best_ms * 1e-3) / 1e12;
  return FMM_OK;
}
