// Copies with the GPU's SMs between device memory and pinned host memory
// (not in the paper; a data-movement helper of the C ABI).  A grid-stride
// kernel of 16-byte loads and stores; every address it forms lies inside
// [src, src + bytes) or [dst, dst + bytes).
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kCopyThreads = 256;

__global__ void __launch_bounds__(kCopyThreads) k_copy16(const float4* __restrict__ src, float4* __restrict__ dst,
                                                         int64_t n16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// The address a kernel on the current device uses for p: device or managed
// memory of this device as it is, pinned or registered host memory through
// its device mapping; FMM_EINVAL for memory CUDA does not know (pageable
// host memory) or memory of another device.
int device_address(const void* p, const void** out) {
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FMM_EINVAL;
  }
  int cur = 0;
  FMM_CUDA_TRY(cudaGetDevice(&cur));
  switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      if (a.device != cur) return FMM_EINVAL;
      *out = p;
      return FMM_OK;
    case cudaMemoryTypeHost:
      if (!a.devicePointer) return FMM_EINVAL;
      *out = a.devicePointer;
      return FMM_OK;
    default:
      return FMM_EINVAL;
  }
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" int fmm_copy(void* dst, const void* src, size_t bytes, void* stream) {
  if (!dst || !src) return FMM_EINVAL;
  if (((uintptr_t)dst | (uintptr_t)src | (uintptr_t)bytes) & 15u) return FMM_EINVAL;
  if (bytes == 0) return FMM_OK;
  const void* s_dev = nullptr;
  const void* d_dev = nullptr;
  if (device_address(src, &s_dev) != FMM_OK || device_address(dst, &d_dev) != FMM_OK) return FMM_EINVAL;
  if (((uintptr_t)s_dev | (uintptr_t)d_dev) & 15u) return FMM_EINVAL;
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  const int64_t n16 = (int64_t)(bytes / 16);
  const int64_t grid = std::min<int64_t>((int64_t)sms * 8, div_up(n16, (int64_t)kCopyThreads));
  k_copy16<<<(unsigned)grid, kCopyThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float4*>(s_dev), static_cast<float4*>(const_cast<void*>(d_dev)), n16);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}
