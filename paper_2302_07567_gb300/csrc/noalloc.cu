// gbar of a beam with no device allocation at all.
//
// Some callers cannot allocate device memory when they need the beam's
// average Lorentz factor:
// - code that runs while a CUDA stream is being captured into a graph, where
//   allocation calls are not permitted;
// - real-time tracking loops that must never wait on an allocator;
// - host applications whose device memory belongs to a pool or budget that
//   forbids driver allocations.
// They cannot attach a workspace either.  fmm_gamma_bar_noalloc gives them
// gbar = sqrt(1 + pbar.pbar) with the same adjacent-pair summation as
// fmm_field, so the two results are identical.  The partial sums live in a
// fixed scratch array compiled into the library (FMM_NOALLOC_MAX_N particles
// at most), not in caller memory.
//
// The scratch array is a file-scope __device__ variable, so every GPU that
// loads the library holds it (about 200 KB) until the process exits.  Host
// code cannot use the array's name as a device address.  The first call on
// each device therefore looks the address up with cudaGetSymbolAddress, with
// that device current, and passes it to the kernels; that first call should
// happen before any stream capture begins.  All calls share the array: every
// partial sum is written before it is read, so nothing has to be cleared
// between calls, but two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it.
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr int64_t kNaChunk = kNaThreads * kNaItems;   // 2048 terms per block
constexpr int64_t kNaMaxN = FMM_NOALLOC_MAX_N;
constexpr int64_t kNaLevel1 = kNaMaxN / kNaChunk;      // partial sums after the first level
constexpr int64_t kNaStride = kNaLevel1 + 64;          // per momentum component
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[3 * kNaStride];

std::mutex g_na_mutex;
double* g_na_addr[kNaMaxDevices] = {};

// Adjacent-pair sum of the aligned 2048-term chunk blockIdx.x of component
// blockIdx.y (terms beyond n are zero): the same binary tree as fmm_field.
__global__ void __launch_bounds__(kNaThreads) k_na_pairwise(const double* __restrict__ in, int64_t n,
                                                           int64_t stride, int64_t comp_in,
                                                           double* __restrict__ out, int64_t comp_out) {
  __shared__ double wsum[kNaThreads / 32];
  const double* src = in + blockIdx.y * comp_in;
  const int64_t base = (int64_t)blockIdx.x * kNaChunk + (int64_t)threadIdx.x * kNaItems;
  double e[kNaItems];
#pragma unroll
  for (int k = 0; k < kNaItems; ++k) e[k] = (base + k < n) ? src[(base + k) * stride] : 0.0;
  double v = __dadd_rn(__dadd_rn(__dadd_rn(e[0], e[1]), __dadd_rn(e[2], e[3])),
                       __dadd_rn(__dadd_rn(e[4], e[5]), __dadd_rn(e[6], e[7])));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    out[blockIdx.y * comp_out + blockIdx.x] =
        __dadd_rn(__dadd_rn(__dadd_rn(wsum[0], wsum[1]), __dadd_rn(wsum[2], wsum[3])),
                  __dadd_rn(__dadd_rn(wsum[4], wsum[5]), __dadd_rn(wsum[6], wsum[7])));
  }
}

__global__ void k_na_gbar(const double* __restrict__ sums, int64_t comp, int64_t N, double* __restrict__ gbar) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double dn = (double)N;
  const double px = __ddiv_rn(sums[0], dn), py = __ddiv_rn(sums[comp], dn), pz = __ddiv_rn(sums[2 * comp], dn);
  const double pp = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
  gbar[0] = __dsqrt_rn(__dadd_rn(1.0, pp));
}

// Device address of the scratch array for the current device (looked up once).
// The stream must belong to that device: the address is only valid there.
int scratch_address(cudaStream_t s, double** out) {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return FMM_EINVAL;
  if (s != nullptr) {
    int sdev = -1;
    FMM_CUDA_TRY(cudaStreamGetDevice(s, &sdev));
    if (sdev != dev) return FMM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* ptr = nullptr;
    FMM_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_na_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_na_addr[dev];
  return FMM_OK;
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_gamma_bar_noalloc(const double* p, int64_t N, double* gbar, void* stream) {
  using namespace fmm;
  if (!p || !gbar || N < 1 || N > kNaMaxN) return FMM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  int rc = scratch_address(s, &scratch);
  if (rc != FMM_OK) return rc;
  // level 1 reads p (stride 3 between particles, 1 between components) into
  // region A; further levels alternate A <-> B until one sum per component is left
  double* region[2] = {scratch, scratch + kNaLevel1};
  const double* src = p;
  int64_t n = N, stride = 3, comp_in = 1;
  int r = 0;
  do {
    const int64_t nb = div_up(n, kNaChunk);
    dim3 grid((unsigned)nb, 3);
    k_na_pairwise<<<grid, kNaThreads, 0, s>>>(src, n, stride, comp_in, region[r], kNaStride);
    FMM_LAUNCH_CHECK();
    src = region[r];
    n = nb;
    stride = 1;
    comp_in = kNaStride;
    r ^= 1;
  } while (n > 1);
  k_na_gbar<<<1, 32, 0, s>>>(src, kNaStride, N, gbar);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}
