// Brute-force field of Section 5 (Alg. 10 with S_t = S_s = S and i != j) in
// FP64, for a list of target rows.  It is the reference the library measures
// its own error against (Eq. 5.1) and allocates nothing.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kDirThreads = 256;

__global__ void __launch_bounds__(kDirThreads) k_direct(const double* __restrict__ x, const double* __restrict__ p,
                                                       const double* __restrict__ q, int64_t N,
                                                       const int64_t* __restrict__ targets, int64_t T,
                                                       double gbar, double* __restrict__ E,
                                                       double* __restrict__ B) {
  __shared__ double sx[kDirThreads][3];
  __shared__ double sm[kDirThreads][4];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < T;
  const int64_t ti = valid ? (targets ? targets[t] : t) : -1;
  double xi[3] = {0, 0, 0};
  if (valid && ti >= 0 && ti < N) {
    xi[0] = x[3 * ti]; xi[1] = x[3 * ti + 1]; xi[2] = x[3 * ti + 2];
  }
  const double g2 = gbar * gbar;
  double acc[6] = {0, 0, 0, 0, 0, 0}, cmp[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t base = 0; base < N; base += kDirThreads) {
    __syncthreads();
    const int64_t j = base + threadIdx.x;
    if (j < N) {
      const double p0 = p[3 * j], p1 = p[3 * j + 1], p2 = p[3 * j + 2];
      const double qj = q[j];
      const double gam = sqrt(1.0 + ((p0 * p0 + p1 * p1) + p2 * p2));
      sx[threadIdx.x][0] = x[3 * j];
      sx[threadIdx.x][1] = x[3 * j + 1];
      sx[threadIdx.x][2] = x[3 * j + 2];
      sm[threadIdx.x][0] = qj * gam;
      sm[threadIdx.x][1] = qj * p0;
      sm[threadIdx.x][2] = qj * p1;
      sm[threadIdx.x][3] = qj * p2;
    }
    __syncthreads();
    const int nj = (int)min64(kDirThreads, N - base);
    double part[6] = {0, 0, 0, 0, 0, 0};
    for (int jj = 0; jj < nj; ++jj) {
      if (base + jj == ti) continue;
      const double rx = xi[0] - sx[jj][0], ry = xi[1] - sx[jj][1], rz = xi[2] - sx[jj][2];
      const double d = rx * rx + ry * ry + g2 * (rz * rz);
      if (!(d > 0.0)) continue;
      const double inv = 1.0 / (d * sqrt(d));
      const double gx = rx * inv, gy = ry * inv, gz = rz * inv;
      const double a = sm[jj][0], bx = sm[jj][1], by = sm[jj][2], bz = sm[jj][3];
      part[0] += a * gx;
      part[1] += a * gy;
      part[2] += a * gz;
      part[3] += by * gz - bz * gy;
      part[4] += bz * gx - bx * gz;
      part[5] += bx * gy - by * gx;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) kahan_add(acc[c], cmp[c], part[c]);
  }
  if (!valid) return;
  const double ke = 1.0 / (4.0 * 3.14159265358979323846 * kEps0);
  for (int c = 0; c < 3; ++c) {
    E[3 * t + c] = ke * acc[c];
    B[3 * t + c] = ke / kC0 * acc[3 + c];
  }
}

// Few targets (fewer than fill the GPU one per thread): a warp per target,
// its lanes striding over the sources; per-lane sums over chunks of 32
// sources are Kahan-added, and the lanes are combined by a fixed butterfly,
// so the result does not depend on scheduling.
__global__ void __launch_bounds__(kDirThreads) k_direct_warp(const double* __restrict__ x,
                                                            const double* __restrict__ p,
                                                            const double* __restrict__ q, int64_t N,
                                                            const int64_t* __restrict__ targets, int64_t T,
                                                            double gbar, double* __restrict__ E,
                                                            double* __restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= T) return;  // whole warps
  const int64_t ti = targets ? targets[t] : t;
  double xi[3] = {0, 0, 0};
  if (ti >= 0 && ti < N) {
    xi[0] = x[3 * ti]; xi[1] = x[3 * ti + 1]; xi[2] = x[3 * ti + 2];
  }
  const double g2 = gbar * gbar;
  double acc[6] = {0, 0, 0, 0, 0, 0}, cmp[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t base = 0; base < N; base += 32 * 32) {
    double part[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 32; ++k) {
      const int64_t j = base + (int64_t)k * 32 + lane;
      if (j >= N || j == ti) continue;
      const double rx = xi[0] - x[3 * j], ry = xi[1] - x[3 * j + 1], rz = xi[2] - x[3 * j + 2];
      const double d = rx * rx + ry * ry + g2 * (rz * rz);
      if (!(d > 0.0)) continue;
      const double p0 = p[3 * j], p1 = p[3 * j + 1], p2 = p[3 * j + 2], qj = q[j];
      const double a = qj * sqrt(1.0 + ((p0 * p0 + p1 * p1) + p2 * p2));
      const double bx = qj * p0, by = qj * p1, bz = qj * p2;
      const double inv = 1.0 / (d * sqrt(d));
      const double gx = rx * inv, gy = ry * inv, gz = rz * inv;
      part[0] += a * gx;
      part[1] += a * gy;
      part[2] += a * gz;
      part[3] += by * gz - bz * gy;
      part[4] += bz * gx - bx * gz;
      part[5] += bx * gy - by * gx;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) kahan_add(acc[c], cmp[c], part[c]);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double v = acc[c] - cmp[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane != 0) return;
  const double ke = 1.0 / (4.0 * 3.14159265358979323846 * kEps0);
  for (int c = 0; c < 3; ++c) {
    E[3 * t + c] = ke * acc[c];
    B[3 * t + c] = ke / kC0 * acc[3 + c];
  }
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_direct_field(const double* x, const double* p, const double* q, int64_t N,
                                const int64_t* targets, int64_t T, double gbar, double* E, double* B,
                                void* stream) {
  if (!x || !p || !q || !E || !B || N < 1 || T < 0) return FMM_EINVAL;
  if (!targets && T != N) return FMM_EINVAL;
  if (!(gbar >= 1.0) || !std::isfinite(gbar)) return FMM_EINVAL;
  if (T == 0) return FMM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (T < 32768) {  // too few targets to fill the GPU one per thread
    fmm::k_direct_warp<<<(unsigned)fmm::div_up(T * 32, fmm::kDirThreads), fmm::kDirThreads, 0, s>>>(
        x, p, q, N, targets, T, gbar, E, B);
  } else {
    fmm::k_direct<<<(unsigned)fmm::div_up(T, fmm::kDirThreads), fmm::kDirThreads, 0, s>>>(x, p, q, N, targets, T,
                                                                                        gbar, E, B);
  }
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}
