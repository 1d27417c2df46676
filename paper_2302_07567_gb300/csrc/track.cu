// Particle tracking: the field of a step that keeps the previous step's tree
// and interaction lists, and the Boris push that moves the beam.  Neither is
// in the paper, whose FMM (Alg. 12) builds the tree and lists for one field
// evaluation; a tracking code calls it every time step, while the particles
// move little between steps.
//
// Reuse.  The tree's membership (which particles form each cluster) and the
// P2P and M2L lists of the last full fmm_field stay; gbar is recomputed from
// the new momenta and every cluster's box is the bounding box (Section 2) of
// its unchanged members at their new positions.  The lists still partition
// all N^2 particle pairs, and if every M2L pair is still admissible under the
// new boxes and gbar (Alg. 8), the FMM of Alg. 12 applies to them as they
// are, with the same error bound (Section 4).  A pair that is no longer
// admissible makes the lists stale: the caller then builds tree and lists
// anew.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kBoxThreads = 256;

// Bounding box of every leaf over its members (slots of the leaf order,
// input rows perm[slot]); min and max are exact, so the box equals the one
// the tree build takes from the sorted coordinates.
__global__ void __launch_bounds__(kBoxThreads) k_leaf_boxes(const double* __restrict__ x,
                                                           const int32_t* __restrict__ perm,
                                                           const int64_t* __restrict__ nstart,
                                                           const int64_t* __restrict__ ncount, int kappa,
                                                           double* __restrict__ nlo, double* __restrict__ nhi) {
  __shared__ double red[2][3][kBoxThreads / 32];
  const int64_t leaf = ((int64_t)1 << kappa) + blockIdx.x;
  const int64_t st = nstart[leaf], cnt = ncount[leaf];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int64_t i = perm[st + j];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = x[3 * i + k];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      red[0][k][w] = lo[k];
      red[1][k][w] = hi[k];
    }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int k = threadIdx.x;
    double a = red[0][k][0], b = red[1][k][0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      a = fmin(a, red[0][k][q]);
      b = fmax(b, red[1][k][q]);
    }
    nlo[3 * leaf + k] = a;
    nhi[3 * leaf + k] = b;
  }
}

// Boxes of one inner level: the union of the two children's boxes, which is
// the bounding box of the node's members.
__global__ void k_parent_boxes(int level, double* __restrict__ nlo, double* __restrict__ nhi) {
  const int64_t first = (int64_t)1 << level;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= first) return;
  const int64_t i = first + t;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nlo[3 * i + k] = fmin(nlo[3 * (2 * i) + k], nlo[3 * (2 * i + 1) + k]);
    nhi[3 * i + k] = fmax(nhi[3 * (2 * i) + k], nhi[3 * (2 * i + 1) + k]);
  }
}

// Per list pair the centre offset under the new boxes (as the traversal
// writes it), and for M2L pairs the admissibility test of the traversal: a
// pair that fails it marks the lists stale (kErrStale), on which the M2L and
// P2P kernels return at once and the host builds tree and lists anew.
template <bool kFP32>
__global__ void k_refresh_lists(const uint64_t* __restrict__ p2p, int64_t np2p, const uint64_t* __restrict__ m2l,
                                int64_t nm2l, int shift, const double* __restrict__ ncen,
                                const double* __restrict__ ndiam, const double* __restrict__ scal, double eta,
                                void* p2p_dc, void* m2l_dc, unsigned int* __restrict__ err) {
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int64_t total = np2p + nm2l;
  bool stale = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const bool is_m2l = e >= np2p;
    const int64_t k = is_m2l ? e - np2p : e;
    const uint64_t key = is_m2l ? m2l[k] : p2p[k];
    const int64_t t = (int64_t)(key >> shift), u = (int64_t)(key & mask);
    store_pair_offset<kFP32>(ncen, scal, t, u, is_m2l ? m2l_dc : p2p_dc, k);
    if (is_m2l && !pair_admissible(ndiam, ncen, scal[0], t, u, eta)) stale = true;
  }
  if (__any_sync(0xffffffffu, stale) && (threadIdx.x & 31) == 0) atomicOr(err, kErrStale);
}

// Relativistic Boris push of every particle over one time step dt, in the
// fields E, B (SI) at the particle.  With u = p = gamma beta (dimensionless),
// a = q dt / (2 m c):
//   u-  = u + a E
//   t   = (a c / gamma(u-)) B,   s = 2 t / (1 + |t|^2)
//   u+  = u- + (u- + u- x t) x s
//   u'  = u+ + a E,              x' = x + c dt u' / gamma(u')
// gamma(u) = sqrt(1 + |u|^2).  The rotation keeps |u| in a pure magnetic
// field to rounding; a pure electric field changes u by 2 a E exactly.
template <typename T>
__global__ void k_boris(double* __restrict__ x, double* __restrict__ p, const double* __restrict__ q, int64_t N,
                        const T* __restrict__ E, const T* __restrict__ B, double qdt_2mc, double dt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = q[i] * qdt_2mc;
    const double e[3] = {(double)E[3 * i], (double)E[3 * i + 1], (double)E[3 * i + 2]};
    const double b[3] = {(double)B[3 * i], (double)B[3 * i + 1], (double)B[3 * i + 2]};
    double um[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = __dadd_rn(p[3 * i + k], __dmul_rn(a, e[k]));
    const double gm = __dsqrt_rn(__dadd_rn(1.0, __dadd_rn(__dadd_rn(__dmul_rn(um[0], um[0]), __dmul_rn(um[1], um[1])),
                                                          __dmul_rn(um[2], um[2]))));
    const double f = __ddiv_rn(__dmul_rn(a, kC0), gm);
    double t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = __dmul_rn(f, b[k]);
    const double t2 = __dadd_rn(__dadd_rn(__dmul_rn(t[0], t[0]), __dmul_rn(t[1], t[1])), __dmul_rn(t[2], t[2]));
    const double g = __ddiv_rn(2.0, __dadd_rn(1.0, t2));
    double s[3], w[3], up[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = __dmul_rn(g, t[k]);
    // w = u- + u- x t
    w[0] = __dadd_rn(um[0], __dsub_rn(__dmul_rn(um[1], t[2]), __dmul_rn(um[2], t[1])));
    w[1] = __dadd_rn(um[1], __dsub_rn(__dmul_rn(um[2], t[0]), __dmul_rn(um[0], t[2])));
    w[2] = __dadd_rn(um[2], __dsub_rn(__dmul_rn(um[0], t[1]), __dmul_rn(um[1], t[0])));
    // u+ = u- + w x s
    up[0] = __dadd_rn(um[0], __dsub_rn(__dmul_rn(w[1], s[2]), __dmul_rn(w[2], s[1])));
    up[1] = __dadd_rn(um[1], __dsub_rn(__dmul_rn(w[2], s[0]), __dmul_rn(w[0], s[2])));
    up[2] = __dadd_rn(um[2], __dsub_rn(__dmul_rn(w[0], s[1]), __dmul_rn(w[1], s[0])));
    double un[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) un[k] = __dadd_rn(up[k], __dmul_rn(a, e[k]));
    const double gn = __dsqrt_rn(__dadd_rn(1.0, __dadd_rn(__dadd_rn(__dmul_rn(un[0], un[0]), __dmul_rn(un[1], un[1])),
                                                          __dmul_rn(un[2], un[2]))));
    const double v = __ddiv_rn(__dmul_rn(kC0, dt), gn);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      p[3 * i + k] = un[k];
      x[3 * i + k] = __dadd_rn(x[3 * i + k], __dmul_rn(v, un[k]));
    }
  }
}

}  // namespace

int run_refresh(fmm_plan_s* P, const double* x, cudaStream_t s) {
  const Layout& L = P->lay;
  double* nlo = ws_ptr<double>(P, L.nlo);
  double* nhi = ws_ptr<double>(P, L.nhi);
  k_leaf_boxes<<<(unsigned)P->nleaves, kBoxThreads, 0, s>>>(x, ws_ptr<int32_t>(P, L.perm),
                                                           ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount),
                                                           P->kappa, nlo, nhi);
  FMM_LAUNCH_CHECK();
  for (int level = P->kappa - 1; level >= 0; --level) {
    const int64_t n = (int64_t)1 << level;
    k_parent_boxes<<<(unsigned)div_up(n, 256), 256, 0, s>>>(level, nlo, nhi);
    FMM_LAUNCH_CHECK();
  }
  return FMM_OK;
}

int run_refresh_lists(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  const int64_t total = P->p2p_count + P->m2l_count;
  if (total == 0) return FMM_OK;
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  const unsigned grid = (unsigned)std::min<int64_t>(div_up(total, 256), (int64_t)8 * sms);
  auto kern = P->precision == FMM_FP32 ? k_refresh_lists<true> : k_refresh_lists<false>;
  kern<<<grid, 256, 0, s>>>(ws_ptr<uint64_t>(P, L.p2p), P->p2p_count, ws_ptr<uint64_t>(P, L.m2l), P->m2l_count,
                            P->kappa + 1, ws_ptr<double>(P, L.ncen), ws_ptr<double>(P, L.ndiam),
                            ws_ptr<double>(P, L.scal), P->eta, P->ws + L.p2p_dc, P->ws + L.m2l_dc,
                            &ws_ptr<Counters>(P, L.counters)->err);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

}  // namespace fmm

using namespace fmm;

extern "C" int fmm_boris_push(double* x, double* p, const double* q, int64_t N, const void* E, const void* B,
                              int field_precision, double mass, double dt, void* stream) {
  if (!x || !p || !q || !E || !B || N < 1) return FMM_EINVAL;
  if (field_precision != FMM_FP32 && field_precision != FMM_FP64) return FMM_EINVAL;
  if (!(mass > 0.0) || !std::isfinite(mass) || !std::isfinite(dt)) return FMM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  const unsigned grid = (unsigned)std::min<int64_t>(div_up(N, 256), (int64_t)16 * sms);
  const double qdt_2mc = dt / (2.0 * mass * kC0);
  if (field_precision == FMM_FP32)
    k_boris<float><<<grid, 256, 0, s>>>(x, p, q, N, static_cast<const float*>(E), static_cast<const float*>(B),
                                        qdt_2mc, dt);
  else
    k_boris<double><<<grid, 256, 0, s>>>(x, p, q, N, static_cast<const double*>(E), static_cast<const double*>(B),
                                         qdt_2mc, dt);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}
