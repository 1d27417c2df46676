// Node geometry, particle preparation and the upward pass (P2M Alg. 3, then
// M2M Alg. 4 / Eq. 2.7 over all levels, Alg. 5).
//
// The interpolation points of a box side [a, b] are xi_k = c + h t_k with
// t_k the Chebyshev points of the second kind; the Lagrange basis is
// evaluated in the barycentric form in the normalised variable t = (x - c)/h.
// A side of zero width carries the basis l_0 = 1.
#include <type_traits>

#include "common.cuh"

namespace fmm {
namespace {

// scal[2] = ell, scal[3] = 1/ell (powers of two near the root box's stretched
// half-diagonal), scal[4] = (1/(4 pi eps0)) mu / ell^2, scal[5] = scal[4] / c0.
__global__ void k_units(const double* __restrict__ nlo, const double* __restrict__ nhi,
                        double* __restrict__ scal, bool poly) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double s[3] = {1.0, 1.0, scal[0]};
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    double v = s[k] * ((nhi[3 + k] - nlo[3 + k]) * 0.5);
    r2 += v * v;
  }
  double r = sqrt(r2);
  int e = (r > 0.0 && isfinite(r)) ? (int)ceil(log2(r)) : 0;
  double ell = ldexp(1.0, e);
  double inv = ldexp(1.0, -e);
  scal[2] = ell;
  scal[3] = inv;
  const double ke = 1.0 / (4.0 * 3.14159265358979323846 * kEps0);
  // internal kernel R'/|R'|^3 = l^2 S R / D^{3/2}, or for the polynomial test
  // kernel R' (1 + l^2 |R'|^2) = S R (1 + D) / l, with S = diag(1, 1, gbar)
  scal[4] = poly ? ke * scal[1] * ell : ke * scal[1] * inv * inv;
  scal[5] = scal[4] / kC0;
}

// Centres and stretched half-diagonals (Algs. 6-7, FP64, fixed operation
// order, no contraction) for the traversal, plus the scaled geometry.
__global__ void k_node_geo(const double* __restrict__ nlo, const double* __restrict__ nhi, int64_t C,
                           const double* __restrict__ scal, double* __restrict__ ncen,
                           double* __restrict__ ndiam, NodeGeo* __restrict__ geo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (i > C) return;
  const double s[3] = {1.0, 1.0, scal[0]};
  const double inv = scal[3];
  double v[3];
  NodeGeo g;
  for (int k = 0; k < 3; ++k) {
    const double lo = nlo[3 * i + k], hi = nhi[3 * i + k];
    const double c = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    ncen[3 * i + k] = c;
    v[k] = __dmul_rn(s[k], __dmul_rn(__dsub_rn(lo, hi), 0.5));
    g.c[k] = __dmul_rn(__dmul_rn(s[k], c), inv);
    g.h[k] = __dmul_rn(__dmul_rn(s[k], __dmul_rn(__dsub_rn(hi, lo), 0.5)), inv);
  }
  ndiam[i] = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])),
                                  __dmul_rn(v[2], v[2])));
  geo[i] = g;
}

// Particles in leaf order: position relative to the leaf centre in stretched,
// scaled coordinates with the scaled mass a' (px), and the scaled momentum
// moment b~' (pb).  The offset from the centre is taken in physical
// coordinates first, s o (x - c) / ell, so that a narrow box far from the
// origin keeps its relative precision.
template <typename T>
__global__ void k_prep(const double* __restrict__ x, const double* __restrict__ p,
                       const double* __restrict__ q, int64_t N, const int32_t* __restrict__ perm,
                       const int64_t* __restrict__ nstart, int kappa, const double* __restrict__ ncen,
                       const double* __restrict__ scal, typename Vec4<T>::type* __restrict__ px,
                       typename Vec4<T>::type* __restrict__ pb, typename Vec4<T>::type* __restrict__ pl) {
  const int64_t first = (int64_t)1 << kappa;
  const double gbar = scal[0], imu = scal[11], inv = scal[3];
  for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < N;
       pos += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = find_node(nstart, first, first, pos);
    const int64_t i = perm[pos];
    const double* c = ncen + 3 * leaf;
    const double xs = (x[3 * i] - c[0]) * inv;
    const double ys = (x[3 * i + 1] - c[1]) * inv;
    const double zs = (gbar * (x[3 * i + 2] - c[2])) * inv;
    const double p0 = p[3 * i], p1 = p[3 * i + 1], p2 = p[3 * i + 2], qi = q[i];
    const double gam = sqrt(1.0 + ((p0 * p0 + p1 * p1) + p2 * p2));
    typename Vec4<T>::type u, w;
    u.x = (T)xs; u.y = (T)ys; u.z = (T)zs; u.w = (T)(qi * gam * imu);
    typename Vec4<T>::type lo;
    if (sizeof(T) == 4) {  // FP32: the rounding remainders, x = hi + lo to ~2^-48
      lo.x = (T)(xs - (double)u.x); lo.y = (T)(ys - (double)u.y); lo.z = (T)(zs - (double)u.z);
    } else {               // FP64: the absolute physical position, for P2P
      lo.x = (T)x[3 * i]; lo.y = (T)x[3 * i + 1]; lo.z = (T)x[3 * i + 2];
    }
    lo.w = (T)0;
    pl[pos] = lo;
    w.x = (T)((qi * p0) / gbar * imu);
    w.y = (T)((qi * p1) / gbar * imu);
    w.z = (T)(qi * p2 * imu);
    w.w = (T)0;
    px[pos] = u;
    pb[pos] = w;
  }
}

// P2M (Alg. 3): one block per leaf, thread per (proxy point, up to NV of them).
// Multipoles M[node][c][nu], c = (a, b~x, b~y, b~z).
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_p2m(const typename Vec4<T>::type* __restrict__ px,
                                             const typename Vec4<T>::type* __restrict__ pb,
                                             const int64_t* __restrict__ nstart,
                                             const int64_t* __restrict__ ncount, int kappa,
                                             const NodeGeo* __restrict__ geo, Cheb ch, int m,
                                             T* __restrict__ M) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  using V4 = typename Vec4<T>::type;
  const int np1 = ch.np1;
  // per particle: the three 1-D bases, then (a, b~) at a 4-aligned offset
  // (one vector load in the inner loop)
  const int boff = (3 * np1 + 3) & ~3;
  const int stride = boff + 4;
  const int64_t leaf = ((int64_t)1 << kappa) + blockIdx.x;
  const int64_t st = nstart[leaf], cnt = ncount[leaf];
  const NodeGeo g = geo[leaf];
  T invh[3];
  bool deg[3];
  for (int k = 0; k < 3; ++k) {
    deg[k] = !(g.h[k] > 0.0);
    invh[k] = deg[k] ? T(0) : (T)(1.0 / g.h[k]);
  }
  T acc[NV][4], cmp[NV][4];
  int nu1[NV], nu2[NV], nu3[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int nu = threadIdx.x + v * blockDim.x;
    nu1[v] = nu % np1;
    nu2[v] = (nu / np1) % np1;
    nu3[v] = nu / (np1 * np1);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[v][c] = cmp[v][c] = T(0);
  }
  for (int64_t base = 0; base < cnt; base += blockDim.x) {
    const int64_t j = base + threadIdx.x;
    T* row = sm + (size_t)threadIdx.x * stride;
    if (j < cnt) {
      const typename Vec4<T>::type u = px[st + j], w = pb[st + j];
      const T rel[3] = {u.x, u.y, u.z};
      for (int k = 0; k < 3; ++k) bary_basis<T>(rel[k] * invh[k], deg[k], ch, row + k * np1);
      V4 mass;
      mass.x = u.w; mass.y = w.x; mass.z = w.y; mass.w = w.z;
      *reinterpret_cast<V4*>(row + boff) = mass;
    }
    __syncthreads();
    const int nj = (int)min64(blockDim.x, cnt - base);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int nu = threadIdx.x + v * blockDim.x;
      if (nu >= m) continue;
      for (int j0 = 0; j0 < nj; j0 += 32) {
        T part[4] = {T(0), T(0), T(0), T(0)};
        const int j1 = min(nj, j0 + 32);
        for (int jj = j0; jj < j1; ++jj) {
          const T* r = sm + (size_t)jj * stride;
          const T wgt = r[nu1[v]] * r[np1 + nu2[v]] * r[2 * np1 + nu3[v]];
          const V4 ms = *reinterpret_cast<const V4*>(r + boff);
          part[0] += wgt * ms.x;
          part[1] += wgt * ms.y;
          part[2] += wgt * ms.z;
          part[3] += wgt * ms.w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) kahan_add(acc[v][c], cmp[v][c], part[c]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int nu = threadIdx.x + v * blockDim.x;
    if (nu >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) M[((size_t)leaf * 4 + c) * m + nu] = acc[v][c];
  }
}

// FP32 P2M with the tensor structure of the basis,
//   M_nu = sum_j l_nu1(x_j) l_nu2(y_j) l_nu3(z_j) m_j   (Alg. 3):
// one block per leaf; a thread owns one (nu2, nu3) and all NP1 values of
// nu1, so per staged particle it forms t_c = l_nu2(y) l_nu3(z) m_c once and
// adds l_nu1(x) t_c for every nu1 (5 multiplies and 4 NP1 FMAs, against 6
// NP1 operations and 4 NP1 shared loads of the point-per-thread form).  The
// particles' 1-D bases and masses are staged a block-width at a time; sums
// over runs of 32 particles are plain and Kahan-compensated across runs, as
// in k_p2m.
constexpr int kP2MSepThreads = 96;
template <int NP1>
__global__ void __launch_bounds__(kP2MSepThreads) k_p2m_sep(const float4* __restrict__ px,
                                                          const float4* __restrict__ pb,
                                                          const int64_t* __restrict__ nstart,
                                                          const int64_t* __restrict__ ncount, int kappa,
                                                          const NodeGeo* __restrict__ geo, Cheb ch,
                                                          float* __restrict__ M) {
  constexpr int m = NP1 * NP1 * NP1;
  constexpr int boff = (3 * NP1 + 3) & ~3;  // (a, b~) at a 16-byte offset
  constexpr int stride = boff + 4;
  static_assert(NP1 * NP1 <= kP2MSepThreads, "one thread per (nu2, nu3)");
  __shared__ __align__(16) float srow[kP2MSepThreads * stride];
  const int64_t leaf = ((int64_t)1 << kappa) + blockIdx.x;
  const int64_t st = nstart[leaf], cnt = ncount[leaf];
  const NodeGeo g = geo[leaf];
  float invh[3];
  bool deg[3];
  for (int k = 0; k < 3; ++k) {
    deg[k] = !(g.h[k] > 0.0);
    invh[k] = deg[k] ? 0.f : (float)(1.0 / g.h[k]);
  }
  const int tid = threadIdx.x;
  const bool own = tid < NP1 * NP1;
  const int nu2 = tid % NP1, nu3 = own ? tid / NP1 : 0;
  float acc[NP1][4], cmp[NP1][4];
#pragma unroll
  for (int a = 0; a < NP1; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = cmp[a][c] = 0.f;
  for (int64_t base = 0; base < cnt; base += kP2MSepThreads) {
    const int64_t j = base + tid;
    if (j < cnt) {
      const float4 u = px[st + j], w = pb[st + j];
      float* row = srow + tid * stride;
      float l[NP1];
      bary_basis_n<NP1>(u.x * invh[0], deg[0], ch, l);
#pragma unroll
      for (int k = 0; k < NP1; ++k) row[k] = l[k];
      bary_basis_n<NP1>(u.y * invh[1], deg[1], ch, l);
#pragma unroll
      for (int k = 0; k < NP1; ++k) row[NP1 + k] = l[k];
      bary_basis_n<NP1>(u.z * invh[2], deg[2], ch, l);
#pragma unroll
      for (int k = 0; k < NP1; ++k) row[2 * NP1 + k] = l[k];
      *reinterpret_cast<float4*>(row + boff) = make_float4(u.w, w.x, w.y, w.z);
    }
    __syncthreads();
    const int nj = (int)min64(kP2MSepThreads, cnt - base);
    if (own) {
      for (int j0 = 0; j0 < nj; j0 += 32) {
        float part[NP1][4];
#pragma unroll
        for (int a = 0; a < NP1; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) part[a][c] = 0.f;
        const int j1 = min(nj, j0 + 32);
        for (int jj = j0; jj < j1; ++jj) {
          const float* r = srow + jj * stride;
          const float t = r[NP1 + nu2] * r[2 * NP1 + nu3];
          const float4 ms = *reinterpret_cast<const float4*>(r + boff);
          const float tc[4] = {t * ms.x, t * ms.y, t * ms.z, t * ms.w};
#pragma unroll
          for (int a = 0; a < NP1; ++a) {
            const float lx = r[a];
#pragma unroll
            for (int c = 0; c < 4; ++c) part[a][c] = fmaf(lx, tc[c], part[a][c]);
          }
        }
#pragma unroll
        for (int a = 0; a < NP1; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) kahan_add(acc[a][c], cmp[a][c], part[a][c]);
      }
    }
    __syncthreads();
  }
  if (!own) return;
#pragma unroll
  for (int a = 0; a < NP1; ++a) {
    const int nu = a + NP1 * (nu2 + NP1 * nu3);
#pragma unroll
    for (int c = 0; c < 4; ++c) M[((size_t)leaf * 4 + c) * m + nu] = acc[a][c];
  }
}

// M2L source table: per node and proxy point, (Y, a) and (b~, 0) with
// Y = h o t_nu the point's offset from the box centre.
template <typename T>
__global__ void k_srctab(const T* __restrict__ M, const NodeGeo* __restrict__ geo, int64_t C, Cheb ch,
                         int m, typename Vec4<T>::type* __restrict__ src) {
  const int64_t total = (C + 1) * (int64_t)m;
  const int np1 = ch.np1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = e / m;
    const int nu = (int)(e % m);
    if (node == 0) continue;
    const NodeGeo g = geo[node];
    const int n1 = nu % np1, n2 = (nu / np1) % np1, n3 = nu / (np1 * np1);
    typename Vec4<T>::type u, w;
    u.x = (T)(g.h[0] * ch.t[n1]);
    u.y = (T)(g.h[1] * ch.t[n2]);
    u.z = (T)(g.h[2] * ch.t[n3]);
    u.w = M[((size_t)node * 4 + 0) * m + nu];
    w.x = M[((size_t)node * 4 + 1) * m + nu];
    w.y = M[((size_t)node * 4 + 2) * m + nu];
    w.z = M[((size_t)node * 4 + 3) * m + nu];
    w.w = T(0);
    src[2 * e] = u;
    src[2 * e + 1] = w;
  }
}

template <typename T, int NV>
int launch_p2m(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  const size_t smem = (size_t)256 * (((3 * P->np1 + 3) & ~3) + 4) * sizeof(T);
  if (int rc = smem_limit(k_p2m<T, NV>, (int)smem)) return rc;
  k_p2m<T, NV><<<(unsigned)P->nleaves, 256, smem, s>>>(
      ws_ptr<typename Vec4<T>::type>(P, L.px), ws_ptr<typename Vec4<T>::type>(P, L.pb),
      ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo),
      P->cheb, P->m, ws_ptr<T>(P, L.mpole));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <int NP1>
int launch_p2m_sep(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  k_p2m_sep<NP1><<<(unsigned)P->nleaves, kP2MSepThreads, 0, s>>>(
      ws_ptr<float4>(P, L.px), ws_ptr<float4>(P, L.pb), ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount),
      P->kappa, ws_ptr<NodeGeo>(P, L.ngeo), P->cheb, ws_ptr<float>(P, L.mpole));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// FP32 with 3, 5, 7 or 9 points per axis: the separable kernel; otherwise
// (FP64, other degrees) the point-per-thread one.
template <typename T>
int launch_p2m_any(fmm_plan_s* P, cudaStream_t s) {
  if (std::is_same<T, float>::value) {
    switch (P->np1) {
      case 3: return launch_p2m_sep<3>(P, s);
      case 5: return launch_p2m_sep<5>(P, s);
      case 7: return launch_p2m_sep<7>(P, s);
      case 9: return launch_p2m_sep<9>(P, s);
      default: break;
    }
  }
  switch (div_up(P->m, 256)) {
    case 1: return launch_p2m<T, 1>(P, s);
    case 2: return launch_p2m<T, 2>(P, s);
    case 3: return launch_p2m<T, 3>(P, s);
    case 4: return launch_p2m<T, 4>(P, s);
    case 5: return launch_p2m<T, 5>(P, s);
    case 6: return launch_p2m<T, 6>(P, s);
    case 7: return launch_p2m<T, 7>(P, s);
    case 8: return launch_p2m<T, 8>(P, s);
    default: return launch_p2m<T, 9>(P, s);
  }
}

template <typename T>
int upward_t(fmm_plan_s* P, cudaStream_t s, int xfer_cap, bool per_level) {
  int rc = launch_p2m_any<T>(P, s);
  if (rc != FMM_OK) return rc;
  // P2M done (stage event of the forward call, not of a recomputation)
  if (!P->have_forward && (rc = record_stage(P, 9, s)) != FMM_OK) return rc;
  const Layout& L = P->lay;
  rc = run_transfer<T, 4, true>(P, ws_ptr<T>(P, L.mpole), s, xfer_cap, per_level);  // M2M, all levels
  if (rc != FMM_OK) return rc;
  if (m2l_specialised(P)) return FMM_OK;  // the specialised M2L reads the multipoles directly
  const int64_t total = (P->C + 1) * (int64_t)P->m;
  k_srctab<T><<<(unsigned)std::min<int64_t>(div_up(total, 256), 8192), 256, 0, s>>>(
      ws_ptr<T>(P, L.mpole), ws_ptr<NodeGeo>(P, L.ngeo), P->C, P->cheb, P->m,
      ws_ptr<typename Vec4<T>::type>(P, L.srct));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

}  // namespace

int run_prep(fmm_plan_s* P, const double* x, const double* p, const double* q, cudaStream_t s) {
  const Layout& L = P->lay;
  double* scal = ws_ptr<double>(P, L.scal);
  k_units<<<1, 32, 0, s>>>(ws_ptr<double>(P, L.nlo), ws_ptr<double>(P, L.nhi), scal,
                           (P->flags & FMM_TEST_POLY_KERNEL) != 0);
  FMM_LAUNCH_CHECK();
  k_node_geo<<<(unsigned)div_up(P->C, 128), 128, 0, s>>>(ws_ptr<double>(P, L.nlo), ws_ptr<double>(P, L.nhi),
                                                          P->C, scal, ws_ptr<double>(P, L.ncen),
                                                          ws_ptr<double>(P, L.ndiam), ws_ptr<NodeGeo>(P, L.ngeo));
  FMM_LAUNCH_CHECK();
  int rc = run_tmats(P, s);
  if (rc != FMM_OK) return rc;
  const int gs = (int)std::min<int64_t>(8192, div_up(P->N, 256));
  if (P->precision == FMM_FP32) {
    k_prep<float><<<gs, 256, 0, s>>>(x, p, q, P->N, ws_ptr<int32_t>(P, L.perm), ws_ptr<int64_t>(P, L.nstart),
                                      P->kappa, ws_ptr<double>(P, L.ncen), scal, ws_ptr<float4>(P, L.px),
                                      ws_ptr<float4>(P, L.pb), ws_ptr<float4>(P, L.pl));
  } else {
    k_prep<double><<<gs, 256, 0, s>>>(x, p, q, P->N, ws_ptr<int32_t>(P, L.perm), ws_ptr<int64_t>(P, L.nstart),
                                       P->kappa, ws_ptr<double>(P, L.ncen), scal, ws_ptr<double4>(P, L.px),
                                       ws_ptr<double4>(P, L.pb), ws_ptr<double4>(P, L.pl));
  }
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int run_upward(fmm_plan_s* P, cudaStream_t s, int xfer_cap, bool per_level) {
  return P->precision == FMM_FP32 ? upward_t<float>(P, s, xfer_cap, per_level)
                                  : upward_t<double>(P, s, xfer_cap, per_level);
}

int run_l2l(fmm_plan_s* P, cudaStream_t s, bool per_level) {
  const int cap = per_level ? kLevelTransferCap : kCoopTransferCap;
  return P->precision == FMM_FP32 ? run_transfer<float, 6, false>(P, ws_ptr<float>(P, P->lay.local), s, cap, per_level)
                                  : run_transfer<double, 6, false>(P, ws_ptr<double>(P, P->lay.local), s, cap, per_level);
}

}  // namespace fmm
