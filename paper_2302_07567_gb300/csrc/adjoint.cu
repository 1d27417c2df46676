// Adjoint of the FMM operator (the paper has no adjoint).
//
// For the loss L = sum_i wE_i . E_i + wB_i . B_i the adjoint returns dL/dx,
// dL/dp and dL/dq of the FMM of Alg. 12 with the tree, boxes, interaction
// lists and gbar held at the values of the forward call.  In the library's
// stretched, scaled units the forward is E'_i = sum_j a'_j K(R'_ij) and
// B'_i = sum_j b~'_j x K(R'_ij) with K(R) = R/|R|^3 (plus the interpolated far
// field), and L = sum_i wE^_i . E'_i + wB^_i . B'_i with the scaled weights
// wE^ = kE diag(1,1,1/gbar) wE, wB^ = kB diag(1,1,gbar) wB.  With
// u_ij = a'_j wE^_i + wB^_i x b~'_j and J(R) = dK/dR (symmetric):
//   near field, pair (i, j):  dL/da'_j += wE^_i . K,  dL/db~'_j += K x wB^_i,
//                             dL/dx'_i += J u_ij,     dL/dx'_j -= J u_ij,
//                             J u = u/|R|^3 - 3 R (R.u)/|R|^5;
//   far field, target side:   dL/dx'_i += sum_mu grad l_mu(x_i) (w^_i . Lc_mu),
//                             Lc the forward's cumulative local of i's leaf;
//   far field, source side:   W = L2P^T(w^) at the leaves, pushed up by the
//                             transposed L2L (an M2M), M2L^T over the
//                             source-major M2L list gives Lambda per source
//                             cluster, pushed down by the transposed M2M (an
//                             L2L); then dL/da'_j += sum_nu l_nu(x_j) Lambda^a_nu,
//                             dL/db~'_j += sum_nu l_nu(x_j) Lambda^b_nu and
//                             dL/dx'_j += sum_nu grad l_nu(x_j) (Lambda_nu . m'_j).
// The basis derivative is l_k'(t) = sum_m l_m(t) D[m][k] (ChebD).  The chain
// rule finally maps (a', b~', x') to (q, p, x) with a = q gamma, b = q p,
// gamma = sqrt(1 + |p|^2).
//
// Buffers: W and Lambda have their own, so the forward's multipoles and
// cumulative locals survive the adjoint (a second adjoint call reuses them),
// and the near field (FP32: both roles of every pair in k_adj_near, after
// k_adj_far has taken the target-side far field from the leaf locals; FP64
// and the gbar term: the target side in k_adj_target) runs on the caller's
// stream while the source side's far field (L2P^T, L2L^T, M2L^T, M2M^T) runs
// on the plan's side stream.  After both, k_adj_final (FP32) or k_adj_source
// adds the source-side far field and applies the chain rule.
#include <type_traits>

#include "common.cuh"

namespace fmm {
namespace {

template <typename T>
__device__ __forceinline__ void basis_deriv(T t, bool deg, const Cheb& ch, const ChebD& cd, T* l, T* dl) {
  bary_basis<T>(t, deg, ch, l);
  const int np1 = ch.np1;
  for (int k = 0; k < np1; ++k) {
    T s = T(0);
    for (int mm = 0; mm < np1; ++mm) s += l[mm] * cheb_diff<T>(cd, mm * np1 + k);
    dl[k] = deg ? T(0) : s;
  }
}

// Scaled loss weights in leaf order.
template <typename T>
__global__ void k_adj_prep(const T* __restrict__ wE, const T* __restrict__ wB, int64_t N,
                           const int32_t* __restrict__ perm, const double* __restrict__ scal,
                           typename Vec4<T>::type* __restrict__ wle, typename Vec4<T>::type* __restrict__ wlb) {
  const double gbar = scal[0], kE = scal[4], kB = scal[5];
  for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < N; pos += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[pos];
    typename Vec4<T>::type e, b;
    e.x = (T)(kE * (double)wE[3 * i]);
    e.y = (T)(kE * (double)wE[3 * i + 1]);
    e.z = (T)(kE * (double)wE[3 * i + 2] / gbar);
    e.w = T(0);
    b.x = (T)(kB * (double)wB[3 * i]);
    b.y = (T)(kB * (double)wB[3 * i + 1]);
    b.z = (T)(kB * (double)wB[3 * i + 2] * gbar);
    b.w = T(0);
    wle[pos] = e;
    wlb[pos] = b;
  }
}

// L2P^T: W[leaf][c][mu] = sum_{i in leaf} l_mu(x_i) w^_i[c], c = (wE^, wB^).
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_l2pt(const typename Vec4<T>::type* __restrict__ px,
                                              const typename Vec4<T>::type* __restrict__ pl,
                                              const typename Vec4<T>::type* __restrict__ wle,
                                              const typename Vec4<T>::type* __restrict__ wlb,
                                              const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount,
                                              int kappa, const NodeGeo* __restrict__ geo, Cheb ch, int m,
                                              T* __restrict__ W) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr bool kSplit = std::is_same<T, float>::value;
  using V4 = typename Vec4<T>::type;
  const int np1 = ch.np1;
  // per particle: the three 1-D bases, then (w^E, w^B) at a 4-aligned offset
  // as two 4-vectors (two vector loads in the inner loop)
  const int boff = (3 * np1 + 3) & ~3;
  const int stride = boff + 8;
  const int64_t leaf = ((int64_t)1 << kappa) + blockIdx.x;
  const int64_t st = nstart[leaf], cnt = ncount[leaf];
  const NodeGeo g = geo[leaf];
  T invh[3];
  bool deg[3];
  for (int k = 0; k < 3; ++k) {
    deg[k] = !(g.h[k] > 0.0);
    invh[k] = deg[k] ? T(0) : (T)(1.0 / g.h[k]);
  }
  T acc[NV][6], cmp[NV][6];
  int nu1[NV], nu2[NV], nu3[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int nu = threadIdx.x + v * blockDim.x;
    nu1[v] = nu % np1;
    nu2[v] = (nu / np1) % np1;
    nu3[v] = nu / (np1 * np1);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[v][c] = cmp[v][c] = T(0);
  }
  for (int64_t base = 0; base < cnt; base += blockDim.x) {
    const int64_t j = base + threadIdx.x;
    T* row = sm + (size_t)threadIdx.x * stride;
    if (j < cnt) {
      const typename Vec4<T>::type u = px[st + j], e = wle[st + j], b = wlb[st + j];
      T rel[3] = {u.x, u.y, u.z};
      if (kSplit) {
        const typename Vec4<T>::type l = pl[st + j];
        rel[0] += l.x; rel[1] += l.y; rel[2] += l.z;
      }
      for (int k = 0; k < 3; ++k) bary_basis<T>(rel[k] * invh[k], deg[k], ch, row + k * np1);
      V4 w0, w1;
      w0.x = e.x; w0.y = e.y; w0.z = e.z; w0.w = b.x;
      w1.x = b.y; w1.y = b.z; w1.z = T(0); w1.w = T(0);
      *reinterpret_cast<V4*>(row + boff) = w0;
      *reinterpret_cast<V4*>(row + boff + 4) = w1;
    }
    __syncthreads();
    const int nj = (int)min64(blockDim.x, cnt - base);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int nu = threadIdx.x + v * blockDim.x;
      if (nu >= m) continue;
      for (int j0 = 0; j0 < nj; j0 += 32) {
        T part[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        const int j1 = min(nj, j0 + 32);
        for (int jj = j0; jj < j1; ++jj) {
          const T* r = sm + (size_t)jj * stride;
          const T wgt = r[nu1[v]] * r[np1 + nu2[v]] * r[2 * np1 + nu3[v]];
          const V4 w0 = *reinterpret_cast<const V4*>(r + boff), w1 = *reinterpret_cast<const V4*>(r + boff + 4);
          part[0] += wgt * w0.x;
          part[1] += wgt * w0.y;
          part[2] += wgt * w0.z;
          part[3] += wgt * w0.w;
          part[4] += wgt * w1.x;
          part[5] += wgt * w1.y;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) kahan_add(acc[v][c], cmp[v][c], part[c]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int nu = threadIdx.x + v * blockDim.x;
    if (nu >= m) continue;
#pragma unroll
    for (int c = 0; c < 6; ++c) W[((size_t)leaf * 6 + c) * m + nu] = acc[v][c];
  }
}

// M2L^T: for source cluster s, Lambda[s][nu] = sum over target clusters S of
// the source-major M2L list and their points mu of (W^E_{S,mu} . K(R),
// K(R) x W^B_{S,mu}) with R = xi_{S,mu} - xi_{s,nu}.
// With GB it also forms the far-field part of gbar dL/dgbar for the cluster,
// sum over nu and the pairs of -3 R_z^2 r^-5 (R . u), u = a_nu W^E + W^B x b_nu:
// Gamma[nu] = sum R_z^2 r^-5 (R . W^E, R x W^B) is contracted with the
// cluster's multipoles (a, b~)_nu and summed over nu in a fixed order into
// gfar[s].
template <typename T, int KPT, bool GB>
__global__ void __launch_bounds__(256) k_adj_m2l(const uint64_t* __restrict__ keys, const int32_t* __restrict__ off,
                                                 int shift, const int32_t* __restrict__ order, int64_t nitems, const NodeGeo* __restrict__ geo,
                                                 const void* __restrict__ sdc, Cheb ch, int m,
                                                 const T* __restrict__ W, T* __restrict__ Lam,
                                                 const T* __restrict__ Mp, double* __restrict__ gfar) {
  using V4 = typename Vec4<T>::type;
  constexpr int NC = GB ? 8 : 4;  // Lambda (4) and Gamma (4)
  extern __shared__ unsigned char smem_raw[];
  V4* sm = reinterpret_cast<V4*>(smem_raw);  // [m][3]
  __shared__ double gred[32];
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {  // sources, longest list first
  const int64_t s = order[w];
  const int np1 = ch.np1;
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int b = off[s], e = off[s + 1];
  const NodeGeo gs = geo[s];
  const int per_pass = KPT * blockDim.x;
  double gsum = 0.0;  // this thread's points: far-field gbar term of the cluster
  for (int pass0 = 0; pass0 < m; pass0 += per_pass) {
    T xh[KPT][3];
    bool valid[KPT];
    T acc[KPT][NC], cmp[KPT][NC];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int nu = pass0 + threadIdx.x + k * blockDim.x;
      valid[k] = nu < m;
      const int nn = valid[k] ? nu : 0;
      xh[k][0] = (T)(gs.h[0] * ch.t[nn % np1]);
      xh[k][1] = (T)(gs.h[1] * ch.t[(nn / np1) % np1]);
      xh[k][2] = (T)(gs.h[2] * ch.t[nn / (np1 * np1)]);
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[k][c] = cmp[k][c] = T(0);
    }
    for (int it = b; it < e; ++it) {
      const int64_t S = (int64_t)(keys[it] & mask);
      T dc0, dc1, dc2;  // c_s - c_S
      if constexpr (sizeof(T) == 4) {
        const float4 dh = static_cast<const float4*>(sdc)[2 * it];
        dc0 = dh.x; dc1 = dh.y; dc2 = dh.z;
      } else {
        const double4 dd = static_cast<const double4*>(sdc)[it];
        dc0 = dd.x; dc1 = dd.y; dc2 = dd.z;
      }
      const NodeGeo gS = geo[S];
      __syncthreads();
      for (int o = threadIdx.x; o < m; o += blockDim.x) {
        const T* w = W + (size_t)S * 6 * m + o;
        V4 r0, r1, r2;
        r0.x = (T)(gS.h[0] * ch.t[o % np1]);
        r0.y = (T)(gS.h[1] * ch.t[(o / np1) % np1]);
        r0.z = (T)(gS.h[2] * ch.t[o / (np1 * np1)]);
        r0.w = w[0];
        r1.x = w[m]; r1.y = w[2 * m]; r1.z = w[3 * m]; r1.w = w[4 * m];
        r2.x = w[5 * m]; r2.y = T(0); r2.z = T(0); r2.w = T(0);
        sm[3 * o] = r0;
        sm[3 * o + 1] = r1;
        sm[3 * o + 2] = r2;
      }
      __syncthreads();
      T Z[KPT][3], part[KPT][NC];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        Z[k][0] = xh[k][0] + dc0;
        Z[k][1] = xh[k][1] + dc1;
        Z[k][2] = xh[k][2] + dc2;
#pragma unroll
        for (int c = 0; c < NC; ++c) part[k][c] = T(0);
      }
      for (int mu = 0; mu < m; ++mu) {
        const V4 r0 = sm[3 * mu], r1 = sm[3 * mu + 1], r2 = sm[3 * mu + 2];
        // r0 = (Y, WE.x), r1 = (WE.y, WE.z, WB.x, WB.y), r2 = (WB.z, ...)
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          const T rx = r0.x - Z[k][0], ry = r0.y - Z[k][1], rz = r0.z - Z[k][2];
          const T d = rx * rx + ry * ry + rz * rz;
          const T inv = d > tiny_sep2<T>() ? rsqrt_t<T>(d) : T(0);
          const T r3 = inv * inv * inv;
          part[k][0] += r3 * (rx * r0.w + ry * r1.x + rz * r1.y);
          part[k][1] += r3 * (ry * r2.x - rz * r1.w);
          part[k][2] += r3 * (rz * r1.z - rx * r2.x);
          part[k][3] += r3 * (rx * r1.w - ry * r1.z);
          if constexpr (GB) {
            const T z2r5 = rz * rz * (r3 * inv * inv);
            part[k][4] += z2r5 * (rx * r0.w + ry * r1.x + rz * r1.y);
            part[k][5] += z2r5 * (ry * r2.x - rz * r1.w);
            part[k][6] += z2r5 * (rz * r1.z - rx * r2.x);
            part[k][7] += z2r5 * (rx * r1.w - ry * r1.z);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) kahan_add(acc[k][c], cmp[k][c], part[k][c]);
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int nu = pass0 + threadIdx.x + k * blockDim.x;
      if (!valid[k]) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) Lam[((size_t)s * 4 + c) * m + nu] = acc[k][c];
      if constexpr (GB) {
        double f = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) f += (double)Mp[((size_t)s * 4 + c) * m + nu] * (double)acc[k][4 + c];
        gsum += -3.0 * f;
      }
    }
  }
  if constexpr (GB) {  // fixed-order block sum: lanes by butterfly, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    __syncthreads();  // gred of the previous cluster is read
    if ((threadIdx.x & 31) == 0) gred[threadIdx.x >> 5] = gsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += gred[w2];
      gfar[s] = t;
    }
  }
  }  // work items
}

// FP32 M2L^T specialised on NP1 = n + 1 (eta <= 1/2), the counterpart of
// k_m2l_fast: a thread owns source points nu with fixed (nu1, nu2), keeps
// R_x[mu1], R_x^2 and R_y[mu2], R_y^2 for R = xi_S,mu - xi_s,nu in registers
// and regroups the sums inside the mu1 loop (R_y, R_z constant there):
//   Lambda^a  += sum r3 W^E_x R_x + R_y sum r3 W^E_y + R_z sum r3 W^E_z
//   Lambda^b  += (R_y sum r3 W^B_z - R_z sum r3 W^B_y,
//                 R_z sum r3 W^B_x - sum r3 W^B_z R_x,
//                 sum r3 W^B_y R_x - R_y sum r3 W^B_x)
template <int NP1, int G, int SPLIT>
__global__ void __launch_bounds__(NP1 * NP1 * G, 3) k_adj_m2l_fast(const uint64_t* __restrict__ keys,
                                                                  const int32_t* __restrict__ off, int shift, const int32_t* __restrict__ order, int64_t nitems, unsigned int* __restrict__ work,
                                                                  const NodeGeo* __restrict__ geo,
                                                                  const float4* __restrict__ sdc, Cheb ch,
                                                                  const float* __restrict__ W, float* __restrict__ Lam) {
  constexpr int KPT = (NP1 + G * SPLIT - 1) / (G * SPLIT);
  constexpr int NT = NP1 * NP1 * G;
  constexpr int m = NP1 * NP1 * NP1;
  __shared__ float4 swa[m];            // (W^E_x, W^E_y, W^E_z, W^B_x)
  __shared__ float2 swb[m];            // (W^B_y, W^B_z)
  __shared__ float syz[NP1];           // target-cluster point offsets along z
  __shared__ float sacc[KPT][8][NT];   // Kahan sums and compensations
  __shared__ int64_t s_item;
  for (;;) {  // items (source, nu3 chunk) fetched in the work order: longest lists first
  if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(work, 1u);
  __syncthreads();
  const int64_t w = s_item;
  __syncthreads();
  if (w >= nitems) break;
  const int64_t s = order[w / SPLIT];
  const int base3 = (int)(w % SPLIT) * G * KPT;
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int b = off[s], e = off[s + 1];
  const NodeGeo gs = geo[s];
  const int tid = threadIdx.x;
  const int nu12 = tid % (NP1 * NP1), g = tid / (NP1 * NP1);
  const int nu1 = nu12 % NP1, nu2 = nu12 / NP1;
  const float xs = (float)(gs.h[0] * ch.t[nu1]), ys = (float)(gs.h[1] * ch.t[nu2]);
  float zs[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int nu3 = base3 + g + k * G;
    zs[k] = (float)(gs.h[2] * ch.t[nu3 < NP1 ? nu3 : 0]);
#pragma unroll
    for (int c = 0; c < 8; ++c) sacc[k][c][tid] = 0.f;
  }
  for (int it = b; it < e; ++it) {
    const int64_t S = (int64_t)(keys[it] & mask);
    const float4 dh = sdc[2 * it];  // c_s - c_S
    const NodeGeo gS = geo[S];
    const float hx = (float)gS.h[0], hy = (float)gS.h[1];
    __syncthreads();
    const float* Ws = W + (size_t)S * 6 * m;
    for (int o = tid; o < m; o += NT) {
      swa[o] = make_float4(Ws[o], Ws[m + o], Ws[2 * m + o], Ws[3 * m + o]);
      swb[o] = make_float2(Ws[4 * m + o], Ws[5 * m + o]);
    }
    if (tid < NP1) syz[tid] = (float)(gS.h[2] * ch.t[tid]);
    __syncthreads();
    const float X = dh.x + xs, Y = dh.y + ys;  // this point relative to the target-cluster centre
    float Rx[NP1], Dx[NP1], Ry[NP1], Dy[NP1];
#pragma unroll
    for (int k = 0; k < NP1; ++k) {
      Rx[k] = hx * (float)ch.t[k] - X;
      Dx[k] = Rx[k] * Rx[k];
      Ry[k] = hy * (float)ch.t[k] - Y;
      Dy[k] = Ry[k] * Ry[k];
    }
    float Z[KPT], part[KPT][4];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      Z[k] = dh.z + zs[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) part[k][c] = 0.f;
    }
    for (int m3 = 0; m3 < NP1; ++m3) {
      const float yz = syz[m3];
      float rz[KPT], dz[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        rz[k] = yz - Z[k];
        dz[k] = rz[k] * rz[k];
      }
      const int row = m3 * NP1 * NP1;
#pragma unroll
      for (int m2 = 0; m2 < NP1; ++m2) {
        float dyz[KPT], T1[KPT], T2[KPT], T3[KPT], T4[KPT], T5[KPT], T5R[KPT], T6[KPT], T6R[KPT];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          dyz[k] = Dy[m2] + dz[k];
          T1[k] = T2[k] = T3[k] = T4[k] = T5[k] = T5R[k] = T6[k] = T6R[k] = 0.f;
        }
#pragma unroll
        for (int m1 = 0; m1 < NP1; ++m1) {
          const float4 wa = swa[row + m2 * NP1 + m1];
          const float2 wb = swb[row + m2 * NP1 + m1];
#pragma unroll
          for (int k = 0; k < KPT; ++k) {
            const float d = fmaxf(Dx[m1] + dyz[k], 5.169878828456423e-26f);
            const float inv = rsqrt_normal(d);
            const float r3 = inv * inv * inv;
            T1[k] = fmaf(wa.x * Rx[m1], r3, T1[k]);
            T2[k] = fmaf(wa.y, r3, T2[k]);
            T3[k] = fmaf(wa.z, r3, T3[k]);
            T4[k] = fmaf(wa.w, r3, T4[k]);
            const float w5 = wb.x * r3;
            T5[k] += w5;
            T5R[k] = fmaf(w5, Rx[m1], T5R[k]);
            const float w6 = wb.y * r3;
            T6[k] += w6;
            T6R[k] = fmaf(w6, Rx[m1], T6R[k]);
          }
        }
        const float ry = Ry[m2];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          part[k][0] += T1[k] + ry * T2[k] + rz[k] * T3[k];
          part[k][1] += ry * T6[k] - rz[k] * T5[k];
          part[k][2] += rz[k] * T4[k] - T6R[k];
          part[k][3] += T5R[k] - ry * T4[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float sum = sacc[k][c][tid], comp = sacc[k][4 + c][tid];
        kahan_add(sum, comp, part[k][c]);
        sacc[k][c][tid] = sum;
        sacc[k][4 + c][tid] = comp;
      }
  }
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int nu3 = base3 + g + k * G;
    if (nu3 >= NP1) continue;
    const int nu = nu1 + NP1 * (nu2 + NP1 * nu3);
#pragma unroll
    for (int c = 0; c < 4; ++c) Lam[((size_t)s * 4 + c) * m + nu] = sacc[k][c][tid];
  }
  }  // work items
}

// FP32 M2L^T with paired arithmetic, the counterpart of k_m2l_pair: a thread
// owns two source points of the cluster, nu_a = P and nu_b = P + H, and
// evaluates both against each target point mu with paired FP32 instructions.
// In the mu1 loop R_x = t_x[mu1] - X is the only varying component
// (R = xi_S,mu - xi_s,nu, its x part held per mu1 in registers), so the sums
// are taken in r3 and r3 R_x and multiplied by R_y, R_z after the loop: of
// Lambda's sums only W^E_x, W^B_y and W^B_z meet R_x, and a point pair costs
// 12 FMA-pipe operations (|R|^2 1, r^-3 2, r3 R_x 1, eight sums) on three
// staged float4 per target point, duplicated for the two lanes:
// (WEx, ., WEy, .), (WEz, ., WBx, .), (WBy, ., WBz, .).  Splitting the R_x
// sums as sum w r3 R_x = sum (w t_x) r3 - X sum w r3 takes as many
// operations on five staged float4 (2^24 core-halo beam, n = 8: 960 ms
// against 853 ms for this form at 3 blocks per SM, 823 ms at 4).
template <int NP1, int NT>
__global__ void __launch_bounds__(NT, 4) k_adj_m2l_pair(const uint64_t* __restrict__ keys,
                                                       const int32_t* __restrict__ off, int shift,
                                                       const int32_t* __restrict__ order, int64_t nitems,
                                                       unsigned int* __restrict__ work,
                                                       const NodeGeo* __restrict__ geo,
                                                       const float4* __restrict__ sdc, Cheb ch,
                                                       const float* __restrict__ W, float* __restrict__ Lam) {
  constexpr int m = NP1 * NP1 * NP1;
  constexpr int H = (m + 1) / 2;
  constexpr int SPLIT = (H + NT - 1) / NT;
  extern __shared__ float4 dsm[];
  float4* sw = dsm;                                        // [m][3] staged target points
  float2* sacc = reinterpret_cast<float2*>(dsm + 3 * m);   // [8][NT] Kahan sums, compensations
  __shared__ float sxyz[3][NP1];                           // target point offsets per axis
  __shared__ int64_t s_item;
  const int tid = threadIdx.x;
  const float2 neg1 = make_float2(-1.f, -1.f);
  for (;;) {  // items (source, chunk of NT point pairs) in the work order: longest lists first
    if (tid == 0) s_item = (int64_t)atomicAdd(work, 1u);
    __syncthreads();
    const int64_t w = s_item;
    __syncthreads();
    if (w >= nitems) break;
    const int64_t s = order[w / SPLIT];
    const int P = (int)(w % SPLIT) * NT + tid;
    const int nua = P < H ? P : 0, nub = P + H < m ? P + H : 0;
    const uint64_t mask = ((uint64_t)1 << shift) - 1;
    const int b = off[s], e = off[s + 1];
    const NodeGeo gs = geo[s];
    const float2 xs = make_float2((float)(gs.h[0] * ch.t[nua % NP1]), (float)(gs.h[0] * ch.t[nub % NP1]));
    const float2 ys = make_float2((float)(gs.h[1] * ch.t[(nua / NP1) % NP1]),
                                  (float)(gs.h[1] * ch.t[(nub / NP1) % NP1]));
    const float2 zs = make_float2((float)(gs.h[2] * ch.t[nua / (NP1 * NP1)]),
                                  (float)(gs.h[2] * ch.t[nub / (NP1 * NP1)]));
#pragma unroll
    for (int c = 0; c < 8; ++c) sacc[c * NT + tid] = make_float2(0.f, 0.f);
    for (int it = b; it < e; ++it) {
      const int64_t S = (int64_t)(keys[it] & mask);
      const float4 dh = sdc[2 * it];  // c_s - c_S
      const NodeGeo gS = geo[S];
      __syncthreads();
      const float* Ws = W + (size_t)S * 6 * m;
      for (int o = tid; o < m; o += NT) {
        const float ex = Ws[o], ey = Ws[m + o], ez = Ws[2 * m + o];
        const float bx = Ws[3 * m + o], by = Ws[4 * m + o], bz = Ws[5 * m + o];
        sw[3 * o] = make_float4(ex, ex, ey, ey);
        sw[3 * o + 1] = make_float4(ez, ez, bx, bx);
        sw[3 * o + 2] = make_float4(by, by, bz, bz);
      }
      if (tid < 3 * NP1) {
        const int d = tid / NP1, k = tid - d * NP1;
        sxyz[d][k] = (float)(gS.h[d] * ch.t[k]);
      }
      __syncthreads();
      // this thread's two source points relative to the target-cluster centre
      const float2 X = __fadd2_rn(make_float2(dh.x, dh.x), xs);
      const float2 Y = __fadd2_rn(make_float2(dh.y, dh.y), ys);
      const float2 Z = __fadd2_rn(make_float2(dh.z, dh.z), zs);
      const float2 nX = __fmul2_rn(X, neg1);
      float2 Rx[NP1];
#pragma unroll
      for (int k = 0; k < NP1; ++k) Rx[k] = __fadd2_rn(make_float2(sxyz[0][k], sxyz[0][k]), nX);
      float2 part[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) part[c] = make_float2(0.f, 0.f);
      for (int m3 = 0; m3 < NP1; ++m3) {
        const float2 rz = __fadd2_rn(make_float2(sxyz[2][m3], sxyz[2][m3]), __fmul2_rn(Z, neg1));
        const float2 nrz = __fmul2_rn(rz, neg1);
        const float2 dz = __fmul2_rn(rz, rz);
        const float4* row = sw + 3 * m3 * NP1 * NP1;
#pragma unroll
        for (int m2 = 0; m2 < NP1; ++m2) {
          const float2 ry = __fadd2_rn(make_float2(sxyz[1][m2], sxyz[1][m2]), __fmul2_rn(Y, neg1));
          const float2 dyz = __ffma2_rn(ry, ry, dz);
          const float2 z0 = make_float2(0.f, 0.f);
          float2 T2 = z0, T3 = z0, T4 = z0, T5 = z0, T6 = z0, U1 = z0, U5 = z0, U6 = z0;
#pragma unroll
          for (int m1 = 0; m1 < NP1; ++m1) {
            const float4* q = row + 3 * (m2 * NP1 + m1);
            const float4 A = q[0], Bq = q[1], C = q[2];
            float2 d = __ffma2_rn(Rx[m1], Rx[m1], dyz);
            d.x = fmaxf(d.x, tiny_sep2<float>());
            d.y = fmaxf(d.y, tiny_sep2<float>());
            const float2 inv = make_float2(rsqrt_normal(d.x), rsqrt_normal(d.y));
            const float2 r3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
            const float2 rr = __fmul2_rn(r3, Rx[m1]);
            U1 = __ffma2_rn(make_float2(A.x, A.y), rr, U1);
            T2 = __ffma2_rn(make_float2(A.z, A.w), r3, T2);
            T3 = __ffma2_rn(make_float2(Bq.x, Bq.y), r3, T3);
            T4 = __ffma2_rn(make_float2(Bq.z, Bq.w), r3, T4);
            T5 = __ffma2_rn(make_float2(C.x, C.y), r3, T5);
            T6 = __ffma2_rn(make_float2(C.z, C.w), r3, T6);
            U5 = __ffma2_rn(make_float2(C.x, C.y), rr, U5);
            U6 = __ffma2_rn(make_float2(C.z, C.w), rr, U6);
          }
          // Lambda^a += sum r3 R_x W^E_x + R_y sum r3 W^E_y + R_z sum r3 W^E_z
          // Lambda^b += (R_y sum r3 W^B_z - R_z sum r3 W^B_y, R_z sum r3 W^B_x - sum r3 R_x W^B_z,
          //              sum r3 R_x W^B_y - R_y sum r3 W^B_x)
          part[0] = __fadd2_rn(part[0], U1);
          part[0] = __ffma2_rn(ry, T2, part[0]);
          part[0] = __ffma2_rn(rz, T3, part[0]);
          part[1] = __ffma2_rn(ry, T6, part[1]);
          part[1] = __ffma2_rn(nrz, T5, part[1]);
          part[2] = __ffma2_rn(rz, T4, part[2]);
          part[2] = __ffma2_rn(U6, neg1, part[2]);
          part[3] = __fadd2_rn(part[3], U5);
          part[3] = __ffma2_rn(__fmul2_rn(ry, neg1), T4, part[3]);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float2 sum = sacc[c * NT + tid], comp = sacc[(4 + c) * NT + tid];
        kahan_add(sum.x, comp.x, part[c].x);
        kahan_add(sum.y, comp.y, part[c].y);
        sacc[c * NT + tid] = sum;
        sacc[(4 + c) * NT + tid] = comp;
      }
    }
    if (P < H) {
#pragma unroll
      for (int c = 0; c < 4; ++c) Lam[((size_t)s * 4 + c) * m + P] = sacc[c * NT + tid].x;
    }
    if (P + H < m) {
#pragma unroll
      for (int c = 0; c < 4; ++c) Lam[((size_t)s * 4 + c) * m + P + H] = sacc[c * NT + tid].y;
    }
  }  // work items
}

template <int NP1, int NT>
int launch_adj_m2l_pair(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  constexpr int m = NP1 * NP1 * NP1, H = (m + 1) / 2, SPLIT = (H + NT - 1) / NT;
  const size_t smem = sizeof(float4) * 3 * m + sizeof(float2) * 8 * NT;
  if (int rc = smem_limit(k_adj_m2l_pair<NP1, NT>, (int)smem)) return rc;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_adj_m2l_pair<NP1, NT>, NT, smem, P->C * SPLIT, &grid)) return rc;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  FMM_CUDA_TRY(cudaMemsetAsync(&cnt->work[1], 0, sizeof(unsigned int), s));
  k_adj_m2l_pair<NP1, NT><<<grid, NT, smem, s>>>(
      ws_ptr<uint64_t>(P, L.m2l_src), ws_ptr<int32_t>(P, L.m2l_soff), P->kappa + 1,
      ws_ptr<int32_t>(P, L.m2l_sorder), P->C * SPLIT, &cnt->work[1], ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.m2l_sdc), P->cheb, ws_ptr<float>(P, L.wbuf), ws_ptr<float>(P, L.lbuf));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <int NP1, int G, int SPLIT>
int launch_adj_m2l_fast(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_adj_m2l_fast<NP1, G, SPLIT>, NP1 * NP1 * G, 0, P->C * SPLIT, &grid)) return rc;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  FMM_CUDA_TRY(cudaMemsetAsync(&cnt->work[1], 0, sizeof(unsigned int), s));
  k_adj_m2l_fast<NP1, G, SPLIT><<<grid, NP1 * NP1 * G, 0, s>>>(
      ws_ptr<uint64_t>(P, L.m2l_src), ws_ptr<int32_t>(P, L.m2l_soff), P->kappa + 1,
      ws_ptr<int32_t>(P, L.m2l_sorder), P->C * SPLIT, &cnt->work[1], ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.m2l_sdc), P->cheb, ws_ptr<float>(P, L.wbuf), ws_ptr<float>(P, L.lbuf));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// Shared-memory bytes ahead of the per-leaf expansion: the staged source rows,
// or the other groups' compensated sums (2 nc values per owned particle) when
// those take more room.
template <typename T>
__host__ __device__ inline size_t stage_bytes(int rows, int kpt, int nc2, int groups, int NT) {
  const size_t a = sizeof(typename Vec4<T>::type) * rows * (size_t)groups * NT;
  const size_t b = sizeof(T) * (size_t)(groups - 1) * kpt * nc2 * NT;
  return a > b ? a : b;
}

// The particle kernels run `groups` groups of NT threads per leaf, every
// group with its own share of the pairs; group 0 adds the compensated sums
// (sum - comp) of groups 1, 2, ... in that order.  cb overlays the staging
// rows, which no thread reads any more.
template <typename T, int KPT, int NC>
__device__ __forceinline__ void combine_groups(T (&acc)[KPT][NC], T (&cmp)[KPT][NC], T* cb, int groups, int grp,
                                               int NT, int lt) {
  if (groups <= 1) return;
  if (grp > 0)
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        cb[(((grp - 1) * KPT + k) * 2 * NC + c) * NT + lt] = acc[k][c];
        cb[(((grp - 1) * KPT + k) * 2 * NC + NC + c) * NT + lt] = cmp[k][c];
      }
  __syncthreads();
  if (grp == 0)
    for (int g2 = 1; g2 < groups; ++g2)
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          kahan_add(acc[k][c], cmp[k][c], cb[(((g2 - 1) * KPT + k) * 2 * NC + c) * NT + lt]);
          kahan_add(acc[k][c], cmp[k][c], -cb[(((g2 - 1) * KPT + k) * 2 * NC + NC + c) * NT + lt]);
        }
  __syncthreads();
}

// Near field at the targets (J u over the target-major P2P list) plus the far
// field at the targets (grad of the forward's cumulative local); writes the
// target-side dL/dx' of every particle (leaf order).  With GB it also sums,
// per target, the near-field part of gbar dL/dgbar: in internal units
// dg/dgbar = -(3/gbar) R_z^2 R / |R|^5, so the pair term is
// -3 R_z^2 r^-5 (R . u), stored in the .w component of the output.
template <typename T, int KPT, bool GB>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 1) k_adj_target(
    const uint64_t* __restrict__ keys, const int32_t* __restrict__ off, int shift,
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int kappa,
    const NodeGeo* __restrict__ geo, const typename Vec4<T>::type* __restrict__ px,
    const typename Vec4<T>::type* __restrict__ pb, const typename Vec4<T>::type* __restrict__ pl,
    const void* __restrict__ pdc_raw, const typename Vec4<T>::type* __restrict__ wle,
    const typename Vec4<T>::type* __restrict__ wlb, const T* __restrict__ Lcum, Cheb ch, ChebD cd, int m,
    int groups, int chunks, int64_t nitems, typename Vec4<T>::type* __restrict__ gout) {
  using V4 = typename Vec4<T>::type;
  constexpr bool kSplit = std::is_same<T, float>::value;
  // FP32: sources staged in pairs, 7 float4 (28 floats) per pair, each of 14
  // components as (source 2q, source 2q+1): -x_hi, -y_hi, -z_hi, a, b~x,
  // b~y, b~z, -b~x, -b~y, -b~z, -x_lo, -y_lo, -z_lo, 0; a thread evaluates
  // both sources of a pair at once with paired FP32 arithmetic
  constexpr int kRow = kSplit ? 4 : 2;
  extern __shared__ unsigned char smem_raw[];
  V4* sp = reinterpret_cast<V4*>(smem_raw);
  const int NT = blockDim.x / groups, grp = threadIdx.x / NT, lt = threadIdx.x - grp * NT;
  constexpr int NC = GB ? 4 : 3;  // dL/dx' (3) and the gbar term
  T* sl = reinterpret_cast<T*>(smem_raw + stage_bytes<T>(kRow, KPT, 2 * NC, groups, NT));  // [6][m]
  const int64_t per_pass = (int64_t)KPT * NT;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {  // (leaf, chunk) items
  __syncthreads();  // the previous item's readers of sl are done
  const int64_t t = ((int64_t)1 << kappa) + item / chunks;
  const int64_t c0 = (int64_t)(item % chunks) * per_pass;
  const int64_t st = nstart[t], cnt = min64(ncount[t], c0 + per_pass);
  if (c0 >= cnt) continue;  // the leaf is smaller than this chunk
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const NodeGeo gt = geo[t];
  const int b = off[t], e = off[t + 1];
  const int np1 = ch.np1;
  T invh[3];
  bool deg[3];
  for (int d = 0; d < 3; ++d) {
    deg[d] = !(gt.h[d] > 0.0);
    invh[d] = deg[d] ? T(0) : (T)(1.0 / gt.h[d]);
  }
  if (kappa > 0) {
    const T* Lt = Lcum + (size_t)t * 6 * m;
    for (int o = threadIdx.x; o < 6 * m; o += blockDim.x) sl[o] = Lt[o];
  }
  for (int64_t pass0 = c0; pass0 < cnt; pass0 += per_pass) {
    T ri[KPT][3], rl[KPT][3], we[KPT][3], wb[KPT][3];
    bool valid[KPT];
    T acc[KPT][NC], cmp[KPT][NC];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int64_t j = pass0 + lt + (int64_t)k * NT;
      valid[k] = j < cnt;
      const int64_t jj = st + (valid[k] ? j : 0);
      const V4 u = px[jj], a = wle[jj], c = wlb[jj];
      ri[k][0] = u.x; ri[k][1] = u.y; ri[k][2] = u.z;
      if constexpr (kSplit) {
        const V4 l = pl[jj];
        rl[k][0] = l.x; rl[k][1] = l.y; rl[k][2] = l.z;
      } else {
        rl[k][0] = rl[k][1] = rl[k][2] = T(0);
      }
      we[k][0] = a.x; we[k][1] = a.y; we[k][2] = a.z;
      wb[k][0] = c.x; wb[k][1] = c.y; wb[k][2] = c.z;
#pragma unroll
      for (int d = 0; d < NC; ++d) acc[k][d] = cmp[k][d] = T(0);
    }
    for (int it = b; it < e; ++it) {
      const int64_t s = (int64_t)(keys[it] & mask);
      const int64_t sst = nstart[s], scnt = ncount[s];
      T X[KPT][3], XL[KPT][3], part[KPT][NC];
      if constexpr (kSplit) {
        const float4* pdc = static_cast<const float4*>(pdc_raw);
        const float4 dh = pdc[2 * it], dl = pdc[2 * it + 1];
        const float dch[3] = {dh.x, dh.y, dh.z}, dcl[3] = {dl.x, dl.y, dl.z};
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float hs, he;
            two_sum(ri[k][d], dch[d], hs, he);
            const float lo = he + (rl[k][d] + dcl[d]);
            X[k][d] = hs + lo;
            XL[k][d] = lo - (X[k][d] - hs);
          }
      } else {
        const double4 dd = static_cast<const double4*>(pdc_raw)[it];
        const T dc[3] = {(T)dd.x, (T)dd.y, (T)dd.z};
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            X[k][d] = ri[k][d] + dc[d];
            XL[k][d] = T(0);
          }
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int d = 0; d < NC; ++d) part[k][d] = T(0);
      float2 pp2[NC];  // paired partial sums (FP32 path): even and odd sources of the leaf
#pragma unroll
      for (int d = 0; d < NC; ++d) pp2[d] = make_float2(0.f, 0.f);
      for (int64_t base = 0; base < scnt; base += blockDim.x) {
        __syncthreads();
        const int64_t j = base + threadIdx.x;
        if constexpr (kSplit && KPT == 1) {
          float c[14];
          if (j < scnt) {
            const float4 u = px[sst + j], w = pb[sst + j], l = pl[sst + j];
            c[0] = -u.x; c[1] = -u.y; c[2] = -u.z; c[3] = u.w;
            c[4] = w.x; c[5] = w.y; c[6] = w.z; c[7] = -w.x; c[8] = -w.y; c[9] = -w.z;
            c[10] = -l.x; c[11] = -l.y; c[12] = -l.z; c[13] = 0.f;
          } else {  // partner of an odd last source: no mass, no contribution
#pragma unroll
            for (int q = 0; q < 14; ++q) c[q] = 0.f;
          }
          float* f = reinterpret_cast<float*>(sp) + (threadIdx.x >> 1) * 28 + (threadIdx.x & 1);
#pragma unroll
          for (int q = 0; q < 14; ++q) f[2 * q] = c[q];
        } else if (j < scnt) {
          sp[kRow * threadIdx.x] = px[sst + j];
          sp[kRow * threadIdx.x + 1] = pb[sst + j];
          if constexpr (kSplit) sp[kRow * threadIdx.x + 2] = pl[sst + j];
        }
        __syncthreads();
        const int nj = (int)min64(blockDim.x, scnt - base);
        if constexpr (kSplit && KPT == 1) {  // source pairs, paired arithmetic
          const int npq = (nj + 1) >> 1;
          const int share2 = (npq + groups - 1) / groups, q1 = min(npq, (grp + 1) * share2);
          const float2 X0 = make_float2(X[0][0], X[0][0]), X1 = make_float2(X[0][1], X[0][1]),
                       X2 = make_float2(X[0][2], X[0][2]);
          const float2 L0 = make_float2(XL[0][0], XL[0][0]), L1 = make_float2(XL[0][1], XL[0][1]),
                       L2 = make_float2(XL[0][2], XL[0][2]);
          const float2 E0 = make_float2(we[0][0], we[0][0]), E1 = make_float2(we[0][1], we[0][1]),
                       E2 = make_float2(we[0][2], we[0][2]);
          const float2 B0 = make_float2(wb[0][0], wb[0][0]), B1 = make_float2(wb[0][1], wb[0][1]),
                       B2 = make_float2(wb[0][2], wb[0][2]);
          const float2 m3 = make_float2(-3.f, -3.f);
          for (int qq = grp * share2; qq < q1; ++qq) {
            const float4* s4 = reinterpret_cast<const float4*>(sp) + 7 * qq;
            const float4 A = s4[0], Bq = s4[1], Cq = s4[2], Dq = s4[3], Eq = s4[4], Fq = s4[5], Gq = s4[6];
            // R = x_i - x_j = (X_hi - x_hi) + (X_lo - x_lo)
            const float2 rx = __fadd2_rn(__fadd2_rn(X0, make_float2(A.x, A.y)), __fadd2_rn(L0, make_float2(Fq.x, Fq.y)));
            const float2 ry = __fadd2_rn(__fadd2_rn(X1, make_float2(A.z, A.w)), __fadd2_rn(L1, make_float2(Fq.z, Fq.w)));
            const float2 rz = __fadd2_rn(__fadd2_rn(X2, make_float2(Bq.x, Bq.y)), __fadd2_rn(L2, make_float2(Gq.x, Gq.y)));
            const float2 d = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
            float2 inv;
            inv.x = d.x > tiny_sep2<float>() ? rsqrt_t<float>(d.x) : 0.f;
            inv.y = d.y > tiny_sep2<float>() ? rsqrt_t<float>(d.y) : 0.f;
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 r3 = __fmul2_rn(inv2, inv);
            const float2 r5 = __fmul2_rn(r3, inv2);
            const float2 aa = make_float2(Bq.z, Bq.w);
            const float2 bx = make_float2(Cq.x, Cq.y), by = make_float2(Cq.z, Cq.w), bz = make_float2(Dq.x, Dq.y);
            const float2 nbx = make_float2(Dq.z, Dq.w), nby = make_float2(Eq.x, Eq.y), nbz = make_float2(Eq.z, Eq.w);
            // u = a'_j wE^_i + wB^_i x b~'_j
            const float2 ux = __ffma2_rn(aa, E0, __ffma2_rn(B1, bz, __fmul2_rn(B2, nby)));
            const float2 uy = __ffma2_rn(aa, E1, __ffma2_rn(B2, bx, __fmul2_rn(B0, nbz)));
            const float2 uz = __ffma2_rn(aa, E2, __ffma2_rn(B0, by, __fmul2_rn(B1, nbx)));
            const float2 ru = __ffma2_rn(rz, uz, __ffma2_rn(ry, uy, __fmul2_rn(rx, ux)));
            const float2 nc3 = __fmul2_rn(__fmul2_rn(r5, m3), ru);
            pp2[0] = __ffma2_rn(nc3, rx, __ffma2_rn(r3, ux, pp2[0]));
            pp2[1] = __ffma2_rn(nc3, ry, __ffma2_rn(r3, uy, pp2[1]));
            pp2[2] = __ffma2_rn(nc3, rz, __ffma2_rn(r3, uz, pp2[2]));
            if constexpr (GB) pp2[NC - 1] = __ffma2_rn(__fmul2_rn(rz, rz), nc3, pp2[NC - 1]);
          }
          continue;
        }
        const int share = (nj + groups - 1) / groups, j1 = min(nj, (grp + 1) * share);
        for (int jj = grp * share; jj < j1; ++jj) {
          const V4 u = sp[kRow * jj], w = sp[kRow * jj + 1];
          V4 ul;
          if constexpr (kSplit) ul = sp[kRow * jj + 2];
#pragma unroll
          for (int k = 0; k < KPT; ++k) {
            T rx, ry, rz;
            if constexpr (kSplit) {
              rx = (X[k][0] - u.x) + (XL[k][0] - ul.x);
              ry = (X[k][1] - u.y) + (XL[k][1] - ul.y);
              rz = (X[k][2] - u.z) + (XL[k][2] - ul.z);
            } else {
              rx = X[k][0] - u.x;
              ry = X[k][1] - u.y;
              rz = X[k][2] - u.z;
            }
            const T d = rx * rx + ry * ry + rz * rz;
            const T inv = d > tiny_sep2<T>() ? rsqrt_t<T>(d) : T(0);
            const T r3 = inv * inv * inv;
            const T r5 = r3 * inv * inv;
            // u = a'_j wE^_i + wB^_i x b~'_j
            const T ux = u.w * we[k][0] + (wb[k][1] * w.z - wb[k][2] * w.y);
            const T uy = u.w * we[k][1] + (wb[k][2] * w.x - wb[k][0] * w.z);
            const T uz = u.w * we[k][2] + (wb[k][0] * w.y - wb[k][1] * w.x);
            const T c3 = T(3) * r5 * (rx * ux + ry * uy + rz * uz);
            part[k][0] += r3 * ux - c3 * rx;
            part[k][1] += r3 * uy - c3 * ry;
            part[k][2] += r3 * uz - c3 * rz;
            if constexpr (GB) part[k][NC - 1] -= rz * rz * c3;
          }
        }
      }
      if constexpr (kSplit && KPT == 1) {
#pragma unroll
        for (int d = 0; d < NC; ++d) part[0][d] = pp2[d].x + pp2[d].y;
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int d = 0; d < NC; ++d) kahan_add(acc[k][d], cmp[k][d], part[k][d]);
    }
    __syncthreads();
    const int a3share = (np1 + groups - 1) / groups;
    const int a3b = min(np1, grp * a3share), a3e = min(np1, a3b + a3share);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (valid[k] && kappa > 0) {  // far field at the target: grad of sum_mu l_mu(x) (w^ . Lc_mu)
        T lx[kMaxNp1], ly[kMaxNp1], lz[kMaxNp1], dx[kMaxNp1], dy[kMaxNp1], dz[kMaxNp1];
        const T lof = kSplit ? T(1) : T(0);
        basis_deriv<T>((ri[k][0] + lof * rl[k][0]) * invh[0], deg[0], ch, cd, lx, dx);
        basis_deriv<T>((ri[k][1] + lof * rl[k][1]) * invh[1], deg[1], ch, cd, ly, dy);
        basis_deriv<T>((ri[k][2] + lof * rl[k][2]) * invh[2], deg[2], ch, cd, lz, dz);
        T G[3] = {T(0), T(0), T(0)};
        int mu = a3b * np1 * np1;
        for (int a3 = a3b; a3 < a3e; ++a3) {
          for (int a2 = 0; a2 < np1; ++a2) {
            T s0 = T(0), sx = T(0);
            for (int a1 = 0; a1 < np1; ++a1, ++mu) {
              const T phi = we[k][0] * sl[mu] + we[k][1] * sl[m + mu] + we[k][2] * sl[2 * m + mu] +
                            wb[k][0] * sl[3 * m + mu] + wb[k][1] * sl[4 * m + mu] + wb[k][2] * sl[5 * m + mu];
              s0 += lx[a1] * phi;
              sx += dx[a1] * phi;
            }
            G[0] += ly[a2] * lz[a3] * sx;
            G[1] += dy[a2] * lz[a3] * s0;
            G[2] += ly[a2] * dz[a3] * s0;
          }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) kahan_add(acc[k][d], cmp[k][d], G[d] * invh[d]);
      }
    }
    combine_groups<T, KPT, NC>(acc, cmp, reinterpret_cast<T*>(smem_raw), groups, grp, NT, lt);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (grp != 0 || !valid[k]) continue;
      const int64_t pos = st + pass0 + lt + (int64_t)k * NT;
      V4 o;
      o.x = acc[k][0]; o.y = acc[k][1]; o.z = acc[k][2]; o.w = GB ? acc[k][NC - 1] : T(0);
      gout[pos] = o;
    }
  }
  }  // items
}

// FP32 near field of both roles in one pass (the default FP32 adjoint).  A
// thread owns particle i of leaf L.  For every P2P partner leaf P of L it
// takes both roles of each pair (i, j), R = x_i - x_j:
//   i as target:  dL/dx'_i += J(R) u_ij,         u_ij = a'_j w^E_i + w^B_i x b~'_j
//   i as source:  dL/dx'_i -= J(R) u_ji,         u_ji = a'_i w^E_j + w^B_j x b~'_i
//                 dL/da'_i -= w^E_j . K(R),  dL/db~'_i -= K(R) x w^B_j,  K = r^-3 R
// with J(R) v = r^-3 v - 3 r^-5 R (R . v) even in R, so the two J terms are
// one J(R)(u_ij - u_ji).  The partners come from merging L's target-major
// list (P is a source of L) with its source-major list (P is a target of L),
// both sorted by partner: a partner in only one list gets only that role,
// by staging its masses (no target role) or its weights (no source role) as
// zero.  Partners are staged in pairs as in k_adj_target and evaluated with
// paired FP32 arithmetic; per partner leaf the two lanes are added and
// Kahan-summed.  With a far field (kappa > 0) the target-side far field that
// k_adj_far left in g1 is added last, so this kernel reads no expansion and
// may run while the far-field chain overwrites the leaf locals.  Output per
// particle (leaf order): g1 = (dL/dx' (3), dL/da'), g2 = (dL/db~' (3), 0);
// the source-side far field and the chain rule follow in k_adj_final.
template <int KPT>
__global__ void __launch_bounds__(128, KPT == 1 ? 5 : 3) k_adj_near(
    const uint64_t* __restrict__ keys, const int32_t* __restrict__ off, const uint64_t* __restrict__ skeys,
    const int32_t* __restrict__ soff, int shift, const int64_t* __restrict__ nstart,
    const int64_t* __restrict__ ncount, int kappa, const float4* __restrict__ px, const float4* __restrict__ pb,
    const float4* __restrict__ pl, const float4* __restrict__ pdc, const float4* __restrict__ sdc,
    const float4* __restrict__ wle, const float4* __restrict__ wlb, int groups, int chunks, int64_t nitems,
    float4* __restrict__ g1, float4* __restrict__ g2) {
  // staged partner pairs: 12 float4 (48 floats) at a 13-float4 stride, 24
  // components as (partner 2q, partner 2q+1): -x_hi (3), -x_lo (3), a, b~ (3),
  // -b~ (3), w^E (3), w^B (3), -w^B (3), 0, 0
  // a staged pair takes 13 float4 (52 floats, 48 used): with a 52-float
  // stride the scattered staging stores of a warp fall into 2 ways of the
  // shared-memory banks instead of 8 (48 = 16 mod 32)
  constexpr int kPairStride = 52;
  constexpr int NC = 7;    // dL/dx' (3), dL/da', dL/db~' (3)
  extern __shared__ unsigned char smem_raw[];
  const int NT = blockDim.x / groups, grp = threadIdx.x / NT, lt = threadIdx.x - grp * NT;
  // per thread and owned particle the running sums and their compensations,
  // [KPT][2 NC][threads]: touched once per partner leaf, so they stay out of
  // the registers of the pair loop
  float* sK = reinterpret_cast<float*>(smem_raw + stage_bytes<float>(7, KPT, 2 * NC, groups, NT)) + threadIdx.x;
  const int kstride = blockDim.x;
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int64_t per_chunk = (int64_t)KPT * NT;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {  // (leaf, chunk) items
  __syncthreads();  // the previous item's readers of the stage are done
  const int64_t L = ((int64_t)1 << kappa) + item / chunks;
  const int64_t c0 = (int64_t)(item % chunks) * per_chunk;
  const int64_t st = nstart[L], cnt = min64(ncount[L], c0 + per_chunk);
  if (c0 >= cnt) continue;  // the leaf is smaller than this chunk
  bool valid[KPT];
  int64_t jj[KPT];
  float4 u0[KPT], l0[KPT];
  float2 WE0[KPT], WE1[KPT], WE2[KPT], WB0[KPT], WB1[KPT], WB2[KPT], NA[KPT], B0[KPT], B1[KPT], B2[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int64_t j0 = c0 + lt + (int64_t)k * NT;
    valid[k] = j0 < cnt;
    jj[k] = st + (valid[k] ? j0 : 0);
    u0[k] = px[jj[k]];
    l0[k] = pl[jj[k]];
    const float4 b0 = pb[jj[k]], e0 = wle[jj[k]], w0 = wlb[jj[k]];
    WE0[k] = make_float2(e0.x, e0.x); WE1[k] = make_float2(e0.y, e0.y); WE2[k] = make_float2(e0.z, e0.z);
    WB0[k] = make_float2(w0.x, w0.x); WB1[k] = make_float2(w0.y, w0.y); WB2[k] = make_float2(w0.z, w0.z);
    NA[k] = make_float2(-u0[k].w, -u0[k].w);
    B0[k] = make_float2(b0.x, b0.x); B1[k] = make_float2(b0.y, b0.y); B2[k] = make_float2(b0.z, b0.z);
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) sK[(k * 2 * NC + c) * kstride] = 0.f;
  }
  const float2 m3 = make_float2(-3.f, -3.f);
  int it1 = off[L], it2 = soff[L];
  const int e1 = off[L + 1], e2 = soff[L + 1];
  while (it1 < e1 || it2 < e2) {  // merge by partner leaf (block-uniform)
    const int64_t P1 = it1 < e1 ? (int64_t)(keys[it1] & mask) : INT64_MAX;
    const int64_t P2 = it2 < e2 ? (int64_t)(skeys[it2] & mask) : INT64_MAX;
    const int64_t P = P1 < P2 ? P1 : P2;
    const bool tgt = P1 == P, src = P2 == P;  // i as target of P's particles / as their source
    // c_L - c_P (scaled), the same in both lists for major L
    const float4 dh = tgt ? pdc[2 * it1] : sdc[2 * it2], dl = tgt ? pdc[2 * it1 + 1] : sdc[2 * it2 + 1];
    if (tgt) ++it1;
    if (src) ++it2;
    float2 X0[KPT], X1[KPT], X2[KPT], L0[KPT], L1[KPT], L2[KPT];  // x_i in P's frame, hi + lo
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const float ri[3] = {u0[k].x, u0[k].y, u0[k].z}, rl[3] = {l0[k].x, l0[k].y, l0[k].z};
      const float dch[3] = {dh.x, dh.y, dh.z}, dcl[3] = {dl.x, dl.y, dl.z};
      float X[3], XL[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float hs, he;
        two_sum(ri[d], dch[d], hs, he);
        const float lo = he + (rl[d] + dcl[d]);
        X[d] = hs + lo;
        XL[d] = lo - (X[d] - hs);
      }
      X0[k] = make_float2(X[0], X[0]); X1[k] = make_float2(X[1], X[1]); X2[k] = make_float2(X[2], X[2]);
      L0[k] = make_float2(XL[0], XL[0]); L1[k] = make_float2(XL[1], XL[1]); L2[k] = make_float2(XL[2], XL[2]);
    }
    const int64_t sst = nstart[P], scnt = ncount[P];
    float2 pp[KPT][NC];
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) pp[k][c] = make_float2(0.f, 0.f);
    for (int64_t base = 0; base < scnt; base += blockDim.x) {
      __syncthreads();
      const int64_t j = base + threadIdx.x;
      {
        float c[24];
        if (j < scnt) {
          const float4 u = px[sst + j], w = pb[sst + j], l = pl[sst + j];
          const float4 e = src ? wle[sst + j] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 v = src ? wlb[sst + j] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float a = tgt ? u.w : 0.f, bx = tgt ? w.x : 0.f, by = tgt ? w.y : 0.f, bz = tgt ? w.z : 0.f;
          c[0] = -u.x; c[1] = -u.y; c[2] = -u.z; c[3] = -l.x; c[4] = -l.y; c[5] = -l.z;
          c[6] = a; c[7] = bx; c[8] = by; c[9] = bz; c[10] = -bx; c[11] = -by; c[12] = -bz;
          c[13] = e.x; c[14] = e.y; c[15] = e.z; c[16] = v.x; c[17] = v.y; c[18] = v.z;
          c[19] = -v.x; c[20] = -v.y; c[21] = -v.z; c[22] = 0.f; c[23] = 0.f;
        } else {  // partner of an odd last particle: no mass, no weight, no contribution
#pragma unroll
          for (int q = 0; q < 24; ++q) c[q] = 0.f;
        }
        float* f = reinterpret_cast<float*>(smem_raw) + (threadIdx.x >> 1) * kPairStride + (threadIdx.x & 1);
#pragma unroll
        for (int q = 0; q < 24; ++q) f[2 * q] = c[q];
      }
      __syncthreads();
      const int nj = (int)min64(blockDim.x, scnt - base);
      const int npq = (nj + 1) >> 1;
      const int share2 = (npq + groups - 1) / groups, q1 = min(npq, (grp + 1) * share2);
      for (int qq = grp * share2; qq < q1; ++qq) {
        const float4* s4 = reinterpret_cast<const float4*>(smem_raw) + (kPairStride / 4) * qq;
        const float4 S0 = s4[0], S1 = s4[1], S2 = s4[2], S3 = s4[3], S4 = s4[4], S5 = s4[5];
        const float4 S6 = s4[6], S7 = s4[7], S8 = s4[8], S9 = s4[9], S10 = s4[10];
        const float2 aj = make_float2(S3.x, S3.y);
        const float2 bx = make_float2(S3.z, S3.w), by = make_float2(S4.x, S4.y), bz = make_float2(S4.z, S4.w);
        const float2 nbx = make_float2(S5.x, S5.y), nby = make_float2(S5.z, S5.w);
        const float2 nbz = make_float2(S6.x, S6.y);
        const float2 ex = make_float2(S6.z, S6.w), ey = make_float2(S7.x, S7.y), ez = make_float2(S7.z, S7.w);
        const float2 wx = make_float2(S8.x, S8.y), wy = make_float2(S8.z, S8.w), wz = make_float2(S9.x, S9.y);
        const float2 nwx = make_float2(S9.z, S9.w), nwy = make_float2(S10.x, S10.y), nwz = make_float2(S10.z, S10.w);
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          const float2 rx = __fadd2_rn(__fadd2_rn(X0[k], make_float2(S0.x, S0.y)), __fadd2_rn(L0[k], make_float2(S1.z, S1.w)));
          const float2 ry = __fadd2_rn(__fadd2_rn(X1[k], make_float2(S0.z, S0.w)), __fadd2_rn(L1[k], make_float2(S2.x, S2.y)));
          const float2 rz = __fadd2_rn(__fadd2_rn(X2[k], make_float2(S1.x, S1.y)), __fadd2_rn(L2[k], make_float2(S2.z, S2.w)));
          const float2 d = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
          float2 inv;
          inv.x = d.x > tiny_sep2<float>() ? rsqrt_t<float>(d.x) : 0.f;
          inv.y = d.y > tiny_sep2<float>() ? rsqrt_t<float>(d.y) : 0.f;
          const float2 inv2 = __fmul2_rn(inv, inv);
          const float2 r3 = __fmul2_rn(inv2, inv);
          // K = R / |R|^3 serves both roles
          const float2 kx = __fmul2_rn(r3, rx), ky = __fmul2_rn(r3, ry), kz = __fmul2_rn(r3, rz);
          // v = u_ij - u_ji = a_j w^E_i + w^B_i x b_j - a_i w^E_j + b_i x w^B_j
          const float2 vx = __ffma2_rn(aj, WE0[k], __ffma2_rn(WB1[k], bz, __ffma2_rn(WB2[k], nby,
                            __ffma2_rn(NA[k], ex, __ffma2_rn(B1[k], wz, __fmul2_rn(B2[k], nwy))))));
          const float2 vy = __ffma2_rn(aj, WE1[k], __ffma2_rn(WB2[k], bx, __ffma2_rn(WB0[k], nbz,
                            __ffma2_rn(NA[k], ey, __ffma2_rn(B2[k], wx, __fmul2_rn(B0[k], nwz))))));
          const float2 vz = __ffma2_rn(aj, WE2[k], __ffma2_rn(WB0[k], by, __ffma2_rn(WB1[k], nbx,
                            __ffma2_rn(NA[k], ez, __ffma2_rn(B0[k], wy, __fmul2_rn(B1[k], nwx))))));
          // J v = r3 v - 3 r5 (R . v) R = r3 v + c K with c = -3 r^-2 (R . v)
          const float2 rv = __ffma2_rn(rz, vz, __ffma2_rn(ry, vy, __fmul2_rn(rx, vx)));
          const float2 c = __fmul2_rn(__fmul2_rn(inv2, m3), rv);
          pp[k][0] = __ffma2_rn(c, kx, __ffma2_rn(r3, vx, pp[k][0]));
          pp[k][1] = __ffma2_rn(c, ky, __ffma2_rn(r3, vy, pp[k][1]));
          pp[k][2] = __ffma2_rn(c, kz, __ffma2_rn(r3, vz, pp[k][2]));
          // source role, summed with the sign flipped at the end: K . w^E_j, K x w^B_j
          pp[k][3] = __ffma2_rn(kz, ez, __ffma2_rn(ky, ey, __ffma2_rn(kx, ex, pp[k][3])));
          pp[k][4] = __ffma2_rn(ky, wz, __ffma2_rn(kz, nwy, pp[k][4]));
          pp[k][5] = __ffma2_rn(kz, wx, __ffma2_rn(kx, nwz, pp[k][5]));
          pp[k][6] = __ffma2_rn(kx, wy, __ffma2_rn(ky, nwx, pp[k][6]));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float* a = sK + (k * 2 * NC + c) * kstride;
        float sum = a[0], comp = a[NC * kstride];
        kahan_add(sum, comp, c < 3 ? pp[k][c].x + pp[k][c].y : -(pp[k][c].x + pp[k][c].y));
        a[0] = sum;
        a[NC * kstride] = comp;
      }
  }
  float acc[KPT][NC], cmp[KPT][NC];
#pragma unroll
  for (int k = 0; k < KPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc[k][c] = sK[(k * 2 * NC + c) * kstride];
      cmp[k][c] = sK[(k * 2 * NC + NC + c) * kstride];
    }
  __syncthreads();
  combine_groups<float, KPT, NC>(acc, cmp, reinterpret_cast<float*>(smem_raw), groups, grp, NT, lt);
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    if (grp == 0 && valid[k]) {
      if (kappa > 0) {  // the target-side far field of k_adj_far
        const float4 f = g1[jj[k]];
        kahan_add(acc[k][0], cmp[k][0], f.x);
        kahan_add(acc[k][1], cmp[k][1], f.y);
        kahan_add(acc[k][2], cmp[k][2], f.z);
      }
      g1[jj[k]] = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
      g2[jj[k]] = make_float4(acc[k][4], acc[k][5], acc[k][6], 0.f);
    }
  }
  }  // items
}

// Source side: near field over the source-major P2P list, far field from the
// pushed-down Lambda, plus the target-side part; then the chain rule to
// physical (x, p, q), written in input order (FP64, and FP32 with the gbar
// term; the FP32 adjoint otherwise uses k_adj_near and k_adj_final).
template <typename T, int KPT>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 7 : 1) k_adj_source(
    const uint64_t* __restrict__ keys, const int32_t* __restrict__ off, int shift,
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int kappa,
    const NodeGeo* __restrict__ geo, const typename Vec4<T>::type* __restrict__ px,
    const typename Vec4<T>::type* __restrict__ pb, const typename Vec4<T>::type* __restrict__ pl,
    const void* __restrict__ sdc_raw, const typename Vec4<T>::type* __restrict__ wle,
    const typename Vec4<T>::type* __restrict__ wlb, const T* __restrict__ Lam, Cheb ch, ChebD cd, int m,
    const typename Vec4<T>::type* __restrict__ gtarget, const int32_t* __restrict__ perm,
    const double* __restrict__ scal, const double* __restrict__ p, const double* __restrict__ q, int groups,
    int chunks, int gbar_term, double* __restrict__ dx_out, double* __restrict__ dp_out,
    double* __restrict__ dq_out) {
  using V4 = typename Vec4<T>::type;
  constexpr bool kSplit = std::is_same<T, float>::value;
  constexpr int kRow = kSplit ? 4 : 3;
  extern __shared__ unsigned char smem_raw[];
  V4* sp = reinterpret_cast<V4*>(smem_raw);
  const int NT = blockDim.x / groups, grp = threadIdx.x / NT, lt = threadIdx.x - grp * NT;
  T* sl = reinterpret_cast<T*>(smem_raw + stage_bytes<T>(kRow, KPT, 14, groups, NT));  // [4][m]
  const int64_t s = ((int64_t)1 << kappa) + blockIdx.x / chunks;
  const int64_t per_pass = (int64_t)KPT * NT;
  const int64_t c0 = (int64_t)(blockIdx.x % chunks) * per_pass;
  const int64_t st = nstart[s], cnt = min64(ncount[s], c0 + per_pass);
  if (c0 >= cnt) return;  // the leaf is smaller than this chunk
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const NodeGeo gs = geo[s];
  const int b = off[s], e = off[s + 1];
  const int np1 = ch.np1;
  T invh[3];
  bool deg[3];
  for (int d = 0; d < 3; ++d) {
    deg[d] = !(gs.h[d] > 0.0);
    invh[d] = deg[d] ? T(0) : (T)(1.0 / gs.h[d]);
  }
  if (kappa > 0) {
    const T* Ls = Lam + (size_t)s * 4 * m;
    for (int o = threadIdx.x; o < 4 * m; o += blockDim.x) sl[o] = Ls[o];
  }
  for (int64_t pass0 = c0; pass0 < cnt; pass0 += per_pass) {
    T rj[KPT][3], rl[KPT][3], aj[KPT], bj[KPT][3];
    bool valid[KPT];
    T acc[KPT][7], cmp[KPT][7];  // (dL/da', dL/db~' x3, dL/dx' x3)
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int64_t j = pass0 + lt + (int64_t)k * NT;
      valid[k] = j < cnt;
      const int64_t jj = st + (valid[k] ? j : 0);
      const V4 u = px[jj], w = pb[jj];
      rj[k][0] = u.x; rj[k][1] = u.y; rj[k][2] = u.z;
      aj[k] = u.w;
      bj[k][0] = w.x; bj[k][1] = w.y; bj[k][2] = w.z;
      if constexpr (kSplit) {
        const V4 l = pl[jj];
        rl[k][0] = l.x; rl[k][1] = l.y; rl[k][2] = l.z;
      } else {
        rl[k][0] = rl[k][1] = rl[k][2] = T(0);
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) acc[k][c] = cmp[k][c] = T(0);
    }
    for (int it = b; it < e; ++it) {
      const int64_t t = (int64_t)(keys[it] & mask);
      const int64_t tst = nstart[t], tcnt = ncount[t];
      T X[KPT][3], XL[KPT][3], part[KPT][7];
      // X = x_j + (c_s - c_t): the source particle in the target leaf's frame
      if constexpr (kSplit) {
        const float4* sdc = static_cast<const float4*>(sdc_raw);
        const float4 dh = sdc[2 * it], dl = sdc[2 * it + 1];
        const float dch[3] = {dh.x, dh.y, dh.z}, dcl[3] = {dl.x, dl.y, dl.z};
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float hs, he;
            two_sum(rj[k][d], dch[d], hs, he);
            const float lo = he + (rl[k][d] + dcl[d]);
            X[k][d] = hs + lo;
            XL[k][d] = lo - (X[k][d] - hs);
          }
      } else {
        const double4 dd = static_cast<const double4*>(sdc_raw)[it];
        const T dc[3] = {(T)dd.x, (T)dd.y, (T)dd.z};
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            X[k][d] = rj[k][d] + dc[d];
            XL[k][d] = T(0);
          }
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 7; ++c) part[k][c] = T(0);
      float2 pp2[7];  // paired partial sums (FP32 path): even and odd targets of the leaf
#pragma unroll
      for (int c = 0; c < 7; ++c) pp2[c] = make_float2(0.f, 0.f);
      for (int64_t base = 0; base < tcnt; base += blockDim.x) {
        __syncthreads();
        const int64_t i = base + threadIdx.x;
        if constexpr (kSplit && KPT == 1) {
          // targets staged in pairs, 8 float4 (32 floats) per pair, each of 16
          // components as (target 2q, target 2q+1): x_hi, y_hi, z_hi, x_lo,
          // y_lo, z_lo, wE^ (3), wB^ (3), -wB^ (3), 0
          float c[16];
          if (i < tcnt) {
            const float4 u = px[tst + i], l = pl[tst + i], e = wle[tst + i], w = wlb[tst + i];
            c[0] = u.x; c[1] = u.y; c[2] = u.z; c[3] = l.x; c[4] = l.y; c[5] = l.z;
            c[6] = e.x; c[7] = e.y; c[8] = e.z; c[9] = w.x; c[10] = w.y; c[11] = w.z;
            c[12] = -w.x; c[13] = -w.y; c[14] = -w.z; c[15] = 0.f;
          } else {  // partner of an odd last target: no weights, no contribution
#pragma unroll
            for (int q = 0; q < 16; ++q) c[q] = 0.f;
          }
          float* f = reinterpret_cast<float*>(sp) + (threadIdx.x >> 1) * 32 + (threadIdx.x & 1);
#pragma unroll
          for (int q = 0; q < 16; ++q) f[2 * q] = c[q];
        } else if (i < tcnt) {
          sp[kRow * threadIdx.x] = px[tst + i];
          sp[kRow * threadIdx.x + 1] = wle[tst + i];
          sp[kRow * threadIdx.x + 2] = wlb[tst + i];
          if constexpr (kSplit) sp[kRow * threadIdx.x + 3] = pl[tst + i];
        }
        __syncthreads();
        const int ni = (int)min64(blockDim.x, tcnt - base);
        if constexpr (kSplit && KPT == 1) {  // target pairs, paired arithmetic
          const int npq = (ni + 1) >> 1;
          const int share2 = (npq + groups - 1) / groups, q1 = min(npq, (grp + 1) * share2);
          const float2 nX0 = make_float2(-X[0][0], -X[0][0]), nX1 = make_float2(-X[0][1], -X[0][1]),
                       nX2 = make_float2(-X[0][2], -X[0][2]);
          const float2 nL0 = make_float2(-XL[0][0], -XL[0][0]), nL1 = make_float2(-XL[0][1], -XL[0][1]),
                       nL2 = make_float2(-XL[0][2], -XL[0][2]);
          const float2 a2 = make_float2(aj[0], aj[0]);
          const float2 b0 = make_float2(bj[0][0], bj[0][0]), b1 = make_float2(bj[0][1], bj[0][1]),
                       b2 = make_float2(bj[0][2], bj[0][2]);
          const float2 m3 = make_float2(-3.f, -3.f);
          for (int qq = grp * share2; qq < q1; ++qq) {
            const float4* s4 = reinterpret_cast<const float4*>(sp) + 8 * qq;
            const float4 P0 = s4[0], P1 = s4[1], P2 = s4[2], P3 = s4[3], P4 = s4[4], P5 = s4[5], P6 = s4[6];
            // R = x_i - x_j = (x_hi - X) + (x_lo - X_lo)
            const float2 rx = __fadd2_rn(__fadd2_rn(make_float2(P0.x, P0.y), nX0), __fadd2_rn(make_float2(P1.z, P1.w), nL0));
            const float2 ry = __fadd2_rn(__fadd2_rn(make_float2(P0.z, P0.w), nX1), __fadd2_rn(make_float2(P2.x, P2.y), nL1));
            const float2 rz = __fadd2_rn(__fadd2_rn(make_float2(P1.x, P1.y), nX2), __fadd2_rn(make_float2(P2.z, P2.w), nL2));
            const float2 d = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
            float2 inv;
            inv.x = d.x > tiny_sep2<float>() ? rsqrt_t<float>(d.x) : 0.f;
            inv.y = d.y > tiny_sep2<float>() ? rsqrt_t<float>(d.y) : 0.f;
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 r3 = __fmul2_rn(inv2, inv);
            const float2 r5 = __fmul2_rn(r3, inv2);
            const float2 kx = __fmul2_rn(r3, rx), ky = __fmul2_rn(r3, ry), kz = __fmul2_rn(r3, rz);
            const float2 ex = make_float2(P3.x, P3.y), ey = make_float2(P3.z, P3.w), ez = make_float2(P4.x, P4.y);
            const float2 wx = make_float2(P4.z, P4.w), wy = make_float2(P5.x, P5.y), wz = make_float2(P5.z, P5.w);
            const float2 nwx = make_float2(P6.x, P6.y), nwy = make_float2(P6.z, P6.w);
            const float4 P7 = s4[7];
            const float2 nwz = make_float2(P7.x, P7.y);
            // dL/da' += wE^ . K,  dL/db~' += K x wB^
            pp2[0] = __ffma2_rn(ez, kz, __ffma2_rn(ey, ky, __ffma2_rn(ex, kx, pp2[0])));
            pp2[1] = __ffma2_rn(kz, nwy, __ffma2_rn(ky, wz, pp2[1]));
            pp2[2] = __ffma2_rn(kx, nwz, __ffma2_rn(kz, wx, pp2[2]));
            pp2[3] = __ffma2_rn(ky, nwx, __ffma2_rn(kx, wy, pp2[3]));
            // u = a'_j wE^ + wB^ x b~'_j;  sum of J u = r^-3 u - 3 r^-5 R (R . u), negated at the end
            const float2 ux = __ffma2_rn(a2, ex, __ffma2_rn(nwz, b1, __fmul2_rn(wy, b2)));
            const float2 uy = __ffma2_rn(a2, ey, __ffma2_rn(nwx, b2, __fmul2_rn(wz, b0)));
            const float2 uz = __ffma2_rn(a2, ez, __ffma2_rn(nwy, b0, __fmul2_rn(wx, b1)));
            const float2 ru = __ffma2_rn(rz, uz, __ffma2_rn(ry, uy, __fmul2_rn(rx, ux)));
            const float2 nc3 = __fmul2_rn(__fmul2_rn(r5, m3), ru);
            pp2[4] = __ffma2_rn(nc3, rx, __ffma2_rn(r3, ux, pp2[4]));
            pp2[5] = __ffma2_rn(nc3, ry, __ffma2_rn(r3, uy, pp2[5]));
            pp2[6] = __ffma2_rn(nc3, rz, __ffma2_rn(r3, uz, pp2[6]));
          }
          continue;
        }
        const int share = (ni + groups - 1) / groups, i1 = min(ni, (grp + 1) * share);
        for (int ii = grp * share; ii < i1; ++ii) {
          const V4 u = sp[kRow * ii], we = sp[kRow * ii + 1], wb = sp[kRow * ii + 2];
          V4 ul;
          if constexpr (kSplit) ul = sp[kRow * ii + 3];
#pragma unroll
          for (int k = 0; k < KPT; ++k) {
            T rx, ry, rz;  // R = x_i - x_j
            if constexpr (kSplit) {
              rx = (u.x - X[k][0]) + (ul.x - XL[k][0]);
              ry = (u.y - X[k][1]) + (ul.y - XL[k][1]);
              rz = (u.z - X[k][2]) + (ul.z - XL[k][2]);
            } else {
              rx = u.x - X[k][0];
              ry = u.y - X[k][1];
              rz = u.z - X[k][2];
            }
            const T d = rx * rx + ry * ry + rz * rz;
            const T inv = d > tiny_sep2<T>() ? rsqrt_t<T>(d) : T(0);
            const T r3 = inv * inv * inv;
            const T r5 = r3 * inv * inv;
            const T kx = r3 * rx, ky = r3 * ry, kz = r3 * rz;
            part[k][0] += we.x * kx + we.y * ky + we.z * kz;
            part[k][1] += ky * wb.z - kz * wb.y;
            part[k][2] += kz * wb.x - kx * wb.z;
            part[k][3] += kx * wb.y - ky * wb.x;
            const T ux = aj[k] * we.x + (wb.y * bj[k][2] - wb.z * bj[k][1]);
            const T uy = aj[k] * we.y + (wb.z * bj[k][0] - wb.x * bj[k][2]);
            const T uz = aj[k] * we.z + (wb.x * bj[k][1] - wb.y * bj[k][0]);
            const T c3 = T(3) * r5 * (rx * ux + ry * uy + rz * uz);
            part[k][4] -= r3 * ux - c3 * rx;
            part[k][5] -= r3 * uy - c3 * ry;
            part[k][6] -= r3 * uz - c3 * rz;
          }
        }
      }
      if constexpr (kSplit && KPT == 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) part[0][c] = pp2[c].x + pp2[c].y;
#pragma unroll
        for (int c = 4; c < 7; ++c) part[0][c] = -(pp2[c].x + pp2[c].y);
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 7; ++c) kahan_add(acc[k][c], cmp[k][c], part[k][c]);
    }
    __syncthreads();
    const double gbar = scal[0], mu_u = scal[1], ell = scal[2];
    const int a3share = (np1 + groups - 1) / groups;
    const int a3b = min(np1, grp * a3share), a3e = min(np1, a3b + a3share);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (valid[k] && kappa > 0) {  // far field at the source: through the P2M basis of its leaf
        T lx[kMaxNp1], ly[kMaxNp1], lz[kMaxNp1], dx[kMaxNp1], dy[kMaxNp1], dz[kMaxNp1];
        const T lof = kSplit ? T(1) : T(0);
        basis_deriv<T>((rj[k][0] + lof * rl[k][0]) * invh[0], deg[0], ch, cd, lx, dx);
        basis_deriv<T>((rj[k][1] + lof * rl[k][1]) * invh[1], deg[1], ch, cd, ly, dy);
        basis_deriv<T>((rj[k][2] + lof * rl[k][2]) * invh[2], deg[2], ch, cd, lz, dz);
        T F[4] = {T(0), T(0), T(0), T(0)}, G[3] = {T(0), T(0), T(0)};
        int nu = a3b * np1 * np1;
        for (int a3 = a3b; a3 < a3e; ++a3) {
          for (int a2 = 0; a2 < np1; ++a2) {
            T f[4] = {T(0), T(0), T(0), T(0)};
            T s0 = T(0), sx = T(0);
            for (int a1 = 0; a1 < np1; ++a1, ++nu) {
              const T L0 = sl[nu], L1 = sl[m + nu], L2 = sl[2 * m + nu], L3 = sl[3 * m + nu];
              const T psi = L0 * aj[k] + L1 * bj[k][0] + L2 * bj[k][1] + L3 * bj[k][2];
              f[0] += lx[a1] * L0;
              f[1] += lx[a1] * L1;
              f[2] += lx[a1] * L2;
              f[3] += lx[a1] * L3;
              s0 += lx[a1] * psi;
              sx += dx[a1] * psi;
            }
            const T wyz = ly[a2] * lz[a3];
#pragma unroll
            for (int c = 0; c < 4; ++c) F[c] += wyz * f[c];
            G[0] += wyz * sx;
            G[1] += dy[a2] * lz[a3] * s0;
            G[2] += ly[a2] * dz[a3] * s0;
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) kahan_add(acc[k][c], cmp[k][c], F[c]);
#pragma unroll
        for (int d = 0; d < 3; ++d) kahan_add(acc[k][4 + d], cmp[k][4 + d], G[d] * invh[d]);
      }
    }
    combine_groups<T, KPT, 7>(acc, cmp, reinterpret_cast<T*>(smem_raw), groups, grp, NT, lt);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (grp != 0 || !valid[k]) continue;
      const int64_t pos = st + pass0 + lt + (int64_t)k * NT;
      const V4 gt = gtarget[pos];
      // internal (a', b~', x') -> physical (a, b, x)
      const double dA = (double)acc[k][0] / mu_u;
      const double dB[3] = {(double)acc[k][1] / (gbar * mu_u), (double)acc[k][2] / (gbar * mu_u),
                            (double)acc[k][3] / mu_u};
      const double dX[3] = {((double)acc[k][4] + (double)gt.x) / ell, ((double)acc[k][5] + (double)gt.y) / ell,
                            gbar * ((double)acc[k][6] + (double)gt.z) / ell};
      const int64_t i = perm[pos];
      const double p0 = p[3 * i], p1 = p[3 * i + 1], p2 = p[3 * i + 2], qi = q[i];
      const double gam = sqrt(1.0 + ((p0 * p0 + p1 * p1) + p2 * p2));
      // a = q gamma, b = q p:  dL/dq = gamma dL/da + p . dL/db,
      //                        dL/dp = q (p/gamma) dL/da + q dL/db
      dq_out[i] = gam * dA + (p0 * dB[0] + p1 * dB[1] + p2 * dB[2]);
      // with gbar(p) live: + dL/dgbar * d gbar/d p_i = scal[10] * pbar
      const double cg = gbar_term ? scal[10] : 0.0;
      dp_out[3 * i + 0] = qi * (p0 / gam) * dA + qi * dB[0] + cg * scal[6];
      dp_out[3 * i + 1] = qi * (p1 / gam) * dA + qi * dB[1] + cg * scal[7];
      dp_out[3 * i + 2] = qi * (p2 / gam) * dA + qi * dB[2] + cg * scal[8];
      dx_out[3 * i + 0] = dX[0];
      dx_out[3 * i + 1] = dX[1];
      dx_out[3 * i + 2] = dX[2];
    }
  }
}

// dL/dgbar from the per-target near-field terms (.w of the target-side
// output, leaf order) and the per-cluster far-field terms gfar[1 .. nfar],
// in two fixed-order passes: block b sums its strided share into
// gpart[b], then one block sums gpart[0 .. nb) and sets
//   scal[9]  = dL/dgbar = (sum of the terms) / gbar,
//   scal[10] = dL/dgbar / (N gbar),
// the factor of pbar in d gbar / d p_i for gbar = sqrt(1 + pbar.pbar),
// pbar = (1/N) sum_j p_j (Section 3).
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gbar_part(const typename Vec4<T>::type* __restrict__ tpart, int64_t N,
                                                   const double* __restrict__ gfar, int64_t nfar,
                                                   double* __restrict__ gpart) {
  __shared__ double red[8];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) v += (double)tpart[i].w;
  for (int64_t c = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nfar; c += stride) v += gfar[c];
  const double t = block_sum_fixed(v, red);
  if (threadIdx.x == 0) gpart[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_gbar_final(const double* __restrict__ gpart, int nb, int64_t N,
                                                    double* __restrict__ scal) {
  __shared__ double red[8];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += gpart[b];
  const double t = block_sum_fixed(v, red);
  if (threadIdx.x != 0) return;
  const double gbar = scal[0], d = t / gbar;
  scal[9] = d;
  scal[10] = d / ((double)N * gbar);
}

// FP32 adjoint after k_adj_near: the source-side far field and the chain
// rule, one thread per particle of a leaf chunk of 128.  Lambda of the leaf is
// staged with its four components side by side (one 16-byte shared load per
// point); then per particle j
//   dL/da'_j += sum_nu l_nu(x_j) Lambda^a_nu,  dL/db~'_j += sum_nu l_nu(x_j) Lambda^b_nu,
//   dL/dx'_j += sum_nu grad l_nu(x_j) psi_nu,  psi_nu = Lambda_nu . (a'_j, b~'_j),
// added to the near field of k_adj_near, and the result is taken to physical
// (x, p, q) as in k_adj_source.
constexpr int kFinalThreads = 128;

// basis_deriv with the points per axis fixed at compile time (the same
// barycentric formula and derivative matrix), so the arrays stay in registers
template <int NP1>
__device__ __forceinline__ void basis_deriv_n(float t, bool deg, const Cheb& ch, const ChebD& cd, float (&l)[NP1],
                                              float (&dl)[NP1]) {
  bary_basis_n<NP1>(t, deg, ch, l);
#pragma unroll
  for (int k = 0; k < NP1; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int mm = 0; mm < NP1; ++mm) acc += l[mm] * cd.Df[mm * NP1 + k];
    dl[k] = deg ? 0.f : acc;
  }
}

template <int NP1>  // 0: points per axis from ch at run time
__global__ void __launch_bounds__(kFinalThreads) k_adj_final(
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int kappa,
    const NodeGeo* __restrict__ geo, const float4* __restrict__ px, const float4* __restrict__ pb,
    const float4* __restrict__ pl, const float* __restrict__ Lam, Cheb ch, ChebD cd, int m, int chunks,
    const float4* __restrict__ g1, const float4* __restrict__ g2, const int32_t* __restrict__ perm,
    const double* __restrict__ scal, const double* __restrict__ p, const double* __restrict__ q,
    double* __restrict__ dx_out, double* __restrict__ dp_out, double* __restrict__ dq_out) {
  extern __shared__ float4 slam[];  // [m]
  const int64_t s = ((int64_t)1 << kappa) + blockIdx.x / chunks;
  const int64_t c0 = (int64_t)(blockIdx.x % chunks) * kFinalThreads;
  const int64_t st = nstart[s], cnt = ncount[s];
  if (c0 >= cnt) return;  // the leaf is smaller than this chunk
  const bool far = kappa > 0;
  if (far) {
    const float* Ls = Lam + (size_t)s * 4 * m;
    for (int o = threadIdx.x; o < m; o += blockDim.x) slam[o] = make_float4(Ls[o], Ls[m + o], Ls[2 * m + o], Ls[3 * m + o]);
  }
  __syncthreads();
  const int64_t j = c0 + threadIdx.x;
  if (j >= cnt) return;
  const int64_t pos = st + j;
  const float4 u = px[pos], b = pb[pos], l = pl[pos];
  float F[4] = {0.f, 0.f, 0.f, 0.f}, G[3] = {0.f, 0.f, 0.f};
  const NodeGeo gs = geo[s];
  float invh[3];
  bool deg[3];
  for (int d = 0; d < 3; ++d) {
    deg[d] = !(gs.h[d] > 0.0);
    invh[d] = deg[d] ? 0.f : (float)(1.0 / gs.h[d]);
  }
  if (far) {
    constexpr int K = NP1 > 0 ? NP1 : kMaxNp1;
    const int np1 = NP1 > 0 ? NP1 : ch.np1;
    float lx[K], ly[K], lz[K], dx[K], dy[K], dz[K];
    if constexpr (NP1 > 0) {
      basis_deriv_n<K>((u.x + l.x) * invh[0], deg[0], ch, cd, lx, dx);
      basis_deriv_n<K>((u.y + l.y) * invh[1], deg[1], ch, cd, ly, dy);
      basis_deriv_n<K>((u.z + l.z) * invh[2], deg[2], ch, cd, lz, dz);
    } else {
      basis_deriv<float>((u.x + l.x) * invh[0], deg[0], ch, cd, lx, dx);
      basis_deriv<float>((u.y + l.y) * invh[1], deg[1], ch, cd, ly, dy);
      basis_deriv<float>((u.z + l.z) * invh[2], deg[2], ch, cd, lz, dz);
    }
    int nu = 0;
    for (int a3 = 0; a3 < np1; ++a3) {
#pragma unroll
      for (int a2 = 0; a2 < (NP1 > 0 ? NP1 : np1); ++a2) {
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, s0 = 0.f, sx = 0.f;
#pragma unroll
        for (int a1 = 0; a1 < (NP1 > 0 ? NP1 : np1); ++a1, ++nu) {
          const float4 L = slam[nu];
          const float psi = L.x * u.w + L.y * b.x + L.z * b.y + L.w * b.z;
          f0 += lx[a1] * L.x;
          f1 += lx[a1] * L.y;
          f2 += lx[a1] * L.z;
          f3 += lx[a1] * L.w;
          s0 += lx[a1] * psi;
          sx += dx[a1] * psi;
        }
        const float wyz = ly[a2] * lz[a3];
        F[0] += wyz * f0;
        F[1] += wyz * f1;
        F[2] += wyz * f2;
        F[3] += wyz * f3;
        G[0] += wyz * sx;
        G[1] += dy[a2] * lz[a3] * s0;
        G[2] += ly[a2] * dz[a3] * s0;
      }
    }
  }
  const float4 h1 = g1[pos], h2 = g2[pos];
  // mu and ell are powers of two: their reciprocals (scal[11], scal[3]) are
  // exact and a product by one equals the quotient; FP64 division runs on
  // the FP64 unit at a small fraction of the FP32 rate
  const double gbar = scal[0], imu = scal[11], iell = scal[3];
  // internal (a', b~', x') -> physical (a, b, x)
  const double dA = ((double)h1.w + (double)F[0]) * imu;
  const double dB[3] = {((double)h2.x + (double)F[1]) * imu / gbar, ((double)h2.y + (double)F[2]) * imu / gbar,
                        ((double)h2.z + (double)F[3]) * imu};
  const double dX[3] = {((double)h1.x + (double)(G[0] * invh[0])) * iell,
                        ((double)h1.y + (double)(G[1] * invh[1])) * iell,
                        gbar * ((double)h1.z + (double)(G[2] * invh[2])) * iell};
  const int64_t i = perm[pos];
  const double p0 = p[3 * i], p1 = p[3 * i + 1], p2 = p[3 * i + 2], qi = q[i];
  const double gam = sqrt(1.0 + ((p0 * p0 + p1 * p1) + p2 * p2));
  const double qa = qi * dA / gam;
  // a = q gamma, b = q p:  dL/dq = gamma dL/da + p . dL/db,
  //                        dL/dp = q (p/gamma) dL/da + q dL/db
  dq_out[i] = gam * dA + (p0 * dB[0] + p1 * dB[1] + p2 * dB[2]);
  dp_out[3 * i + 0] = p0 * qa + qi * dB[0];
  dp_out[3 * i + 1] = p1 * qa + qi * dB[1];
  dp_out[3 * i + 2] = p2 * qa + qi * dB[2];
  dx_out[3 * i + 0] = dX[0];
  dx_out[3 * i + 1] = dX[1];
  dx_out[3 * i + 2] = dX[2];
}

// FP32 target-side far field of the adjoint (FP64 and the gbar term take it
// in k_adj_target): per particle i of leaf L, in internal units,
//   dL/dx'_i = sum_mu grad l_mu(x_i) (w^_i . Lc_mu),
// the L2P of Alg. 14 (Eq. 2.8) differentiated in x_i, with Lc the forward's
// cumulative local of L.  One thread per particle of a leaf chunk of 128,
// the six components of Lc staged side by side as in the forward's L2P.
// Written to g1 as (dL/dx', 0) before the near field, which adds it, so the
// far-field chain may overwrite the locals (FMM_RECOMPUTE) while the near
// field runs.
template <int NP1>  // 0: points per axis from ch at run time
__global__ void __launch_bounds__(kFinalThreads) k_adj_far(
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int kappa,
    const NodeGeo* __restrict__ geo, const float4* __restrict__ px, const float4* __restrict__ pl,
    const float4* __restrict__ wle, const float4* __restrict__ wlb, const float* __restrict__ Lcum, Cheb ch,
    ChebD cd, int m, int chunks, float4* __restrict__ g1) {
  extern __shared__ float4 slc[];  // [m][2]: (L0, L1, L2, L3), (L4, L5, 0, 0)
  const int64_t t = ((int64_t)1 << kappa) + blockIdx.x / chunks;
  const int64_t c0 = (int64_t)(blockIdx.x % chunks) * kFinalThreads;
  const int64_t st = nstart[t], cnt = ncount[t];
  if (c0 >= cnt) return;  // the leaf is smaller than this chunk
  const float* Lt = Lcum + (size_t)t * 6 * m;
  for (int o = threadIdx.x; o < m; o += blockDim.x) {
    slc[2 * o] = make_float4(Lt[o], Lt[m + o], Lt[2 * m + o], Lt[3 * m + o]);
    slc[2 * o + 1] = make_float4(Lt[4 * m + o], Lt[5 * m + o], 0.f, 0.f);
  }
  __syncthreads();
  const int64_t j = c0 + threadIdx.x;
  if (j >= cnt) return;
  const int64_t pos = st + j;
  const float4 u = px[pos], l = pl[pos], e = wle[pos], w = wlb[pos];
  const NodeGeo g = geo[t];
  float invh[3];
  bool deg[3];
  for (int d = 0; d < 3; ++d) {
    deg[d] = !(g.h[d] > 0.0);
    invh[d] = deg[d] ? 0.f : (float)(1.0 / g.h[d]);
  }
  constexpr int K = NP1 > 0 ? NP1 : kMaxNp1;
  const int np1 = NP1 > 0 ? NP1 : ch.np1;
  float lx[K], ly[K], lz[K], dx[K], dy[K], dz[K];
  if constexpr (NP1 > 0) {
    basis_deriv_n<K>((u.x + l.x) * invh[0], deg[0], ch, cd, lx, dx);
    basis_deriv_n<K>((u.y + l.y) * invh[1], deg[1], ch, cd, ly, dy);
    basis_deriv_n<K>((u.z + l.z) * invh[2], deg[2], ch, cd, lz, dz);
  } else {
    basis_deriv<float>((u.x + l.x) * invh[0], deg[0], ch, cd, lx, dx);
    basis_deriv<float>((u.y + l.y) * invh[1], deg[1], ch, cd, ly, dy);
    basis_deriv<float>((u.z + l.z) * invh[2], deg[2], ch, cd, lz, dz);
  }
  float G[3] = {0.f, 0.f, 0.f};
  int mu = 0;
  for (int a3 = 0; a3 < np1; ++a3) {
#pragma unroll
    for (int a2 = 0; a2 < (NP1 > 0 ? NP1 : np1); ++a2) {
      float s0 = 0.f, sx = 0.f;
#pragma unroll
      for (int a1 = 0; a1 < (NP1 > 0 ? NP1 : np1); ++a1, ++mu) {
        const float4 A = slc[2 * mu], Bv = slc[2 * mu + 1];
        const float phi = e.x * A.x + e.y * A.y + e.z * A.z + w.x * A.w + w.y * Bv.x + w.z * Bv.y;
        s0 += lx[a1] * phi;
        sx += dx[a1] * phi;
      }
      G[0] += ly[a2] * lz[a3] * sx;
      G[1] += dy[a2] * lz[a3] * s0;
      G[2] += ly[a2] * dz[a3] * s0;
    }
  }
  g1[pos] = make_float4(G[0] * invh[0], G[1] * invh[1], G[2] * invh[2], 0.f);
}

// ---------------------------------------------------------------- launchers
// Raise the kernel's dynamic shared-memory limit to what this launch needs.
template <typename K>
int set_smem(K* kernel, size_t smem) {
  return smem_limit(kernel, (int)smem);
}

template <typename T, int NV>
int launch_l2pt(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  const size_t smem = (size_t)256 * (((3 * P->np1 + 3) & ~3) + 8) * sizeof(T);
  if (int rc = set_smem(k_l2pt<T, NV>, smem)) return rc;
  using V4 = typename Vec4<T>::type;
  k_l2pt<T, NV><<<(unsigned)P->nleaves, 256, smem, s>>>(ws_ptr<V4>(P, L.px), ws_ptr<V4>(P, L.pl), ws_ptr<V4>(P, L.wle),
                                                        ws_ptr<V4>(P, L.wlb), ws_ptr<int64_t>(P, L.nstart),
                                                        ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo),
                                                        P->cheb, P->m, ws_ptr<T>(P, L.wbuf));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T>
int l2pt(fmm_plan_s* P, cudaStream_t s) {
  switch (div_up(P->m, 256)) {
    case 1: return launch_l2pt<T, 1>(P, s);
    case 2: return launch_l2pt<T, 2>(P, s);
    case 3: return launch_l2pt<T, 3>(P, s);
    case 4: return launch_l2pt<T, 4>(P, s);
    case 5: return launch_l2pt<T, 5>(P, s);
    case 6: return launch_l2pt<T, 6>(P, s);
    case 7: return launch_l2pt<T, 7>(P, s);
    case 8: return launch_l2pt<T, 8>(P, s);
    default: return launch_l2pt<T, 9>(P, s);
  }
}

template <typename T, int KPT, bool GB>
int launch_adj_m2l(fmm_plan_s* P, int nt, cudaStream_t s) {
  const Layout& L = P->lay;
  const size_t smem = (size_t)3 * P->m * sizeof(typename Vec4<T>::type);
  if (int rc = set_smem(k_adj_m2l<T, KPT, GB>, smem)) return rc;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_adj_m2l<T, KPT, GB>, nt, smem, P->C, &grid)) return rc;
  k_adj_m2l<T, KPT, GB><<<grid, nt, smem, s>>>(
      ws_ptr<uint64_t>(P, L.m2l_src), ws_ptr<int32_t>(P, L.m2l_soff), P->kappa + 1, ws_ptr<int32_t>(P, L.m2l_sorder),
      P->C, ws_ptr<NodeGeo>(P, L.ngeo), P->ws + L.m2l_sdc, P->cheb, P->m, ws_ptr<T>(P, L.wbuf), ws_ptr<T>(P, L.lbuf),
      ws_ptr<T>(P, L.mpole), ws_ptr<double>(P, L.gfar));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T, bool GB>
int adj_m2l_generic(fmm_plan_s* P, cudaStream_t s) {
  // the same thread shape rule as the forward M2L
  int best_nt = 256, best_k = 4;
  int64_t best_waste = -1, best_passes = 0;
  for (int k = 1; k <= 4; ++k) {
    int t = (int)(div_up(div_up(P->m, k), 32) * 32);
    if (t > 256) t = 256;
    const int64_t passes = div_up(P->m, (int64_t)t * k);
    const int64_t waste = passes * t * k - P->m;
    if (best_waste < 0 || waste < best_waste || (waste == best_waste && passes < best_passes)) {
      best_waste = waste;
      best_passes = passes;
      best_nt = t;
      best_k = k;
    }
  }
  switch (best_k) {
    case 1: return launch_adj_m2l<T, 1, GB>(P, best_nt, s);
    case 2: return launch_adj_m2l<T, 2, GB>(P, best_nt, s);
    case 3: return launch_adj_m2l<T, 3, GB>(P, best_nt, s);
    default: return launch_adj_m2l<T, 4, GB>(P, best_nt, s);
  }
}

// With the gbar term the generic kernel runs (it also forms the far-field
// part of dL/dgbar); otherwise FP32 at eta <= 1/2 takes the specialised one.
template <typename T>
int adj_m2l(fmm_plan_s* P, bool gbar_term, cudaStream_t s) {
  if (gbar_term) return adj_m2l_generic<T, true>(P, s);
  if (std::is_same<T, float>::value && P->eta <= 0.5) {
    switch (P->np1) {
      case 3: return launch_adj_m2l_fast<3, 3, 1>(P, s);
      // paired kernels, the block sizes of the forward M2L
      case 5: return launch_adj_m2l_pair<5, 64>(P, s);
      case 7: return launch_adj_m2l_pair<7, 64>(P, s);
      case 9: return launch_adj_m2l_pair<9, 128>(P, s);
      case 11: return launch_adj_m2l_pair<11, 128>(P, s);
      default: break;
    }
  }
  return adj_m2l_generic<T, false>(P, s);
}

template <typename T, bool GB>
int launch_adj_target(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  using V4 = typename Vec4<T>::type;
  constexpr bool kSplit = std::is_same<T, float>::value;
  int NT, groups, chunks;
  particle_shape(P->leaf, 1, &NT, &groups, &chunks);  // as the forward P2P
  const int nt = groups * NT;
  const int64_t items = P->nleaves * chunks;
  unsigned grid = (unsigned)items;
  const size_t smem = stage_bytes<T>(kSplit ? 4 : 2, 1, GB ? 8 : 6, groups, NT) + sizeof(T) * 6 * P->m;
  if (int rc = set_smem(k_adj_target<T, 1, GB>, smem)) return rc;
  // beside the source side's far field (side stream) the target side keeps
  // to half of the SMs' block slots, so the other branch finds room; alone
  // it takes every resident slot
  if (P->kappa > 0 && P->adj_overlap) {
    int sms = 0;
    if (int rc = device_sms(&sms)) return rc;
    grid = (unsigned)std::min<int64_t>(items, (int64_t)4 * sms);  // 3-4 measured best at 2^9 leaves
  } else if (int rc = resident_blocks(k_adj_target<T, 1, GB>, nt, smem, items, &grid)) {
    return rc;
  }
  k_adj_target<T, 1, GB><<<grid, nt, smem, s>>>(
      ws_ptr<uint64_t>(P, L.p2p), ws_ptr<int32_t>(P, L.p2p_off), P->kappa + 1, ws_ptr<int64_t>(P, L.nstart),
      ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo), ws_ptr<V4>(P, L.px), ws_ptr<V4>(P, L.pb),
      ws_ptr<V4>(P, L.pl), P->ws + L.p2p_dc, ws_ptr<V4>(P, L.wle), ws_ptr<V4>(P, L.wlb), ws_ptr<T>(P, L.local),
      P->cheb, P->chebd, P->m, groups, chunks, items, ws_ptr<V4>(P, L.adj_part));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// FP32 before the near field: the target-side far field (k_adj_far) into g1.
int launch_adj_far(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  const int64_t most = *std::max_element(P->node_count.begin() + P->nleaves, P->node_count.end());
  const int chunks = (int)div_up(most, kFinalThreads);
  const size_t smem = sizeof(float4) * 2 * P->m;
  auto kern = k_adj_far<0>;
  switch (P->np1) {
    case 3: kern = k_adj_far<3>; break;
    case 5: kern = k_adj_far<5>; break;
    case 7: kern = k_adj_far<7>; break;
    case 9: kern = k_adj_far<9>; break;
    case 11: kern = k_adj_far<11>; break;
    default: break;
  }
  if (int rc = smem_limit(kern, (int)smem)) return rc;
  kern<<<(unsigned)(P->nleaves * chunks), kFinalThreads, smem, s>>>(
      ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.px), ws_ptr<float4>(P, L.pl), ws_ptr<float4>(P, L.wle), ws_ptr<float4>(P, L.wlb),
      ws_ptr<float>(P, L.local), P->cheb, P->chebd, P->m, chunks, ws_ptr<float4>(P, L.adj_part));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// FP32 after k_adj_near: source-side far field and chain rule.
int launch_adj_final(fmm_plan_s* P, const double* p, const double* q, double* dx, double* dp, double* dq,
                     cudaStream_t s) {
  const Layout& L = P->lay;
  const int64_t most = *std::max_element(P->node_count.begin() + P->nleaves, P->node_count.end());
  const int chunks = (int)div_up(most, kFinalThreads);
  const size_t smem = sizeof(float4) * P->m;
  auto kern = k_adj_final<0>;
  switch (P->np1) {
    case 3: kern = k_adj_final<3>; break;
    case 5: kern = k_adj_final<5>; break;
    case 7: kern = k_adj_final<7>; break;
    case 9: kern = k_adj_final<9>; break;
    case 11: kern = k_adj_final<11>; break;
    default: break;
  }
  if (int rc = smem_limit(kern, (int)smem)) return rc;
  kern<<<(unsigned)(P->nleaves * chunks), kFinalThreads, smem, s>>>(
      ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.px), ws_ptr<float4>(P, L.pb), ws_ptr<float4>(P, L.pl), ws_ptr<float>(P, L.lbuf), P->cheb,
      P->chebd, P->m, chunks, ws_ptr<float4>(P, L.adj_part), ws_ptr<float4>(P, L.adj_part2),
      ws_ptr<int32_t>(P, L.perm), ws_ptr<double>(P, L.scal), p, q, dx, dp, dq);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T>
int adj_source(fmm_plan_s* P, const double* p, const double* q, double* dx, double* dp, double* dq, bool gbar_term,
               bool fused, cudaStream_t s) {
  if (fused) return launch_adj_final(P, p, q, dx, dp, dq, s);
  const Layout& L = P->lay;
  using V4 = typename Vec4<T>::type;
  constexpr bool kSplit = std::is_same<T, float>::value;
  int NT, groups, chunks;
  particle_shape(P->leaf, 1, &NT, &groups, &chunks);  // as the forward P2P
  const int nt = groups * NT;
  const unsigned grid = (unsigned)(P->nleaves * chunks);
  const size_t smem = stage_bytes<T>(kSplit ? 4 : 3, 1, 14, groups, NT) + sizeof(T) * 4 * P->m;
  if (int rc = set_smem(k_adj_source<T, 1>, smem)) return rc;
  k_adj_source<T, 1><<<grid, nt, smem, s>>>(
      ws_ptr<uint64_t>(P, L.p2p_src), ws_ptr<int32_t>(P, L.p2p_soff), P->kappa + 1, ws_ptr<int64_t>(P, L.nstart),
      ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo), ws_ptr<V4>(P, L.px), ws_ptr<V4>(P, L.pb),
      ws_ptr<V4>(P, L.pl), P->ws + L.p2p_sdc, ws_ptr<V4>(P, L.wle), ws_ptr<V4>(P, L.wlb), ws_ptr<T>(P, L.lbuf),
      P->cheb, P->chebd, P->m, ws_ptr<V4>(P, L.adj_part), ws_ptr<int32_t>(P, L.perm), ws_ptr<double>(P, L.scal), p,
      q, groups, chunks, gbar_term ? 1 : 0, dx, dp, dq);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// FP32 near field of both roles (k_adj_near), on the caller's stream beside
// the source side's far field; like the target side it keeps to part of the
// SMs' block slots.
template <int KPT>
int launch_adj_near_k(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  int NT, groups, chunks;
  particle_shape(P->leaf, KPT, &NT, &groups, &chunks);  // as the forward P2P
  const int nt = groups * NT;
  const int64_t items = P->nleaves * chunks;
  unsigned grid = (unsigned)items;
  const size_t smem = stage_bytes<float>(7, KPT, 14, groups, NT)  // 7 float4 per thread: half a 52-float pair
                      + sizeof(float) * KPT * 14 * nt;            // running sums and compensations
  if (int rc = set_smem(k_adj_near<KPT>, smem)) return rc;
  if (P->kappa > 0 && P->adj_overlap) {  // 3 per SM measured best at 2^9 leaves (4: +0.4%, one per item: +2%, 5: +4%)
    int sms = 0;
    if (int rc = device_sms(&sms)) return rc;
    grid = (unsigned)std::min<int64_t>(items, (int64_t)3 * sms);
  } else if (int rc = resident_blocks(k_adj_near<KPT>, nt, smem, items, &grid)) {  // alone: every resident slot
    return rc;
  }
  k_adj_near<KPT><<<grid, nt, smem, s>>>(
      ws_ptr<uint64_t>(P, L.p2p), ws_ptr<int32_t>(P, L.p2p_off), ws_ptr<uint64_t>(P, L.p2p_src),
      ws_ptr<int32_t>(P, L.p2p_soff), P->kappa + 1, ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount),
      P->kappa, ws_ptr<float4>(P, L.px), ws_ptr<float4>(P, L.pb), ws_ptr<float4>(P, L.pl),
      ws_ptr<float4>(P, L.p2p_dc), ws_ptr<float4>(P, L.p2p_sdc), ws_ptr<float4>(P, L.wle), ws_ptr<float4>(P, L.wlb),
      groups, chunks, items, ws_ptr<float4>(P, L.adj_part), ws_ptr<float4>(P, L.adj_part2));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// Two targets per thread on leaves of 256 or more, as the forward P2P: each
// staged partner pair feeds two independent chains (2^24 core-halo beam,
// N0 = 256: alone 1124 -> 1079 ms; at N0 = 128 the 2^16 cylinder is slower).
int launch_adj_near(fmm_plan_s* P, cudaStream_t s) {
  return P->leaf >= 256 ? launch_adj_near_k<2>(P, s) : launch_adj_near_k<1>(P, s);
}

// dL/dgbar into scal[9], scal[10] (after the target side and M2L^T).
template <typename T>
int gbar_sum(fmm_plan_s* P, bool far, cudaStream_t s) {
  const Layout& L = P->lay;
  using V4 = typename Vec4<T>::type;
  const int64_t nfar = far ? P->C : 0;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kGbarBlocks, div_up(std::max(P->N, nfar), 256 * 8)));
  k_gbar_part<T><<<nb, 256, 0, s>>>(ws_ptr<V4>(P, L.adj_part), P->N, ws_ptr<double>(P, L.gfar), nfar,
                                    ws_ptr<double>(P, L.gpart));
  FMM_LAUNCH_CHECK();
  k_gbar_final<<<1, 256, 0, s>>>(ws_ptr<double>(P, L.gpart), nb, P->N, ws_ptr<double>(P, L.scal));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int record(fmm_plan_s* P, int k, cudaStream_t s) { return record_stage(P, k, s); }

template <typename T>
int adjoint_t(fmm_plan_s* P, const double* x, const double* p, const double* q, const void* wE, const void* wB,
              double* dx, double* dp, double* dq, cudaStream_t s) {
  const Layout& L = P->lay;
  using V4 = typename Vec4<T>::type;
  int rc;
  if ((rc = record(P, 15, s)) != FMM_OK) return rc;
  if (!P->transposed_valid) {
    if ((rc = run_list_transpose(P, s)) != FMM_OK) return rc;
    if ((P->flags & FMM_BOUNDS_CHECK) && (rc = run_bounds_check(P, true, s)) != FMM_OK) return rc;
    P->transposed_valid = true;
  }
  // the forward's multipoles and locals again, where an FMM_RECOMPUTE
  // adjoint has overwritten them (W over L, Lambda over M)
  if (!P->locals_valid) {
    if ((rc = run_upward(P, s)) != FMM_OK) return rc;
    if ((rc = run_m2l(P, s)) != FMM_OK) return rc;
    if ((rc = run_l2l(P, s)) != FMM_OK) return rc;
    P->locals_valid = true;
  }
  const int gs = (int)std::min<int64_t>(8192, div_up(P->N, 256));
  k_adj_prep<T><<<gs, 256, 0, s>>>(static_cast<const T*>(wE), static_cast<const T*>(wB), P->N,
                                    ws_ptr<int32_t>(P, L.perm), ws_ptr<double>(P, L.scal), ws_ptr<V4>(P, L.wle),
                                    ws_ptr<V4>(P, L.wlb));
  FMM_LAUNCH_CHECK();
  // Two independent branches from here: the far field of the source side
  // (L2P^T, L2L^T, M2L^T, M2M^T, mostly latency-bound transfers) on the
  // plan's side stream, the near-field particle kernel (ALU-bound) on the
  // caller's stream.  They share no buffer that either writes, and only
  // the target-side far field reads the forward's leaf locals: in FP32
  // without the gbar term k_adj_far takes it before the branches, so
  // FMM_RECOMPUTE may write W over the locals beside the near field; where
  // the near-field kernel itself reads them (k_adj_target) FMM_RECOMPUTE
  // runs it first and the chain after it, on the caller's stream.  With
  // FMM_SERIAL the chain runs first on the caller's stream.
  const bool chain = P->kappa > 0;
  const bool gb = (P->flags & FMM_GBAR_TERM) != 0;
  const bool rec = (P->flags & FMM_RECOMPUTE) != 0;
  const bool fused = std::is_same<T, float>::value && !gb;  // FP32 without the gbar term: both roles in one kernel
  const bool near_first = rec && !fused;
  const bool ov = chain && P->overlap && !near_first;
  P->adj_overlap = ov;
  if (fused && chain && (rc = launch_adj_far(P, s)) != FMM_OK) return rc;
  if ((rc = record(P, 16, s)) != FMM_OK) return rc;
  auto near = [&]() -> int {
    int r;
    if (fused) r = launch_adj_near(P, s);
    else if constexpr (std::is_same<T, float>::value) r = launch_adj_target<T, true>(P, s);  // FP32: only with the gbar term
    else r = gb ? launch_adj_target<T, true>(P, s) : launch_adj_target<T, false>(P, s);
    if (r != FMM_OK) return r;
    return record(P, 10, s);
  };
  if (near_first && (rc = near()) != FMM_OK) return rc;
  if (chain) {
    cudaStream_t t = s;
    if (ov) {
      if ((rc = ensure_side(P)) != FMM_OK) return rc;
      t = P->side;
      FMM_CUDA_TRY(cudaEventRecord(P->fork_ev, s));
      FMM_CUDA_TRY(cudaStreamWaitEvent(t, P->fork_ev, 0));
    }
    // beside the particle kernel the transfers are launched once per level: a
    // cooperative launch would wait for the particle kernel to end
    const int cap = ov ? kLevelTransferCap : kCoopTransferCap;
    if ((rc = l2pt<T>(P, t)) != FMM_OK) return rc;
    if ((rc = run_transfer<T, 6, true>(P, ws_ptr<T>(P, L.wbuf), t, cap, ov)) != FMM_OK) return rc;  // L2L^T
    if ((rc = record(P, 11, t)) != FMM_OK) return rc;
    if ((rc = adj_m2l<T>(P, gb, t)) != FMM_OK) return rc;
    if ((rc = record(P, 12, t)) != FMM_OK) return rc;
    if ((rc = run_transfer<T, 4, false>(P, ws_ptr<T>(P, L.lbuf), t, cap, ov)) != FMM_OK) return rc;  // M2M^T
    if ((rc = record(P, 13, t)) != FMM_OK) return rc;
    if (ov) FMM_CUDA_TRY(cudaEventRecord(P->join_ev, t));
    if (rec) P->locals_valid = false;  // W and Lambda now hold what L and M held
  }
  if (!near_first && (rc = near()) != FMM_OK) return rc;
  if (ov) FMM_CUDA_TRY(cudaStreamWaitEvent(s, P->join_ev, 0));
  if (gb && (rc = gbar_sum<T>(P, chain, s)) != FMM_OK) return rc;
  if ((rc = adj_source<T>(P, p, q, dx, dp, dq, gb, fused, s)) != FMM_OK) return rc;
  if ((rc = record(P, 14, s)) != FMM_OK) return rc;
  (void)x;
  P->adj_timed = (P->flags & FMM_TIMING) != 0;
  P->adj_chain = chain;
  P->adj_order = ov ? 0 : (near_first ? 2 : 1);
  return FMM_OK;
}

}  // namespace

int run_adjoint(fmm_plan_s* P, const double* x, const double* p, const double* q, const void* wE, const void* wB,
                double* dx, double* dp, double* dq, cudaStream_t s) {
  return P->precision == FMM_FP32 ? adjoint_t<float>(P, x, p, q, wE, wB, dx, dp, dq, s)
                                  : adjoint_t<double>(P, x, p, q, wE, wB, dx, dp, dq, s);
}

}  // namespace fmm
