// P2P (Alg. 10) fused with L2P (Alg. 14) and the output transform.
//
// A block takes a chunk of KPT NT targets of one leaf and drains the leaf's
// P2P list (sorted by target, so each particle's fields are written by
// exactly one thread; Section 10).  Chunks of a few dozen targets give some
// thousand blocks even for ~500 leaves, which keeps every SM busy to the
// end.  The block is `groups` groups of NT threads; in every group a thread
// owns KPT target particles.  Source leaves are contiguous slot ranges of the
// leaf-ordered particle arrays, staged through shared memory a block-width
// at a time; each group takes its own share of every staged batch (and of
// the far-field sum), and group 0 adds the other groups' compensated sums in
// group order, so the result does not depend on scheduling.  A pair whose squared stretched, scaled
// separation is at or below tiny_sep2 (the particle itself, or two particles
// at the same position, which the leaf-relative coordinates may place a few
// units of the last place apart) contributes nothing.  Per-source-leaf partial sums are added with Kahan compensation.
//
// Separations in FP32: positions are stored relative to their leaf's centre
// as unevaluated sums hi + lo of two floats, and the centre offset c_t - c_s
// of every pair likewise, so R = (X_hi - x_hi) + (X_lo - x_lo) with
// X = x_i + (c_t - c_s) keeps the relative precision of R itself even for
// two particles much closer to each other than to their leaf centres.
// (With single floats the absolute position error, ~2^-24 of the leaf size,
// dominates the field of such close pairs.)
//
// Separations in FP64: positions are absolute physical coordinates and R is
// x_i - x_j with the stretch applied inside D, exactly as Eq. 3.2 is written
// (exact for close pairs); the summed near field is then converted to the
// stretched, scaled convention of the far field.
//
// Afterwards each thread adds the far field of its particles from the
// leaf's cumulative local field (Eq. 2.8), converts from stretched, scaled
// units to SI (E_z / gbar, B_z * gbar, prefactors 1/(4 pi eps0) and 1/c0) and
// writes the row of the particle's input index.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int kP2PPairLeaf = 256;  // near-field P2P with two targets per thread from this leaf size

template <typename T, int KPT, bool POLY>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (KPT == 1 ? 8 : 5) : 1) k_p2p_l2p(
    const uint64_t* __restrict__ keys, const int32_t* __restrict__ off, int shift, const unsigned int* __restrict__ err,
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int kappa,
    const NodeGeo* __restrict__ geo, const typename Vec4<T>::type* __restrict__ px,
    const typename Vec4<T>::type* __restrict__ pb, const float4* __restrict__ pl,  // Vec4<T> rows
    const void* __restrict__ pdc_raw, const T* __restrict__ Lcum, Cheb ch, int m,
    const int32_t* __restrict__ perm, const double* __restrict__ scal, int groups, int chunks, T* __restrict__ Eout,
    T* __restrict__ Bout, float4* __restrict__ near_out, float4* __restrict__ near_out2) {
  using V4 = typename Vec4<T>::type;
  constexpr bool kSplit = std::is_same<T, float>::value;  // hi + lo separations
  constexpr int kRow = kSplit ? 4 : 2;                      // V4 per staged source particle
  // FP32: sources are staged in pairs, 7 float4 (28 floats) per pair, each of
  // 14 components as (source 2q, source 2q+1): -x_hi, -y_hi, -z_hi, a, b~x,
  // b~y, b~z, -b~x, -b~y, -b~z, -x_lo, -y_lo, -z_lo, 0.  A thread evaluates
  // both sources of a pair at once with paired FP32 arithmetic (__fadd2_rn,
  // __fmul2_rn, __ffma2_rn: two lanes per instruction).
  extern __shared__ unsigned char smem_raw[];
  V4* sp = reinterpret_cast<V4*>(smem_raw);                                // [blockDim][kRow]
  if (*err) return;  // the traversal failed: the lists are incomplete
  const size_t stage = max(sizeof(V4) * kRow * blockDim.x,
                           sizeof(T) * (size_t)(groups - 1) * KPT * 12 * (blockDim.x / groups));
  T* sl = reinterpret_cast<T*>(smem_raw + stage);  // [6][m]
  const int64_t t = ((int64_t)1 << kappa) + blockIdx.x / chunks;
  const int NT = blockDim.x / groups, grp = threadIdx.x / NT, lt = threadIdx.x - grp * NT;
  const int64_t per_pass = (int64_t)KPT * NT;
  const int64_t c0 = (int64_t)(blockIdx.x % chunks) * per_pass;
  const int64_t st = nstart[t], cnt = min64(ncount[t], c0 + per_pass);
  if (c0 >= cnt) return;  // the leaf is smaller than this chunk
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const NodeGeo gt = geo[t];
  const int b = off[t], e = off[t + 1];
  const int np1 = ch.np1;
  const double gbar = scal[0], kE = scal[4], kB = scal[5];
  T invh[3];
  bool deg[3];
  for (int d = 0; d < 3; ++d) {
    deg[d] = !(gt.h[d] > 0.0);
    invh[d] = deg[d] ? T(0) : (T)(1.0 / gt.h[d]);
  }
  // near_out (FP32): near field only, written per particle in leaf order as
  // (E'x, E'y, E'z, B'x) and (B'y, B'z, 0, 0) in near_out2; L2P and the
  // output follow in k_l2p_far
  const bool far = kappa > 0 && near_out == nullptr;
  if (far) {  // the leaf's cumulative local field, for L2P below
    const T* Lt = Lcum + (size_t)t * 6 * m;
    for (int o = threadIdx.x; o < 6 * m; o += blockDim.x) sl[o] = Lt[o];
  }
  const double ell2 = scal[2] * scal[2];
  const T g2 = (T)(gbar * gbar);
  for (int64_t pass0 = c0; pass0 < cnt; pass0 += per_pass) {
    T ri[KPT][3], rl[KPT][3];
    bool valid[KPT];
    T acc[KPT][6], cmp[KPT][6];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int64_t j = pass0 + lt + (int64_t)k * NT;
      valid[k] = j < cnt;
      const int64_t jj = st + (valid[k] ? j : 0);
      const V4 u = px[jj];
      ri[k][0] = u.x; ri[k][1] = u.y; ri[k][2] = u.z;
      // FP32: low parts of the leaf-relative position; FP64: absolute physical position
      const V4 l = reinterpret_cast<const V4*>(pl)[jj];
      rl[k][0] = l.x; rl[k][1] = l.y; rl[k][2] = l.z;
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[k][c] = cmp[k][c] = T(0);
    }
    for (int it = b; it < e; ++it) {
      const int64_t s = (int64_t)(keys[it] & mask);
      const int64_t sst = nstart[s], scnt = ncount[s];
      T X[KPT][3], XL[KPT][3], part[KPT][6];
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
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            X[k][d] = rl[k][d];
            XL[k][d] = T(0);
          }
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) part[k][c] = T(0);
      float2 pp2[KPT][6];  // paired partial sums (FP32 path): even and odd sources of the leaf
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) pp2[k][c] = make_float2(0.f, 0.f);
      for (int64_t base = 0; base < scnt; base += blockDim.x) {
        __syncthreads();
        const int64_t j = base + threadIdx.x;
        if constexpr (kSplit) {
          float c[14];
          if (j < scnt) {
            const float4 u = px[sst + j], w = pb[sst + j], l = pl[sst + j];
            c[0] = -u.x; c[1] = -u.y; c[2] = -u.z; c[3] = u.w;
            c[4] = w.x; c[5] = w.y; c[6] = w.z; c[7] = -w.x; c[8] = -w.y; c[9] = -w.z;
            c[10] = -l.x; c[11] = -l.y; c[12] = -l.z; c[13] = 0.f;
          } else {  // partner of an odd last source: no mass, no field
#pragma unroll
            for (int q = 0; q < 14; ++q) c[q] = 0.f;
          }
          float* f = reinterpret_cast<float*>(sp) + (threadIdx.x >> 1) * 28 + (threadIdx.x & 1);
#pragma unroll
          for (int q = 0; q < 14; ++q) f[2 * q] = c[q];
        }
        if (j < scnt) {
          if constexpr (!kSplit) {  // absolute physical position with a', and b' = (b~x gbar, b~y gbar, b~z)
            const V4 a = reinterpret_cast<const V4*>(pl)[sst + j], u = px[sst + j], w = pb[sst + j];
            V4 r0, r1;
            r0.x = a.x; r0.y = a.y; r0.z = a.z; r0.w = u.w;
            r1.x = w.x * (T)gbar; r1.y = w.y * (T)gbar; r1.z = w.z; r1.w = T(0);
            sp[kRow * threadIdx.x] = r0;
            sp[kRow * threadIdx.x + 1] = r1;
          }
        }
        __syncthreads();
        const int nj = (int)min64(blockDim.x, scnt - base);
        if constexpr (kSplit) {  // source pairs, paired arithmetic, KPT targets per thread
          const int npq = (nj + 1) >> 1;
          const int share2 = (npq + groups - 1) / groups, q1 = min(npq, (grp + 1) * share2);
          float2 X0[KPT], X1[KPT], X2[KPT], L0[KPT], L1[KPT], L2[KPT];
#pragma unroll
          for (int k = 0; k < KPT; ++k) {
            X0[k] = make_float2(X[k][0], X[k][0]);
            X1[k] = make_float2(X[k][1], X[k][1]);
            X2[k] = make_float2(X[k][2], X[k][2]);
            L0[k] = make_float2(XL[k][0], XL[k][0]);
            L1[k] = make_float2(XL[k][1], XL[k][1]);
            L2[k] = make_float2(XL[k][2], XL[k][2]);
          }
          for (int q = grp * share2; q < q1; ++q) {
            const float4* s4 = reinterpret_cast<const float4*>(sp) + 7 * q;
            const float4 A = s4[0], Bq = s4[1], Cq = s4[2], Dq = s4[3], Eq = s4[4], Fq = s4[5], Gq = s4[6];
#pragma unroll
            for (int k = 0; k < KPT; ++k) {
              const float2 rx = __fadd2_rn(__fadd2_rn(X0[k], make_float2(A.x, A.y)), __fadd2_rn(L0[k], make_float2(Fq.x, Fq.y)));
              const float2 ry = __fadd2_rn(__fadd2_rn(X1[k], make_float2(A.z, A.w)), __fadd2_rn(L1[k], make_float2(Fq.z, Fq.w)));
              const float2 rz = __fadd2_rn(__fadd2_rn(X2[k], make_float2(Bq.x, Bq.y)), __fadd2_rn(L2[k], make_float2(Gq.x, Gq.y)));
              const float2 d = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
              float2 inv;
              inv.x = d.x > tiny_sep2<float>() ? rsqrt_t<float>(d.x) : 0.f;
              inv.y = d.y > tiny_sep2<float>() ? rsqrt_t<float>(d.y) : 0.f;
              // K = R / |R|^3; E += a K, B += b~ x K (12 operations per source pair)
              const float2 r3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
              const float2 kx = __fmul2_rn(r3, rx), ky = __fmul2_rn(r3, ry), kz = __fmul2_rn(r3, rz);
              const float2 aa = make_float2(Bq.z, Bq.w);
              pp2[k][0] = __ffma2_rn(aa, kx, pp2[k][0]);
              pp2[k][1] = __ffma2_rn(aa, ky, pp2[k][1]);
              pp2[k][2] = __ffma2_rn(aa, kz, pp2[k][2]);
              pp2[k][3] = __ffma2_rn(make_float2(Eq.z, Eq.w), ky, __ffma2_rn(make_float2(Cq.z, Cq.w), kz, pp2[k][3]));
              pp2[k][4] = __ffma2_rn(make_float2(Dq.z, Dq.w), kz, __ffma2_rn(make_float2(Dq.x, Dq.y), kx, pp2[k][4]));
              pp2[k][5] = __ffma2_rn(make_float2(Eq.x, Eq.y), kx, __ffma2_rn(make_float2(Cq.x, Cq.y), ky, pp2[k][5]));
            }
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
            T rx, ry, rz, d, inv;
            if constexpr (kSplit) {
              rx = (X[k][0] - u.x) + (XL[k][0] - ul.x);
              ry = (X[k][1] - u.y) + (XL[k][1] - ul.y);
              rz = (X[k][2] - u.z) + (XL[k][2] - ul.z);
              d = rx * rx + ry * ry + rz * rz;
              inv = d > tiny_sep2<T>() ? rsqrt_t<T>(d) : T(0);
            } else {  // Eq. 3.2 as written, in physical coordinates
              rx = X[k][0] - u.x;
              ry = X[k][1] - u.y;
              rz = X[k][2] - u.z;
              d = rx * rx + ry * ry + g2 * (rz * rz);
              inv = d > T(0) ? rsqrt_t<T>(d) : T(0);
            }
            T r3;
            if constexpr (POLY) r3 = T(1) + d;  // the polynomial test kernel R (1 + D), FP64 only
            else r3 = inv * inv * inv;
            const T ar3 = u.w * r3;
            part[k][0] += ar3 * rx;
            part[k][1] += ar3 * ry;
            part[k][2] += ar3 * rz;
            part[k][3] += r3 * (w.y * rz - w.z * ry);
            part[k][4] += r3 * (w.z * rx - w.x * rz);
            part[k][5] += r3 * (w.x * ry - w.y * rx);
          }
        }
      }
      if constexpr (kSplit) {
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int c = 0; c < 6; ++c) part[k][c] = pp2[k][c].x + pp2[k][c].y;
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) kahan_add(acc[k][c], cmp[k][c], part[k][c]);
    }
    if constexpr (!kSplit) {  // physical near field -> stretched, scaled convention of the far field
      // normal kernel: l^2 S R / D^{3/2};  polynomial test kernel: S R (1 + D) / l
      const double c = POLY ? scal[3] : ell2;
      const T fe[6] = {(T)c, (T)c, (T)(c * gbar), (T)c, (T)c, (T)(c / gbar)};
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          acc[k][c] *= fe[c];
          cmp[k][c] *= fe[c];
        }
    }
    __syncthreads();  // sl (loaded above) is visible to every thread from here on

    const int a3share = (np1 + groups - 1) / groups;
    const int a3b = min(np1, grp * a3share), a3e = min(np1, a3b + a3share);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (valid[k] && far) {  // far field: L2P from the cumulative local field of the leaf
        T lx[kMaxNp1], ly[kMaxNp1], lz[kMaxNp1];
        const T lof = kSplit ? T(1) : T(0);
        bary_basis<T>((ri[k][0] + lof * rl[k][0]) * invh[0], deg[0], ch, lx);
        bary_basis<T>((ri[k][1] + lof * rl[k][1]) * invh[1], deg[1], ch, ly);
        bary_basis<T>((ri[k][2] + lof * rl[k][2]) * invh[2], deg[2], ch, lz);
        T f[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        int mu = a3b * np1 * np1;
        for (int a3 = a3b; a3 < a3e; ++a3) {
          for (int a2 = 0; a2 < np1; ++a2) {
            const T w = lz[a3] * ly[a2];
            T g[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            for (int a1 = 0; a1 < np1; ++a1, ++mu) {
#pragma unroll
              for (int c = 0; c < 6; ++c) g[c] += lx[a1] * sl[c * m + mu];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] += w * g[c];
          }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) kahan_add(acc[k][c], cmp[k][c], f[c]);
      }
    }
    if (groups > 1) {  // group 0 adds the other groups' sums, in group order
      T* cb = reinterpret_cast<T*>(smem_raw);  // [groups - 1][KPT][12][NT], over the staging rows
      if (grp > 0)
#pragma unroll
        for (int k = 0; k < KPT; ++k)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            cb[(((grp - 1) * KPT + k) * 12 + c) * NT + lt] = acc[k][c];
            cb[(((grp - 1) * KPT + k) * 12 + 6 + c) * NT + lt] = cmp[k][c];
          }
      __syncthreads();
      if (grp == 0)
        for (int g2 = 1; g2 < groups; ++g2)
#pragma unroll
          for (int k = 0; k < KPT; ++k)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              kahan_add(acc[k][c], cmp[k][c], cb[(((g2 - 1) * KPT + k) * 12 + c) * NT + lt]);
              kahan_add(acc[k][c], cmp[k][c], -cb[(((g2 - 1) * KPT + k) * 12 + 6 + c) * NT + lt]);
            }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (grp != 0 || !valid[k]) continue;
      const int64_t pos = st + pass0 + lt + (int64_t)k * NT;
      if (near_out != nullptr) {
        near_out[pos] = make_float4((float)acc[k][0], (float)acc[k][1], (float)acc[k][2], (float)acc[k][3]);
        near_out2[pos] = make_float4((float)acc[k][4], (float)acc[k][5], 0.f, 0.f);
        continue;
      }
      const int64_t i = perm[pos];
      Eout[3 * i + 0] = (T)(kE * (double)acc[k][0]);
      Eout[3 * i + 1] = (T)(kE * (double)acc[k][1]);
      Eout[3 * i + 2] = (T)(kE * (double)acc[k][2] / gbar);
      Bout[3 * i + 0] = (T)(kB * (double)acc[k][3]);
      Bout[3 * i + 1] = (T)(kB * (double)acc[k][4]);
      Bout[3 * i + 2] = (T)(kB * (double)acc[k][5] * gbar);
    }
  }
}

// FP32 far field after the near-field-only P2P (which ran beside M2L and
// L2L): L2P (Alg. 14, Eq. 2.8) from the leaf's cumulative local field, one
// thread per particle of a leaf chunk of 128, the local field staged with
// its six components side by side (two 16-byte shared loads per point); the
// near field is added and the sum converted to SI and written to the
// particle's input row as in k_p2p_l2p.  NP1 > 0 fixes the points per axis
// at compile time (basis values in registers); 0 reads them from ch.
constexpr int kFarThreads = 128;
template <int NP1>
__global__ void __launch_bounds__(kFarThreads) k_l2p_far(
    const unsigned int* __restrict__ err, const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount,
    int kappa, const NodeGeo* __restrict__ geo, const float4* __restrict__ px, const float4* __restrict__ pl,
    const float* __restrict__ Lcum, Cheb ch, int m, int chunks, const float4* __restrict__ near,
    const float4* __restrict__ near2, const int32_t* __restrict__ perm, const double* __restrict__ scal, float* __restrict__ Eout,
    float* __restrict__ Bout) {
  extern __shared__ float4 slc[];  // [m][2]: (L0, L1, L2, L3), (L4, L5, 0, 0)
  if (*err) return;  // the traversal failed: nothing is written
  const int64_t t = ((int64_t)1 << kappa) + blockIdx.x / chunks;
  const int64_t c0 = (int64_t)(blockIdx.x % chunks) * kFarThreads;
  const int64_t st = nstart[t], cnt = ncount[t];
  if (c0 >= cnt) return;  // the leaf is smaller than this chunk
  const bool far = kappa > 0;
  if (far) {
    const float* Lt = Lcum + (size_t)t * 6 * m;
    for (int o = threadIdx.x; o < m; o += blockDim.x) {
      slc[2 * o] = make_float4(Lt[o], Lt[m + o], Lt[2 * m + o], Lt[3 * m + o]);
      slc[2 * o + 1] = make_float4(Lt[4 * m + o], Lt[5 * m + o], 0.f, 0.f);
    }
  }
  __syncthreads();
  const int64_t j = c0 + threadIdx.x;
  if (j >= cnt) return;
  const int64_t pos = st + j;
  float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (far) {
    const NodeGeo g = geo[t];
    const float4 u = px[pos], l = pl[pos];
    const float xr[3] = {u.x + l.x, u.y + l.y, u.z + l.z};
    constexpr int K = NP1 > 0 ? NP1 : kMaxNp1;
    const int np1 = NP1 > 0 ? NP1 : ch.np1;
    float lx[K], ly[K], lz[K];
    float* lb[3] = {lx, ly, lz};
    for (int d = 0; d < 3; ++d) {
      const bool deg = !(g.h[d] > 0.0);
      const float tt = deg ? 0.f : xr[d] * (float)(1.0 / g.h[d]);
      if constexpr (NP1 > 0) {
        if (d == 0) bary_basis_n<K>(tt, deg, ch, lx);
        else if (d == 1) bary_basis_n<K>(tt, deg, ch, ly);
        else bary_basis_n<K>(tt, deg, ch, lz);
      } else {
        bary_basis<float>(tt, deg, ch, lb[d]);
      }
    }
    int mu = 0;
    for (int a3 = 0; a3 < np1; ++a3) {
#pragma unroll
      for (int a2 = 0; a2 < (NP1 > 0 ? NP1 : np1); ++a2) {
        const float w = lz[a3] * ly[a2];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f;
#pragma unroll
        for (int a1 = 0; a1 < (NP1 > 0 ? NP1 : np1); ++a1, ++mu) {
          const float4 A = slc[2 * mu], Bv = slc[2 * mu + 1];
          g0 += lx[a1] * A.x;
          g1 += lx[a1] * A.y;
          g2 += lx[a1] * A.z;
          g3 += lx[a1] * A.w;
          g4 += lx[a1] * Bv.x;
          g5 += lx[a1] * Bv.y;
        }
        f[0] += w * g0;
        f[1] += w * g1;
        f[2] += w * g2;
        f[3] += w * g3;
        f[4] += w * g4;
        f[5] += w * g5;
      }
    }
  }
  const float4 n0 = near[pos], n1 = near2[pos];
  const double gbar = scal[0], kE = scal[4], kB = scal[5];
  const int64_t i = perm[pos];
  Eout[3 * i + 0] = (float)(kE * (double)(n0.x + f[0]));
  Eout[3 * i + 1] = (float)(kE * (double)(n0.y + f[1]));
  Eout[3 * i + 2] = (float)(kE * (double)(n0.z + f[2]) / gbar);
  Bout[3 * i + 0] = (float)(kB * (double)(n0.w + f[3]));
  Bout[3 * i + 1] = (float)(kB * (double)(n1.x + f[4]));
  Bout[3 * i + 2] = (float)(kB * (double)(n1.y + f[5]) * gbar);
}

template <typename T, int KPT, bool POLY>
int launch(fmm_plan_s* P, void* E, void* B, cudaStream_t s, float4* near_out = nullptr,
           float4* near_out2 = nullptr) {
  const Layout& L = P->lay;
  int NT, groups, chunks;
  particle_shape(P->leaf, KPT, &NT, &groups, &chunks);
  const int nt = groups * NT;
  const int row = std::is_same<T, float>::value ? 4 : 2;
  const size_t stage = std::max(sizeof(typename Vec4<T>::type) * row * nt,
                                sizeof(T) * (size_t)(groups - 1) * KPT * 12 * NT);
  const size_t smem = stage + sizeof(T) * 6 * P->m;
  if (int rc = smem_limit(k_p2p_l2p<T, KPT, POLY>, (int)smem)) return rc;
  k_p2p_l2p<T, KPT, POLY><<<(unsigned)(P->nleaves * chunks), nt, smem, s>>>(
      ws_ptr<uint64_t>(P, L.p2p), ws_ptr<int32_t>(P, L.p2p_off), P->kappa + 1,
      &ws_ptr<Counters>(P, L.counters)->err, ws_ptr<int64_t>(P, L.nstart),
      ws_ptr<int64_t>(P, L.ncount), P->kappa, ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<typename Vec4<T>::type>(P, L.px), ws_ptr<typename Vec4<T>::type>(P, L.pb), ws_ptr<float4>(P, L.pl),
      P->ws + L.p2p_dc, ws_ptr<T>(P, L.local), P->cheb, P->m, ws_ptr<int32_t>(P, L.perm),
      ws_ptr<double>(P, L.scal), groups, chunks, static_cast<T*>(E), static_cast<T*>(B), near_out, near_out2);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T>
int p2p_t(fmm_plan_s* P, void* E, void* B, cudaStream_t s) {
  // one target per thread (two per thread measured slower: the extra
  // registers cost more occupancy than the shared loads they save)
  if constexpr (sizeof(T) == 8)
    if (P->flags & FMM_TEST_POLY_KERNEL) return launch<T, 1, true>(P, E, B, s);
  return launch<T, 1, false>(P, E, B, s);
}

}  // namespace

int run_p2p_l2p(fmm_plan_s* P, void* E, void* B, cudaStream_t s) {
  return P->precision == FMM_FP32 ? p2p_t<float>(P, E, B, s) : p2p_t<double>(P, E, B, s);
}

int run_p2p_near(fmm_plan_s* P, cudaStream_t s) {
  if (P->precision != FMM_FP32) return FMM_EINVAL;
  // two targets per thread on leaves of 256 or more: each staged source pair
  // then feeds two independent chains (2^24 core-halo beam, N0 = 256: P2P
  // alone 457.6 -> 424.5 ms)
  if (P->leaf >= kP2PPairLeaf)
    return launch<float, 2, false>(P, nullptr, nullptr, s, ws_ptr<float4>(P, P->lay.adj_part),
                                   ws_ptr<float4>(P, P->lay.adj_part2));
  return launch<float, 1, false>(P, nullptr, nullptr, s, ws_ptr<float4>(P, P->lay.adj_part),
                                 ws_ptr<float4>(P, P->lay.adj_part2));
}

int run_l2p_far(fmm_plan_s* P, void* E, void* B, cudaStream_t s) {
  if (P->precision != FMM_FP32) return FMM_EINVAL;
  const Layout& L = P->lay;
  const int64_t most = *std::max_element(P->node_count.begin() + P->nleaves, P->node_count.end());
  const int chunks = (int)div_up(most, kFarThreads);
  const size_t smem = sizeof(float4) * 2 * P->m;
  auto kern = k_l2p_far<0>;
  switch (P->np1) {
    case 3: kern = k_l2p_far<3>; break;
    case 5: kern = k_l2p_far<5>; break;
    case 7: kern = k_l2p_far<7>; break;
    case 9: kern = k_l2p_far<9>; break;
    case 11: kern = k_l2p_far<11>; break;
    default: break;
  }
  if (int rc = smem_limit(kern, (int)smem)) return rc;
  kern<<<(unsigned)(P->nleaves * chunks), kFarThreads, smem, s>>>(
      &ws_ptr<Counters>(P, L.counters)->err, ws_ptr<int64_t>(P, L.nstart), ws_ptr<int64_t>(P, L.ncount), P->kappa,
      ws_ptr<NodeGeo>(P, L.ngeo), ws_ptr<float4>(P, L.px), ws_ptr<float4>(P, L.pl), ws_ptr<float>(P, L.local),
      P->cheb, P->m, chunks, ws_ptr<float4>(P, L.adj_part), ws_ptr<float4>(P, L.adj_part2), ws_ptr<int32_t>(P, L.perm),
      ws_ptr<double>(P, L.scal),
      static_cast<float*>(E), static_cast<float*>(B));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

}  // namespace fmm
