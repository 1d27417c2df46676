// M2L (Alg. 9, Eq. 2.5 with the effective masses of Section 3).
//
// One block per target cluster t drains t's M2L list (sorted by target, so no
// two blocks write the same locals and no atomics are needed, Section 10).
// Each thread owns KPT proxy points mu of t.  For every source cluster the
// source's proxy table (point offsets Y_nu and effective masses a_nu, b~_nu)
// is staged in shared memory and every owned point accumulates
//   E_mu += a_nu R / |R|^3,  B_mu += b~_nu x R / |R|^3,  R = xi_t,mu - xi_s,nu
// in stretched, scaled coordinates.  The centre difference c_t - c_s is
// formed in FP64 once per list pair and rounded once; per-source partial sums are added to the
// running sums with Kahan compensation.  Locals of clusters without M2L
// sources are written as zeros.
#include "common.cuh"

namespace fmm {
namespace {

template <typename T, int KPT, bool POLY>
__global__ void __launch_bounds__(256) k_m2l(const uint64_t* __restrict__ keys, const int32_t* __restrict__ off,
                                             int shift, const unsigned int* __restrict__ err, const int32_t* __restrict__ order, int64_t nitems, const NodeGeo* __restrict__ geo,
                                             const void* __restrict__ pdc, Cheb ch, int m, const double* __restrict__ scal,
                                             const typename Vec4<T>::type* __restrict__ src, T* __restrict__ Lout) {
  using V4 = typename Vec4<T>::type;
  extern __shared__ unsigned char smem_raw[];
  V4* sm = reinterpret_cast<V4*>(smem_raw);
  if (*err) return;  // the traversal failed: the lists are incomplete
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {  // targets, longest list first
  const int64_t t = order[w];
  const int np1 = ch.np1;
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int b = off[t], e = off[t + 1];
  const NodeGeo gt = geo[t];
  const int per_pass = KPT * blockDim.x;
  for (int pass0 = 0; pass0 < m; pass0 += per_pass) {
    T xh[KPT][3];
    bool valid[KPT];
    T acc[KPT][6], cmp[KPT][6];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int mu = pass0 + threadIdx.x + k * blockDim.x;
      valid[k] = mu < m;
      const int mm = valid[k] ? mu : 0;
      const int m1 = mm % np1, m2 = (mm / np1) % np1, m3 = mm / (np1 * np1);
      xh[k][0] = (T)(gt.h[0] * ch.t[m1]);
      xh[k][1] = (T)(gt.h[1] * ch.t[m2]);
      xh[k][2] = (T)(gt.h[2] * ch.t[m3]);
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[k][c] = cmp[k][c] = T(0);
    }
    for (int it = b; it < e; ++it) {
      const int64_t s = (int64_t)(keys[it] & mask);
      T dc0, dc1, dc2;
      if constexpr (sizeof(T) == 4) {  // FP32: the pair's centre offset, rounded once from FP64
        const float4 dh = static_cast<const float4*>(pdc)[2 * it];
        dc0 = dh.x; dc1 = dh.y; dc2 = dh.z;
      } else {
        const double4 dd = static_cast<const double4*>(pdc)[it];
        dc0 = dd.x; dc1 = dd.y; dc2 = dd.z;
      }
      const V4* tab = src + (size_t)s * m * 2;
      __syncthreads();
      for (int o = threadIdx.x; o < 2 * m; o += blockDim.x) sm[o] = tab[o];
      __syncthreads();
      T X[KPT][3], part[KPT][6];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        X[k][0] = dc0 + xh[k][0];
        X[k][1] = dc1 + xh[k][1];
        X[k][2] = dc2 + xh[k][2];
#pragma unroll
        for (int c = 0; c < 6; ++c) part[k][c] = T(0);
      }
      for (int nu = 0; nu < m; ++nu) {
        const V4 ya = sm[2 * nu], bb = sm[2 * nu + 1];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          const T rx = X[k][0] - ya.x, ry = X[k][1] - ya.y, rz = X[k][2] - ya.z;
          const T d = rx * rx + ry * ry + rz * rz;
          T r3;
          if constexpr (POLY) {  // the polynomial test kernel R' (1 + l^2 |R'|^2)
            r3 = T(1) + (T)(scal[2] * scal[2]) * d;
          } else {
            const T inv = d > tiny_sep2<T>() ? rsqrt_t<T>(d) : T(0);
            r3 = inv * inv * inv;
          }
          const T ar3 = ya.w * r3;
          part[k][0] += ar3 * rx;
          part[k][1] += ar3 * ry;
          part[k][2] += ar3 * rz;
          part[k][3] += r3 * (bb.y * rz - bb.z * ry);
          part[k][4] += r3 * (bb.z * rx - bb.x * rz);
          part[k][5] += r3 * (bb.x * ry - bb.y * rx);
        }
      }
#pragma unroll
      for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) kahan_add(acc[k][c], cmp[k][c], part[k][c]);
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int mu = pass0 + threadIdx.x + k * blockDim.x;
      if (!valid[k]) continue;
#pragma unroll
      for (int c = 0; c < 6; ++c) Lout[((size_t)t * 6 + c) * m + mu] = acc[k][c];
    }
  }
  }  // work items
}

// FP32 M2L specialised on the points per axis NP1 = n + 1 (for eta <= 1/2).
//
// A thread owns the target points mu = (mu1, mu2, mu3) with fixed (mu1, mu2)
// and mu3 = g, g + G, ... (KPT of them).  For a source s the separation
// R = xi_t,mu - xi_s,nu splits per axis: R_x depends on (mu1, nu1) only, so
// the thread keeps R_x[nu1], R_x^2 and R_y[nu2], R_y^2 in registers, and
// |R|^2 = R_x^2[nu1] + (R_y^2[nu2] + R_z^2[nu3]) costs one add per point
// pair.  Inside the nu1 loop R_y and R_z are constant, so the sums regroup:
//   E  += (sum a r3 R_x,  R_y sum a r3,  R_z sum a r3)
//   B  += (R_z sum b_y r3 - R_y sum b_z r3,  sum b_z r3 R_x - R_z sum b_x r3,
//          R_y sum b_x r3 - sum b_y r3 R_x)
// with seven running sums per target point (13 FP32 operations and one
// rsqrt per point pair instead of 21).  A block takes one of SPLIT chunks of
// a target's mu3 points at a time, fetching (target, chunk) items from an
// atomic counter in the work order (longest source lists first), so the
// SMs finish together even when a few targets have the longest lists.  The same terms are added, in the same
// per-source groups, as in the generic kernel.  For eta <= 1/2 admissible
// boxes are disjoint (r_t + r_s < d), so |R|^2 > 0 and a clamp replaces the
// zero mask.  The running Kahan sums across sources live in shared memory.
template <int NP1, int G, int SPLIT>
__global__ void __launch_bounds__(NP1 * NP1 * G, 3) k_m2l_fast(const uint64_t* __restrict__ keys,
                                                              const int32_t* __restrict__ off, int shift, const unsigned int* __restrict__ err, const int32_t* __restrict__ order, int64_t nitems, unsigned int* __restrict__ work,
                                                              const NodeGeo* __restrict__ geo,
                                                              const float4* __restrict__ pdc, Cheb ch,
                                                              const float* __restrict__ M, float* __restrict__ Lout) {
  constexpr int KPT = (NP1 + G * SPLIT - 1) / (G * SPLIT);
  constexpr int NT = NP1 * NP1 * G;
  constexpr int m = NP1 * NP1 * NP1;
  __shared__ float4 sm[m];              // source effective masses (a, b~x, b~y, b~z)
  __shared__ float syz[NP1];            // source point offsets along z
  __shared__ float sacc[KPT][12][NT];   // Kahan sums and compensations
  if (*err) return;  // the traversal failed: the lists are incomplete
  __shared__ int64_t s_item;
  for (;;) {  // items (target, mu3 chunk) fetched in the work order: longest lists first
  if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(work, 1u);
  __syncthreads();
  const int64_t w = s_item;
  __syncthreads();
  if (w >= nitems) break;
  const int64_t t = order[w / SPLIT];
  const int base3 = (int)(w % SPLIT) * G * KPT;
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int b = off[t], e = off[t + 1];
  const NodeGeo gt = geo[t];
  const int tid = threadIdx.x;
  const int mu12 = tid % (NP1 * NP1), g = tid / (NP1 * NP1);
  const int mu1 = mu12 % NP1, mu2 = mu12 / NP1;
  const float xt = (float)(gt.h[0] * ch.t[mu1]), yt = (float)(gt.h[1] * ch.t[mu2]);
  float zt[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int mu3 = base3 + g + k * G;
    zt[k] = (float)(gt.h[2] * ch.t[mu3 < NP1 ? mu3 : 0]);
#pragma unroll
    for (int c = 0; c < 12; ++c) sacc[k][c][tid] = 0.f;
  }
  for (int it = b; it < e; ++it) {
    const int64_t s = (int64_t)(keys[it] & mask);
    const float4 dh = pdc[2 * it];
    const NodeGeo gs = geo[s];
    const float hsx = (float)gs.h[0], hsy = (float)gs.h[1];
    __syncthreads();
    const float* Ms = M + (size_t)s * 4 * m;
    for (int o = tid; o < m; o += NT) sm[o] = make_float4(Ms[o], Ms[m + o], Ms[2 * m + o], Ms[3 * m + o]);
    if (tid < NP1) syz[tid] = (float)(gs.h[2] * ch.t[tid]);
    __syncthreads();
    const float X = dh.x + xt, Y = dh.y + yt;
    float Rx[NP1], Dx[NP1], Ry[NP1], Dy[NP1];
#pragma unroll
    for (int k = 0; k < NP1; ++k) {
      Rx[k] = X - hsx * (float)ch.t[k];
      Dx[k] = Rx[k] * Rx[k];
      Ry[k] = Y - hsy * (float)ch.t[k];
      Dy[k] = Ry[k] * Ry[k];
    }
    float Z[KPT], part[KPT][6];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      Z[k] = dh.z + zt[k];
#pragma unroll
      for (int c = 0; c < 6; ++c) part[k][c] = 0.f;
    }
    for (int n3 = 0; n3 < NP1; ++n3) {
      const float yz = syz[n3];
      float rz[KPT], dz[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        rz[k] = Z[k] - yz;
        dz[k] = rz[k] * rz[k];
      }
      const float4* row = sm + n3 * NP1 * NP1;
#pragma unroll
      for (int n2 = 0; n2 < NP1; ++n2) {
        float dyz[KPT], Ta[KPT], TaR[KPT], Tbx[KPT], Tby[KPT], TbyR[KPT], Tbz[KPT], TbzR[KPT];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          dyz[k] = Dy[n2] + dz[k];
          Ta[k] = TaR[k] = Tbx[k] = Tby[k] = TbyR[k] = Tbz[k] = TbzR[k] = 0.f;
        }
#pragma unroll
        for (int n1 = 0; n1 < NP1; ++n1) {
          const float4 src = row[n2 * NP1 + n1];
#pragma unroll
          for (int k = 0; k < KPT; ++k) {
            const float d = fmaxf(Dx[n1] + dyz[k], 5.169878828456423e-26f);
            const float inv = rsqrt_normal(d);
            const float r3 = inv * inv * inv;
            const float ar3 = src.x * r3;
            Ta[k] += ar3;
            TaR[k] = fmaf(ar3, Rx[n1], TaR[k]);
            Tbx[k] = fmaf(src.y, r3, Tbx[k]);
            const float byr3 = src.z * r3;
            Tby[k] += byr3;
            TbyR[k] = fmaf(byr3, Rx[n1], TbyR[k]);
            const float bzr3 = src.w * r3;
            Tbz[k] += bzr3;
            TbzR[k] = fmaf(bzr3, Rx[n1], TbzR[k]);
          }
        }
        const float ry = Ry[n2];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          part[k][0] += TaR[k];
          part[k][1] += ry * Ta[k];
          part[k][2] += rz[k] * Ta[k];
          part[k][3] += rz[k] * Tby[k] - ry * Tbz[k];
          part[k][4] += TbzR[k] - rz[k] * Tbx[k];
          part[k][5] += ry * Tbx[k] - TbyR[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float sum = sacc[k][c][tid], comp = sacc[k][6 + c][tid];
        kahan_add(sum, comp, part[k][c]);
        sacc[k][c][tid] = sum;
        sacc[k][6 + c][tid] = comp;
      }
  }
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int mu3 = base3 + g + k * G;
    if (mu3 >= NP1) continue;
    const int mu = mu1 + NP1 * (mu2 + NP1 * mu3);
#pragma unroll
    for (int c = 0; c < 6; ++c) Lout[((size_t)t * 6 + c) * m + mu] = sacc[k][c][tid];
  }
  }  // work items
}

// FP32 M2L with paired arithmetic and the R_x products held per point
// (eta <= 1/2, points per axis NP1 fixed).
//
// Two changes against k_m2l_fast, which issues about 18 instructions per
// point pair, 14 of them on the FMA pipe:
// - A thread owns two target points of the cluster, mu_a = P and
//   mu_b = P + H (H = ceil(m / 2)), and evaluates both against each source
//   point with paired FP32 instructions (__fadd2_rn, __fmul2_rn,
//   __ffma2_rn: two lanes per instruction), so one instruction stream serves
//   two point pairs.
// - In the nu1 loop R_x = X - s_x[nu1] is the only varying component (held
//   per nu1 in registers), so the sums are taken in r3 and r3 R_x and
//   multiplied by R_y, R_z after the loop: a point pair costs 11 FMA-pipe
//   operations (|R|^2 1, r^-3 2, r3 R_x 1, seven sums) on two staged float4.
//   Splitting the R_x sums instead (sum q r3 R_x = X sum q r3 - sum (q s_x)
//   r3, with q s_x staged) saves the r3 R_x product but doubles the shared
//   loads; measured on the 2^24 core-halo beam (n = 8) at 4 blocks per SM
//   this form takes 743 ms against the split form's 791 ms at 3 blocks.
// Staged per source point, every value duplicated for the two lanes:
// (a, a, b~x, b~x), (b~y, b~y, b~z, b~z).  The running sums across sources
// are Kahan-compensated in shared memory, in the same per-source groups as
// the other M2L kernels.
// Items are (target, chunk of NT point pairs), fetched from the work counter
// in the work order (longest source lists first).
template <int NP1, int NT>
__global__ void __launch_bounds__(NT, 4) k_m2l_pair(const uint64_t* __restrict__ keys, const int32_t* __restrict__ off,
                                                   int shift, const unsigned int* __restrict__ err,
                                                   const int32_t* __restrict__ order, int64_t nitems,
                                                   unsigned int* __restrict__ work, const NodeGeo* __restrict__ geo,
                                                   const float4* __restrict__ pdc, Cheb ch,
                                                   const float* __restrict__ M, float* __restrict__ Lout) {
  constexpr int m = NP1 * NP1 * NP1;
  constexpr int H = (m + 1) / 2;               // point pairs per cluster
  constexpr int SPLIT = (H + NT - 1) / NT;     // items per cluster
  extern __shared__ float4 dsm[];
  float4* sm = dsm;                                           // [m][2] staged source points
  float2* sacc = reinterpret_cast<float2*>(dsm + 2 * m);      // [12][NT] Kahan sums, compensations
  __shared__ float sxyz[3][NP1];               // source point offsets per axis
  __shared__ int64_t s_item;
  if (*err) return;  // the traversal failed: the lists are incomplete
  const int tid = threadIdx.x;
  const float2 neg1 = make_float2(-1.f, -1.f);
  for (;;) {
    if (tid == 0) s_item = (int64_t)atomicAdd(work, 1u);
    __syncthreads();
    const int64_t w = s_item;
    __syncthreads();
    if (w >= nitems) break;
    const int64_t t = order[w / SPLIT];
    const int P = (int)(w % SPLIT) * NT + tid;
    const int mua = P < H ? P : 0, mub = P + H < m ? P + H : 0;
    const uint64_t mask = ((uint64_t)1 << shift) - 1;
    const int b = off[t], e = off[t + 1];
    const NodeGeo gt = geo[t];
    // target point offsets from the cluster centre, lanes (mu_a, mu_b)
    const float2 xt = make_float2((float)(gt.h[0] * ch.t[mua % NP1]), (float)(gt.h[0] * ch.t[mub % NP1]));
    const float2 yt = make_float2((float)(gt.h[1] * ch.t[(mua / NP1) % NP1]),
                                  (float)(gt.h[1] * ch.t[(mub / NP1) % NP1]));
    const float2 zt = make_float2((float)(gt.h[2] * ch.t[mua / (NP1 * NP1)]),
                                  (float)(gt.h[2] * ch.t[mub / (NP1 * NP1)]));
#pragma unroll
    for (int c = 0; c < 12; ++c) sacc[c * NT + tid] = make_float2(0.f, 0.f);
    for (int it = b; it < e; ++it) {
      const int64_t s = (int64_t)(keys[it] & mask);
      const float4 dh = pdc[2 * it];
      const NodeGeo gs = geo[s];
      __syncthreads();
      const float* Ms = M + (size_t)s * 4 * m;
      for (int o = tid; o < m; o += NT) {
        const float a = Ms[o], bx = Ms[m + o], by = Ms[2 * m + o], bz = Ms[3 * m + o];
        sm[2 * o] = make_float4(a, a, bx, bx);
        sm[2 * o + 1] = make_float4(by, by, bz, bz);
      }
      if (tid < 3 * NP1) {
        const int d = tid / NP1, k = tid - d * NP1;
        sxyz[d][k] = (float)(gs.h[d] * ch.t[k]);
      }
      __syncthreads();
      // this thread's two target points relative to the source-cluster centre
      const float2 X = __fadd2_rn(make_float2(dh.x, dh.x), xt);
      const float2 Y = __fadd2_rn(make_float2(dh.y, dh.y), yt);
      const float2 Z = __fadd2_rn(make_float2(dh.z, dh.z), zt);
      float2 Rx[NP1];
#pragma unroll
      for (int k = 0; k < NP1; ++k) Rx[k] = __fadd2_rn(X, make_float2(-sxyz[0][k], -sxyz[0][k]));
      float2 part[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) part[c] = make_float2(0.f, 0.f);
      for (int n3 = 0; n3 < NP1; ++n3) {
        const float2 rz = __fadd2_rn(Z, make_float2(-sxyz[2][n3], -sxyz[2][n3]));
        const float2 nrz = __fmul2_rn(rz, neg1);
        const float2 dz = __fmul2_rn(rz, rz);
        const float4* row = sm + 2 * n3 * NP1 * NP1;
#pragma unroll
        for (int n2 = 0; n2 < NP1; ++n2) {
          const float2 ry = __fadd2_rn(Y, make_float2(-sxyz[1][n2], -sxyz[1][n2]));
          const float2 dyz = __ffma2_rn(ry, ry, dz);
          const float2 z0 = make_float2(0.f, 0.f);
          float2 Ta = z0, Ua = z0, Tbx = z0, Tby = z0, Uby = z0, Tbz = z0, Ubz = z0;
#pragma unroll
          for (int n1 = 0; n1 < NP1; ++n1) {
            const float4* q = row + 2 * (n2 * NP1 + n1);
            const float4 A = q[0], Bq = q[1];
            float2 d = __ffma2_rn(Rx[n1], Rx[n1], dyz);
            d.x = fmaxf(d.x, tiny_sep2<float>());
            d.y = fmaxf(d.y, tiny_sep2<float>());
            const float2 inv = make_float2(rsqrt_normal(d.x), rsqrt_normal(d.y));
            const float2 r3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
            Ta = __ffma2_rn(make_float2(A.x, A.y), r3, Ta);
            Tbx = __ffma2_rn(make_float2(A.z, A.w), r3, Tbx);
            Tby = __ffma2_rn(make_float2(Bq.x, Bq.y), r3, Tby);
            Tbz = __ffma2_rn(make_float2(Bq.z, Bq.w), r3, Tbz);
            const float2 rr = __fmul2_rn(r3, Rx[n1]);
            Ua = __ffma2_rn(make_float2(A.x, A.y), rr, Ua);
            Uby = __ffma2_rn(make_float2(Bq.x, Bq.y), rr, Uby);
            Ubz = __ffma2_rn(make_float2(Bq.z, Bq.w), rr, Ubz);
          }
          const float2 TaR = Ua, TbyR = Uby, TbzR = Ubz;
          // E += (sum a r3 R_x, R_y sum a r3, R_z sum a r3)
          // B += (R_z sum b~y r3 - R_y sum b~z r3, sum b~z r3 R_x - R_z sum b~x r3,
          //       R_y sum b~x r3 - sum b~y r3 R_x)
          part[0] = __fadd2_rn(part[0], TaR);
          part[1] = __ffma2_rn(ry, Ta, part[1]);
          part[2] = __ffma2_rn(rz, Ta, part[2]);
          part[3] = __ffma2_rn(rz, Tby, part[3]);
          part[3] = __ffma2_rn(__fmul2_rn(ry, neg1), Tbz, part[3]);
          part[4] = __fadd2_rn(part[4], TbzR);
          part[4] = __ffma2_rn(nrz, Tbx, part[4]);
          part[5] = __ffma2_rn(ry, Tbx, part[5]);
          part[5] = __ffma2_rn(TbyR, neg1, part[5]);
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float2 sum = sacc[c * NT + tid], comp = sacc[(6 + c) * NT + tid];
        kahan_add(sum.x, comp.x, part[c].x);
        kahan_add(sum.y, comp.y, part[c].y);
        sacc[c * NT + tid] = sum;
        sacc[(6 + c) * NT + tid] = comp;
      }
    }
    if (P < H) {
#pragma unroll
      for (int c = 0; c < 6; ++c) Lout[((size_t)t * 6 + c) * m + P] = sacc[c * NT + tid].x;
    }
    if (P + H < m) {
#pragma unroll
      for (int c = 0; c < 6; ++c) Lout[((size_t)t * 6 + c) * m + P + H] = sacc[c * NT + tid].y;
    }
  }  // work items
}

template <int NP1, int NT>
int launch_pair(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  constexpr int m = NP1 * NP1 * NP1, H = (m + 1) / 2, SPLIT = (H + NT - 1) / NT;
  const size_t smem = sizeof(float4) * 2 * m + sizeof(float2) * 12 * NT;
  if (int rc = smem_limit(k_m2l_pair<NP1, NT>, (int)smem)) return rc;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_m2l_pair<NP1, NT>, NT, smem, P->C * SPLIT, &grid)) return rc;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  FMM_CUDA_TRY(cudaMemsetAsync(&cnt->work[0], 0, sizeof(unsigned int), s));
  k_m2l_pair<NP1, NT><<<grid, NT, smem, s>>>(
      ws_ptr<uint64_t>(P, L.m2l), ws_ptr<int32_t>(P, L.m2l_off), P->kappa + 1, &cnt->err,
      ws_ptr<int32_t>(P, L.m2l_order), P->C * SPLIT, &cnt->work[0], ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.m2l_dc), P->cheb, ws_ptr<float>(P, L.mpole), ws_ptr<float>(P, L.local));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <int NP1, int G, int SPLIT>
int launch_fast(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_m2l_fast<NP1, G, SPLIT>, NP1 * NP1 * G, 0, P->C * SPLIT, &grid)) return rc;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  FMM_CUDA_TRY(cudaMemsetAsync(&cnt->work[0], 0, sizeof(unsigned int), s));
  k_m2l_fast<NP1, G, SPLIT><<<grid, NP1 * NP1 * G, 0, s>>>(
      ws_ptr<uint64_t>(P, L.m2l), ws_ptr<int32_t>(P, L.m2l_off), P->kappa + 1, &cnt->err,
      ws_ptr<int32_t>(P, L.m2l_order), P->C * SPLIT, &cnt->work[0], ws_ptr<NodeGeo>(P, L.ngeo),
      ws_ptr<float4>(P, L.m2l_dc), P->cheb, ws_ptr<float>(P, L.mpole), ws_ptr<float>(P, L.local));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// Block shape: threads nt <= 256 (a multiple of 32) owning KPT points each,
// chosen to waste the fewest thread slots, then to need the fewest passes.
void pick_shape(int m, int* nt, int* kpt) {
  int best_nt = 256, best_k = 4;
  int64_t best_waste = -1, best_passes = 0;
  for (int k = 1; k <= 4; ++k) {
    int t = (int)(div_up(div_up(m, k), 32) * 32);
    if (t > 256) t = 256;
    const int64_t passes = div_up(m, (int64_t)t * k);
    const int64_t waste = passes * t * k - m;
    if (best_waste < 0 || waste < best_waste || (waste == best_waste && passes < best_passes)) {
      best_waste = waste;
      best_passes = passes;
      best_nt = t;
      best_k = k;
    }
  }
  *nt = best_nt;
  *kpt = best_k;
}

template <typename T, int KPT, bool POLY>
int launch(fmm_plan_s* P, int nt, cudaStream_t s) {
  const Layout& L = P->lay;
  const size_t smem = (size_t)2 * P->m * sizeof(typename Vec4<T>::type);
  if (int rc = smem_limit(k_m2l<T, KPT, POLY>, (int)smem)) return rc;
  unsigned grid = 0;
  if (int rc = resident_blocks(k_m2l<T, KPT, POLY>, nt, smem, P->C, &grid)) return rc;
  k_m2l<T, KPT, POLY><<<grid, nt, smem, s>>>(ws_ptr<uint64_t>(P, L.m2l), ws_ptr<int32_t>(P, L.m2l_off),
                                        P->kappa + 1, &ws_ptr<Counters>(P, L.counters)->err,
                                        ws_ptr<int32_t>(P, L.m2l_order), P->C,
                                        ws_ptr<NodeGeo>(P, L.ngeo), P->ws + L.m2l_dc, P->cheb, P->m,
                                        ws_ptr<double>(P, L.scal),
                                                  ws_ptr<typename Vec4<T>::type>(P, L.srct), ws_ptr<T>(P, L.local));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T, bool POLY>
int m2l_t(fmm_plan_s* P, cudaStream_t s) {
  int nt, kpt;
  pick_shape(P->m, &nt, &kpt);
  switch (kpt) {
    case 1: return launch<T, 1, POLY>(P, nt, s);
    case 2: return launch<T, 2, POLY>(P, nt, s);
    case 3: return launch<T, 3, POLY>(P, nt, s);
    default: return launch<T, 4, POLY>(P, nt, s);
  }
}

}  // namespace

bool m2l_specialised(const fmm_plan_s* P) {
  return P->precision == FMM_FP32 && P->eta <= 0.5 && !(P->flags & FMM_TEST_POLY_KERNEL) &&
         (P->np1 == 3 || P->np1 == 5 || P->np1 == 7 || P->np1 == 9 || P->np1 == 11);
}

int run_m2l(fmm_plan_s* P, cudaStream_t s) {
  if (m2l_specialised(P)) {
    switch (P->np1) {
      case 3: return launch_fast<3, 3, 1>(P, s);
      // paired kernels, block sizes from sweeps of fwd+adj steps: n = 4 (64
      // threads) 33.2 -> 32.1 ms on the 1.28e6 cube; n = 6 (64) 1.465 ->
      // 1.432 ms at 2^16, 14.9 -> 14.3 ms at 2^18 (192: 14.0, 96: 14.6);
      // n = 8 (128) with the x sums split 3.91 -> 3.47 s at 2^24; n = 10
      // (128): M2L 11.4 -> 4.9 ms on the 1.28e6 cube at eta = 0.3
      case 5: return launch_pair<5, 64>(P, s);
      case 7: return launch_pair<7, 64>(P, s);
      case 9: return launch_pair<9, 128>(P, s);
      case 11: return launch_pair<11, 128>(P, s);
      default: break;
    }
  }
  if (P->flags & FMM_TEST_POLY_KERNEL) return m2l_t<double, true>(P, s);  // FP64 plans only
  return P->precision == FMM_FP32 ? m2l_t<float, false>(P, s) : m2l_t<double, false>(P, s);
}

}  // namespace fmm
