// Separable transfers between tree levels: M2M (Eq. 2.7, Alg. 4) and L2L
// (Eq. 2.9, Alg. 13), and their transposes in the adjoint.
//
// For a child c of parent p and axis d, T_{c,d}[a][b] = l^d_{p,a}(xi^d_{c,b})
// is the parent's 1-D basis at the child's points.  All matrices are formed
// once per forward (k_tmats, FP64 from the physical boxes, the oracle's
// formula xi = c + h t_k, t = (xi - c_p)/h_p) and stored in the working
// precision.  A transfer applies T_x, T_y, T_z one axis at a time:
//   UP   (M2M, and L2L^T):  parent[a]  = sum_children sum_b T[a][b] child[b]
//   DOWN (L2L, and M2M^T):  child[b]  += sum_a T[a][b] parent[a]
// Each block handles one parent with both children and a group of
// components at once, so a parent costs three synchronised stages.  One
// cooperative launch walks all levels (deepest first for UP, root first for
// DOWN) with a grid-wide barrier between levels; beside another cooperative
// kernel (which the driver would run first) the same kernel is launched once
// per level instead.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace fmm {
namespace {

// tm[(c * 3 + d) * q + a * np1 + b] = l^d_{parent(c), a}(xi^d_{c, b})
template <typename T>
__global__ void k_tmats(const double* __restrict__ nlo, const double* __restrict__ nhi, int64_t C, Cheb ch,
                        T* __restrict__ tm) {
  const int np1 = ch.np1, q = np1 * np1;
  const int64_t total = (C - 1) * 3 * np1;  // nodes 2..C, axes, child points
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = 2 + e / (3 * np1);
    const int d = (int)((e / np1) % 3), b = (int)(e % np1);
    const int64_t p = c / 2;
    const double clo = nlo[3 * c + d], chi = nhi[3 * c + d];
    const double plo = nlo[3 * p + d], phi = nhi[3 * p + d];
    const double xc = chi > clo ? (clo + chi) / 2.0 + ((chi - clo) / 2.0) * ch.t[b] : clo;
    const bool deg = !(phi > plo);
    const double t = deg ? 0.0 : (xc - (plo + phi) / 2.0) / ((phi - plo) / 2.0);
    double l[kMaxNp1];
    bary_basis<double>(t, deg, ch, l);
    T* out = tm + ((size_t)c * 3 + d) * q;
    for (int a = 0; a < np1; ++a) out[a * np1 + b] = (T)l[a];
  }
}

template <typename T, int NC, bool UP>
__global__ void __launch_bounds__(256) k_transfer_all(int level_first, int level_last, int group, const T* __restrict__ tm,
                                                      Cheb ch, int m, T* __restrict__ buf) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  cg::grid_group grid = cg::this_grid();
  const int np1 = ch.np1, q = np1 * np1, pl = q;
  T* mats = sm;                       // [2 children][3 axes][q]
  T* in = mats + 6 * q;               // UP: [2][group][m]; DOWN: [group][m]
  T* t1 = in + 2 * group * m;         // [2][group][m]
  T* t2 = t1 + 2 * group * m;         // [2][group][m]
  const int ngroups = (NC + group - 1) / group;
  const int step = UP ? -1 : 1;
  for (int level = level_first;; level += step) {
    const int64_t nparents = (int64_t)1 << level;
    const int64_t items = nparents * ngroups;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const int64_t parent = nparents + it / ngroups;
      const int c0 = (int)(it % ngroups) * group;
      const int gc = min(group, NC - c0);
      __syncthreads();
      for (int o = threadIdx.x; o < 6 * q; o += blockDim.x) mats[o] = tm[(size_t)(2 * parent) * 3 * q + o];
      if (UP) {
        for (int o = threadIdx.x; o < 2 * gc * m; o += blockDim.x) {
          const int c = o / (gc * m), r = o % (gc * m);
          in[o] = buf[((size_t)(2 * parent + c) * NC + c0) * m + r];
        }
      } else {
        for (int o = threadIdx.x; o < gc * m; o += blockDim.x) in[o] = buf[((size_t)parent * NC + c0) * m + o];
      }
      __syncthreads();
      const int n1 = 2 * gc * m;
      // x axis
      for (int o = threadIdx.x; o < n1; o += blockDim.x) {
        const int c = o / (gc * m), r = o % (gc * m), comp = r / m, idx = r % m;
        const int a = idx % np1, rest = idx / np1;
        const T* M = mats + (c * 3 + 0) * q;
        const T* src = UP ? in + (c * gc + comp) * m : in + comp * m;
        T s = T(0);
        for (int k = 0; k < np1; ++k) s += (UP ? M[a * np1 + k] : M[k * np1 + a]) * src[rest * np1 + k];
        t1[o] = s;
      }
      __syncthreads();
      // y axis
      for (int o = threadIdx.x; o < n1; o += blockDim.x) {
        const int c = o / (gc * m), r = o % (gc * m), comp = r / m, idx = r % m;
        const int a = idx % np1, bb = (idx / np1) % np1, cz = idx / q;
        const T* M = mats + (c * 3 + 1) * q;
        const T* src = t1 + (c * gc + comp) * m;
        T s = T(0);
        for (int k = 0; k < np1; ++k) s += (UP ? M[bb * np1 + k] : M[k * np1 + bb]) * src[(cz * np1 + k) * np1 + a];
        t2[o] = s;
      }
      __syncthreads();
      // z axis, then sum the children into the parent (UP) or add into each child (DOWN)
      if (UP) {
        for (int o = threadIdx.x; o < gc * m; o += blockDim.x) {
          const int comp = o / m, idx = o % m;
          const int ab = idx % pl, cz = idx / pl;
          T s = T(0);
          for (int c = 0; c < 2; ++c) {
            const T* M = mats + (c * 3 + 2) * q;
            const T* src = t2 + (c * gc + comp) * m;
            for (int k = 0; k < np1; ++k) s += M[cz * np1 + k] * src[k * pl + ab];
          }
          buf[((size_t)parent * NC + c0 + comp) * m + idx] = s;
        }
      } else {
        for (int o = threadIdx.x; o < n1; o += blockDim.x) {
          const int c = o / (gc * m), r = o % (gc * m), comp = r / m, idx = r % m;
          const int ab = idx % pl, cz = idx / pl;
          const T* M = mats + (c * 3 + 2) * q;
          const T* src = t2 + (c * gc + comp) * m;
          T s = T(0);
          for (int k = 0; k < np1; ++k) s += M[k * np1 + cz] * src[k * pl + ab];
          buf[((size_t)(2 * parent + c) * NC + c0 + comp) * m + idx] += s;
        }
      }
    }
    if (level == level_last) break;
    grid.sync();
  }
}

// The same transfer specialised on the number of points per axis, with one
// (parent, component) pair per work item: compile-time extents turn the index
// arithmetic into shifts and multiplies, and the extra items shorten the
// per-level critical path near the root where only a few parents exist.
template <typename T, int NP1, bool UP>
__global__ void __launch_bounds__(256) k_transfer_np(int level_first, int level_last, int nc, const T* __restrict__ tm,
                                                     T* __restrict__ buf) {
  constexpr int Q = NP1 * NP1, M = Q * NP1;
  __shared__ T mats[6 * Q];  // [2 children][3 axes][Q]
  __shared__ T in[2 * M];    // UP: both children; DOWN: the parent in the first M
  __shared__ T t1[2 * M];
  __shared__ T t2[2 * M];
  cg::grid_group grid = cg::this_grid();
  const int step = UP ? -1 : 1;
  for (int level = level_first;; level += step) {
    const int64_t nparents = (int64_t)1 << level;
    const int64_t items = nparents * nc;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const int64_t parent = nparents + it / nc;
      const int comp = (int)(it % nc);
      __syncthreads();
      for (int o = threadIdx.x; o < 6 * Q; o += blockDim.x) mats[o] = tm[(size_t)(2 * parent) * 3 * Q + o];
      if (UP) {
        for (int o = threadIdx.x; o < 2 * M; o += blockDim.x) {
          const int c = o / M, idx = o - c * M;
          in[o] = buf[((size_t)(2 * parent + c) * nc + comp) * M + idx];
        }
      } else {
        for (int o = threadIdx.x; o < M; o += blockDim.x) in[o] = buf[((size_t)parent * nc + comp) * M + o];
      }
      __syncthreads();
      for (int o = threadIdx.x; o < 2 * M; o += blockDim.x) {  // x axis
        const int c = o / M, idx = o - c * M;
        const int a = idx % NP1, rest = idx / NP1;
        const T* Mx = mats + (c * 3 + 0) * Q;
        const T* src = (UP ? in + c * M : in) + rest * NP1;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NP1; ++k) s += (UP ? Mx[a * NP1 + k] : Mx[k * NP1 + a]) * src[k];
        t1[o] = s;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < 2 * M; o += blockDim.x) {  // y axis
        const int c = o / M, idx = o - c * M;
        const int a = idx % NP1, bb = (idx / NP1) % NP1, cz = idx / Q;
        const T* My = mats + (c * 3 + 1) * Q;
        const T* src = t1 + c * M + cz * Q + a;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NP1; ++k) s += (UP ? My[bb * NP1 + k] : My[k * NP1 + bb]) * src[k * NP1];
        t2[o] = s;
      }
      __syncthreads();
      if (UP) {  // z axis, summed over the two children into the parent
        for (int o = threadIdx.x; o < M; o += blockDim.x) {
          const int ab = o % Q, cz = o / Q;
          T s = T(0);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const T* Mz = mats + (c * 3 + 2) * Q;
            const T* src = t2 + c * M + ab;
#pragma unroll
            for (int k = 0; k < NP1; ++k) s += Mz[cz * NP1 + k] * src[k * Q];
          }
          buf[((size_t)parent * nc + comp) * M + o] = s;
        }
      } else {  // z axis, added into each child
        for (int o = threadIdx.x; o < 2 * M; o += blockDim.x) {
          const int c = o / M, idx = o - c * M;
          const int ab = idx % Q, cz = idx / Q;
          const T* Mz = mats + (c * 3 + 2) * Q;
          const T* src = t2 + c * M + ab;
          T s = T(0);
#pragma unroll
          for (int k = 0; k < NP1; ++k) s += Mz[k * NP1 + cz] * src[k * Q];
          buf[((size_t)(2 * parent + c) * nc + comp) * M + idx] += s;
        }
      }
    }
    if (level == level_last) break;
    grid.sync();
  }
}

template <typename T, int NP1, bool UP>
int launch_np(fmm_plan_s* P, int nc, T* buf, cudaStream_t s, int cap_per_sm, bool per_level) {
  int per_sm = 0, sms = 0;
  auto kern = k_transfer_np<T, NP1, UP>;
  if (int rc = device_sms(&sms)) return rc;
  if (int rc = blocks_per_sm(kern, 256, 0, &per_sm)) return rc;
  if (per_sm < 1) return FMM_EINVAL;
  // at most cap_per_sm blocks per SM (kCoopTransferCap for the cooperative
  // launch, kLevelTransferCap for the per-level launches)
  const int64_t most = ((int64_t)1 << (P->kappa - 1)) * nc;
  const int64_t blocks = (int64_t)std::min(per_sm, cap_per_sm) * sms;
  const T* tm = ws_ptr<T>(P, P->lay.tmat);
  if (per_level) {  // one ordinary launch per level (no grid barrier is reached)
    for (int i = 0; i < P->kappa; ++i) {
      const int level = UP ? P->kappa - 1 - i : i;
      const int grid = (int)std::min<int64_t>(blocks, ((int64_t)1 << level) * nc);
      kern<<<grid, 256, 0, s>>>(level, level, nc, tm, buf);
      FMM_LAUNCH_CHECK();
    }
    return FMM_OK;
  }
  const int grid = (int)std::min<int64_t>(blocks, most);
  int first = UP ? P->kappa - 1 : 0, last = UP ? 0 : P->kappa - 1;
  void* args[] = {&first, &last, &nc, (void*)&tm, &buf};
  FMM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(256), args, 0, s));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T, int NC, bool UP>
int launch_all(fmm_plan_s* P, T* buf, cudaStream_t s) {
  if (P->kappa == 0) return FMM_OK;
  const int q = P->np1 * P->np1;
  const size_t budget = 200 * 1024;
  const size_t mats = (size_t)6 * q * sizeof(T);
  int group = NC;
  while (group > 1 && mats + (size_t)6 * group * P->m * sizeof(T) > budget) --group;
  const size_t smem = mats + (size_t)6 * group * P->m * sizeof(T);
  int per_sm = 0, sms = 0;
  auto kern = k_transfer_all<T, NC, UP>;
  if (int rc = smem_limit(kern, (int)budget)) return rc;
  if (int rc = device_sms(&sms)) return rc;
  if (int rc = blocks_per_sm(kern, 256, smem, &per_sm)) return rc;
  if (per_sm < 1) return FMM_EINVAL;
  const int ngroups = (NC + group - 1) / group;
  const int64_t most = ((int64_t)1 << (P->kappa - 1)) * ngroups;
  const int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, most);
  int first = UP ? P->kappa - 1 : 0, last = UP ? 0 : P->kappa - 1;
  const T* tm = ws_ptr<T>(P, P->lay.tmat);
  Cheb ch = P->cheb;
  int m = P->m;
  void* args[] = {&first, &last, &group, (void*)&tm, &ch, &m, &buf};
  FMM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(256), args, smem, s));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

}  // namespace

int run_tmats(fmm_plan_s* P, cudaStream_t s) {
  if (P->kappa == 0) return FMM_OK;
  const int64_t total = (P->C - 1) * 3 * P->np1;
  const unsigned g = (unsigned)std::min<int64_t>(div_up(total, 128), 8192);
  if (P->precision == FMM_FP32)
    k_tmats<float><<<g, 128, 0, s>>>(ws_ptr<double>(P, P->lay.nlo), ws_ptr<double>(P, P->lay.nhi), P->C, P->cheb,
                                     ws_ptr<float>(P, P->lay.tmat));
  else
    k_tmats<double><<<g, 128, 0, s>>>(ws_ptr<double>(P, P->lay.nlo), ws_ptr<double>(P, P->lay.nhi), P->C, P->cheb,
                                      ws_ptr<double>(P, P->lay.tmat));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

template <typename T, int NC, bool UP>
int run_transfer(fmm_plan_s* P, T* buf, cudaStream_t s, int max_blocks_per_sm, bool per_level) {
  if (P->kappa == 0) return FMM_OK;
  const int c = std::max(1, max_blocks_per_sm);
  switch (P->np1) {
    case 3: return launch_np<T, 3, UP>(P, NC, buf, s, c, per_level);
    case 5: return launch_np<T, 5, UP>(P, NC, buf, s, c, per_level);
    case 7: return launch_np<T, 7, UP>(P, NC, buf, s, c, per_level);
    case 9: return launch_np<T, 9, UP>(P, NC, buf, s, c, per_level);
    default: return launch_all<T, NC, UP>(P, buf, s);
  }
}

template int run_transfer<float, 4, true>(fmm_plan_s*, float*, cudaStream_t, int, bool);
template int run_transfer<double, 4, true>(fmm_plan_s*, double*, cudaStream_t, int, bool);
template int run_transfer<float, 6, false>(fmm_plan_s*, float*, cudaStream_t, int, bool);
template int run_transfer<double, 6, false>(fmm_plan_s*, double*, cudaStream_t, int, bool);
template int run_transfer<float, 6, true>(fmm_plan_s*, float*, cudaStream_t, int, bool);
template int run_transfer<double, 6, true>(fmm_plan_s*, double*, cudaStream_t, int, bool);
template int run_transfer<float, 4, false>(fmm_plan_s*, float*, cudaStream_t, int, bool);
template int run_transfer<double, 4, false>(fmm_plan_s*, double*, cudaStream_t, int, bool);

}  // namespace fmm
