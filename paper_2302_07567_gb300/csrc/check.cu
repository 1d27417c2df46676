// Device checks of a plan's indices (FMM_BOUNDS_CHECK).
//
// After the traversal (and, in the adjoint, after the source-major lists are
// built) the checks below run on the device; any violation sets kErrBounds,
// and the call returns FMM_EBOUNDS before a kernel indexes through the bad
// value.  What they verify:
//   - node tables: every node non-empty and inside [0, N); the two children
//     of an inner node split its slot range (Alg. 2, Appendix B: first child
//     ceil(|S|/2));
//   - the leaf order is a permutation of 0 .. N-1, and the M2L work order
//     (target-major, or source-major in the adjoint) one of the nodes 1 .. C;
//   - every list pair names nodes 1 .. C, P2P pairs name leaves (Algs. 11,
//     17: only leaf-leaf pairs go to P2P), the keys are strictly increasing
//     (sorted by (major, minor), no duplicate pair) and agree with the CSR
//     offsets of their major node;
//   - the lists cover every ordered particle pair exactly once:
//     sum over P2P and M2L pairs of |S_t| |S_s| = N^2 (the dual traversal
//     partitions the interaction matrix, Section 4).
#include "common.cuh"

namespace fmm {
namespace {

__device__ __forceinline__ void bad(Counters* cnt) { atomicOr(&cnt->err, kErrBounds); }

__global__ void k_check_nodes(const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int64_t C,
                              int kappa, int64_t N, Counters* cnt) {
  const int64_t inner = ((int64_t)1 << kappa) - 1;  // nodes 1 .. inner have children
  for (int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= C; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t st = nstart[i], c = ncount[i];
    if (c < 1 || st < 0 || st + c > N) bad(cnt);
    if (i <= inner) {
      const int64_t h1 = (c + 1) / 2;
      if (nstart[2 * i] != st || ncount[2 * i] != h1 || nstart[2 * i + 1] != st + h1 || ncount[2 * i + 1] != c - h1)
        bad(cnt);
    }
  }
}

__global__ void k_check_perm_count(const int32_t* __restrict__ perm, int64_t N, uint32_t* __restrict__ seen,
                                   Counters* cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = perm[k];
    if (i < 0 || (int64_t)i >= N) bad(cnt);
    else atomicAdd(&seen[i], 1u);
  }
}

__global__ void k_check_perm_once(const uint32_t* __restrict__ seen, int64_t N, Counters* cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    if (seen[i] != 1u) bad(cnt);
}

// A work order: nodes 1 .. C, each exactly once, in C slots.
__global__ void k_check_order_count(const int32_t* __restrict__ order, int64_t C, uint32_t* __restrict__ seen,
                                    Counters* cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < C; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[k];
    if (v < 1 || (int64_t)v > C) bad(cnt);
    else atomicAdd(&seen[v - 1], 1u);
  }
}

// One list: keys (major << shift | minor), CSR offsets by major [C + 2].
__global__ void k_check_list(const uint64_t* __restrict__ keys, int64_t count, const int32_t* __restrict__ off,
                             int64_t C, int shift, bool leaves_only, int kappa, const int64_t* __restrict__ ncount,
                             Counters* cnt) {
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const int64_t leaf0 = (int64_t)1 << kappa;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = tid; t <= C; t += stride)  // offsets non-decreasing, from 0 to count
    if (off[t] > off[t + 1]) bad(cnt);
  if (tid == 0 && (off[0] != 0 || (int64_t)off[C + 1] != count)) bad(cnt);
  for (int64_t e = tid; e < count; e += stride) {
    const uint64_t k = keys[e];
    const int64_t a = (int64_t)(k >> shift), b = (int64_t)(k & mask);
    if (a < 1 || a > C || b < 1 || b > C || (leaves_only && (a < leaf0 || b < leaf0))) {
      bad(cnt);
      continue;
    }
    if (e + 1 < count && !(keys[e + 1] > k)) bad(cnt);
    if (!((int64_t)off[a] <= e && e < (int64_t)off[a + 1])) bad(cnt);
    atomicAdd(&cnt->cover, (unsigned long long)ncount[a] * (unsigned long long)ncount[b]);
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(div_up(n, 256), 2048)); }

}  // namespace

int run_bounds_check(fmm_plan_s* P, bool source_major, cudaStream_t s) {
  const Layout& L = P->lay;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  const int64_t* nstart = ws_ptr<int64_t>(P, L.nstart);
  const int64_t* ncount = ws_ptr<int64_t>(P, L.ncount);
  const int shift = P->kappa + 1;
  FMM_CUDA_TRY(cudaMemsetAsync(&cnt->cover, 0, sizeof(cnt->cover), s));
  if (!source_major) {
    k_check_nodes<<<grid_for(P->C), 256, 0, s>>>(nstart, ncount, P->C, P->kappa, P->N, cnt);
    FMM_LAUNCH_CHECK();
    // the rank arrays are free once the tree is built: N counters
    uint32_t* seen = ws_ptr<uint32_t>(P, L.rank);
    FMM_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(uint32_t) * P->N, s));
    k_check_perm_count<<<grid_for(P->N), 256, 0, s>>>(ws_ptr<int32_t>(P, L.perm), P->N, seen, cnt);
    FMM_LAUNCH_CHECK();
    k_check_perm_once<<<grid_for(P->N), 256, 0, s>>>(seen, P->N, cnt);
    FMM_LAUNCH_CHECK();
  }
  {  // the M2L work order of this list direction is a permutation of the nodes
    uint32_t* seen = ws_ptr<uint32_t>(P, L.rank);
    FMM_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(uint32_t) * P->C, s));
    k_check_order_count<<<grid_for(P->C), 256, 0, s>>>(ws_ptr<int32_t>(P, source_major ? L.m2l_sorder : L.m2l_order),
                                                        P->C, seen, cnt);
    FMM_LAUNCH_CHECK();
    k_check_perm_once<<<grid_for(P->C), 256, 0, s>>>(seen, P->C, cnt);
    FMM_LAUNCH_CHECK();
  }
  const size_t kp = source_major ? L.p2p_src : L.p2p, km = source_major ? L.m2l_src : L.m2l;
  const size_t op = source_major ? L.p2p_soff : L.p2p_off, om = source_major ? L.m2l_soff : L.m2l_off;
  k_check_list<<<grid_for(std::max<int64_t>(P->p2p_count, P->C + 2)), 256, 0, s>>>(
      ws_ptr<uint64_t>(P, kp), P->p2p_count, ws_ptr<int32_t>(P, op), P->C, shift, true, P->kappa, ncount, cnt);
  FMM_LAUNCH_CHECK();
  k_check_list<<<grid_for(std::max<int64_t>(P->m2l_count, P->C + 2)), 256, 0, s>>>(
      ws_ptr<uint64_t>(P, km), P->m2l_count, ws_ptr<int32_t>(P, om), P->C, shift, false, P->kappa, ncount, cnt);
  FMM_LAUNCH_CHECK();
  Counters hc;
  FMM_CUDA_TRY(cudaMemcpyAsync(&hc, cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned long long n2 = (unsigned long long)P->N * (unsigned long long)P->N;
  if ((hc.err & kErrBounds) || hc.cover != n2) return FMM_EBOUNDS;
  return FMM_OK;
}

}  // namespace fmm
