// Dual tree traversal (Algs. 11 and 17) producing the P2P and M2L interaction
// lists, sorted by (target, source) and indexed by target (Section 10).
//
// The recursion of Alg. 17 is run level-synchronously: a frontier of node
// pairs starts at (1, 1); every step classifies each pair exactly as Alg. 17
// does (leaf-leaf -> P2P; admissible -> M2L; else split the leaf's partner,
// or the pair member with the larger stretched diameter, the source on a
// tie) and appends the two child pairs to the next frontier.  Each step adds
// one level to one member of a pair, so 2 kappa + 1 steps empty the frontier.
// Appends go through atomic counters (order unspecified); the radix sort by
// (target << bits | source) afterwards makes the lists deterministic.
//
// The admissibility test is Alg. 8 with diam and dist of Algs. 6-7 in FP64
// with round-to-nearest operations in a fixed order and no contraction:
// max(r_t, r_s) / d < eta, d = sqrt((v_x^2 + v_y^2) + v_z^2), v = s o (c_t - c_s).
#include "common.cuh"

namespace fmm {
namespace {

__global__ void k_trav_init(Counters* cnt, int2* f0) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    f0[0] = make_int2(1, 1);
    cnt->frontier_count[0] = 1;
    cnt->frontier_count[1] = 0;
    cnt->frontier_count[2] = 0;
    cnt->p2p_count = 0;
    cnt->m2l_count = 0;
  }
}

__device__ __forceinline__ void push(unsigned long long* counter, int64_t cap, uint64_t* list, uint64_t key,
                                     unsigned int* err, unsigned flag) {
  unsigned long long at = atomicAdd(counter, 1ull);
  if ((int64_t)at < cap) list[at] = key;
  else atomicOr(err, flag);
}

__global__ void k_trav_step(const int2* __restrict__ fin, int it, int2* __restrict__ fout, Counters* cnt,
                            int64_t cap_front, uint64_t* __restrict__ p2p, int64_t cap_p2p,
                            uint64_t* __restrict__ m2l, int64_t cap_m2l, const double* __restrict__ ncen,
                            const double* __restrict__ ndiam, const double* __restrict__ scal, double eta,
                            int kappa, int shift) {
  const unsigned long long nin = cnt->frontier_count[it % 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt->frontier_count[(it + 2) % 3] = 0;
  unsigned long long* nout = &cnt->frontier_count[(it + 1) % 3];
  const int64_t n = min64((int64_t)nin, cap_front);
  const int leaf0 = 1 << kappa;
  const double s[3] = {1.0, 1.0, scal[0]};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = fin[e];
    const int t = pr.x, u = pr.y;
    const bool lt = t >= leaf0, lu = u >= leaf0;
    if (lt && lu) {
      push(&cnt->p2p_count, cap_p2p, p2p, ((uint64_t)t << shift) | (uint64_t)u, &cnt->err, kErrOvfP2P);
      continue;
    }
    const double rt = ndiam[t], ru = ndiam[u];
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = __dmul_rn(s[k], __dsub_rn(ncen[3 * t + k], ncen[3 * u + k]));
    const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])),
                                          __dmul_rn(v[2], v[2])));
    const double ratio = __ddiv_rn(rt >= ru ? rt : ru, d);
    if (ratio < eta) {
      push(&cnt->m2l_count, cap_m2l, m2l, ((uint64_t)t << shift) | (uint64_t)u, &cnt->err, kErrOvfM2L);
      continue;
    }
    int2 c0, c1;
    if (lt || (!lu && !(rt > ru))) {  // split the source
      c0 = make_int2(t, 2 * u);
      c1 = make_int2(t, 2 * u + 1);
    } else {                          // split the target
      c0 = make_int2(2 * t, u);
      c1 = make_int2(2 * t + 1, u);
    }
    unsigned long long at = atomicAdd(nout, 2ull);
    if ((int64_t)at + 1 < cap_front) {
      fout[at] = c0;
      fout[at + 1] = c1;
    } else {
      atomicOr(&cnt->err, kErrOvfFrontier);
    }
  }
}

// off[t] = first list index whose target is >= t, for t = 0 .. C+1.
__global__ void k_csr(const uint64_t* __restrict__ keys, int64_t count, int shift, int64_t C,
                      int32_t* __restrict__ off) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > C + 1) return;
  const uint64_t key = (uint64_t)t << shift;
  int64_t lo = 0, hi = count;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  off[t] = (int32_t)lo;
}

// Source-major copy of a list: (t << shift | s) -> (s << shift | t).
__global__ void k_swap_pairs(const uint64_t* __restrict__ in, int64_t count, int shift,
                             uint64_t* __restrict__ out) {
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = in[e];
    out[e] = ((k & mask) << shift) | (k >> shift);
  }
}

// Centre offset c_t - c_s of every list pair in stretched, scaled units,
// s o (c_t - c_s) / ell with the difference taken in physical FP64
// coordinates.  FP32 plans store it as an unevaluated sum hi + lo of two
// float4 rows, FP64 plans as one double4.
template <bool kFP32>
__global__ void k_pair_dc(const uint64_t* __restrict__ keys, int64_t count, int shift,
                          const double* __restrict__ ncen, const double* __restrict__ scal, void* __restrict__ out) {
  const uint64_t mask = ((uint64_t)1 << shift) - 1;
  const double s[3] = {1.0, 1.0, scal[0]};
  const double inv = scal[3];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[e];
    const double* ct = ncen + 3 * (k >> shift);
    const double* cs = ncen + 3 * (k & mask);
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = (s[d] * (ct[d] - cs[d])) * inv;
    if (kFP32) {
      float h[3], l[3];
      for (int d = 0; d < 3; ++d) {
        h[d] = (float)dc[d];
        l[d] = (float)(dc[d] - (double)h[d]);
      }
      float4* o = static_cast<float4*>(out);
      o[2 * e] = make_float4(h[0], h[1], h[2], 0.f);
      o[2 * e + 1] = make_float4(l[0], l[1], l[2], 0.f);
    } else {
      static_cast<double4*>(out)[e] = make_double4(dc[0], dc[1], dc[2], 0.0);
    }
  }
}

}  // namespace

int pair_offsets(fmm_plan_s* P, size_t keys_off, int64_t count, size_t out_off, cudaStream_t s) {
  if (count <= 0) return FMM_OK;
  const Layout& L = P->lay;
  const int shift = P->kappa + 1;
  const unsigned g = (unsigned)std::min<int64_t>(div_up(count, 256), 4096);
  if (P->precision == FMM_FP32)
    k_pair_dc<true><<<g, 256, 0, s>>>(ws_ptr<uint64_t>(P, keys_off), count, shift, ws_ptr<double>(P, L.ncen),
                                      ws_ptr<double>(P, L.scal), P->ws + out_off);
  else
    k_pair_dc<false><<<g, 256, 0, s>>>(ws_ptr<uint64_t>(P, keys_off), count, shift, ws_ptr<double>(P, L.ncen),
                                       ws_ptr<double>(P, L.scal), P->ws + out_off);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int run_pair_offsets(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  int rc = pair_offsets(P, L.p2p, P->p2p_count, L.p2p_dc, s);
  if (rc != FMM_OK) return rc;
  return pair_offsets(P, L.m2l, P->m2l_count, L.m2l_dc, s);
}

int run_traverse(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  int2* f[2] = {ws_ptr<int2>(P, L.front0), ws_ptr<int2>(P, L.front1)};
  k_trav_init<<<1, 32, 0, s>>>(cnt, f[0]);
  FMM_LAUNCH_CHECK();
  const int shift = P->kappa + 1;
  const int steps = 2 * P->kappa + 1;
  for (int it = 0; it < steps; ++it) {
    k_trav_step<<<152 * 4, 256, 0, s>>>(f[it & 1], it, f[(it + 1) & 1], cnt, P->cap_frontier,
                                         ws_ptr<uint64_t>(P, L.p2p), P->cap_p2p, ws_ptr<uint64_t>(P, L.m2l),
                                         P->cap_m2l, ws_ptr<double>(P, L.ncen), ws_ptr<double>(P, L.ndiam),
                                         ws_ptr<double>(P, L.scal), P->eta, P->kappa, shift);
    FMM_LAUNCH_CHECK();
  }
  return FMM_OK;
}

// Sort one list in place (keys sorted by the packed pair), build its CSR.
static int sort_list(fmm_plan_s* P, uint64_t* list, int64_t count, int32_t* off, cudaStream_t s) {
  const Layout& L = P->lay;
  const int shift = P->kappa + 1;
  bool alt = false;
  int rc = radix_sort(list, ws_ptr<uint64_t>(P, L.keys_alt), nullptr, nullptr, count, 0, 2 * shift,
                      ws_ptr<uint32_t>(P, L.hist), ws_ptr<uint32_t>(P, L.scan_tmp), (int64_t)L.nblk_sort, s, &alt);
  if (rc != FMM_OK) return rc;
  if (alt && count > 0) {
    FMM_CUDA_TRY(cudaMemcpyAsync(list, ws_ptr<uint64_t>(P, L.keys_alt), sizeof(uint64_t) * count,
                                 cudaMemcpyDeviceToDevice, s));
  }
  k_csr<<<(unsigned)div_up(P->C + 2, 256), 256, 0, s>>>(list, count, shift, P->C, off);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int run_list_sort(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  int rc = sort_list(P, ws_ptr<uint64_t>(P, L.p2p), P->p2p_count, ws_ptr<int32_t>(P, L.p2p_off), s);
  if (rc != FMM_OK) return rc;
  return sort_list(P, ws_ptr<uint64_t>(P, L.m2l), P->m2l_count, ws_ptr<int32_t>(P, L.m2l_off), s);
}

// Source-major lists for the adjoint: the transposed pairs, sorted, with CSR by source.
int run_list_transpose(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  const int shift = P->kappa + 1;
  const int gs = 1024;
  if (P->p2p_count > 0) {
    k_swap_pairs<<<gs, 256, 0, s>>>(ws_ptr<uint64_t>(P, L.p2p), P->p2p_count, shift, ws_ptr<uint64_t>(P, L.p2p_src));
    FMM_LAUNCH_CHECK();
  }
  if (P->m2l_count > 0) {
    k_swap_pairs<<<gs, 256, 0, s>>>(ws_ptr<uint64_t>(P, L.m2l), P->m2l_count, shift, ws_ptr<uint64_t>(P, L.m2l_src));
    FMM_LAUNCH_CHECK();
  }
  int rc = sort_list(P, ws_ptr<uint64_t>(P, L.p2p_src), P->p2p_count, ws_ptr<int32_t>(P, L.p2p_soff), s);
  if (rc != FMM_OK) return rc;
  rc = sort_list(P, ws_ptr<uint64_t>(P, L.m2l_src), P->m2l_count, ws_ptr<int32_t>(P, L.m2l_soff), s);
  if (rc != FMM_OK) return rc;
  // offsets c_s - c_t of the source-major pairs (s, t)
  rc = pair_offsets(P, L.p2p_src, P->p2p_count, L.p2p_sdc, s);
  if (rc != FMM_OK) return rc;
  return pair_offsets(P, L.m2l_src, P->m2l_count, L.m2l_sdc, s);
}

}  // namespace fmm
