// Shared definitions of the CUDA translation units of the GB300 FMM.
//
// Coordinates inside the library.  After the tree is built every stage works
// in "stretched, scaled" coordinates: x' = (x, y, gbar z) / ell, with ell a
// power of two near the root box size.  In these coordinates the relativistic
// kernel of Eq. 3.2 becomes the Coulomb kernel R'/|R'|^3 followed by a
// diagonal rescale: g = ell^-2 diag(1, 1, 1/gbar) R'/|R'|^3.  The masses are
// scaled by a power of two mu near max|q|: a' = q gamma / mu and
// b~' = (q p_x / gbar, q p_y / gbar, q p_z) / mu, for which
// b x g = ell^-2 diag(1, 1, gbar) (b~' x R') / |R'|^3 * mu.  Powers of two
// make the scaling exact in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fmm.h"

namespace fmm {

constexpr int kMaxDegree = 12;
constexpr int kMaxNp1 = kMaxDegree + 1;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kC0 = 299792458.0;

// device error bits (Counters::err)
enum : unsigned {
  kErrNonFinite = 1u,
  kErrOvfFrontier = 2u,
  kErrOvfP2P = 4u,
  kErrOvfM2L = 8u,
  kErrBounds = 16u,
  kErrStale = 32u,  // field with reuse: an M2L pair is no longer admissible
};

// Device-resident counters of one call (first bytes of the workspace).
// Blocks a cooperative traversal launch may use (scan partials reserved per list).
constexpr int64_t kTravPartials = 4096;
constexpr int kGbarBlocks = 512;  // most blocks of the dL/dgbar partial sums
// Blocks per SM of the transfer launches (M2M, L2L and their transposes):
// the cooperative launch over all levels takes at most 4 (more make its
// grid-wide barriers dearer than the extra blocks help the deepest levels),
// the per-level launches beside another kernel at most 8 (no grid barrier;
// measured at 2^9 leaves: 1.2% faster step than 4, 2 slower).
constexpr int kCoopTransferCap = 4;
constexpr int kLevelTransferCap = 8;

struct Counters {
  unsigned long long p2p_count;
  unsigned long long m2l_count;
  unsigned long long frontier_count[3];  // rotating: step k reads [k%3], appends to [(k+1)%3]
  unsigned int err;
  unsigned int work[2];  // item counters of the dynamically scheduled M2L and M2L^T launches
  unsigned int pad[1];
  unsigned long long cover;  // FMM_BOUNDS_CHECK: sum of |S_t| |S_s| over the list pairs
  unsigned long long p2p_work;  // sum of |S_t| |S_s| over the P2P pairs (traversal)
};

// Chebyshev points of the second kind t_k = cos(k pi / n) and their
// barycentric weights w_k = (-1)^k delta_k (delta = 1/2 at both ends), passed
// to kernels by value.
struct Cheb {
  int n;
  int np1;
  double t[kMaxNp1];
  double w[kMaxNp1];
  // the same nodes and weights rounded to FP32 on the host: the FP32
  // kernels read them as they are (a conversion from FP64 runs on the FP64
  // unit, a small fraction of the FP32 rate)
  float tf[kMaxNp1];
  float wf[kMaxNp1];
};

// Differentiation matrix of the Lagrange basis on the Chebyshev points:
// D[m][k] = l_k'(t_m), so l_k'(t) = sum_m l_m(t) D[m][k] exactly (l_k' has
// degree n - 1 and is reproduced by the interpolation, Theorem 1).
struct ChebD {
  double D[kMaxNp1 * kMaxNp1];
  float Df[kMaxNp1 * kMaxNp1];  // D rounded to FP32 on the host
};

// The tables in the arithmetic's precision.
template <typename T>
__device__ __forceinline__ T cheb_node(const Cheb& ch, int k);
template <>
__device__ __forceinline__ float cheb_node<float>(const Cheb& ch, int k) { return ch.tf[k]; }
template <>
__device__ __forceinline__ double cheb_node<double>(const Cheb& ch, int k) { return ch.t[k]; }
template <typename T>
__device__ __forceinline__ T cheb_weight(const Cheb& ch, int k);
template <>
__device__ __forceinline__ float cheb_weight<float>(const Cheb& ch, int k) { return ch.wf[k]; }
template <>
__device__ __forceinline__ double cheb_weight<double>(const Cheb& ch, int k) { return ch.w[k]; }
template <typename T>
__device__ __forceinline__ T cheb_diff(const ChebD& cd, int i);
template <>
__device__ __forceinline__ float cheb_diff<float>(const ChebD& cd, int i) { return cd.Df[i]; }
template <>
__device__ __forceinline__ double cheb_diff<double>(const ChebD& cd, int i) { return cd.D[i]; }

// Per-node geometry in stretched, scaled coordinates (FP64).
struct NodeGeo {
  double c[3];  // box centre
  double h[3];  // half widths (0 for a side of zero width)
};

// ------------------------------------------------------------- workspace
struct Layout {
  size_t total = 0;
  // every field is a byte offset into the workspace
  size_t counters, scal, psum_part, qmax_part;
  size_t keys, keys_alt, vals, vals_alt, hist, scan_tmp;
  size_t A, A_alt, rank, blocksum;
  size_t nstart, ncount, nleftpre, nlo, nhi, naxis, nmed, ncen, ndiam, ngeo;
  size_t perm, px, pb, pl;         // leaf-order particles (pl: low parts, FP32 only)
  size_t p2p_dc, m2l_dc;           // per list pair: centre offset c_t - c_s as (hi, lo)
  size_t mpole, local, srct, tmat;
  size_t front0, front1, p2p, m2l, p2p_off, m2l_off, p2p_src, m2l_src, p2p_soff, m2l_soff;
  size_t adj_part;                 // per particle: target-side position gradient (leaf order)
  size_t wbuf, lbuf;               // adjoint expansions: W [C+1][6][m] and Lambda [C+1][4][m]
  size_t wle, wlb;                 // per particle: scaled loss weights (leaf order)
  size_t p2p_sdc, m2l_sdc;         // centre offsets of the source-major lists
  size_t tcnt, tpart;               // list ordering: per-node counts and fills, scan partials
  size_t thist, m2l_order, m2l_sorder;  // M2L work orders: count buckets, targets, sources
  size_t gfar, gpart;  // adjoint with the gbar term: per-cluster far-field sums, block partials
  size_t adj_part2;    // FP32 adjoint: dL/db~' of the fused near field, per particle
  size_t nblk_sort;   // radix tiles of the three presorts
  size_t nblk_part;   // partition blocks at N
};

}  // namespace fmm

struct fmm_plan_s {
  int64_t N = 0;
  int n = 0, np1 = 0, m = 0, leaf = 0, precision = 0;
  unsigned flags = 0;
  double eta = 0.0;
  int kappa = 0;
  int64_t C = 0, nleaves = 0;
  int64_t cap_p2p = 0, cap_m2l = 0, cap_frontier = 0;
  std::vector<int64_t> node_start, node_count, node_leftpre;  // index 0 unused
  fmm::Layout lay;
  fmm::Cheb cheb;
  fmm::ChebD chebd;
  bool transposed_valid = false;  // source-major lists built for the current forward
  bool locals_valid = false;      // multipole / local buffers hold the forward's values (an
                                  // FMM_RECOMPUTE adjoint overwrites them with W and Lambda)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool have_forward = false;
  int64_t p2p_count = 0, m2l_count = 0;
  double p2p_work = 0.0;          // sum |S_t| |S_s| over the P2P pairs of the last forward
  double gbar = 0.0, lunit = 1.0, munit = 1.0;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[20] = {};
  bool ev_made = false;
  cudaStream_t side = nullptr;    // second stream for independent branches (higher priority)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  void* hpin = nullptr;           // pinned host copy of the counters and scalars after the traversal
  cudaEvent_t trav_ev = nullptr;  // recorded after that copy
  double stage_ms[18] = {};
  bool overlap = true;     // independent branches on two streams (no FMM_SERIAL)
  bool split_fwd = false;  // the last forward ran the FP32 near field and L2P as kernels of their own
  bool reuse_stale = false;  // the last fmm_field_reuse found the kept lists stale
  bool adj_timed = false;  // the last adjoint recorded its stage events
  bool adj_chain = false;  // ... and had a far-field chain (kappa > 0)
  bool adj_overlap = false;  // the running adjoint has its two branches on two streams
  int adj_order = 0;       // stage order of the last adjoint: 0 branches overlapped, 1 chain then
                           // near field (FMM_SERIAL), 2 near field then chain (FMM_RECOMPUTE)
  // a recorded step (fmm_step_graph_*): the forward and, if recorded, the adjoint
  cudaGraphExec_t graph_fwd = nullptr, graph_adj = nullptr;
  long long graph_fwd_kernels = 0, graph_adj_kernels = 0;  // kernel launches of one replay
  bool graph_locals_valid = false;  // locals_valid after a replayed step
  bool capturing = false;           // forward / adjoint are being recorded: no host waits
};

namespace fmm {

template <typename T>
inline T* ws_ptr(const fmm_plan_s* p, size_t off) {
  return reinterpret_cast<T*>(p->ws + off);
}

void set_last_cuda_error(cudaError_t e);
void count_launch();

#define FMM_CUDA_TRY(expr)                          \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) {                        \
      ::fmm::set_last_cuda_error(_e);               \
      return FMM_ECUDA;                             \
    }                                               \
  } while (0)

#define FMM_LAUNCH_CHECK()                          \
  do {                                              \
    ::fmm::count_launch();                          \
    cudaError_t _e = cudaGetLastError();            \
    if (_e != cudaSuccess) {                        \
      ::fmm::set_last_cuda_error(_e);               \
      return FMM_ECUDA;                             \
    }                                               \
  } while (0)

inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// ------------------------------------------------------------- device helpers
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
// 1/sqrt(x) by the hardware approximation (rsqrt.approx) for a normal
// positive float.  rsqrtf also rescales subnormal inputs, which costs extra
// instructions in the inner loops; every FP32 caller here passes
// x >= tiny_sep2<float>() = 2^-84 (masked or clamped), far above the
// subnormal range, where the flush-to-zero form returns the same value.
__device__ __forceinline__ float rsqrt_normal(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrt_normal(x); }
// 1/x by the hardware approximation (rcp.approx) for a normal positive
// float, on the transcendental unit instead of the FMA pipe: r^-3 as
// rsqrt(d) rcp(d) takes one FMA-pipe multiply instead of two.
__device__ __forceinline__ float rcp_normal(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

// Squared separations (stretched, scaled units) at or below this count as a
// coincident pair whose contribution is zero: 2^-84 in FP32 (below it r^-3
// would overflow), 2^-100 in FP64.  Distinct particles closer than
// 2^-42 (FP32) or 2^-50 (FP64) of the length unit are treated as coincident.
template <typename T>
__host__ __device__ __forceinline__ T tiny_sep2();
template <>
__host__ __device__ __forceinline__ float tiny_sep2<float>() { return 5.169878828456423e-26f; }
template <>
__host__ __device__ __forceinline__ double tiny_sep2<double>() { return 7.888609052210118e-31; }

// Values of the n+1 Lagrange basis polynomials at the normalised coordinate
// t in [-1, 1] (second, "true" barycentric form).  `degenerate` marks a box
// side of zero width, whose basis is l_0 = 1, l_k = 0.  A coordinate that
// coincides with a point t_k (to within `tiny`) gives the cardinal vector e_k.
template <typename T>
__device__ __forceinline__ void bary_basis(T t, bool degenerate, const Cheb& ch, T* out) {
  const int np1 = ch.np1;
  const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-300);
  int hit = degenerate ? 0 : -1;
  if (!degenerate) {
    for (int k = 0; k < np1; ++k) {
      T d = t - cheb_node<T>(ch, k);
      if (hit < 0 && fabs(d) <= tiny) hit = k;
    }
  }
  if (hit >= 0) {
    for (int k = 0; k < np1; ++k) out[k] = (k == hit) ? T(1) : T(0);
    return;
  }
  T s = T(0);
  for (int k = 0; k < np1; ++k) {
    T v = cheb_weight<T>(ch, k) / (t - cheb_node<T>(ch, k));
    out[k] = v;
    s += v;
  }
  T inv = T(1) / s;
  for (int k = 0; k < np1; ++k) out[k] *= inv;
}

// bary_basis in FP32 with the points per axis fixed at compile time (the
// same formula), so that callers keep the values in registers.
template <int NP1>
__device__ __forceinline__ void bary_basis_n(float t, bool degenerate, const Cheb& ch, float (&out)[NP1]) {
  int hit = degenerate ? 0 : -1;
  if (!degenerate) {
#pragma unroll
    for (int k = 0; k < NP1; ++k)
      if (hit < 0 && fabsf(t - ch.tf[k]) <= 1e-30f) hit = k;
  }
  if (hit >= 0) {
#pragma unroll
    for (int k = 0; k < NP1; ++k) out[k] = (k == hit) ? 1.f : 0.f;
    return;
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < NP1; ++k) {
    out[k] = ch.wf[k] / (t - ch.tf[k]);
    sum += out[k];
  }
  const float inv = 1.f / sum;
#pragma unroll
  for (int k = 0; k < NP1; ++k) out[k] *= inv;
}

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Kahan-compensated accumulation: (sum, comp) += v.
template <typename T>
__device__ __forceinline__ void kahan_add(T& sum, T& comp, T v) {
  T y = v - comp;
  T t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Launch facts of kernels on the current device.  A kernel's attributes
// (the raised dynamic shared-memory limit) and its occupancy belong to one
// device context, so they are kept per (device, kernel) in tables guarded by
// a mutex: plans on several devices of one process, or on several host
// threads, each get their own.  Every function works on the device that is
// current in the calling thread.
int device_sms(int* sms);
// Raise the kernel's dynamic shared-memory limit to at least `bytes` (once
// per device and kernel).
int smem_limit_raw(const void* kern, int bytes);
// Resident blocks per SM of the kernel at `threads` threads and `smem`
// dynamic shared bytes (computed once per device, kernel and shape).
int blocks_per_sm_raw(const void* kern, int threads, size_t smem, int* per_sm);

template <typename K>
inline int smem_limit(K* kern, int bytes) {
  return smem_limit_raw(reinterpret_cast<const void*>(kern), bytes);
}
template <typename K>
inline int blocks_per_sm(K* kern, int threads, size_t smem, int* per_sm) {
  return blocks_per_sm_raw(reinterpret_cast<const void*>(kern), threads, smem, per_sm);
}

// Blocks of a grid-stride launch of `kern`: as many as are resident at once
// at `threads` threads and `smem` dynamic shared bytes, at most `items`.
template <typename K>
inline int resident_blocks(K* kern, int threads, size_t smem, int64_t items, unsigned* grid) {
  int sms = 0, per_sm = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (int rc = blocks_per_sm(kern, threads, smem, &per_sm)) return rc;
  if (per_sm < 1) return FMM_EINVAL;
  *grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, items));
  return FMM_OK;
}

// Thread shape of the particle-pair kernels (forward P2P, adjoint target and
// source sides): blocks of `groups` groups of NT threads over chunks of
// kpt NT targets of a leaf, `chunks` blocks per leaf.
inline void particle_shape(int64_t leaf, int kpt, int* NT, int* groups, int* chunks) {
  const int64_t per_thread = (leaf + kpt - 1) / kpt;
  *NT = (int)std::min<int64_t>(64, (per_thread + 31) / 32 * 32);
  *groups = *NT <= 32 ? 4 : 2;
  *chunks = (int)((leaf + (int64_t)kpt * *NT - 1) / ((int64_t)kpt * *NT));
}

// Admissibility of the cluster pair (t, u) (Alg. 8 with Algs. 6-7):
// max(r_t, r_u) / d < eta in FP64 with the operations in a fixed order and
// no contraction, d the stretched centre distance; d = 0 gives inf or NaN,
// not admissible.  The traversal and the tracking refresh share it, so both
// take the same decision to the last bit.
__device__ __forceinline__ bool pair_admissible(const double* __restrict__ ndiam, const double* __restrict__ ncen,
                                                double gbar, int64_t t, int64_t u, double eta) {
  const double s[3] = {1.0, 1.0, gbar};
  const double rt = ndiam[t], ru = ndiam[u];
  double v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = __dmul_rn(s[k], __dsub_rn(ncen[3 * t + k], ncen[3 * u + k]));
  const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])),
                                        __dmul_rn(v[2], v[2])));
  const double ratio = __ddiv_rn(rt >= ru ? rt : ru, d);
  return ratio < eta;
}

// Centre offset s o (c_a - c_b) / ell of a list pair in stretched, scaled
// units, stored as hi + lo floats (FP32 plans) or a double4 (FP64 plans).
template <bool kFP32>
__device__ __forceinline__ void store_pair_offset(const double* __restrict__ ncen, const double* __restrict__ scal,
                                                  int64_t a, int64_t b, void* dc, int64_t dst) {
  const double s3[3] = {1.0, 1.0, scal[0]};
  const double inv = scal[3];
  const double* ca = ncen + 3 * a;
  const double* cb = ncen + 3 * b;
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = __dmul_rn(__dmul_rn(s3[k], __dsub_rn(ca[k], cb[k])), inv);
  if (kFP32) {
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      h[k] = (float)d[k];
      l[k] = (float)(d[k] - (double)h[k]);
    }
    float4* o = static_cast<float4*>(dc);
    o[2 * dst] = make_float4(h[0], h[1], h[2], 0.f);
    o[2 * dst + 1] = make_float4(l[0], l[1], l[2], 0.f);
  } else {
    static_cast<double4*>(dc)[dst] = make_double4(d[0], d[1], d[2], 0.0);
  }
}

// Node of a breadth-first tree level containing slot `pos`: binary search in
// the first slots of the 2^level nodes [first, first + count).
__device__ __forceinline__ int64_t find_node(const int64_t* __restrict__ nstart, int64_t first,
                                             int64_t count, int64_t pos) {
  int64_t lo = 0, hi = count - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (nstart[first + mid] <= pos) lo = mid; else hi = mid - 1;
  }
  return first + lo;
}

}  // namespace fmm

// ------------------------------------------------------------- stage entry points
namespace fmm {
int run_setup(fmm_plan_s* P, const double* x, const double* p, const double* q, cudaStream_t s);
int run_tree(fmm_plan_s* P, const double* x, cudaStream_t s);
int run_prep(fmm_plan_s* P, const double* x, const double* p, const double* q, cudaStream_t s);
// P2M, M2M (at most xfer_cap blocks per SM in the transfer) and the M2L source table
int run_upward(fmm_plan_s* P, cudaStream_t s, int xfer_cap = kCoopTransferCap, bool per_level = false);
// traversal and both target-major lists (sorted, CSR, centre offsets), one launch
int run_traverse(fmm_plan_s* P, cudaStream_t s);
int run_list_transpose(fmm_plan_s* P, cudaStream_t s);
// the plan's side stream and its fork / join events (created on first use)
int ensure_side(fmm_plan_s* P);
// FMM_TIMING: record the plan's stage event k on stream s (no-op otherwise)
int record_stage(fmm_plan_s* P, int k, cudaStream_t s);
// FMM_BOUNDS_CHECK: node tables, leaf order and lists (target- or source-major);
// synchronises the stream, FMM_EBOUNDS on any violation
int run_bounds_check(fmm_plan_s* P, bool source_major, cudaStream_t s);
int run_m2l(fmm_plan_s* P, cudaStream_t s);
// field with reuse (track.cu): the boxes of the kept tree membership at the
// new positions, then the lists' centre offsets and the admissibility of
// every M2L pair under them (kErrStale on failure)
int run_refresh(fmm_plan_s* P, const double* x, cudaStream_t s);
int run_refresh_lists(fmm_plan_s* P, cudaStream_t s);
// FP32 M2L with a kernel specialised on the points per axis (reads the
// multipoles directly); otherwise the generic kernel reads the source table
bool m2l_specialised(const fmm_plan_s* P);
int run_l2l(fmm_plan_s* P, cudaStream_t s, bool per_level = false);
int run_p2p_l2p(fmm_plan_s* P, void* E, void* B, cudaStream_t s);
// FP32 forward split: near-field P2P into the adjoint's per-particle buffers
// (free during the forward call), then L2P with the output transform
int run_p2p_near(fmm_plan_s* P, cudaStream_t s);
int run_l2p_far(fmm_plan_s* P, void* E, void* B, cudaStream_t s);
int run_adjoint(fmm_plan_s* P, const double* x, const double* p, const double* q, const void* wE,
                const void* wB, double* dx, double* dp, double* dq, cudaStream_t s);
// stable LSD radix sort of 64-bit keys with 32-bit values over bits
// [begin_bit, end_bit): nbatch independent sorts of n keys each, batch k at
// keys + k * stride; returns in `*in_alt` whether the result sits in the
// alternate buffers.
int radix_sort_batched(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t stride,
                       int nbatch, int64_t n, int begin_bit, int end_bit, uint32_t* hist, uint32_t* scan_tmp,
                       int64_t max_tiles, cudaStream_t s, bool* in_alt);
int scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s);
// per-node 1-D transfer matrices, and the separable transfers over all
// levels (see transfer.cu)
int run_tmats(fmm_plan_s* P, cudaStream_t s);
template <typename T, int NC, bool UP>
int run_transfer(fmm_plan_s* P, T* buf, cudaStream_t s, int max_blocks_per_sm, bool per_level);
int64_t radix_tiles(int64_t n);
int64_t scan_tmp_words(int64_t n);
}  // namespace fmm
