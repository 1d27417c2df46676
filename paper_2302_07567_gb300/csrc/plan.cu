// C ABI: plans, workspace, forward pass driver (Alg. 12), statistics, export.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "common.cuh"

namespace fmm {

static thread_local std::string g_last_cuda_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_last_cuda_error(cudaError_t e) {
  g_last_cuda_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
}

namespace {

std::mutex g_launch_mutex;
std::map<int, int> g_sms;                                           // device -> SMs
std::map<std::pair<int, const void*>, int> g_smem_limit;           // (device, kernel) -> raised limit
std::map<std::tuple<int, const void*, int, size_t>, int> g_per_sm;  // (device, kernel, threads, smem)

}  // namespace

int device_sms(int* sms) {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_launch_mutex);
  auto it = g_sms.find(dev);
  if (it == g_sms.end()) {
    int v = 0;
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    it = g_sms.emplace(dev, v).first;
  }
  *sms = it->second;
  return FMM_OK;
}

int smem_limit_raw(const void* kern, int bytes) {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_launch_mutex);
  int& cur = g_smem_limit[{dev, kern}];
  if (cur < bytes) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    cur = bytes;
  }
  return FMM_OK;
}

int blocks_per_sm_raw(const void* kern, int threads, size_t smem, int* per_sm) {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_launch_mutex);
  const auto key = std::make_tuple(dev, kern, threads, smem);
  auto it = g_per_sm.find(key);
  if (it == g_per_sm.end()) {
    int v = 0;
    FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem));
    it = g_per_sm.emplace(key, v).first;
  }
  *per_sm = it->second;
  return FMM_OK;
}

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

void make_layout(fmm_plan_s* P) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t N = (size_t)P->N, C1 = (size_t)P->C + 1, m = (size_t)P->m;
  const size_t R = P->precision == FMM_FP32 ? sizeof(float) : sizeof(double);
  const size_t V4 = 4 * R;
  // keys: the three presorts; keys_alt: their alternate buffer, then the
  // interaction lists grouped by major node while they are ordered
  const int64_t sort_n = std::max<int64_t>(3 * P->N, 1);
  const int64_t alt_n = std::max<int64_t>({3 * P->N, P->cap_p2p + P->cap_m2l, 1});
  const int64_t tiles = 3 * radix_tiles(P->N);
  const int64_t nblk_part = div_up(P->N, 2048);
  L.nblk_sort = (size_t)tiles;
  L.nblk_part = (size_t)nblk_part;
  L.counters = take(sizeof(Counters));
  L.scal = take(16 * sizeof(double));
  const size_t np0 = (size_t)div_up(P->N, 2048);
  L.psum_part = take(3 * 2 * (np0 + 2) * sizeof(double));
  L.qmax_part = take((np0 + 2) * sizeof(double));
  L.keys = take(sort_n * 8);
  L.keys_alt = take(alt_n * 8);
  L.vals = take(3 * N * 4);
  L.vals_alt = take(3 * N * 4);
  L.hist = take((size_t)256 * tiles * 4);
  L.scan_tmp = take((size_t)scan_tmp_words(std::max<int64_t>(256 * tiles, nblk_part)) * 4 + 1024);
  L.A = take(3 * N * 4);
  L.A_alt = take(3 * N * 4);
  L.rank = take(3 * N * 4);
  L.blocksum = take(3 * (size_t)nblk_part * 4);
  L.nstart = take(C1 * 8);
  L.ncount = take(C1 * 8);
  L.nleftpre = take(C1 * 8);
  L.nlo = take(C1 * 3 * 8);
  L.nhi = take(C1 * 3 * 8);
  L.naxis = take(C1 * 4);
  L.nmed = take(C1 * 4);
  L.ncen = take(C1 * 3 * 8);
  L.ndiam = take(C1 * 8);
  L.ngeo = take(C1 * sizeof(NodeGeo));
  L.perm = take(N * 4);
  L.px = take(N * V4);
  L.pb = take(N * V4);
  L.pl = take(N * V4);
  // Expansions.  FMM_RECOMPUTE keeps one set: the adjoint's node weights W
  // overwrite the locals L (both [C+1][6][m]) and its adjoint moments Lambda
  // the multipoles M (both [C+1][4][m]; with the gbar term M2L^T reads M, so
  // Lambda keeps a buffer of its own).  The M2L source table exists only for
  // the generic M2L kernel.
  const bool rec = (P->flags & FMM_RECOMPUTE) != 0;
  L.mpole = take(C1 * 4 * m * R);
  L.local = take(C1 * 6 * m * R);
  L.srct = take(m2l_specialised(P) ? 0 : C1 * m * 2 * V4);
  L.tmat = take(C1 * 3 * (size_t)P->np1 * P->np1 * R);
  L.front0 = take((size_t)P->cap_frontier * 8);
  L.front1 = take((size_t)P->cap_frontier * 8);
  L.p2p = take((size_t)P->cap_p2p * 8);
  L.m2l = take((size_t)P->cap_m2l * 8);
  L.p2p_off = take((C1 + 1) * 4);
  L.m2l_off = take((C1 + 1) * 4);
  L.p2p_src = take((size_t)P->cap_p2p * 8);
  L.m2l_src = take((size_t)P->cap_m2l * 8);
  L.p2p_soff = take((C1 + 1) * 4);
  L.p2p_dc = take((size_t)P->cap_p2p * 32);
  L.m2l_dc = take((size_t)P->cap_m2l * 32);
  L.m2l_soff = take((C1 + 1) * 4);
  // adjoint: per particle the scaled weights and the target-side position
  // gradient, per source-major list pair a centre offset; the node weights W
  // and adjoint moments Lambda have buffers of their own (wbuf, lbuf below)
  L.adj_part = take(N * V4);
  L.wle = take(N * V4);
  L.wlb = take(N * V4);
  L.tcnt = take(4 * (C1 + 1) * 4);
  L.tpart = take(2 * (size_t)kTravPartials * 4);
  L.thist = take(4 * 256 * 4);
  L.m2l_order = take(C1 * 4);
  L.m2l_sorder = take(C1 * 4);
  L.wbuf = rec ? L.local : take(C1 * 6 * m * R);
  L.lbuf = rec && !(P->flags & FMM_GBAR_TERM) ? L.mpole : take(C1 * 4 * m * R);
  L.p2p_sdc = take((size_t)P->cap_p2p * 32);
  L.m2l_sdc = take((size_t)P->cap_m2l * 32);
  L.gfar = take(C1 * 8);
  L.adj_part2 = take(N * V4);
  L.gpart = take((size_t)kGbarBlocks * 8);
  L.total = off;
  P->lay = L;
}

void make_tables(fmm_plan_s* P) {
  const int64_t C = P->C;
  P->node_start.assign(C + 1, 0);
  P->node_count.assign(C + 1, 0);
  P->node_leftpre.assign(C + 1, 0);
  P->node_start[1] = 0;
  P->node_count[1] = P->N;
  for (int l = 0; l < P->kappa; ++l) {
    int64_t pre = 0;
    for (int64_t i = (int64_t)1 << l; i < ((int64_t)2 << l); ++i) {
      const int64_t c = P->node_count[i], h1 = (c + 1) / 2;
      P->node_leftpre[i] = pre;
      pre += h1;
      P->node_start[2 * i] = P->node_start[i];
      P->node_count[2 * i] = h1;
      P->node_start[2 * i + 1] = P->node_start[i] + h1;
      P->node_count[2 * i + 1] = c - h1;
    }
  }
  Cheb& ch = P->cheb;
  std::memset(&ch, 0, sizeof(ch));
  ch.n = P->n;
  ch.np1 = P->np1;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k <= P->n; ++k) {
    // cos(k pi / n) written as sin(pi (n - 2k) / (2n)): exact symmetry, exact 0
    ch.t[k] = std::sin(pi * (double)(P->n - 2 * k) / (2.0 * P->n));
    ch.w[k] = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == P->n) ? 0.5 : 1.0);
  }
  ChebD& cd = P->chebd;
  std::memset(&cd, 0, sizeof(cd));
  const int np1 = P->np1;
  for (int a = 0; a < np1; ++a) {
    double diag = 0.0;
    for (int k = 0; k < np1; ++k) {
      if (k == a) continue;
      const double v = (ch.w[k] / ch.w[a]) / (ch.t[a] - ch.t[k]);
      cd.D[a * np1 + k] = v;
      diag -= v;
    }
    cd.D[a * np1 + a] = diag;
  }
  for (int k = 0; k < np1; ++k) {
    ch.tf[k] = (float)ch.t[k];
    ch.wf[k] = (float)ch.w[k];
  }
  for (int k = 0; k < np1 * np1; ++k) cd.Df[k] = (float)cd.D[k];
}

// Default list capacities (cluster pairs): 128 P2P partners per leaf and 64
// M2L pairs per cluster (the 2^24 core-halo beam at gamma 200 needs 114 and
// 24; the gamma-50 cylinder 12 and 1).  A list that overflows is grown by
// the caller (fmm_plan_set_capacity) and the call repeated.
void default_caps(fmm_plan_s* P) {
  if (P->cap_p2p <= 0) P->cap_p2p = 128 * P->nleaves + 1024;
  if (P->cap_m2l <= 0) P->cap_m2l = 64 * P->C + 1024;
  if (P->cap_frontier <= 0) P->cap_frontier = P->cap_p2p + P->cap_m2l;
}

int ensure_events(fmm_plan_s* P) {
  if (P->ev_made) return FMM_OK;
  for (auto& e : P->ev) FMM_CUDA_TRY(cudaEventCreate(&e));
  P->ev_made = true;
  return FMM_OK;
}

int record(fmm_plan_s* P, int k, cudaStream_t s) { return record_stage(P, k, s); }

// Drops the recorded step (fmm_step_graph_*).
void drop_graphs(fmm_plan_s* P) {
  if (P->graph_fwd) cudaGraphExecDestroy(P->graph_fwd);
  if (P->graph_adj) cudaGraphExecDestroy(P->graph_adj);
  P->graph_fwd = P->graph_adj = nullptr;
  P->graph_fwd_kernels = P->graph_adj_kernels = 0;
}

}  // namespace

int record_stage(fmm_plan_s* P, int k, cudaStream_t s) {
  if (!(P->flags & FMM_TIMING) || !P->ev_made) return FMM_OK;
  FMM_CUDA_TRY(cudaEventRecord(P->ev[k], s));
  return FMM_OK;
}

int ensure_side(fmm_plan_s* P) {
  if (P->side) return FMM_OK;
  int least = 0, greatest = 0;
  FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  FMM_CUDA_TRY(cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, greatest));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming));
  return FMM_OK;
}
}  // namespace fmm

using namespace fmm;

extern "C" {

int fmm_version(void) { return 1; }

size_t fmm_stats_bytes(void) { return sizeof(fmm_stats); }

int64_t fmm_kernel_launches(void) { return (int64_t)g_launches.load(); }

const char* fmm_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

const char* fmm_strerror(int status) {
  switch (status) {
    case FMM_OK: return "ok";
    case FMM_EINVAL: return "invalid argument";
    case FMM_ENOWORKSPACE: return "no or too small workspace attached";
    case FMM_EOVERFLOW: return "interaction-list capacity exceeded";
    case FMM_ENONFINITE: return "non-finite value in x or p";
    case FMM_ESTATE: return "adjoint called without a successful forward call";
    case FMM_ECUDA: return "CUDA runtime error";
    case FMM_EBOUNDS: return "device index check failed";
    default: return "unknown status";
  }
}

int fmm_plan_create(fmm_plan_t* out, int64_t N, int degree, int leaf_size, double eta, int precision,
                    unsigned flags) {
  if (!out) return FMM_EINVAL;
  *out = nullptr;
  if (N < 1 || N > ((int64_t)1 << 30)) return FMM_EINVAL;
  if (degree < 1 || degree > kMaxDegree) return FMM_EINVAL;
  if (leaf_size < 2 || leaf_size > 4096) return FMM_EINVAL;
  if (!(eta > 0.0) || !std::isfinite(eta)) return FMM_EINVAL;
  if (precision != FMM_FP32 && precision != FMM_FP64) return FMM_EINVAL;
  if (flags & ~(unsigned)(FMM_RECOMPUTE | FMM_BOUNDS_CHECK | FMM_TIMING | FMM_SIZE_AWARE | FMM_TEST_POLY_KERNEL |
                          FMM_GBAR_TERM | FMM_SERIAL))
    return FMM_EINVAL;
  if ((flags & FMM_TEST_POLY_KERNEL) && precision != FMM_FP64) return FMM_EINVAL;
  fmm_plan_s* P = new (std::nothrow) fmm_plan_s();
  if (!P) return FMM_EINVAL;
  P->N = N;
  P->n = degree;
  P->np1 = degree + 1;
  P->m = P->np1 * P->np1 * P->np1;
  P->leaf = leaf_size;
  P->eta = eta;
  P->precision = precision;
  P->flags = flags;
  int kappa = 0;
  if (N > leaf_size) {
    while ((int64_t)leaf_size * ((int64_t)1 << kappa) < N) ++kappa;
  }
  P->kappa = kappa;
  P->C = ((int64_t)2 << kappa) - 1;
  P->nleaves = (int64_t)1 << kappa;
  P->overlap = !(flags & FMM_SERIAL);
  default_caps(P);
  make_tables(P);
  make_layout(P);
  *out = P;
  return FMM_OK;
}

int fmm_plan_set_capacity(fmm_plan_t P, int64_t p2p_pairs, int64_t m2l_pairs, int64_t frontier_pairs) {
  if (!P || p2p_pairs < 0 || m2l_pairs < 0 || frontier_pairs < 0) return FMM_EINVAL;
  if (p2p_pairs > 0) P->cap_p2p = p2p_pairs;
  if (m2l_pairs > 0) P->cap_m2l = m2l_pairs;
  if (frontier_pairs > 0) P->cap_frontier = frontier_pairs;
  default_caps(P);
  make_layout(P);
  drop_graphs(P);  // they record the old workspace's addresses
  P->ws = nullptr;
  P->ws_bytes = 0;
  P->have_forward = false;
  return FMM_OK;
}

int fmm_plan_workspace_bytes(fmm_plan_t P, size_t* bytes) {
  if (!P || !bytes) return FMM_EINVAL;
  *bytes = P->lay.total;
  return FMM_OK;
}

int fmm_plan_set_workspace(fmm_plan_t P, void* dev, size_t bytes) {
  if (!P || !dev) return FMM_EINVAL;
  if (bytes < P->lay.total || ((uintptr_t)dev & 255u)) return FMM_ENOWORKSPACE;
  drop_graphs(P);  // they record the old workspace's addresses
  P->ws = static_cast<char*>(dev);
  P->ws_bytes = bytes;
  P->have_forward = false;
  const size_t tb = sizeof(int64_t) * (size_t)(P->C + 1);
  FMM_CUDA_TRY(cudaMemcpy(P->ws + P->lay.nstart, P->node_start.data(), tb, cudaMemcpyHostToDevice));
  FMM_CUDA_TRY(cudaMemcpy(P->ws + P->lay.ncount, P->node_count.data(), tb, cudaMemcpyHostToDevice));
  FMM_CUDA_TRY(cudaMemcpy(P->ws + P->lay.nleftpre, P->node_leftpre.data(), tb, cudaMemcpyHostToDevice));
  return FMM_OK;
}

}  // extern "C"

namespace fmm {
namespace {
// Alg. 12.  With reuse the tree's membership and the lists of the last
// forward stay: the boxes, gbar and everything after them are recomputed,
// and kStaleLists is returned (E, B unwritten) if an M2L pair is no longer
// admissible.
constexpr int kStaleLists = -1;

// The list sizes, device error flags and scalars a forward copied to the
// pinned slot after its traversal (the copy must have completed).
int check_counters(fmm_plan_s* P, bool reuse) {
  const Counters* hc = static_cast<const Counters*>(P->hpin);
  const double* hs = reinterpret_cast<const double*>(static_cast<const char*>(P->hpin) + 256);
  if (!reuse) {  // with reuse the lists, their sizes and pair counts stay those of the last forward
    P->p2p_count = (int64_t)hc->p2p_count;
    P->m2l_count = (int64_t)hc->m2l_count;
    P->p2p_work = (double)hc->p2p_work;
  }
  if (hc->err & kErrNonFinite) return FMM_ENONFINITE;
  if (hc->err & kErrStale) return kStaleLists;
  if ((hc->err & (kErrOvfFrontier | kErrOvfP2P | kErrOvfM2L)) || P->p2p_count > P->cap_p2p ||
      P->m2l_count > P->cap_m2l)
    return FMM_EOVERFLOW;
  P->gbar = hs[0];
  P->munit = hs[1];
  P->lunit = hs[2];
  return FMM_OK;
}

int forward(fmm_plan_s* P, const double* x, const double* p, const double* q, void* E, void* B, cudaStream_t s,
            bool reuse) {
  P->have_forward = false;
  P->last_stream = s;
  int rc;
  if (P->flags & FMM_TIMING) {
    if ((rc = ensure_events(P)) != FMM_OK) return rc;
  }
  if ((rc = record(P, 0, s)) != FMM_OK) return rc;
  if ((rc = run_setup(P, x, p, q, s)) != FMM_OK) return rc;
  if ((rc = record(P, 1, s)) != FMM_OK) return rc;
  if ((rc = reuse ? run_refresh(P, x, s) : run_tree(P, x, s)) != FMM_OK) return rc;
  if ((rc = run_prep(P, x, p, q, s)) != FMM_OK) return rc;
  if ((rc = record(P, 2, s)) != FMM_OK) return rc;
  // The upward pass and the traversal are independent, but the traversal is
  // one cooperative launch, which the GPU does not run beside other kernels
  // (measured: a side-stream upward pass then waits for it), so they run in turn.
  if ((rc = run_upward(P, s)) != FMM_OK) return rc;
  if ((rc = record(P, 17, s)) != FMM_OK) return rc;
  if ((rc = reuse ? run_refresh_lists(P, s) : run_traverse(P, s)) != FMM_OK) return rc;
  if ((rc = record(P, 3, s)) != FMM_OK) return rc;
  // The list sizes, error flags and scalars go to pinned host memory right
  // after the traversal, and M2L, L2L and P2P are queued at once: the host
  // waits only for that copy, the GPU not at all.  On an error the M2L and
  // P2P kernels return at their first instruction (they read the device error
  // word), so nothing indexes through an incomplete list and E, B stay
  // unwritten.  FMM_BOUNDS_CHECK needs the sizes first and waits before.
  if (!P->hpin) {
    FMM_CUDA_TRY(cudaHostAlloc(&P->hpin, 256 + 8 * sizeof(double), cudaHostAllocDefault));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&P->trav_ev, cudaEventDisableTiming));
  }
  Counters* hc = static_cast<Counters*>(P->hpin);
  double* hs = reinterpret_cast<double*>(static_cast<char*>(P->hpin) + 256);
  static_assert(sizeof(Counters) <= 256, "counters fit the pinned slot");
  FMM_CUDA_TRY(cudaMemcpyAsync(hc, P->ws + P->lay.counters, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaMemcpyAsync(hs, P->ws + P->lay.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  // (not while recording: an event recorded into a graph cannot be waited on
  // afterwards, and the replay is waited on as a whole)
  if (!P->capturing) FMM_CUDA_TRY(cudaEventRecord(P->trav_ev, s));
  auto read_back = [&]() -> int {
    FMM_CUDA_TRY(cudaEventSynchronize(P->trav_ev));
    return check_counters(P, reuse);
  };
  const bool wait_first = (P->flags & FMM_BOUNDS_CHECK) != 0;
  if (wait_first) {
    if ((rc = read_back()) != FMM_OK) return rc;
    if ((rc = run_bounds_check(P, false, s)) != FMM_OK) return rc;
  }
  if ((rc = record(P, 4, s)) != FMM_OK) return rc;
  if ((rc = record(P, 5, s)) != FMM_OK) return rc;
  // FP32: the near-field P2P needs only the lists, so it runs on the
  // caller's stream while M2L and L2L (launched per level, as a cooperative
  // launch would wait for the P2P kernel) run on the plan's high-priority
  // side stream (with FMM_SERIAL the three run in turn on the caller's
  // stream).  L2P and the output follow when both are done.  FP64 and the
  // polynomial test kernel keep the fused P2P + L2P after M2L and L2L.
  const bool split = P->precision == FMM_FP32 && !(P->flags & FMM_TEST_POLY_KERNEL) && P->kappa > 0;
  if (split) {
    cudaStream_t t = s;
    if (P->overlap) {
      if ((rc = ensure_side(P)) != FMM_OK) return rc;
      t = P->side;
      FMM_CUDA_TRY(cudaEventRecord(P->fork_ev, s));
      FMM_CUDA_TRY(cudaStreamWaitEvent(t, P->fork_ev, 0));
      if ((rc = record(P, 5, t)) != FMM_OK) return rc;
    }
    if ((rc = run_m2l(P, t)) != FMM_OK) return rc;
    if ((rc = record(P, 6, t)) != FMM_OK) return rc;
    if ((rc = run_l2l(P, t, P->overlap)) != FMM_OK) return rc;
    if ((rc = record(P, 7, t)) != FMM_OK) return rc;
    if (P->overlap) FMM_CUDA_TRY(cudaEventRecord(P->join_ev, t));
    if ((rc = run_p2p_near(P, s)) != FMM_OK) return rc;
    if ((rc = record(P, 18, s)) != FMM_OK) return rc;
    if (P->overlap) FMM_CUDA_TRY(cudaStreamWaitEvent(s, P->join_ev, 0));
    if ((rc = record(P, 19, s)) != FMM_OK) return rc;
    if ((rc = run_l2p_far(P, E, B, s)) != FMM_OK) return rc;
    if ((rc = record(P, 8, s)) != FMM_OK) return rc;
  } else {
    if ((rc = run_m2l(P, s)) != FMM_OK) return rc;
    if ((rc = record(P, 6, s)) != FMM_OK) return rc;
    if ((rc = run_l2l(P, s)) != FMM_OK) return rc;
    if ((rc = record(P, 7, s)) != FMM_OK) return rc;
    if ((rc = run_p2p_l2p(P, E, B, s)) != FMM_OK) return rc;
    if ((rc = record(P, 8, s)) != FMM_OK) return rc;
  }
  P->split_fwd = split;
  // while recording a step the host waits for nothing: fmm_step_graph_launch
  // reads the counters after the replay
  if (!wait_first && !P->capturing && (rc = read_back()) != FMM_OK) return rc;
  P->have_forward = true;
  P->transposed_valid = false;
  P->locals_valid = true;
  return FMM_OK;
}

}  // namespace
}  // namespace fmm

extern "C" {

int fmm_field(fmm_plan_t P, const double* x, const double* p, const double* q, void* E, void* B, void* stream) {
  if (!P || !x || !p || !q || !E || !B) return FMM_EINVAL;
  if (!P->ws) return FMM_ENOWORKSPACE;
  P->reuse_stale = false;
  return forward(P, x, p, q, E, B, static_cast<cudaStream_t>(stream), false);
}

int fmm_field_reuse(fmm_plan_t P, const double* x, const double* p, const double* q, void* E, void* B, void* stream,
                    int* rebuilt) {
  if (!P || !x || !p || !q || !E || !B) return FMM_EINVAL;
  if (!P->ws) return FMM_ENOWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rebuilt) *rebuilt = 0;
  // A call right after a stale attempt builds at once instead of trying
  // again: where the kept lists go stale every step the wasted attempts are
  // then every second step only.
  const bool attempt = P->have_forward && !P->reuse_stale;
  P->reuse_stale = false;
  if (attempt) {
    const int rc = forward(P, x, p, q, E, B, s, true);
    if (rc != kStaleLists) return rc;
    P->reuse_stale = true;
  }
  if (rebuilt) *rebuilt = 1;
  return forward(P, x, p, q, E, B, s, false);
}

int fmm_field_adjoint(fmm_plan_t P, const double* x, const double* p, const double* q, const void* wE,
                      const void* wB, double* dx, double* dp, double* dq, void* stream) {
  if (!P || !x || !p || !q || !wE || !wB || !dx || !dp || !dq) return FMM_EINVAL;
  if (!P->ws) return FMM_ENOWORKSPACE;
  if (!P->have_forward) return FMM_ESTATE;
  if (P->flags & FMM_TEST_POLY_KERNEL) return FMM_EINVAL;  // the adjoint is of the physical kernel only
  return run_adjoint(P, x, p, q, wE, wB, dx, dp, dq, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace fmm {
namespace {
// Records what `body` queues on s into an instantiated graph; the kernel
// launches it counted are taken back off the launch counter (recorded, not
// run) and returned in *kernels.
template <typename F>
int record_graph(fmm_plan_s* P, cudaStream_t s, F body, cudaGraphExec_t* out, long long* kernels) {
  *out = nullptr;
  const long long before = g_launches.load();
  FMM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  P->capturing = true;
  const int rc = body();
  P->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  const long long n = g_launches.load() - before;
  g_launches.fetch_sub(n);
  if (rc != FMM_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc != FMM_OK) return rc;
    set_last_cuda_error(ce);
    return FMM_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *out = nullptr;
    set_last_cuda_error(ie);
    return FMM_ECUDA;
  }
  *kernels = n;
  return FMM_OK;
}
}  // namespace
}  // namespace fmm

extern "C" {

int fmm_step_graph_create(fmm_plan_t P, const double* x, const double* p, const double* q, const void* wE,
                          const void* wB, void* E, void* B, double* dx, double* dp, double* dq, void* stream) {
  if (!P || !x || !p || !q || !E || !B) return FMM_EINVAL;
  const bool adj = wE != nullptr;
  if (adj && (!wB || !dx || !dp || !dq)) return FMM_EINVAL;
  if (!P->ws) return FMM_ENOWORKSPACE;
  if (P->flags & (FMM_TIMING | FMM_BOUNDS_CHECK)) return FMM_EINVAL;  // host-side timing or waits
  if (adj && (P->flags & FMM_TEST_POLY_KERNEL)) return FMM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return FMM_EINVAL;  // not recordable
  drop_graphs(P);
  // the step once as usual: it makes the plan's events, side stream and
  // pinned slot, the per-device launch facts, and returns the step's errors
  int rc = fmm_field(P, x, p, q, E, B, stream);
  if (rc == FMM_OK && adj) rc = fmm_field_adjoint(P, x, p, q, wE, wB, dx, dp, dq, stream);
  if (rc != FMM_OK) return rc;
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  P->reuse_stale = false;
  rc = record_graph(P, s, [&]() { return forward(P, x, p, q, E, B, s, false); }, &P->graph_fwd,
                    &P->graph_fwd_kernels);
  if (rc == FMM_OK && adj)
    rc = record_graph(P, s, [&]() { return run_adjoint(P, x, p, q, wE, wB, dx, dp, dq, s); }, &P->graph_adj,
                      &P->graph_adj_kernels);
  if (rc != FMM_OK) {
    drop_graphs(P);
    P->have_forward = false;
    return rc;
  }
  P->graph_locals_valid = P->locals_valid;
  return FMM_OK;
}

int fmm_step_graph_launch(fmm_plan_t P, void* stream) {
  if (!P) return FMM_EINVAL;
  if (!P->graph_fwd || !P->ws) return FMM_ESTATE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  P->have_forward = false;
  FMM_CUDA_TRY(cudaGraphLaunch(P->graph_fwd, s));
  g_launches.fetch_add(P->graph_fwd_kernels);
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  P->last_stream = s;
  int rc = check_counters(P, false);
  if (rc != FMM_OK) return rc;
  P->have_forward = true;
  P->transposed_valid = false;
  P->locals_valid = true;
  if (P->graph_adj) {
    FMM_CUDA_TRY(cudaGraphLaunch(P->graph_adj, s));
    g_launches.fetch_add(P->graph_adj_kernels);
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    P->transposed_valid = true;
    P->locals_valid = P->graph_locals_valid;
  }
  return FMM_OK;
}

int fmm_step_graph_destroy(fmm_plan_t P) {
  if (!P) return FMM_EINVAL;
  drop_graphs(P);
  return FMM_OK;
}

int fmm_plan_stats(fmm_plan_t P, fmm_stats* out) {
  if (!P || !out) return FMM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->N = P->N;
  out->nodes = P->C;
  out->leaves = P->nleaves;
  out->degree = P->n;
  out->leaf_size = P->leaf;
  out->kappa = P->kappa;
  out->precision = P->precision;
  out->eta = P->eta;
  out->gbar = P->gbar;
  out->length_unit = P->lunit;
  out->mass_unit = P->munit;
  out->p2p_pairs = P->p2p_count;
  out->m2l_pairs = P->m2l_count;
  out->cap_p2p = P->cap_p2p;
  out->cap_m2l = P->cap_m2l;
  out->cap_frontier = P->cap_frontier;
  out->m2l_interactions = (double)P->m2l_count * (double)P->m * (double)P->m;
  // sum |S_t| |S_s| over the P2P pairs, counted by the traversal kernel
  if (P->have_forward) out->p2p_interactions = P->p2p_work - (double)P->N;
  if ((P->flags & FMM_TIMING) && P->ev_made) {
    FMM_CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    for (int k = 0; k < 16; ++k) P->stage_ms[k] = 0.0;
    auto el = [&](int a, int b) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, P->ev[a], P->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
      }
      return (double)ms;
    };
    P->stage_ms[0] = el(0, 1);
    P->stage_ms[1] = el(1, 2);
    P->stage_ms[2] = el(2, 17);  // upward pass
    P->stage_ms[17] = el(2, 9);  // its P2M
    P->stage_ms[3] = el(17, 3);  // traversal and lists
    P->stage_ms[4] = el(3, 5);   // copy of the list sizes to the host
    P->stage_ms[5] = el(5, 6);
    P->stage_ms[6] = el(6, 7);
    if (P->split_fwd) {
      // near-field P2P: beside M2L and L2L, or after them
      P->stage_ms[7] = P->overlap ? el(5, 18) : el(7, 18);
      P->stage_ms[16] = el(19, 8);  // L2P and the output
    } else {
      P->stage_ms[7] = el(7, 8);
      P->stage_ms[16] = 0.0;
    }
    P->stage_ms[13] = el(0, 8);
    if (P->adj_timed) {
      // the near-field kernel runs on the caller's stream from event 16 while
      // L2P^T .. M2M^T run on the side stream (order 0), after them (order
      // 1, FMM_SERIAL) or before them (order 2, FMM_RECOMPUTE where the
      // near-field kernel reads the leaf locals: FP64, the gbar term); the
      // source side starts when both have finished
      const int ord = P->adj_chain ? P->adj_order : 2;
      P->stage_ms[11] = ord == 1 ? el(13, 10) : el(16, 10);  // near-field particle kernel
      if (P->adj_chain) {
        P->stage_ms[8] = ord == 2 ? el(10, 11) : el(16, 11);  // L2P^T + L2L^T
        P->stage_ms[9] = el(11, 12);   // M2L^T
        P->stage_ms[10] = el(12, 13);  // M2M^T
        P->stage_ms[12] = ord == 0 ? std::min(el(10, 14), el(13, 14)) : (ord == 1 ? el(10, 14) : el(13, 14));
      } else {
        P->stage_ms[12] = el(10, 14);
      }
      P->stage_ms[14] = el(15, 14);  // whole adjoint call
      P->stage_ms[15] = el(15, 16);  // source-major lists, recompute if asked, weights, FP32 target-side far field
    }
    for (int k = 0; k < 18; ++k) out->stage_ms[k] = P->stage_ms[k];
  }
  return FMM_OK;
}

int fmm_plan_export(fmm_plan_t P, int what, void* host, size_t bytes) {
  if (!P || !host) return FMM_EINVAL;
  if (!P->ws || !P->have_forward) return FMM_ESTATE;
  const int64_t C = P->C, N = P->N, m = P->m;
  FMM_CUDA_TRY(cudaStreamSynchronize(P->last_stream));
  const Layout& L = P->lay;
  const bool f32 = P->precision == FMM_FP32;
  auto need = [&](size_t b) { return bytes >= b; };
  switch (what) {
    case FMM_EXPORT_GBAR: {
      if (!need(8)) return FMM_EINVAL;
      std::memcpy(host, &P->gbar, 8);
      return FMM_OK;
    }
    case FMM_EXPORT_PERM: {
      if (!need(4 * N)) return FMM_EINVAL;
      FMM_CUDA_TRY(cudaMemcpy(host, P->ws + L.perm, 4 * N, cudaMemcpyDeviceToHost));
      return FMM_OK;
    }
    case FMM_EXPORT_NODES: {
      if (!need(16 * C)) return FMM_EINVAL;
      int64_t* o = static_cast<int64_t*>(host);
      for (int64_t i = 1; i <= C; ++i) {
        o[2 * (i - 1)] = P->node_start[i];
        o[2 * (i - 1) + 1] = P->node_count[i];
      }
      return FMM_OK;
    }
    case FMM_EXPORT_BBOX: {
      if (!need(48 * C)) return FMM_EINVAL;
      std::vector<double> lo(3 * (C + 1)), hi(3 * (C + 1));
      FMM_CUDA_TRY(cudaMemcpy(lo.data(), P->ws + L.nlo, 8 * lo.size(), cudaMemcpyDeviceToHost));
      FMM_CUDA_TRY(cudaMemcpy(hi.data(), P->ws + L.nhi, 8 * hi.size(), cudaMemcpyDeviceToHost));
      double* o = static_cast<double*>(host);
      for (int64_t i = 1; i <= C; ++i)
        for (int k = 0; k < 3; ++k) {
          o[6 * (i - 1) + k] = lo[3 * i + k];
          o[6 * (i - 1) + 3 + k] = hi[3 * i + k];
        }
      return FMM_OK;
    }
    case FMM_EXPORT_AXIS: {
      if (!need(4 * C)) return FMM_EINVAL;
      std::vector<int32_t> ax(C + 1);
      FMM_CUDA_TRY(cudaMemcpy(ax.data(), P->ws + L.naxis, 4 * ax.size(), cudaMemcpyDeviceToHost));
      std::memcpy(host, ax.data() + 1, 4 * C);
      return FMM_OK;
    }
    case FMM_EXPORT_P2P:
    case FMM_EXPORT_M2L: {
      const int64_t n = what == FMM_EXPORT_P2P ? P->p2p_count : P->m2l_count;
      if (!need(8 * n)) return FMM_EINVAL;
      std::vector<uint64_t> keys((size_t)n);
      if (n > 0)
        FMM_CUDA_TRY(cudaMemcpy(keys.data(), P->ws + (what == FMM_EXPORT_P2P ? L.p2p : L.m2l), 8 * n,
                                cudaMemcpyDeviceToHost));
      const int shift = P->kappa + 1;
      const uint64_t mask = ((uint64_t)1 << shift) - 1;
      int32_t* o = static_cast<int32_t*>(host);
      for (int64_t e = 0; e < n; ++e) {
        o[2 * e] = (int32_t)(keys[e] >> shift);
        o[2 * e + 1] = (int32_t)(keys[e] & mask);
      }
      return FMM_OK;
    }
    case FMM_EXPORT_MULTIPOLE:
    case FMM_EXPORT_LOCAL: {
      if (!P->locals_valid) return FMM_ESTATE;  // an FMM_RECOMPUTE adjoint overwrote them
      const int nc = what == FMM_EXPORT_MULTIPOLE ? 4 : 6;
      if (!need(sizeof(double) * C * nc * m)) return FMM_EINVAL;
      const size_t cnt = (size_t)(C + 1) * nc * m;
      std::vector<double> buf(cnt);
      const size_t off = what == FMM_EXPORT_MULTIPOLE ? L.mpole : L.local;
      if (f32) {
        std::vector<float> tmp(cnt);
        FMM_CUDA_TRY(cudaMemcpy(tmp.data(), P->ws + off, 4 * cnt, cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < cnt; ++e) buf[e] = tmp[e];
      } else {
        FMM_CUDA_TRY(cudaMemcpy(buf.data(), P->ws + off, 8 * cnt, cudaMemcpyDeviceToHost));
      }
      const double mu = P->munit, g = P->gbar, il2 = 1.0 / (P->lunit * P->lunit);
      double sc[6];
      if (nc == 4) {
        sc[0] = mu; sc[1] = g * mu; sc[2] = g * mu; sc[3] = mu;
      } else {
        sc[0] = mu * il2; sc[1] = mu * il2; sc[2] = mu * il2 / g;
        sc[3] = mu * il2; sc[4] = mu * il2; sc[5] = mu * il2 * g;
      }
      double* o = static_cast<double*>(host);
      for (int64_t i = 1; i <= C; ++i)
        for (int c = 0; c < nc; ++c)
          for (int64_t v = 0; v < m; ++v)
            o[((i - 1) * nc + c) * m + v] = sc[c] * buf[((size_t)i * nc + c) * m + v];
      return FMM_OK;
    }
    default:
      return FMM_EINVAL;
  }
}

void fmm_plan_destroy(fmm_plan_t P) {
  if (!P) return;
  drop_graphs(P);
  if (P->ev_made)
    for (auto& e : P->ev) cudaEventDestroy(e);
  if (P->hpin) {
    cudaEventSynchronize(P->trav_ev);
    cudaEventDestroy(P->trav_ev);
    cudaFreeHost(P->hpin);
  }
  if (P->side) {
    cudaStreamSynchronize(P->side);
    cudaStreamDestroy(P->side);
    cudaEventDestroy(P->fork_ev);
    cudaEventDestroy(P->join_ev);
  }
  (void)cudaGetLastError();  // the teardown is best effort: leave no error for the next call to report
  delete P;
}

}  // extern "C"
