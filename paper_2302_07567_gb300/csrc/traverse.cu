// Dual tree traversal (Algs. 11 and 17) producing the P2P and M2L interaction
// lists, sorted by (target, source) and indexed by target (Section 10), and
// the source-major lists the adjoint reads.
//
// The recursion of Alg. 17 is run level-synchronously: a frontier of node
// pairs starts at (1, 1); every step classifies each pair exactly as Alg. 17
// does (leaf-leaf -> P2P; admissible -> M2L; else split the leaf's partner,
// or the pair member with the larger stretched diameter, the source on a
// tie) and appends the two child pairs to the next frontier.  Each step adds
// one level to one member of a pair, so 2 kappa + 1 steps empty the frontier.
// All steps run in one cooperative launch with a grid-wide barrier between
// them.  Appends go through atomic counters (order unspecified); the same
// launch then orders both lists: pairs are counted per target, the counts
// scanned into the CSR offsets, the pairs scattered into their target's
// segment, and every segment ranked by source (a pair's rank is the number of
// smaller keys in its segment, the keys being distinct).  The result is the
// order a sort by (target << bits | source) gives, whatever the append order.
// The centre offset of each pair is written as it reaches its final slot.
//
// Size-aware variant (FMM_SIZE_AWARE, not in the paper): an admissible pair
// with |S_t| |S_s| < m^2 particle pairs is cheaper and exact as a direct sum,
// so every leaf pair under it goes to the P2P list instead of M2L.
//
// The admissibility test is Alg. 8 with diam and dist of Algs. 6-7 in FP64
// with round-to-nearest operations in a fixed order and no contraction:
// max(r_t, r_s) / d < eta, d = sqrt((v_x^2 + v_y^2) + v_z^2), v = s o (c_t - c_s).
#include <cooperative_groups.h>

#include "common.cuh"

namespace fmm {
namespace {

namespace cg = cooperative_groups;

constexpr int kTravThreads = 256;
constexpr int kSegStage = 128;  // keys of one segment a warp ranks from shared memory
// Work order of a list's major nodes: counting sort by pair count, longest
// lists first (counts of kOrderBuckets - 1 and more share the first bucket).
// Kernels that give a block per major node walk this order, so the long
// lists start first and the short ones fill in behind them.
constexpr int kOrderBuckets = kTravThreads;
static_assert(kOrderBuckets == kTravThreads, "one bucket per thread in the bucket scan");

__device__ __forceinline__ int order_bucket(uint32_t count) {
  return kOrderBuckets - 1 - (int)min(count, (uint32_t)(kOrderBuckets - 1));
}

// One list to order: pairs key = (major << shift | minor), optionally swapped
// from (minor << shift | major), grouped and sorted by key.  Arrays written
// earlier in the same launch are read through L2 (__ldcg).
struct ListJob {
  const uint64_t* in;               // pairs to order
  const unsigned long long* n;      // their number (device counter)
  int64_t cap;                      // capacity of in, tmp, out and dc
  uint32_t* cnt;                    // [C + 2] pairs per major node
  uint32_t* fill;                   // [C + 2] pairs placed per major node
  int32_t* off;                     // [C + 2] CSR: first pair whose major is >= t
  uint64_t* tmp;                    // pairs grouped by major
  uint64_t* out;                    // pairs sorted by key
  void* dc;                         // s o (c_major - c_minor) / ell per pair
  int32_t* order;                   // [C] nodes 1..C by decreasing pair count, or null
  uint32_t* hb;                     // [kOrderBuckets] nodes per count bucket, then placed per bucket
};

struct ListArgs {
  ListJob job[2];
  bool swap;                        // order by source: key = (s << shift | t)
  int shift;
  int64_t C;
  const double* ncen;
  const double* scal;
  uint32_t* partial;                // [2][gridDim.x] scan partials
};

struct TravArgs {
  Counters* cnt;
  int2* front[2];
  int64_t cap_front;
  uint64_t* p2p;                    // unordered appends
  int64_t cap_p2p;
  uint64_t* m2l;
  int64_t cap_m2l;
  const double* ndiam;
  const int64_t* ncount;
  int64_t m2sub;                    // size-aware: admissible pairs below this many particle pairs go to P2P
  double eta;
  int kappa;
  ListArgs lists;
};

__device__ __forceinline__ void push(unsigned long long* counter, int64_t cap, uint64_t* list, uint64_t key,
                                     unsigned int* err, unsigned flag) {
  unsigned long long at = atomicAdd(counter, 1ull);
  if ((int64_t)at < cap) list[at] = key;
  else atomicOr(err, flag);
}

__device__ __forceinline__ uint64_t list_key(const ListArgs& a, const uint64_t* in, int64_t e) {
  const uint64_t k = __ldcg(reinterpret_cast<const unsigned long long*>(in) + e);
  if (!a.swap) return k;
  const uint64_t mask = ((uint64_t)1 << a.shift) - 1;
  return ((k & mask) << a.shift) | (k >> a.shift);
}

__device__ __forceinline__ int64_t list_count(const ListJob& j) {
  const int64_t n = (int64_t)__ldcg(j.n);
  return n < j.cap ? n : j.cap;
}

// Exclusive scan of one value per thread over the block; returns the block total.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* wt, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < nw ? wt[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) wt[lane] = wi - w;
    if (lane == nw - 1) wt[32] = wi;
  }
  __syncthreads();
  const uint32_t r = wt[warp] + inc - v;
  total = wt[32];
  __syncthreads();
  return r;
}

// Count, scan, scatter and rank both lists of `a` (every block of the grid).
template <bool kFP32>
__device__ void order_lists(cg::grid_group& grid, const ListArgs& a) {
  __shared__ uint32_t wt[33];
  __shared__ uint64_t stage[kTravThreads / 32][kSegStage];
  const int64_t M = a.C + 2;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int j = 0; j < 2; ++j) {
    for (int64_t i = gtid; i < M; i += gstride) {
      a.job[j].cnt[i] = 0;
      a.job[j].fill[i] = 0;
    }
    if (a.job[j].order)
      for (int64_t i = gtid; i < 2 * kOrderBuckets; i += gstride) a.job[j].hb[i] = 0;
  }
  grid.sync();
  for (int j = 0; j < 2; ++j) {
    const ListJob& J = a.job[j];
    const int64_t n = list_count(J);
    for (int64_t e = gtid; e < n; e += gstride) atomicAdd(&J.cnt[list_key(a, J.in, e) >> a.shift], 1u);
  }
  grid.sync();
  // CSR offsets: block b scans the chunk [b chunk, (b + 1) chunk) after the
  // partial sums of the chunks before it
  const int64_t chunk = (M + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * chunk, c1 = min64(M, c0 + chunk);
  for (int j = 0; j < 2; ++j) {
    uint32_t v = 0;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      const uint32_t c = __ldcg(a.job[j].cnt + i);
      v += c;
      if (a.job[j].order && i >= 1 && i <= a.C) atomicAdd(&a.job[j].hb[order_bucket(c)], 1u);
    }
    uint32_t tot;
    block_scan_excl(v, wt, tot);
    if (threadIdx.x == 0) a.partial[j * gridDim.x + blockIdx.x] = tot;
  }
  grid.sync();
  for (int j = 0; j < 2; ++j) {
    const ListJob& J = a.job[j];
    uint32_t v = 0;
    for (int64_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) v += __ldcg(a.partial + j * gridDim.x + b);
    uint32_t base;
    block_scan_excl(v, wt, base);
    for (int64_t i0 = c0; i0 < c1; i0 += blockDim.x) {
      const int64_t i = i0 + threadIdx.x;
      const uint32_t c = i < c1 ? __ldcg(J.cnt + i) : 0u;
      uint32_t t;
      const uint32_t ex = block_scan_excl(c, wt, t);
      if (i < c1) J.off[i] = (int32_t)(base + ex);
      base += t;
    }
    if (J.order) {  // place this chunk's nodes in the work order
      uint32_t tot;
      const uint32_t bstart = block_scan_excl(__ldcg(J.hb + threadIdx.x), wt, tot);
      __shared__ uint32_t bofs[kOrderBuckets];
      bofs[threadIdx.x] = bstart;
      __syncthreads();
      for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        if (i < 1 || i > a.C) continue;
        const int bk = order_bucket(__ldcg(J.cnt + i));
        J.order[bofs[bk] + atomicAdd(&J.hb[kOrderBuckets + bk], 1u)] = (int32_t)i;
      }
      __syncthreads();
    }
  }
  grid.sync();
  for (int j = 0; j < 2; ++j) {
    const ListJob& J = a.job[j];
    const int64_t n = list_count(J);
    for (int64_t e = gtid; e < n; e += gstride) {
      const uint64_t k = list_key(a, J.in, e);
      const int64_t t = (int64_t)(k >> a.shift);
      const int64_t pos = (int64_t)__ldcg(J.off + t) + atomicAdd(&J.fill[t], 1u);
      J.tmp[pos] = k;
    }
  }
  grid.sync();
  // rank every segment by key; one warp per major node
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = gtid >> 5, nwarps = gstride >> 5;
  const uint64_t mask = ((uint64_t)1 << a.shift) - 1;
  for (int64_t w = gw; w < 2 * M; w += nwarps) {
    const int j = w >= M ? 1 : 0;
    const int64_t t = w - j * M;
    if (t >= M - 1) continue;
    const ListJob& J = a.job[j];
    const int64_t lo = __ldcg(J.off + t), hi = __ldcg(J.off + t + 1);
    const int n = (int)(hi - lo);
    if (n <= 0) continue;
    const unsigned long long* seg = reinterpret_cast<const unsigned long long*>(J.tmp) + lo;
    const bool staged = n <= kSegStage;
    if (staged)
      for (int i = lane; i < n; i += 32) stage[wib][i] = __ldcg(seg + i);
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint64_t ki = staged ? stage[wib][i] : __ldcg(seg + i);
      int r = 0;
      for (int q = 0; q < n; ++q) r += (staged ? stage[wib][q] : __ldcg(seg + q)) < ki ? 1 : 0;
      const int64_t dst = lo + r;
      J.out[dst] = ki;
      store_pair_offset<kFP32>(a.ncen, a.scal, (int64_t)(ki >> a.shift), (int64_t)(ki & mask), J.dc, dst);
    }
    __syncwarp();
  }
}

template <bool kFP32>
__global__ void __launch_bounds__(kTravThreads) k_traverse(TravArgs a) {
  cg::grid_group grid = cg::this_grid();
  Counters* cnt = a.cnt;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.front[0][0] = make_int2(1, 1);
    cnt->frontier_count[0] = 1;
    cnt->frontier_count[1] = 0;
    cnt->frontier_count[2] = 0;
    cnt->p2p_count = 0;
    cnt->m2l_count = 0;
    cnt->p2p_work = 0;
  }
  grid.sync();
  unsigned long long work = 0;  // this thread's share of sum |S_t| |S_s| over the P2P pairs
  const int leaf0 = 1 << a.kappa;
  const int shift = a.lists.shift;
  const double* ncen = a.lists.ncen;
  const double s[3] = {1.0, 1.0, a.lists.scal[0]};
  const int steps = 2 * a.kappa + 1;
  for (int it = 0; it < steps; ++it) {
    const int2* fin = a.front[it & 1];
    int2* fout = a.front[(it + 1) & 1];
    const int64_t nin = (int64_t)__ldcg(&cnt->frontier_count[it % 3]);
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt->frontier_count[(it + 2) % 3] = 0;
    unsigned long long* nout = &cnt->frontier_count[(it + 1) % 3];
    const int64_t n = min64(nin, a.cap_front);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const int2 pr = __ldcg(fin + e);
      const int t = pr.x, u = pr.y;
      const bool lt = t >= leaf0, lu = u >= leaf0;
      if (lt && lu) {
        push(&cnt->p2p_count, a.cap_p2p, a.p2p, ((uint64_t)t << shift) | (uint64_t)u, &cnt->err, kErrOvfP2P);
        work += (unsigned long long)(a.ncount[t] * a.ncount[u]);
        continue;
      }
      const double rt = a.ndiam[t], ru = a.ndiam[u];
      if (pair_admissible(a.ndiam, ncen, s[2], t, u, a.eta)) {
        if (a.m2sub > 0 && a.ncount[t] * a.ncount[u] < a.m2sub) {
          // fewer particle pairs than proxy-point pairs: every leaf pair under
          // (t, u) goes to P2P instead (all leaves sit at depth kappa)
          const int dt = a.kappa - (31 - __clz(t)), du = a.kappa - (31 - __clz(u));
          const int64_t t0 = (int64_t)t << dt, u0 = (int64_t)u << du;
          const int64_t nt = (int64_t)1 << dt, nu = (int64_t)1 << du;
          const unsigned long long at = atomicAdd(&cnt->p2p_count, (unsigned long long)(nt * nu));
          work += (unsigned long long)(a.ncount[t] * a.ncount[u]);  // all leaf pairs under (t, u)
          if ((int64_t)at + nt * nu <= a.cap_p2p) {
            for (int64_t i = 0; i < nt; ++i)
              for (int64_t k = 0; k < nu; ++k)
                a.p2p[at + i * nu + k] = ((uint64_t)(t0 + i) << shift) | (uint64_t)(u0 + k);
          } else {
            atomicOr(&cnt->err, kErrOvfP2P);
          }
          continue;
        }
        push(&cnt->m2l_count, a.cap_m2l, a.m2l, ((uint64_t)t << shift) | (uint64_t)u, &cnt->err, kErrOvfM2L);
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
      if ((int64_t)at + 1 < a.cap_front) {
        fout[at] = c0;
        fout[at + 1] = c1;
      } else {
        atomicOr(&cnt->err, kErrOvfFrontier);
      }
    }
    grid.sync();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
  if ((threadIdx.x & 31) == 0 && work) atomicAdd(&cnt->p2p_work, work);
  // every block sees the same final flags: on any error no list is ordered
  if (__ldcg(&cnt->err) != 0u) return;
  order_lists<kFP32>(grid, a.lists);
}

template <bool kFP32>
__global__ void __launch_bounds__(kTravThreads) k_lists_src(ListArgs a) {
  cg::grid_group grid = cg::this_grid();
  order_lists<kFP32>(grid, a);
}

// Blocks of a cooperative launch of `kern`: all co-resident, at most `cap`,
// about one per `per_block` work items but at least one per SM.  A grid-wide
// barrier costs more the more blocks arrive at it, and a small tree's
// frontier fits in few blocks.
template <typename K>
int coop_grid(K* kern, int64_t cap, int64_t items, int64_t per_block, int* grid) {
  int sms = 0, per_sm = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (int rc = blocks_per_sm(kern, kTravThreads, 0, &per_sm)) return rc;
  if (per_sm < 1) return FMM_EINVAL;
  const int64_t want = std::max<int64_t>(sms, div_up(items, per_block));
  *grid = (int)std::min<int64_t>({(int64_t)per_sm * sms, cap, want});
  return FMM_OK;
}

ListArgs list_args(fmm_plan_s* P, bool swap) {
  const Layout& L = P->lay;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  ListArgs a;
  a.swap = swap;
  a.shift = P->kappa + 1;
  a.C = P->C;
  a.ncen = ws_ptr<double>(P, L.ncen);
  a.scal = ws_ptr<double>(P, L.scal);
  a.partial = ws_ptr<uint32_t>(P, L.tpart);
  uint32_t* tc = ws_ptr<uint32_t>(P, L.tcnt);
  const int64_t M = P->C + 2;
  uint64_t* tmp = ws_ptr<uint64_t>(P, L.keys_alt);
  for (int j = 0; j < 2; ++j) {
    ListJob& J = a.job[j];
    const bool p2p = j == 0;
    J.n = p2p ? &cnt->p2p_count : &cnt->m2l_count;
    J.cap = p2p ? P->cap_p2p : P->cap_m2l;
    J.cnt = tc + (2 * j) * M;
    J.fill = tc + (2 * j + 1) * M;
    J.tmp = tmp + (p2p ? 0 : P->cap_p2p);
    J.order = p2p ? nullptr : ws_ptr<int32_t>(P, swap ? L.m2l_sorder : L.m2l_order);
    J.hb = ws_ptr<uint32_t>(P, L.thist) + (size_t)(swap ? 2 : 0) * kOrderBuckets;
    if (!swap) {  // forward: raw appends (in the source-major buffers) -> target-major lists
      J.in = ws_ptr<uint64_t>(P, p2p ? L.p2p_src : L.m2l_src);
      J.out = ws_ptr<uint64_t>(P, p2p ? L.p2p : L.m2l);
      J.off = ws_ptr<int32_t>(P, p2p ? L.p2p_off : L.m2l_off);
      J.dc = P->ws + (p2p ? L.p2p_dc : L.m2l_dc);
    } else {      // adjoint: target-major lists -> source-major lists
      J.in = ws_ptr<uint64_t>(P, p2p ? L.p2p : L.m2l);
      J.out = ws_ptr<uint64_t>(P, p2p ? L.p2p_src : L.m2l_src);
      J.off = ws_ptr<int32_t>(P, p2p ? L.p2p_soff : L.m2l_soff);
      J.dc = P->ws + (p2p ? L.p2p_sdc : L.m2l_sdc);
    }
  }
  return a;
}

}  // namespace

int run_traverse(fmm_plan_s* P, cudaStream_t s) {
  const Layout& L = P->lay;
  TravArgs a;
  a.cnt = ws_ptr<Counters>(P, L.counters);
  a.front[0] = ws_ptr<int2>(P, L.front0);
  a.front[1] = ws_ptr<int2>(P, L.front1);
  a.cap_front = P->cap_frontier;
  a.p2p = ws_ptr<uint64_t>(P, L.p2p_src);
  a.cap_p2p = P->cap_p2p;
  a.m2l = ws_ptr<uint64_t>(P, L.m2l_src);
  a.cap_m2l = P->cap_m2l;
  a.ndiam = ws_ptr<double>(P, L.ndiam);
  a.ncount = ws_ptr<int64_t>(P, L.ncount);
  a.m2sub = (P->flags & FMM_SIZE_AWARE) ? (int64_t)P->m * P->m : 0;
  a.eta = P->eta;
  a.kappa = P->kappa;
  a.lists = list_args(P, false);
  const bool f32 = P->precision == FMM_FP32;
  void* kern = f32 ? (void*)k_traverse<true> : (void*)k_traverse<false>;
  int grid = 0;
  int rc = f32 ? coop_grid(k_traverse<true>, kTravPartials, P->nleaves, 8, &grid)
               : coop_grid(k_traverse<false>, kTravPartials, P->nleaves, 8, &grid);
  if (rc != FMM_OK) return rc;
  void* args[] = {&a};
  FMM_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kTravThreads), args, 0, s));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

// Source-major lists for the adjoint: pairs (s, t) sorted by (source,
// target), CSR by source, offsets c_s - c_t.
int run_list_transpose(fmm_plan_s* P, cudaStream_t s) {
  ListArgs a = list_args(P, true);
  const bool f32 = P->precision == FMM_FP32;
  void* kern = f32 ? (void*)k_lists_src<true> : (void*)k_lists_src<false>;
  int grid = 0;
  int rc = f32 ? coop_grid(k_lists_src<true>, kTravPartials, P->nleaves, 8, &grid)
               : coop_grid(k_lists_src<false>, kTravPartials, P->nleaves, 8, &grid);
  if (rc != FMM_OK) return rc;
  void* args[] = {&a};
  FMM_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kTravThreads), args, 0, s));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

}  // namespace fmm
