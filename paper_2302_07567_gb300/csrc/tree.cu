// Setup and cluster tree (Section 3 averages; Algs. 1-2; Appendix B; Section 8).
//
// gbar: the mean momentum is summed by the adjacent-pair binary tree over
// 2^ceil(log2 N) zero-padded terms, so gbar is the same to the last bit
// whatever the launch shape, and the tree and traversal decisions that depend
// on it are reproducible.
//
// Tree: the particles are sorted once along each axis by (coordinate, input
// index).  Three index arrays A_x, A_y, A_z are kept, each holding every
// node's members as a contiguous slot range sorted along its own axis.  For a
// node the bounding box of Section 2 is then read off the end slots of the
// three arrays, the split axis of Alg. 1 is argmax_k s_k (b_k - a_k), and the
// median of Appendix B is the element at slot first + ceil(|S|/2) - 1 of the
// split axis' array.  Each array is then stably partitioned inside every
// node by "rank along the split axis <= rank of the median", which keeps all
// three arrays sorted inside the children.  Node slot ranges depend only on
// N and N0 (balanced halving, ceil to the first child), so they are tables
// computed when the plan is created.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedItems = 8;
constexpr int kRedChunk = kRedThreads * kRedItems;  // 2048 = 2^11

constexpr int kPartThreads = 256;
constexpr int kPartItems = 8;
constexpr int kPartChunk = kPartThreads * kPartItems;

// Adjacent-pair (binary tree) sum of the aligned chunk `chunk` of 2048
// terms in[i * stride], zero beyond n, by the whole block; the result is
// valid in thread 0.  Eight terms per thread, then the warp butterfly
// (adjacent lanes first), then the eight warp sums: one fixed binary tree.
__device__ __forceinline__ double chunk_pairwise(const double* __restrict__ in, int64_t n, int64_t stride,
                                                 int64_t chunk, double* wsum) {
  const int64_t base = chunk * kRedChunk + (int64_t)threadIdx.x * kRedItems;
  double e[kRedItems];
#pragma unroll
  for (int k = 0; k < kRedItems; ++k) e[k] = (base + k < n) ? in[(base + k) * stride] : 0.0;
  double v = __dadd_rn(__dadd_rn(__dadd_rn(e[0], e[1]), __dadd_rn(e[2], e[3])),
                       __dadd_rn(__dadd_rn(e[4], e[5]), __dadd_rn(e[6], e[7])));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    r = __dadd_rn(__dadd_rn(__dadd_rn(wsum[0], wsum[1]), __dadd_rn(wsum[2], wsum[3])),
                  __dadd_rn(__dadd_rn(wsum[4], wsum[5]), __dadd_rn(wsum[6], wsum[7])));
  __syncthreads();
  return r;
}

// First level of the three momentum sums (grid.y = component k): chunk sums
// of p[i][k]; the same blocks flag non-finite x, p, q and (k = 0) take the
// chunk's max |q|.
__global__ void __launch_bounds__(kRedThreads) k_setup_first(const double* __restrict__ x,
                                                            const double* __restrict__ p,
                                                            const double* __restrict__ q, int64_t N,
                                                            double* __restrict__ part, int64_t comp_step,
                                                            double* __restrict__ qmax, Counters* cnt) {
  __shared__ double wsum[kRedThreads / 32];
  const int k = blockIdx.y;
  const int64_t base = (int64_t)blockIdx.x * kRedChunk + (int64_t)threadIdx.x * kRedItems;
  bool bad = false;
  double m = 0.0;
#pragma unroll
  for (int j = 0; j < kRedItems; ++j) {
    const int64_t i = base + j;
    if (i >= N) break;
    bad |= !isfinite(x[3 * i + k]) || !isfinite(p[3 * i + k]);
    if (k == 0) {
      bad |= !isfinite(q[i]);
      m = fmax(m, fabs(q[i]));
    }
  }
  if (bad) atomicOr(&cnt->err, kErrNonFinite);
  const double r = chunk_pairwise(p + k, N, 3, blockIdx.x, wsum);
  if (threadIdx.x == 0) part[k * comp_step + blockIdx.x] = r;
  if (k == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kRedThreads / 32; ++w) t = fmax(t, wsum[w]);
      qmax[blockIdx.x] = t;
    }
  }
}

// A further level of the three sums (more than 2048 partials left).
__global__ void __launch_bounds__(kRedThreads) k_pairwise(const double* __restrict__ in, int64_t n,
                                                         int64_t comp_step, double* __restrict__ out) {
  __shared__ double wsum[kRedThreads / 32];
  const double r = chunk_pairwise(in + blockIdx.y * comp_step, n, 1, blockIdx.x, wsum);
  if (threadIdx.x == 0) out[blockIdx.y * comp_step + blockIdx.x] = r;
}

// Last level (at most 2048 partials per component), max |q| and
// scal[0] = gbar, scal[1] = mass unit mu (power of two near max|q|), scal[11] = 1/mu,
// scal[6..8] = pbar (for the adjoint's gbar term).
__global__ void __launch_bounds__(kRedThreads) k_setup_final(const double* __restrict__ part, int64_t n,
                                                            int64_t comp_step, int64_t N,
                                                            const double* __restrict__ qmax, int64_t nq,
                                                            double* __restrict__ scal) {
  __shared__ double wsum[kRedThreads / 32];
  double sum[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sum[k] = chunk_pairwise(part + k * comp_step, n, 1, 0, wsum);
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < nq; i += blockDim.x) m = fmax(m, qmax[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 0; w < kRedThreads / 32; ++w) m = fmax(m, wsum[w]);
  const double dn = (double)N;
  const double px = __ddiv_rn(sum[0], dn), py = __ddiv_rn(sum[1], dn), pz = __ddiv_rn(sum[2], dn);
  const double pp = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
  scal[0] = __dsqrt_rn(__dadd_rn(1.0, pp));
  const int me = (m > 0.0 && isfinite(m)) ? (int)rint(log2(m)) : 0;
  scal[1] = ldexp(1.0, me);
  scal[11] = ldexp(1.0, -me);  // 1/mu, exact
  scal[6] = px;
  scal[7] = py;
  scal[8] = pz;
}

// Order-preserving 64-bit key of a double; -0 is folded onto +0.
__device__ __forceinline__ uint64_t dkey(double v) {
  if (v == 0.0) v = 0.0;
  uint64_t u = (uint64_t)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Sort keys of all three axes (grid.y = axis): keys[axis][i], vals[axis][i] = i.
__global__ void k_make_keys(const double* __restrict__ x, int64_t N, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int axis = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[axis * N + i] = dkey(x[3 * i + axis]);
    vals[axis * N + i] = (uint32_t)i;
  }
}

__global__ void k_store_axis(const uint32_t* __restrict__ sorted, int64_t N, int32_t* __restrict__ A,
                             int32_t* __restrict__ rank) {
  const int64_t o = (int64_t)blockIdx.y * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = sorted[o + i];
    A[o + i] = (int32_t)v;
    rank[o + v] = (int32_t)i;
  }
}

// Boxes of the nodes of one level; for inner levels also the split axis
// (Alg. 1) and the rank of the median element (Appendix B).
__global__ void k_node_split(const double* __restrict__ x, const int32_t* __restrict__ A,
                             const int32_t* __restrict__ rank, int64_t N, const int64_t* __restrict__ nstart,
                             const int64_t* __restrict__ ncount, int level, int kappa,
                             const double* __restrict__ scal, double* __restrict__ nlo,
                             double* __restrict__ nhi, int32_t* __restrict__ naxis,
                             int32_t* __restrict__ nmed) {
  const int64_t first = (int64_t)1 << level;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= first) return;
  const int64_t i = first + t;
  const int64_t st = nstart[i], c = ncount[i];
  const double s[3] = {1.0, 1.0, scal[0]};
  double w[3];
  for (int k = 0; k < 3; ++k) {
    double lo = x[3 * (int64_t)A[k * N + st] + k];
    double hi = x[3 * (int64_t)A[k * N + st + c - 1] + k];
    nlo[3 * i + k] = lo;
    nhi[3 * i + k] = hi;
    w[k] = __dmul_rn(s[k], __dsub_rn(hi, lo));
  }
  if (level == kappa) {
    naxis[i] = -1;
    nmed[i] = -1;
    return;
  }
  int ax = 0;
  if (w[1] > w[ax]) ax = 1;
  if (w[2] > w[ax]) ax = 2;
  const int64_t h1 = (c + 1) / 2;
  naxis[i] = ax;
  nmed[i] = rank[ax * N + A[ax * N + st + h1 - 1]];
}

// Flags "goes to the first child" (rank along the node's split axis <= the
// median's rank) of the kPartItems slots from `base` on, and their nodes.
// The loads of one phase are independent, so they are all in flight at once.
__device__ __forceinline__ uint32_t part_flags(const int32_t* __restrict__ Ak, const int32_t* __restrict__ rank,
                                               int64_t N, const int64_t* __restrict__ nstart, int64_t first,
                                               const int32_t* __restrict__ naxis, const int32_t* __restrict__ nmed,
                                               int64_t base, int64_t (&nd)[kPartItems]) {
  int32_t id[kPartItems];
#pragma unroll
  for (int j = 0; j < kPartItems; ++j) id[j] = base + j < N ? Ak[base + j] : 0;
  int64_t node = -1, node_end = -1;
#pragma unroll
  for (int j = 0; j < kPartItems; ++j) {
    const int64_t pos = base + j;
    if (pos < N && pos >= node_end) {
      node = find_node(nstart, first, first, pos);
      node_end = (node + 1 < 2 * first) ? nstart[node + 1] : N;
    }
    nd[j] = pos < N ? node : -1;
  }
  int ax[kPartItems], med[kPartItems];
#pragma unroll
  for (int j = 0; j < kPartItems; ++j) {
    ax[j] = nd[j] >= 0 ? naxis[nd[j]] : 0;
    med[j] = nd[j] >= 0 ? nmed[nd[j]] : -1;
  }
  uint32_t f = 0;
#pragma unroll
  for (int j = 0; j < kPartItems; ++j)
    if (nd[j] >= 0 && rank[(int64_t)ax[j] * N + id[j]] <= med[j]) f |= 1u << j;
  return f;
}

// Per-chunk count of elements going to the first child (grid.y = array k).
__global__ void __launch_bounds__(kPartThreads) k_part_count(
    const int32_t* __restrict__ A, const int32_t* __restrict__ rank, int64_t N,
    const int64_t* __restrict__ nstart, int level, const int32_t* __restrict__ naxis,
    const int32_t* __restrict__ nmed, int64_t nblk, uint32_t* __restrict__ bsum) {
  __shared__ uint32_t red[kPartThreads / 32];
  const int k = blockIdx.y;
  const int32_t* Ak = A + (int64_t)k * N;
  const int64_t first = (int64_t)1 << level;
  const int64_t base = (int64_t)blockIdx.x * kPartChunk + (int64_t)threadIdx.x * kPartItems;
  int64_t nd[kPartItems];
  uint32_t c = __popc(part_flags(Ak, rank, N, nstart, first, naxis, nmed, base, nd));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kPartThreads / 32; ++w) t += red[w];
    bsum[(int64_t)k * nblk + blockIdx.x] = t;
  }
}

// Stable partition of every node's slot range (grid.y = array k).
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(
    const int32_t* __restrict__ A, const int32_t* __restrict__ rank, int64_t N,
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount,
    const int64_t* __restrict__ nleftpre, int level, const int32_t* __restrict__ naxis,
    const int32_t* __restrict__ nmed, int64_t nblk, const uint32_t* __restrict__ bscan, bool fused,
    int32_t* __restrict__ Aout) {
  __shared__ uint32_t wt[33];
  __shared__ uint32_t sbase;
  const int k = blockIdx.y;
  const int32_t* Ak = A + (int64_t)k * N;
  int32_t* Ok = Aout + (int64_t)k * N;
  const int64_t first = (int64_t)1 << level;
  const int64_t base = (int64_t)blockIdx.x * kPartChunk + (int64_t)threadIdx.x * kPartItems;
  int64_t nd[kPartItems];
  const uint32_t fm = part_flags(Ak, rank, N, nstart, first, naxis, nmed, base, nd);
  const uint32_t c = __popc(fm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {  // first-child elements before this chunk
    uint32_t b0;
    if (fused) {     // raw per-chunk counts: sum those of the earlier chunks
      b0 = 0;
      for (int64_t j = lane; j < (int64_t)blockIdx.x; j += 32) b0 += bscan[(int64_t)k * nblk + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) b0 += __shfl_xor_sync(0xffffffffu, b0, o);
    } else {         // already an exclusive scan
      b0 = bscan[(int64_t)k * nblk + blockIdx.x];
    }
    if (lane == 0) sbase = b0;
  }
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = kPartThreads / 32;
    uint32_t w = lane < nw ? wt[lane] : 0u, wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) wt[lane] = wi - w;
  }
  __syncthreads();
  int64_t P = (int64_t)sbase + wt[warp] + (inc - c);
#pragma unroll
  for (int j = 0; j < kPartItems; ++j) {
    const int64_t pos = base + j;
    if (pos >= N) break;
    const int64_t n0 = nd[j];
    const bool f = (fm >> j) & 1u;
    const int64_t st = nstart[n0], cnt = ncount[n0], h1 = (cnt + 1) / 2;
    const int64_t lb = P - nleftpre[n0];  // first-child elements before pos inside the node
    const int64_t dst = f ? st + lb : st + h1 + ((pos - st) - lb);
    Ok[dst] = Ak[pos];
    P += f ? 1 : 0;
  }
}

// Deep levels in one block per subtree.  Once a node holds at most
// kSubSlots slots, one block finishes every level below it in shared memory:
// the node's members get local ids (their slot in the x-array), the three
// slot arrays hold local ids, and a level is one box/axis/median step per
// node followed by the stable partition of every node's slot ranges.  Inside
// a node the split axis' array is in rank order, so "rank <= median rank" is
// "slot among the first ceil(c/2) of that array": each member's flag is read
// off the split axis' array and no rank is looked up but the median's.  The
// children's slot ranges follow from the parent's by the same halving rule
// as the plan's node tables (first child ceil(c/2)).
constexpr int kSubSlots = 4096;
constexpr int kSubThreads = 1024;
constexpr int kSubPer = kSubSlots / kSubThreads;  // consecutive slots per thread, in each array
constexpr int kSubNodes = kSubSlots / 2;          // a node above the leaves has >= 2 members

struct SubtreeSmem {
  uint16_t arr[2][3][kSubSlots];  // local ids by slot, current and next level
                                  // (arr[1] holds 4-byte x-ranks before the first level)
  int32_t gid[kSubSlots];         // local id -> input index
  uint16_t seg[kSubSlots];        // slot -> node of the current level (relative)
  uint8_t flag[kSubSlots];        // local id -> goes to the first child
  uint16_t nst[2][kSubNodes], ncnt[2][kSubNodes];  // node slot ranges, current and previous level
  uint8_t nax[kSubNodes];
  uint64_t npre[kSubNodes];       // first-child elements before each node's start, 16 bits per array
  uint64_t wt[33];
};
static_assert(sizeof(uint16_t) * 3 * kSubSlots >= sizeof(int32_t) * kSubSlots, "x-ranks fit in arr[1]");

__device__ __forceinline__ uint64_t sub_block_scan(uint64_t v, uint64_t* wt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = wt[lane];
    uint64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    wt[lane] = wi - w;
  }
  __syncthreads();
  return wt[warp] + inc - v;
}

__global__ void __launch_bounds__(kSubThreads) k_subtree(
    const double* __restrict__ x, int32_t* A, const int32_t* __restrict__ rank, int64_t N,
    const int64_t* __restrict__ nstart, const int64_t* __restrict__ ncount, int ls, int kappa,
    const double* __restrict__ scal, double* __restrict__ nlo, double* __restrict__ nhi,
    int32_t* __restrict__ naxis, int32_t* __restrict__ nmed) {
  extern __shared__ __align__(16) unsigned char sub_raw[];
  SubtreeSmem& S = *reinterpret_cast<SubtreeSmem*>(sub_raw);
  const int64_t root = ((int64_t)1 << ls) + blockIdx.x;
  const int64_t st0 = nstart[root];
  const int c = (int)ncount[root];
  const double sz = scal[0];
  // local ids: slot in the x-array; the y- and z-arrays find theirs by the
  // x-rank, which increases along the x-array's slots
  int32_t* xr = reinterpret_cast<int32_t*>(&S.arr[1][0][0]);
  for (int j = threadIdx.x; j < c; j += kSubThreads) {
    const int32_t e = A[st0 + j];
    S.gid[j] = e;
    xr[j] = rank[e];
    S.arr[0][0][j] = (uint16_t)j;
    S.seg[j] = 0;
  }
  if (threadIdx.x == 0) {
    S.nst[1][0] = 0;
    S.ncnt[1][0] = (uint16_t)c;
  }
  __syncthreads();
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    for (int j = threadIdx.x; j < c; j += kSubThreads) {
      const int32_t rx = rank[A[(int64_t)k * N + st0 + j]];
      int lo = 0, hi = c - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (xr[mid] < rx) lo = mid + 1; else hi = mid;
      }
      S.arr[0][k][j] = (uint16_t)lo;
    }
  }
  const int j0 = threadIdx.x * kSubPer;  // this thread's slots j0 .. j0 + kSubPer - 1
  int cur = 0, pb = 1;                   // slot buffer; node buffer of the previous level
  for (int l = ls;; ++l) {
    __syncthreads();
    const int64_t first = root << (l - ls);
    const int nodes = 1 << (l - ls);
    for (int u = threadIdx.x; u < nodes; u += kSubThreads) {  // boxes, Alg. 1 axis, Appendix B median
      int st, cnt;
      if (l == ls) {
        st = 0;
        cnt = c;
      } else {
        const int pst = S.nst[pb][u >> 1], pc = S.ncnt[pb][u >> 1], ph = (pc + 1) / 2;
        st = (u & 1) ? pst + ph : pst;
        cnt = (u & 1) ? pc - ph : ph;
      }
      const int64_t g = first + u;
      double w[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double lo = x[3 * (int64_t)S.gid[S.arr[cur][k][st]] + k];
        const double hi = x[3 * (int64_t)S.gid[S.arr[cur][k][st + cnt - 1]] + k];
        nlo[3 * g + k] = lo;
        nhi[3 * g + k] = hi;
        w[k] = __dmul_rn(k == 2 ? sz : 1.0, __dsub_rn(hi, lo));
      }
      if (l == kappa) {
        naxis[g] = -1;
        nmed[g] = -1;
        continue;
      }
      int ax = 0;
      if (w[1] > w[ax]) ax = 1;
      if (w[2] > w[ax]) ax = 2;
      const int h1 = (cnt + 1) / 2;
      naxis[g] = ax;
      nmed[g] = rank[(int64_t)ax * N + S.gid[S.arr[cur][ax][st + h1 - 1]]];
      S.nst[pb ^ 1][u] = (uint16_t)st;
      S.ncnt[pb ^ 1][u] = (uint16_t)cnt;
      S.nax[u] = (uint8_t)ax;
    }
    if (l == kappa) break;
    pb ^= 1;
    const uint16_t* nst = S.nst[pb];
    const uint16_t* ncnt = S.ncnt[pb];
    __syncthreads();
    int su[kSubPer];
#pragma unroll
    for (int i = 0; i < kSubPer; ++i) {
      const int j = j0 + i;
      su[i] = j < c ? S.seg[j] : 0;
      if (j < c) {
        const int u = su[i];
        S.flag[S.arr[cur][S.nax[u]][j]] = (uint8_t)(j - nst[u] < (ncnt[u] + 1) / 2);
      }
    }
    __syncthreads();
    // stable partition of the three arrays; one scan, 16 bits per array
    uint32_t fm = 0;
    uint64_t cnt3 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < kSubPer; ++i) {
        const int j = j0 + i;
        const uint32_t f = j < c ? S.flag[S.arr[cur][k][j]] : 0u;
        fm |= f << (k * kSubPer + i);
        cnt3 += (uint64_t)f << (16 * k);
      }
    const uint64_t pre = sub_block_scan(cnt3, S.wt);
    uint64_t run = pre;
#pragma unroll
    for (int i = 0; i < kSubPer; ++i) {
      const int j = j0 + i;
      if (j < c && j == nst[su[i]]) S.npre[su[i]] = run;
#pragma unroll
      for (int k = 0; k < 3; ++k) run += (uint64_t)((fm >> (k * kSubPer + i)) & 1u) << (16 * k);
    }
    __syncthreads();
    run = pre;
#pragma unroll
    for (int i = 0; i < kSubPer; ++i) {
      const int j = j0 + i;
      if (j < c) {
        const int u = su[i];
        const int st = nst[u], h1 = (ncnt[u] + 1) / 2;
        const uint64_t np = S.npre[u];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int lb = (int)(((run >> (16 * k)) - (np >> (16 * k))) & 0xffffu);
          const bool f = (fm >> (k * kSubPer + i)) & 1u;
          const int dst = f ? st + lb : st + h1 + ((j - st) - lb);
          S.arr[cur ^ 1][k][dst] = S.arr[cur][k][j];
        }
        S.seg[j] = (uint16_t)(2 * u + (j - st >= h1 ? 1 : 0));
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) run += (uint64_t)((fm >> (k * kSubPer + i)) & 1u) << (16 * k);
    }
    cur ^= 1;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k)
    for (int j = threadIdx.x; j < c; j += kSubThreads) A[(int64_t)k * N + st0 + j] = S.gid[S.arr[cur][k][j]];
}

}  // namespace

int run_setup(fmm_plan_s* P, const double* x, const double* p, const double* q, cudaStream_t s) {
  const Layout& L = P->lay;
  const int64_t N = P->N;
  Counters* cnt = ws_ptr<Counters>(P, L.counters);
  FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(Counters), s));
  // pairwise momentum sums: per component two ping-pong arrays of partials
  const int64_t np0 = div_up(N, kRedChunk);
  const int64_t comp_step = 2 * (np0 + 2);
  double* a = ws_ptr<double>(P, L.psum_part);
  double* b = a + (np0 + 2);
  double* qmax = ws_ptr<double>(P, L.qmax_part);
  k_setup_first<<<dim3((unsigned)np0, 3), kRedThreads, 0, s>>>(x, p, q, N, a, comp_step, qmax, cnt);
  FMM_LAUNCH_CHECK();
  int64_t n = np0;
  while (n > kRedChunk) {
    const int64_t nb = div_up(n, kRedChunk);
    k_pairwise<<<dim3((unsigned)nb, 3), kRedThreads, 0, s>>>(a, n, comp_step, b);
    FMM_LAUNCH_CHECK();
    std::swap(a, b);
    n = nb;
  }
  k_setup_final<<<1, kRedThreads, 0, s>>>(a, n, comp_step, N, qmax, np0, ws_ptr<double>(P, L.scal));
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int run_tree(fmm_plan_s* P, const double* x, cudaStream_t s) {
  const Layout& L = P->lay;
  const int64_t N = P->N;
  uint64_t* keys = ws_ptr<uint64_t>(P, L.keys);
  uint64_t* keys_alt = ws_ptr<uint64_t>(P, L.keys_alt);
  uint32_t* vals = ws_ptr<uint32_t>(P, L.vals);
  uint32_t* vals_alt = ws_ptr<uint32_t>(P, L.vals_alt);
  uint32_t* hist = ws_ptr<uint32_t>(P, L.hist);
  uint32_t* stmp = ws_ptr<uint32_t>(P, L.scan_tmp);
  int32_t* A = ws_ptr<int32_t>(P, L.A);
  int32_t* Aalt = ws_ptr<int32_t>(P, L.A_alt);
  int32_t* rank = ws_ptr<int32_t>(P, L.rank);
  const double* scal = ws_ptr<double>(P, L.scal);
  const int64_t* nstart = ws_ptr<int64_t>(P, L.nstart);
  const int64_t* ncount = ws_ptr<int64_t>(P, L.ncount);
  const int64_t* nleftpre = ws_ptr<int64_t>(P, L.nleftpre);
  double* nlo = ws_ptr<double>(P, L.nlo);
  double* nhi = ws_ptr<double>(P, L.nhi);
  int32_t* naxis = ws_ptr<int32_t>(P, L.naxis);
  int32_t* nmed = ws_ptr<int32_t>(P, L.nmed);
  const int gs = (int)std::min<int64_t>(4096, div_up(N, 256));

  {  // the three presorts by (coordinate, input index), batched
    k_make_keys<<<dim3(gs, 3), 256, 0, s>>>(x, N, keys, vals);
    FMM_LAUNCH_CHECK();
    bool alt = false;
    int rc = radix_sort_batched(keys, keys_alt, vals, vals_alt, N, 3, N, 0, 64, hist, stmp, (int64_t)L.nblk_sort, s,
                                &alt);
    if (rc != FMM_OK) return rc;
    k_store_axis<<<dim3(gs, 3), 256, 0, s>>>(alt ? vals_alt : vals, N, A, rank);
    FMM_LAUNCH_CHECK();
  }

  const int64_t nblk = div_up(N, kPartChunk);
  uint32_t* bsum = ws_ptr<uint32_t>(P, L.blocksum);
  int32_t* cur = A;
  int32_t* nxt = Aalt;
  // first level whose nodes one block finishes alone (the leftmost node of a
  // level is its largest)
  int ls = 0;
  while (ls < P->kappa && P->node_count[(size_t)1 << ls] > kSubSlots) ++ls;
  for (int l = 0; l < ls; ++l) {
    const int64_t nodes = (int64_t)1 << l;
    k_node_split<<<(unsigned)div_up(nodes, 128), 128, 0, s>>>(x, cur, rank, N, nstart, ncount, l, P->kappa,
                                                             scal, nlo, nhi, naxis, nmed);
    FMM_LAUNCH_CHECK();
    dim3 g((unsigned)nblk, 3);
    k_part_count<<<g, kPartThreads, 0, s>>>(cur, rank, N, nstart, l, naxis, nmed, nblk, bsum);
    FMM_LAUNCH_CHECK();
    const bool fused = nblk <= 64;  // the scatter sums the earlier chunk counts itself
    if (!fused) {
      for (int k = 0; k < 3; ++k) {
        int rc = scan_exclusive(bsum + k * nblk, bsum + k * nblk, nblk, stmp, s);
        if (rc != FMM_OK) return rc;
      }
    }
    k_part_scatter<<<g, kPartThreads, 0, s>>>(cur, rank, N, nstart, ncount, nleftpre, l, naxis, nmed, nblk,
                                              bsum, fused, nxt);
    FMM_LAUNCH_CHECK();
    int32_t* t = cur; cur = nxt; nxt = t;
  }
  {
    if (int rc = smem_limit(k_subtree, (int)sizeof(SubtreeSmem))) return rc;
    k_subtree<<<(unsigned)((int64_t)1 << ls), kSubThreads, sizeof(SubtreeSmem), s>>>(
        x, cur, rank, N, nstart, ncount, ls, P->kappa, scal, nlo, nhi, naxis, nmed);
    FMM_LAUNCH_CHECK();
  }
  // leaf order: the x-array's slot order (members of each leaf sorted by x)
  FMM_CUDA_TRY(cudaMemcpyAsync(ws_ptr<int32_t>(P, L.perm), cur, sizeof(int32_t) * N,
                               cudaMemcpyDeviceToDevice, s));
  return FMM_OK;
}

}  // namespace fmm
