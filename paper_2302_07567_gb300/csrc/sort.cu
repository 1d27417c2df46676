// Device-wide exclusive scan and stable LSD radix sort (64-bit keys).
//
// Used by the tree build: one presort of the particles along each axis, so
// that equal coordinates stay in input-index order, which is the tie rule of
// the median split.
#include <cooperative_groups.h>

#include "common.cuh"

namespace fmm {
namespace {

namespace cg = cooperative_groups;

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;
// up to this many tiles per batch every pass runs in one cooperative launch
constexpr int64_t kFusedTiles = 64;

// Exclusive prefix of `v` over the block (blocked arrangement); returns the
// block total through `total`.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == nw - 1) warp_tot[32] = wi;
  }
  __syncthreads();
  uint32_t res = warp_tot[warp] + inc - v;
  total = warp_tot[32];
  __syncthreads();
  return res;
}

__global__ void k_chunk_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[33];
  int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += (base + k < n) ? in[base + k] : 0u;
  uint32_t tot;
  block_exclusive_scan(s, wt, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// In-place safe: every thread reads its items before the block-wide scan.
__global__ void k_chunk_scan(const uint32_t* in, int64_t n, uint32_t* out,
                             const uint32_t* __restrict__ offsets) {
  __shared__ uint32_t wt[33];
  int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan(s, wt, tot) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block state of the stable scatter of one tile.
struct ScatterSmem {
  uint32_t wcnt[kSortWarps][256];  // per warp and digit: keys of the current round
  uint32_t run[256];               // per digit: keys of the tile placed so far
  uint32_t gbase[256];             // per digit: first output slot of this tile
  uint32_t cnt[256];               // per digit: keys of this tile
  uint32_t loff[256];              // per digit: first slot of its run in the tile, reordered
  uint32_t wt[33];
  uint64_t skey[kSortTile];        // the tile in digit order (stable)
  uint32_t sval[kSortTile];
};

// The tile's keys (and values) in registers, thread-strided within each round.
template <bool kCG>
__device__ __forceinline__ void load_tile(const uint64_t* keys, const uint32_t* vals, int64_t base, int64_t n,
                                          uint64_t (&kk)[kSortRounds], uint32_t (&vv)[kSortRounds]) {
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (kCG) {
      kk[r] = i < n ? (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(keys) + i) : 0ull;
      vv[r] = (i < n && vals) ? __ldcg(vals + i) : 0u;
    } else {
      kk[r] = i < n ? keys[i] : 0ull;
      vv[r] = (i < n && vals) ? vals[i] : 0u;
    }
  }
}

// Digit counts of the tile into cnt[256] (valid after the call).
__device__ __forceinline__ void tile_histogram(const uint64_t (&kk)[kSortRounds], int64_t base, int64_t n,
                                               int shift, uint32_t* cnt) {
  cnt[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const unsigned d = valid ? (unsigned)((kk[r] >> shift) & 0xffu) : 0x100u + (threadIdx.x & 31);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && (peers & lanemask_lt()) == 0u) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
}

// Stable scatter of the tile by its digit; S.gbase holds the tile's first
// output slot of every digit and S.cnt its count of every digit.  Rounds go
// in input order, warps in order inside a round and lanes in order inside a
// warp.  The tile is first reordered by digit in shared memory, then written
// out in that order, so that consecutive threads write consecutive slots of
// one digit's run (coalesced) instead of slots of up to 32 different runs.
__device__ __forceinline__ void tile_scatter(const uint64_t (&kk)[kSortRounds], const uint32_t (&vv)[kSortRounds],
                                             int64_t base, int64_t n, int shift, bool with_vals, ScatterSmem& S,
                                             uint64_t* keys_out, uint32_t* vals_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kSortWarps; ++w) S.wcnt[w][threadIdx.x] = 0;
  S.run[threadIdx.x] = 0;
  {
    uint32_t tot;
    S.loff[threadIdx.x] = block_exclusive_scan(S.cnt[threadIdx.x], S.wt, tot);  // synchronises
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const unsigned d = valid ? (unsigned)((kk[r] >> shift) & 0xffu) : 0x100u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned wr = __popc(peers & lanemask_lt());
    if (valid && wr == 0u) S.wcnt[warp][d] = (uint32_t)__popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pre = S.run[d];
      for (int w = 0; w < warp; ++w) pre += S.wcnt[w][d];
      const uint32_t lpos = S.loff[d] + pre + wr;
      S.skey[lpos] = kk[r];
      S.sval[lpos] = vv[r];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      tot += S.wcnt[w][threadIdx.x];
      S.wcnt[w][threadIdx.x] = 0;
    }
    S.run[threadIdx.x] += tot;
    __syncthreads();
  }
  const int nv = (int)(n - base < kSortTile ? n - base : kSortTile);
  for (int e = threadIdx.x; e < nv; e += kSortThreads) {
    const uint64_t key = S.skey[e];
    const unsigned d = (unsigned)((key >> shift) & 0xffu);
    const uint32_t pos = S.gbase[d] + ((uint32_t)e - S.loff[d]);
    keys_out[pos] = key;
    if (with_vals) vals_out[pos] = S.sval[e];
  }
}

// Digit histogram of one tile of one batch: hist[batch][digit][tile].
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint64_t* __restrict__ keys, int64_t stride,
                                                               int64_t n, int shift, int64_t ntiles,
                                                               uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  keys += blockIdx.y * stride;
  hist += (int64_t)blockIdx.y * 256 * ntiles;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  uint64_t kk[kSortRounds];
  uint32_t vv[kSortRounds];
  load_tile<false>(keys, nullptr, base, n, kk, vv);
  tile_histogram(kk, base, n, shift, cnt);
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile by its digit; `hist` holds the exclusive scan
// over (digit, tile).
__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t stride, int64_t n, int shift,
    int64_t ntiles, const uint32_t* __restrict__ hist, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
  __shared__ ScatterSmem S;
  const int64_t boff = blockIdx.y * stride;
  keys += boff;
  keys_out += boff;
  if (vals) {
    vals += boff;
    vals_out += boff;
  }
  hist += (int64_t)blockIdx.y * 256 * ntiles;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  uint64_t kk[kSortRounds];
  uint32_t vv[kSortRounds];
  load_tile<false>(keys, vals, base, n, kk, vv);
  // hist is the exclusive scan over (digit, tile), digit-major: the next
  // entry (the next tile, or the next digit's first tile) ends this one
  const int64_t f = (int64_t)threadIdx.x * ntiles + blockIdx.x;
  const uint32_t g0 = hist[f];
  S.gbase[threadIdx.x] = g0;
  S.cnt[threadIdx.x] = (f + 1 < 256 * ntiles ? hist[f + 1] : (uint32_t)n) - g0;
  tile_scatter(kk, vv, base, n, shift, vals != nullptr, S, keys_out, vals_out);
}

// Every pass of a sort of at most kFusedTiles tiles per batch in one
// cooperative launch: per pass, tile histograms hist[batch][tile][digit],
// a grid-wide barrier, then every tile forms its digit offsets from the
// histograms (digit totals scanned, plus the counts of the earlier tiles)
// and scatters; a barrier again before the next digit.
__global__ void __launch_bounds__(kSortThreads) k_radix_coop(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                                                            uint32_t* vals_alt, int64_t stride, int nbatch,
                                                            int64_t n, int begin_bit, int end_bit, int64_t ntiles,
                                                            uint32_t* hist) {
  __shared__ ScatterSmem S;
  cg::grid_group grid = cg::this_grid();
  const bool with_vals = vals != nullptr;
  uint64_t* kin = keys;
  uint64_t* kout = keys_alt;
  uint32_t* vin = vals;
  uint32_t* vout = vals_alt;
  const int64_t items = ntiles * nbatch;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const int64_t batch = it / ntiles, tile = it - batch * ntiles, base = tile * kSortTile;
      uint64_t kk[kSortRounds];
      uint32_t vv[kSortRounds];
      load_tile<true>(kin + batch * stride, nullptr, base, n, kk, vv);
      tile_histogram(kk, base, n, shift, S.cnt);
      hist[it * 256 + threadIdx.x] = S.cnt[threadIdx.x];
    }
    grid.sync();
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const int64_t batch = it / ntiles, tile = it - batch * ntiles, base = tile * kSortTile;
      uint64_t kk[kSortRounds];
      uint32_t vv[kSortRounds];
      load_tile<true>(kin + batch * stride, with_vals ? vin + batch * stride : nullptr, base, n, kk, vv);
      const uint32_t* h = hist + batch * ntiles * 256 + threadIdx.x;
      uint32_t tot = 0, before = 0;
      for (int64_t t0 = 0; t0 < ntiles; t0 += 16) {
        uint32_t c[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) c[u] = t0 + u < ntiles ? __ldcg(h + (t0 + u) * 256) : 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          tot += c[u];
          before += t0 + u < tile ? c[u] : 0u;
        }
      }
      uint32_t all;
      S.gbase[threadIdx.x] = block_exclusive_scan(tot, S.wt, all) + before;
      S.cnt[threadIdx.x] = __ldcg(h + tile * 256);
      tile_scatter(kk, vv, base, n, shift, with_vals, S, kout + batch * stride,
                   with_vals ? vout + batch * stride : nullptr);
    }
    grid.sync();
    uint64_t* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
}

}  // namespace

int64_t scan_tmp_words(int64_t n) {
  int64_t nc = div_up(n, kScanChunk);
  if (nc <= 1) return 1;
  return nc + scan_tmp_words(nc);
}

int scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s) {
  if (n <= 0) return FMM_OK;
  int64_t nc = div_up(n, kScanChunk);
  if (nc == 1) {
    k_chunk_scan<<<1, kScanThreads, 0, s>>>(in, n, out, nullptr);
    FMM_LAUNCH_CHECK();
    return FMM_OK;
  }
  k_chunk_sums<<<(unsigned)nc, kScanThreads, 0, s>>>(in, n, tmp);
  FMM_LAUNCH_CHECK();
  int rc = scan_exclusive(tmp, tmp, nc, tmp + nc, s);
  if (rc != FMM_OK) return rc;
  k_chunk_scan<<<(unsigned)nc, kScanThreads, 0, s>>>(in, n, out, tmp);
  FMM_LAUNCH_CHECK();
  return FMM_OK;
}

int64_t radix_tiles(int64_t n) { return div_up(n > 0 ? n : 1, kSortTile); }

int radix_sort_batched(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t stride,
                       int nbatch, int64_t n, int begin_bit, int end_bit, uint32_t* hist, uint32_t* scan_tmp,
                       int64_t max_tiles, cudaStream_t s, bool* in_alt) {
  *in_alt = false;
  if (n <= 1 || nbatch < 1) return FMM_OK;
  const int64_t nt = radix_tiles(n);
  if (nt * nbatch > max_tiles) return FMM_EINVAL;
  const int passes = (end_bit - begin_bit + 7) / 8;
  if (nt <= kFusedTiles) {  // one cooperative launch for every pass
    int per_sm = 0, sms = 0;
    if (int rc = device_sms(&sms)) return rc;
    if (int rc = blocks_per_sm(k_radix_coop, kSortThreads, 0, &per_sm)) return rc;
    if (per_sm < 1) return FMM_EINVAL;
    int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, nt * nbatch);
    void* args[] = {&keys, &keys_alt, &vals, &vals_alt, &stride, &nbatch, &n, &begin_bit, &end_bit,
                    (void*)&nt, &hist};
    FMM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_radix_coop, dim3(grid), dim3(kSortThreads), args, 0, s));
    FMM_LAUNCH_CHECK();
    *in_alt = (passes & 1) != 0;
    return FMM_OK;
  }
  uint64_t* k_in = keys;
  uint64_t* k_out = keys_alt;
  uint32_t* v_in = vals;
  uint32_t* v_out = vals_alt;
  bool alt = false;
  const dim3 grid((unsigned)nt, (unsigned)nbatch);
  for (int b = begin_bit; b < end_bit; b += 8) {
    k_radix_upsweep<<<grid, kSortThreads, 0, s>>>(k_in, stride, n, b, nt, hist);
    FMM_LAUNCH_CHECK();
    for (int k = 0; k < nbatch; ++k) {
      uint32_t* h = hist + (int64_t)k * 256 * nt;
      int rc = scan_exclusive(h, h, 256 * nt, scan_tmp, s);
      if (rc != FMM_OK) return rc;
    }
    k_radix_downsweep<<<grid, kSortThreads, 0, s>>>(k_in, v_in, stride, n, b, nt, hist, k_out, v_out);
    FMM_LAUNCH_CHECK();
    uint64_t* tk = k_in; k_in = k_out; k_out = tk;
    uint32_t* tv = v_in; v_in = v_out; v_out = tv;
    alt = !alt;
  }
  *in_alt = alt;
  return FMM_OK;
}

}  // namespace fmm
