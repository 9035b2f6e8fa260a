// K2-K3: the depth sort of one splat (camera or light) and the records in
// depth-rank order; the paper bins the light view with the same splatting
// pipeline as the camera view (Sec. 3, Sec. 4.2).
//
//   1. stable radix sort of the N FP32 depth keys (index payload, emitted in
//      index order), one pass per 8-bit digit with decoupled look-back
//      -> rank r, order[r]
//   2. records gathered into rank order, tile counts per rank, and the counts
//      per (tile row, block of ranks) that the binning by counting
//      (tile_bin.cu) starts from
// Ties in depth keep index order, so a tile's list is ascending (depth bits,
// index), as a stable sort of 64-bit (tile << 32 | depth) keys emitted in
// index order would give.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

// ---------------------------------------------------------------------------
// Device-wide exclusive scan: reduce, scan of block sums, down-sweep.  No
// block ever waits on another block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* in, uint32_t n, uint32_t* part) {
  __shared__ uint32_t red[8];
  const uint32_t base = blockIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll 4
  for (int r = 0; r < kScanItems / 256; ++r) {
    uint32_t i = base + r * 256 + threadIdx.x;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the block sums, any length
__global__ void __launch_bounds__(1024) k_scan_part(uint32_t* part, uint32_t nb, uint32_t* total) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < nb; base += 1024) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < nb ? part[i] : 0;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    uint32_t incl = x + (warp ? wsum[warp - 1] : 0u);
    if (i < nb) part[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t* in, uint32_t* out, uint32_t n,
                                                   const uint32_t* part) {
  __shared__ uint32_t sm[kScanItems];
  __shared__ uint32_t wsum[8];
  const uint32_t base = blockIdx.x * kScanItems;
  for (int r = 0; r < kScanItems / 256; ++r) {
    uint32_t i = base + r * 256 + threadIdx.x;
    sm[r * 256 + threadIdx.x] = i < n ? in[i] : 0u;
  }
  __syncthreads();
  constexpr int per = kScanItems / 256;  // 16 consecutive items per thread
  uint32_t loc[per];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    loc[j] = s;
    s += sm[threadIdx.x * per + j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0;
    for (int w = 0; w < 8; ++w) { uint32_t t = wsum[w]; wsum[w] = a; a += t; }
  }
  __syncthreads();
  const uint32_t off = part[blockIdx.x] + wsum[warp] + (x - s);
#pragma unroll
  for (int j = 0; j < per; ++j) sm[threadIdx.x * per + j] = off + loc[j];
  __syncthreads();
  for (int r = 0; r < kScanItems / 256; ++r) {
    uint32_t i = base + r * 256 + threadIdx.x;
    if (i < n) out[i] = sm[r * 256 + threadIdx.x];
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort pass, 8-bit digit, u32 key + u32 value.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t load_n(const uint32_t* n_ptr, uint32_t n_fixed) {
  return n_ptr ? *n_ptr : n_fixed;
}

// Per block of kSortThreads * ROUNDS consecutive items: the count of each
// digit.  Warp w counts its own 32 * ROUNDS consecutive items (all keys loaded
// first) into its own row of counters; the rows are added at the end.
template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* n_ptr, uint32_t n_fixed,
                                                             int shift, uint32_t* hist, int nblocks) {
  __shared__ uint32_t cnt[kSortThreads / 32][256];
  const uint32_t n = load_n(n_ptr, n_fixed);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) cnt[w][t] = 0;
  __syncthreads();
  const uint32_t wbase = blockIdx.x * (uint32_t)(kSortThreads * ROUNDS) + (uint32_t)warp * (32u * ROUNDS);
  uint32_t d[ROUNDS];
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const uint32_t i = wbase + r * 32 + lane;
    d[r] = i < n ? (keys[i] >> shift) & 255u : 256u;
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const uint32_t peers = __match_any_sync(0xffffffffu, d[r]);
    if (d[r] < 256u && lane == __ffs(peers) - 1) cnt[warp][d[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) c += cnt[w][t];
  hist[t * nblocks + blockIdx.x] = c;
}

// The block's items are ranked within their digit and staged in shared
// memory sorted by digit, then written out by consecutive threads, so each
// digit's run of the block leaves as contiguous stores instead of one
// scattered store per item.  Warp w ranks its own 32 * ROUNDS consecutive
// items against its own digit counters (no block barrier per round); a
// block scan over (digit, warp) then places the warps' runs, so the order
// within a digit is the items' order (stable).
template <int ROUNDS>
struct ScatterSmem {
  uint32_t base[256];    // the block's first output slot per digit (scanned histogram)
  uint32_t start[256];   // first staging slot per digit
  uint32_t cnt[kSortThreads / 32][256];  // per warp and digit: items so far, then the warp's first slot
  uint32_t wsum[kSortThreads / 32];
  uint32_t key[kSortThreads * ROUNDS], val[kSortThreads * ROUNDS];
};

template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* n_ptr, uint32_t n_fixed, int shift,
    const uint32_t* __restrict__ hist, int nblocks) {
  constexpr int kItems = kSortThreads * ROUNDS;
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ uint4 scatter_raw[];
  ScatterSmem<ROUNDS>& S = *reinterpret_cast<ScatterSmem<ROUNDS>*>(scatter_raw);
  const uint32_t n = load_n(n_ptr, n_fixed);
  const uint32_t base = blockIdx.x * (uint32_t)kItems;
  if (base >= n) return;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t lt = (1u << lane) - 1u;
  S.base[t] = hist[t * nblocks + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; ++w) S.cnt[w][t] = 0;
  const uint32_t wbase = base + (uint32_t)warp * (32u * ROUNDS);
  uint32_t kk[ROUNDS], vv[ROUNDS];
  uint32_t rk[(ROUNDS + 1) / 2];  // two 16-bit ranks per word (a warp ranks at most 32 * ROUNDS items)
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const uint32_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    kk[r] = valid ? kin[i] : 0u;
    vv[r] = valid ? (vin ? vin[i] : i) : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const bool valid = wbase + r * 32 + lane < n;
    const uint32_t d = valid ? (kk[r] >> shift) & 255u : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t c = 0;
    if (valid && lane == leader) c = S.cnt[warp][d];
    c = __shfl_sync(0xffffffffu, c, leader);
    const uint32_t rank = c + __popc(peers & lt);  // rank within the digit among the warp's items
    rk[r >> 1] = (r & 1) ? (rk[r >> 1] | (rank << 16)) : rank;
    if (valid && lane == leader) S.cnt[warp][d] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread t = digit t: the warps' first slots within the digit, the digit's
  // total, then an exclusive scan of the totals over the digits
  {
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.cnt[w][t];
      S.cnt[w][t] = tot;
      tot += c;
    }
    uint32_t x = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += S.wsum[w];
    const uint32_t st = before + x - tot;
    S.start[t] = st;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) S.cnt[w][t] += st;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    if (wbase + r * 32 + lane < n) {
      const uint32_t lp = S.cnt[warp][(kk[r] >> shift) & 255u] + ((rk[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
      S.key[lp] = kk[r];
      S.val[lp] = vv[r];
    }
  }
  __syncthreads();
  const uint32_t cnt = min((uint32_t)kItems, n - base);
  for (uint32_t i = t; i < cnt; i += kSortThreads) {
    const uint32_t k = S.key[i];
    const uint32_t d = (k >> shift) & 255u;
    const uint32_t pos = S.base[d] + (i - S.start[d]);
    if (pos < n) {
      kout[pos] = k;
      vout[pos] = S.val[i];
    }
  }
}

// ---------------------------------------------------------------------------
// The tile and depth sorts, one kernel per digit pass (decoupled look-back).
// Each block takes the next kSortThreads * ROUNDS items in order by a ticket
// (4096 tile pairs, 1024 depth keys), ranks them as k_radix_scatter does,
// publishes its count of every digit, and adds up the
// counts of the blocks before it from their published words: a block's own
// count (kLookAgg) or, once that block finished its look-back, the count of
// it and of every block before it (kLookPre).  A block waits only on blocks
// with smaller tickets, which have started and never wait on it; every wait
// is bounded: past kLookSpin polls the block records GS3_ERR_TIMEOUT in the
// header and goes on.  The digits' global starts come from totals counted once
// before the first pass, so no histogram pass or device-wide scan runs between
// the passes.  The result is that of the stable LSD passes above.
// ---------------------------------------------------------------------------
constexpr unsigned long long kLookAgg = 1ull << 32;
constexpr unsigned long long kLookPre = 2ull << 32;
constexpr int kLookSpin = 1 << 20;

// Every digit of every pass (PASSES <= 4 eight-bit digits), counted over the
// n keys.  Warp-private counters; a warp whose 32 keys share a digit (the
// usual case for a tile key's second digit, a splat's tiles being
// neighbours, and for the top digits of the depth keys) adds it once.
template <int PASSES>
__global__ void __launch_bounds__(256) k_digit_totals(const uint32_t* __restrict__ keys, const uint32_t* n_ptr,
                                                      uint32_t n_fixed, int passes, uint32_t* __restrict__ totals) {
  __shared__ uint32_t h[PASSES][kSortThreads / 32][256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
#pragma unroll
  for (int p = 0; p < PASSES; ++p)
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) h[p][w][t] = 0;
  __syncthreads();
  const uint32_t n = load_n(n_ptr, n_fixed);
  // each warp takes 128 consecutive keys per step, four coalesced loads in flight per lane
  for (uint32_t wb = (blockIdx.x * (kSortThreads / 32) + warp) * 128u; wb < n; wb += gridDim.x * kSortThreads * 4u) {
    uint32_t k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = wb + 32u * u + lane;
      k[u] = i < n ? keys[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool valid = wb + 32u * u + lane < n;
      const uint32_t vm = __ballot_sync(0xffffffffu, valid);
      if (!vm) break;
#pragma unroll
      for (int p = 0; p < PASSES; ++p) {
        if (p >= passes) break;
        const uint32_t d = (k[u] >> (8 * p)) & 255u;
        const uint32_t first = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, !valid || d == first)) {
          if (lane == 0) h[p][warp][first] += __popc(vm);
        } else if (valid) {
          atomicAdd(&h[p][warp][d], 1u);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) c += h[p][w][t];
    if (c) atomicAdd(&totals[p * 256 + t], c);
  }
}

template <int ROUNDS>
struct OnesweepSmem {
  uint32_t base[256];    // the block's first output slot per digit
  uint32_t start[256];   // first staging slot per digit
  uint32_t cnt[kSortThreads / 32][256];  // per warp and digit: items so far, then the warp's first slot
  uint32_t wsum[kSortThreads / 32], gsum[kSortThreads / 32];
  uint32_t ticket;
  uint32_t key[kSortThreads * ROUNDS], val[kSortThreads * ROUNDS];
};

template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* n_ptr, uint32_t n_fixed, int shift,
    const uint32_t* __restrict__ totals, unsigned long long* look, uint32_t* ticket, uint32_t* header) {
  constexpr int kItems = kSortThreads * ROUNDS;
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ uint4 onesweep_raw[];
  OnesweepSmem<ROUNDS>& S = *reinterpret_cast<OnesweepSmem<ROUNDS>*>(onesweep_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t n = load_n(n_ptr, n_fixed);
  if (t == 0) S.ticket = atomicAdd(ticket, 1u);
#pragma unroll
  for (int w = 0; w < kWarps; ++w) S.cnt[w][t] = 0;
  __syncthreads();
  const uint32_t blk = S.ticket;
  const uint32_t base = blk * (uint32_t)kItems;
  if (base >= n) return;  // every later ticket is past the end as well
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t wbase = base + (uint32_t)warp * (32u * ROUNDS);
  uint32_t kk[ROUNDS], vv[ROUNDS];
  uint32_t rk[(ROUNDS + 1) / 2];  // two 16-bit ranks per word
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const uint32_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    kk[r] = valid ? kin[i] : 0u;
    vv[r] = valid ? (vin ? vin[i] : i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const bool valid = wbase + r * 32 + lane < n;
    const uint32_t d = valid ? (kk[r] >> shift) & 255u : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t c = 0;
    if (valid && lane == leader) c = S.cnt[warp][d];
    c = __shfl_sync(0xffffffffu, c, leader);
    const uint32_t rank = c + __popc(peers & lt);
    rk[r >> 1] = (r & 1) ? (rk[r >> 1] | (rank << 16)) : rank;
    if (valid && lane == leader) S.cnt[warp][d] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread t = digit t: the block's count, published at once
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.cnt[w][t];
      S.cnt[w][t] = tot;
      tot += c;
    }
    volatile unsigned long long* mine = look + (size_t)blk * 256 + t;
    *mine = (blk == 0 ? kLookPre : kLookAgg) | tot;
    // staging starts (scan of the block's counts) and the digit's start over
    // all items (scan of the totals)
    const uint32_t g = totals[t];
    uint32_t x = tot, y = g;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t a = __shfl_up_sync(0xffffffffu, x, o);
      const uint32_t b = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) { x += a; y += b; }
    }
    if (lane == 31) { S.wsum[warp] = x; S.gsum[warp] = y; }
    // the blocks before this one
    uint32_t excl = 0;
    if (blk > 0) {
      uint32_t j = blk - 1;
      int spins = 0;
      for (;;) {
        const unsigned long long v = *(volatile const unsigned long long*)(look + (size_t)j * 256 + t);
        const uint32_t flag = (uint32_t)(v >> 32);
        if (flag == 0u) {
          if (++spins > kLookSpin) {
            atomicCAS(header + H_STATUS, 0u, (uint32_t)GS3_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += (uint32_t)v;
        if (flag == 2u || j == 0u) break;
        --j;
      }
      *mine = kLookPre | (unsigned long long)(excl + tot);
    }
    __syncthreads();
    uint32_t before = 0, gbefore = 0;
    for (int w = 0; w < warp; ++w) { before += S.wsum[w]; gbefore += S.gsum[w]; }
    const uint32_t st = before + x - tot;
    S.start[t] = st;
    S.base[t] = gbefore + y - g + excl;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) S.cnt[w][t] += st;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    if (wbase + r * 32 + lane < n) {
      const uint32_t lp = S.cnt[warp][(kk[r] >> shift) & 255u] + ((rk[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
      S.key[lp] = kk[r];
      S.val[lp] = vv[r];
    }
  }
  __syncthreads();
  const uint32_t cnt = min((uint32_t)kItems, n - base);
  for (uint32_t i = t; i < cnt; i += kSortThreads) {
    const uint32_t k = S.key[i];
    const uint32_t d = (k >> shift) & 255u;
    const uint32_t pos = S.base[d] + (i - S.start[d]);
    if (pos < n) {
      kout[pos] = k;
      vout[pos] = S.val[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Rank order and counts
// ---------------------------------------------------------------------------
// Records into depth-rank order and the tile count of each rank.  Also
// counts, for the block's kBinBlock ranks, the ranks whose rectangle covers
// each tile row y (a difference array over the rows, then its running sum),
// into row_cnt[y][block].
__global__ void __launch_bounds__(kBinBlock) k_reorder(int n, const uint32_t* __restrict__ order,
                                                       const SplatRec* __restrict__ rec, SplatRec* __restrict__ rrec,
                                                       uint32_t* __restrict__ rank_of, uint32_t* __restrict__ cnt,
                                                       const float4* __restrict__ shade, float4* __restrict__ ccol,
                                                       uint32_t* __restrict__ row_cnt, int gy) {
  __shared__ int d[kMaxTileAxis + 1];
  for (int y = threadIdx.x; y <= gy; y += blockDim.x) d[y] = 0;
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t g = r < n ? order[r] : 0xFFFFFFFFu;
  if (g < (uint32_t)n) {
    const SplatRec q = rec[g];
    rrec[r] = q;
    rank_of[g] = r;
    const bool in = q.r.x >= 0;
    cnt[r] = in ? (uint32_t)(q.r.z - q.r.x + 1) * (uint32_t)(q.r.w - q.r.y + 1) : 0u;
    if (in) {
      atomicAdd(&d[q.r.y], 1);
      atomicAdd(&d[q.r.w + 1], -1);
    }
    if (ccol) {
      float4 c = shade[g];
      ccol[2 * r] = make_float4(c.x, c.y, c.z, 0.f);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int run = 0;
    for (int y0 = 0; y0 < gy; y0 += 32) {
      const int y = y0 + lane;
      int v = y < gy ? d[y] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (y < gy) row_cnt[(size_t)y * gridDim.x + blockIdx.x] = (uint32_t)(run + v);
      run += __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

// gs3_depth_order_static: 4096 items per block, three-kernel scans
void radix_sort(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                uint32_t* v1, const uint32_t* n_ptr, uint32_t n_fixed, int nblocks, int passes,
                uint32_t* hist, uint32_t* scan_part, cudaStream_t s) {
  static DeviceOnce once;
  once.run([] {
    return cudaFuncSetAttribute(k_radix_scatter<kSortRounds>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ScatterSmem<kSortRounds>)) == cudaSuccess;
  });
  const uint32_t* ki = kin;
  const uint32_t* vi = vin;
  for (int p = 0; p < passes; ++p) {
    uint32_t* ko = (p & 1) ? k1 : k0;
    uint32_t* vo = (p & 1) ? v1 : v0;
    k_radix_hist<kSortRounds><<<nblocks, kSortThreads, 0, s>>>(ki, n_ptr, n_fixed, 8 * p, hist, nblocks);
    device_exclusive_scan(hist, hist, 256u * nblocks, nullptr, scan_part, s);
    k_radix_scatter<kSortRounds><<<nblocks, kSortThreads, sizeof(ScatterSmem<kSortRounds>), s>>>(
        ki, vi, ko, vo, n_ptr, n_fixed, 8 * p, hist, nblocks);
    count_launch(2);
    ki = ko;
    vi = vo;
  }
}

// Stable LSD sort of (key, value) pairs (vin null: values are the input
// positions) on the low 8 * passes key bits (passes <= PASSES): one
// k_digit_totals, then one k_onesweep per pass.  Even passes write (k0, v0),
// odd passes (k1, v1), each reading the previous pass's output (pass 0 reads
// (kin, vin)).  look_region: onesweep_bytes(nblocks, PASSES) bytes, zeroed here.
template <int ROUNDS, int PASSES>
void onesweep_sort(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                   uint32_t* v1, const uint32_t* n_ptr, uint32_t n_fixed, int nblocks, int passes,
                   unsigned char* look_region, uint32_t* header, cudaStream_t s) {
  static DeviceOnce once;
  once.run([] {
    return cudaFuncSetAttribute(k_onesweep<ROUNDS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(OnesweepSmem<ROUNDS>)) == cudaSuccess;
  });
  unsigned long long* look = reinterpret_cast<unsigned long long*>(look_region);
  uint32_t* tickets = reinterpret_cast<uint32_t*>(look + (size_t)PASSES * 256 * (size_t)nblocks);
  uint32_t* totals = tickets + PASSES;
  cudaMemsetAsync(look_region, 0, onesweep_bytes(nblocks, PASSES), s);
  const int tb_cap = device_sm_count() * 4;
  int tb = n_ptr ? tb_cap : (int)((n_fixed + 1023) / 1024);
  if (tb < 1) tb = 1;
  if (tb > tb_cap) tb = tb_cap;
  k_digit_totals<PASSES><<<tb, kSortThreads, 0, s>>>(kin, n_ptr, n_fixed, passes, totals);
  const uint32_t* ki = kin;
  const uint32_t* vi = vin;
  for (int p = 0; p < passes; ++p) {
    uint32_t* ko = (p & 1) ? k1 : k0;
    uint32_t* vo = (p & 1) ? v1 : v0;
    k_onesweep<ROUNDS><<<nblocks, kSortThreads, sizeof(OnesweepSmem<ROUNDS>), s>>>(
        ki, vi, ko, vo, n_ptr, n_fixed, 8 * p, totals + 256 * p, look + (size_t)p * 256 * nblocks, tickets + p,
        header);
    ki = ko;
    vi = vo;
  }
  count_launch(1 + passes);
}

}  // namespace

size_t scan_scratch_words(size_t n) { return (n + kScanItems - 1) / kScanItems + 1; }

void radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                      uint32_t* v1, uint32_t n, int passes, uint32_t* hist, uint32_t* scan_part,
                      cudaStream_t s) {
  const int nblocks = (int)((n + kSortTileItems - 1) / kSortTileItems);
  radix_sort(kin, vin, k0, v0, k1, v1, nullptr, n, nblocks, passes, hist, scan_part, s);
}

void device_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total,
                           uint32_t* scratch, cudaStream_t s) {
  const uint32_t nb = (n + kScanItems - 1) / kScanItems;
  if (nb == 0) return;
  k_scan_reduce<<<nb, 256, 0, s>>>(in, n, scratch);
  k_scan_part<<<1, 1024, 0, s>>>(scratch, nb, total);
  k_scan_down<<<nb, 256, 0, s>>>(in, out, n, scratch);
  count_launch(3);
}

void launch_depth_sort(const FrameArgs& f, int sp, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[sp];
  unsigned char* ws = f.ws;
  const int n = f.sc.n;
  // 1024 keys per block: four times the blocks of the pair sorts, for a
  // sort of a few hundred thousand keys that would otherwise leave SMs idle
  onesweep_sort<kDepthSortRounds, 4>(at<uint32_t>(ws, b.key), nullptr, at<uint32_t>(ws, b.sk[0]),
                                     at<uint32_t>(ws, b.sv[0]), at<uint32_t>(ws, b.sk[1]), at<uint32_t>(ws, b.sv[1]),
                                     nullptr, (uint32_t)n, f.L->nb_n, 4, at<unsigned char>(ws, b.dlook),
                                     at<uint32_t>(ws, f.L->header), s);
  // 4 passes end in buffer 1: sv[1] holds the index of each depth rank
  k_reorder<<<f.L->nb_rows, kBinBlock, 0, s>>>(
      n, at<uint32_t>(ws, b.sv[1]), at<SplatRec>(ws, b.rec), at<SplatRec>(ws, b.rrec),
      at<uint32_t>(ws, b.rank_of), at<uint32_t>(ws, b.cnt), at<float4>(ws, f.L->shade),
      sp == 0 ? at<float4>(ws, f.L->ccol) : nullptr, at<uint32_t>(ws, b.row_cnt), f.L->gy);
  count_launch();
}

}  // namespace gs3

// Self-test of the bounded waits: one look-back pass over n zero keys whose
// tickets start at 1, so every block's look-back reaches ticket 0's words,
// which no block writes.  Each such wait must give up after kLookSpin polls
// and record GS3_ERR_TIMEOUT; the pass then finishes.
extern "C" gs3_status gs3_selftest_wait_timeout(uint32_t n, uint32_t* status_out) {
  using namespace gs3;
  if (!status_out || n <= (uint32_t)kTileSortItems || n > (1u << 20)) {
    set_last_error("gs3_selftest_wait_timeout: need status_out and 4096 < n <= 1 << 20");
    return GS3_ERR_INVALID_ARG;
  }
  const int nblocks = (int)((n + kTileSortItems - 1) / kTileSortItems);
  const size_t look = onesweep_bytes(nblocks, 1);
  const size_t bytes = 16ull * n + look + 16;
  unsigned char* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    set_last_error("gs3_selftest_wait_timeout: cudaMalloc failed");
    return GS3_ERR_OOM;
  }
  uint32_t* kin = reinterpret_cast<uint32_t*>(d);
  uint32_t* vin = kin + n;
  uint32_t* kout = vin + n;
  uint32_t* vout = kout + n;
  unsigned long long* lk = reinterpret_cast<unsigned long long*>(d + 16ull * n);
  uint32_t* tickets = reinterpret_cast<uint32_t*>(lk + 256ull * nblocks);
  uint32_t* totals = tickets + 1;
  uint32_t* status = reinterpret_cast<uint32_t*>(d + 16ull * n + look);
  const uint32_t first_ticket = 1;
  cudaError_t e = cudaMemset(d, 0, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(tickets, &first_ticket, 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    cudaFuncSetAttribute(k_onesweep<kTileSortRounds>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(OnesweepSmem<kTileSortRounds>));
    k_onesweep<kTileSortRounds><<<nblocks, kSortThreads, sizeof(OnesweepSmem<kTileSortRounds>)>>>(
        kin, vin, kout, vout, nullptr, n, 0, totals, lk, tickets, status);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status_out, status, 4, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_last_error("gs3_selftest_wait_timeout: CUDA call failed");
    return GS3_ERR_CUDA;
  }
  return GS3_OK;
}
