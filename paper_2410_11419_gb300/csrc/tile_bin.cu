// K4-K5: tile binning of one splat (camera or light): for every tile, the
// depth ranks of the Gaussians whose tile rectangle covers it, in rank order,
// and the tiles' [start, end) ranges (Sec. 3; the light view is binned the
// same way, Sec. 4.2).
//
// A rank's (tile, rank) pairs are the tiles of its rectangle, so the lists
// are built from the rectangles by two stable counting passes instead of
// emitting the pairs and sorting them on the tile bits:
//   rows     the ranks covering tile row y, for every y, in rank order: the
//            counts per (row, block of kBinBlock ranks) come from k_reorder;
//            k_bin_plan scans them (row-major), k_bin_rows places the ranks;
//   columns  each row's rank sequence is cut into chunks of bin_chunk(gx)
//            items; k_bin_count counts the items per (row, column, chunk);
//            k_bin_rowscan scans each row's counts in (column, chunk) order,
//            after the pairs of the rows above, which gives every tile's
//            start and every chunk's offset in each of its tiles; k_bin_place
//            writes the list entries.
// Inside a block of 256 items the position of an item among the items
// covering the same row (or column) is the count of earlier warps plus the
// popcount of the lower lanes in a ballot, each warp sweeping the union of
// its lanes' spans once.  Every list is therefore in rank order, the result
// a stable sort of the pairs by tile would give, and no step depends on
// timing or waits on another block.
#include <climits>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kBinThreads = 256;  // 8 warps
constexpr int kBinWarps = kBinThreads / 32;

// Exclusive scan of v[0, len) in place, starting at carry, by one block of
// NT threads (four consecutive words per thread per step); returns carry plus
// the sum.  sm: 32 words of shared memory.  Every thread must call it.
template <int NT>
__device__ uint32_t block_scan_inplace(uint32_t* v, size_t len, uint32_t carry, uint32_t* sm) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  constexpr int kWarps = NT / 32;
  for (size_t base = 0; base < len; base += 4 * NT) {
    uint32_t x[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t i = base + 4 * (size_t)t + j;
      x[j] = i < len ? v[i] : 0u;
      s += x[j];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
      uint32_t u = lane < kWarps ? sm[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t z = __shfl_up_sync(0xffffffffu, u, o);
        if (lane >= o) u += z;
      }
      if (lane < kWarps) sm[lane] = u;
    }
    __syncthreads();
    uint32_t pre = carry + (w ? sm[w - 1] : 0u) + inc - s;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t i = base + 4 * (size_t)t + j;
      if (i < len) v[i] = pre;
      pre += x[j];
    }
    carry += sm[kWarps - 1];
    __syncthreads();  // sm is rewritten by the next step
  }
  return carry;
}

// the sum of every thread's x over a block of kBinThreads (all threads get it)
__device__ uint32_t block_sum(uint32_t x, uint32_t* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kBinWarps; ++k) s += sm[k];
  __syncthreads();
  return s;
}

// The plan words: rs[gy + 1] row starts in the row sequence, cb[gy + 1]
// chunk starts (every row has at least one chunk), pairs[gy] list entries
// per row, ok (the pairs fit the capacity).
struct BinPlan {
  uint32_t *rs, *cb, *pairs, *ok;
  __device__ BinPlan(uint32_t* p, int gy) : rs(p), cb(p + gy + 1), pairs(p + 2 * gy + 2), ok(p + 3 * gy + 2) {}
};

// the row of chunk kg: the largest y with cb[y] <= kg (cb[0] = 0 <= kg < cb[gy])
__device__ __forceinline__ int chunk_row(const uint32_t* cb, int gy, uint32_t kg) {
  int lo = 0, hi = gy;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cb[mid] <= kg) lo = mid; else hi = mid;
  }
  return lo;
}

// One block of 1024 threads: scans the row counts (row-major, so that the
// counts of row y start at the row's place in the row sequence), cuts every
// row into chunks, and checks that the pairs fit the capacity.
__global__ void __launch_bounds__(1024) k_bin_plan(uint32_t* __restrict__ row_cnt, int nb, int gy, uint32_t ch,
                                                  size_t tab_words, int gx, uint32_t* __restrict__ plan,
                                                  uint32_t* header, int h_need, int h_pairs, size_t cap) {
  __shared__ uint32_t sm[32];
  const uint32_t M = block_scan_inplace<1024>(row_cnt, (size_t)gy * nb, 0u, sm);
  BinPlan P(plan, gy);
  const int y = threadIdx.x, lane = y & 31, w = y >> 5;
  uint32_t nch = 0;
  if (y < gy) {
    const uint32_t a = row_cnt[(size_t)y * nb];
    const uint32_t e = y + 1 < gy ? row_cnt[(size_t)(y + 1) * nb] : M;
    P.rs[y] = a;
    P.pairs[y] = 0u;
    const uint32_t c = (uint32_t)(((uint64_t)(e - a) + ch - 1) / ch);
    nch = c > 1u ? c : 1u;
  }
  if (y == 0) P.rs[gy] = M;
  uint32_t inc = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t u = sm[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += z;
    }
    sm[lane] = u;
  }
  __syncthreads();
  if (y < gy) P.cb[y] = (w ? sm[w - 1] : 0u) + inc - nch;
  if (y == 0) {
    const uint32_t C = sm[31];
    P.cb[gy] = C;
    const uint32_t need = header[h_need];
    const bool ok = need <= cap && (size_t)C * (size_t)gx <= tab_words;
    header[h_pairs] = ok ? need : 0u;
    if (!ok) atomicCAS(&header[H_STATUS], 0u, (uint32_t)GS3_ERR_CAPACITY);
    *P.ok = ok ? 1u : 0u;
  }
}

// The row sequence: rank r goes to every row of its rectangle, at the row's
// offset for r's block, plus the ranks of earlier warps and lower lanes of
// the block covering that row.
__global__ void __launch_bounds__(kBinThreads) k_bin_rows(int n, const SplatRec* __restrict__ rrec,
                                                          const uint32_t* __restrict__ row_cnt, int nb, int gy,
                                                          const uint32_t* __restrict__ plan,
                                                          uint32_t* __restrict__ rowseq, size_t cap) {
  __shared__ uint32_t wc[kBinWarps][kMaxTileAxis];
  __shared__ int wlo[kBinWarps], whi[kBinWarps];
  if (plan[3 * gy + 2] == 0u) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kBinThreads + threadIdx.x;
  int a = 0, b = -1;  // the rank's rows
  if (r < n) {
    const int4 q = rrec[r].r;
    if (q.x >= 0) {
      a = q.y;
      b = q.w;
    }
  }
  const int lo = __reduce_min_sync(0xffffffffu, a <= b ? a : INT_MAX);
  const int hi = __reduce_max_sync(0xffffffffu, a <= b ? b : -1);
  for (int y = lo; y <= hi; ++y) {
    const uint32_t m = __ballot_sync(0xffffffffu, a <= y && y <= b);
    if (lane == 0) wc[w][y] = (uint32_t)__popc(m);
  }
  if (lane == 0) {
    wlo[w] = lo;
    whi[w] = hi;
  }
  __syncthreads();
  for (int y = threadIdx.x; y < gy; y += kBinThreads) {
    uint32_t run = row_cnt[(size_t)y * nb + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kBinWarps; ++k) {
      const uint32_t c = (y >= wlo[k] && y <= whi[k]) ? wc[k][y] : 0u;
      wc[k][y] = run;
      run += c;
    }
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (int y = lo; y <= hi; ++y) {
    const bool cov = a <= y && y <= b;
    const uint32_t m = __ballot_sync(0xffffffffu, cov);
    if (cov) {
      const uint32_t pos = wc[w][y] + (uint32_t)__popc(m & lt);
      if (pos < cap) rowseq[pos] = (uint32_t)r;
    }
  }
}

// Counts per (row, column, chunk): a difference array over the columns of
// the chunk's rectangles, then its running sum, at tab[cb[y] gx + x nch + k]
// (row y's counts in (column, chunk) order); adds the chunk's list entries
// to the row's pairs.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const SplatRec* __restrict__ rrec,
                                                           const uint32_t* __restrict__ rowseq,
                                                           uint32_t* __restrict__ plan, int gx, int gy, uint32_t ch,
                                                           uint32_t* __restrict__ tab) {
  __shared__ int d[kMaxTileAxis + 1];
  __shared__ uint32_t sm[32];
  BinPlan P(plan, gy);
  if (*P.ok == 0u) return;
  const uint32_t C = P.cb[gy];
  for (uint32_t kg = blockIdx.x; kg < C; kg += gridDim.x) {
    const int y = chunk_row(P.cb, gy, kg);
    const uint32_t c0 = P.cb[y], nch = P.cb[y + 1] - c0, k = kg - c0;
    const uint32_t i0 = P.rs[y] + k * ch, i1 = min(P.rs[y + 1], i0 + ch);
    for (int x = threadIdx.x; x <= gx; x += kBinThreads) d[x] = 0;
    __syncthreads();
    uint32_t width = 0;
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += kBinThreads) {
      const int4 q = rrec[rowseq[i]].r;
      atomicAdd(&d[q.x], 1);
      atomicAdd(&d[q.z + 1], -1);
      width += (uint32_t)(q.z - q.x + 1);
    }
    const uint32_t total = block_sum(width, sm);  // also orders the difference array's updates
    if (threadIdx.x == 0 && total) atomicAdd(P.pairs + y, total);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      uint32_t* out = tab + (size_t)c0 * gx + k;
      int run = 0;
      for (int x0 = 0; x0 < gx; x0 += 32) {
        const int x = x0 + lane;
        int v = x < gx ? d[x] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += t;
        }
        if (x < gx) out[(size_t)x * nch] = (uint32_t)(run + v);
        run += __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();  // d is cleared for the next chunk
  }
}

// One block per row: the row's counts scanned in (column, chunk) order after
// the list entries of the rows above; tile (y, x) starts at the scanned count
// of its first chunk.  The last row also writes the end of the last tile.
__global__ void __launch_bounds__(kBinThreads) k_bin_rowscan(uint32_t* __restrict__ tab,
                                                             const uint32_t* __restrict__ plan, int gx, int gy,
                                                             uint32_t* __restrict__ tile_start) {
  __shared__ uint32_t sm[32];
  const int y = blockIdx.x;
  const uint32_t* cb = plan + gy + 1;
  const uint32_t* pairs = plan + 2 * gy + 2;
  uint32_t* ts = tile_start + (size_t)y * gx;
  if (plan[3 * gy + 2] == 0u) {  // over capacity: every list empty
    for (int x = threadIdx.x; x < gx; x += kBinThreads) ts[x] = 0u;
    if (y == gy - 1 && threadIdx.x == 0) tile_start[(size_t)gx * gy] = 0u;
    return;
  }
  uint32_t above = 0;
  for (int t = threadIdx.x; t < y; t += kBinThreads) above += pairs[t];
  above = block_sum(above, sm);
  const uint32_t c0 = cb[y], nch = cb[y + 1] - c0;
  uint32_t* seg = tab + (size_t)c0 * gx;
  const uint32_t end = block_scan_inplace<kBinThreads>(seg, (size_t)nch * gx, above, sm);
  for (int x = threadIdx.x; x < gx; x += kBinThreads) ts[x] = seg[(size_t)x * nch];
  if (y == gy - 1 && threadIdx.x == 0) tile_start[(size_t)gx * gy] = end;
}

// The list entries: each chunk in sub-chunks of 256 items; column x of a
// sub-chunk's warp k starts at the chunk's running offset in tile (y, x)
// plus the items of warps 0..k-1 covering x, and an item at the popcount of
// the lower lanes covering x.
__global__ void __launch_bounds__(kBinThreads) k_bin_place(const SplatRec* __restrict__ rrec,
                                                           const uint32_t* __restrict__ rowseq,
                                                           const uint32_t* __restrict__ plan,
                                                           const uint32_t* __restrict__ tab, int gx, int gy,
                                                           uint32_t ch, uint32_t* __restrict__ list, size_t cap) {
  __shared__ uint32_t wc[kBinWarps][kMaxTileAxis];
  __shared__ uint32_t run[kMaxTileAxis];
  __shared__ int wlo[kBinWarps], whi[kBinWarps];
  const uint32_t* rs = plan;
  const uint32_t* cb = plan + gy + 1;
  if (plan[3 * gy + 2] == 0u) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t C = cb[gy];
  for (uint32_t kg = blockIdx.x; kg < C; kg += gridDim.x) {
    const int y = chunk_row(cb, gy, kg);
    const uint32_t c0 = cb[y], nch = cb[y + 1] - c0, k = kg - c0;
    const uint32_t i0 = rs[y] + k * ch, i1 = min(rs[y + 1], i0 + ch);
    // each thread reads back only the columns it wrote
    for (int x = threadIdx.x; x < gx; x += kBinThreads) run[x] = tab[(size_t)c0 * gx + (size_t)x * nch + k];
    for (uint32_t sub = i0; sub < i1; sub += kBinThreads) {
      const uint32_t i = sub + threadIdx.x;
      int a = 0, b = -1;  // the item's columns
      uint32_t r = 0;
      if (i < i1) {
        r = rowseq[i];
        const int4 q = rrec[r].r;
        a = q.x;
        b = q.z;
      }
      const int lo = __reduce_min_sync(0xffffffffu, a <= b ? a : INT_MAX);
      const int hi = __reduce_max_sync(0xffffffffu, a <= b ? b : -1);
      for (int x = lo; x <= hi; ++x) {
        const uint32_t m = __ballot_sync(0xffffffffu, a <= x && x <= b);
        if (lane == 0) wc[w][x] = (uint32_t)__popc(m);
      }
      if (lane == 0) {
        wlo[w] = lo;
        whi[w] = hi;
      }
      __syncthreads();
      for (int x = threadIdx.x; x < gx; x += kBinThreads) {
        uint32_t base = run[x];
#pragma unroll
        for (int kk = 0; kk < kBinWarps; ++kk) {
          const uint32_t c = (x >= wlo[kk] && x <= whi[kk]) ? wc[kk][x] : 0u;
          wc[kk][x] = base;
          base += c;
        }
        run[x] = base;
      }
      __syncthreads();
      for (int x = lo; x <= hi; ++x) {
        const bool cov = a <= x && x <= b;
        const uint32_t m = __ballot_sync(0xffffffffu, cov);
        if (cov) {
          const uint32_t pos = wc[w][x] + (uint32_t)__popc(m & lt);
          if (pos < cap) list[pos] = r;
        }
      }
      __syncthreads();  // wc, wlo and whi are rewritten by the next sub-chunk
    }
  }
}

}  // namespace

void launch_binning(const FrameArgs& f, int sp, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[sp];
  unsigned char* ws = f.ws;
  const int n = f.sc.n;
  const int gx = f.L->gx, gy = f.L->gy, nb = f.L->nb_rows;
  const size_t cap = f.L->cap;
  uint32_t* header = at<uint32_t>(ws, f.L->header);
  const int h_need = sp ? H_NEED_LIGHT : H_NEED_CAM;
  const int h_pairs = sp ? H_PAIRS_LIGHT : H_PAIRS_CAM;
  // every rank's first list slot in rank order (the shadow partials' slots) and the total
  device_exclusive_scan(at<uint32_t>(ws, b.cnt), at<uint32_t>(ws, b.off), (uint32_t)n, header + h_need,
                        at<uint32_t>(ws, b.scan_part), s);
  // the lists go where the composites and the backward read them
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  uint32_t* rowseq = at<uint32_t>(ws, b.tk[fin]);
  uint32_t* list = at<uint32_t>(ws, b.tv[fin]);
  uint32_t* row_cnt = at<uint32_t>(ws, b.row_cnt);
  uint32_t* plan = at<uint32_t>(ws, b.bin_plan);
  uint32_t* tab = at<uint32_t>(ws, b.bin_tab);
  const SplatRec* rrec = at<SplatRec>(ws, b.rrec);
  const uint32_t ch = bin_chunk(gx);
  k_bin_plan<<<1, 1024, 0, s>>>(row_cnt, nb, gy, ch, bin_tab_words(cap, gx, gy), gx, plan, header, h_need, h_pairs,
                                cap);
  k_bin_rows<<<nb, kBinThreads, 0, s>>>(n, rrec, row_cnt, nb, gy, plan, rowseq, cap);
  const size_t chunks = cap / ch + (size_t)gy + 1;
  int grid = device_sm_count() * 6;
  if ((size_t)grid > chunks) grid = (int)chunks;
  k_bin_count<<<grid, kBinThreads, 0, s>>>(rrec, rowseq, plan, gx, gy, ch, tab);
  k_bin_rowscan<<<gy, kBinThreads, 0, s>>>(tab, plan, gx, gy, at<uint32_t>(ws, b.tile_start));
  k_bin_place<<<grid, kBinThreads, 0, s>>>(rrec, rowseq, plan, tab, gx, gy, ch, list, cap);
  count_launch(5);
}

}  // namespace gs3
