// K4-K5: tile binning of one splat (camera or light): for every tile, the
// depth ranks of the Gaussians whose tile rectangle covers it, in rank order,
// and the tiles' [start, end) ranges (Sec. 3; the light view is binned the
// same way, Sec. 4.2).
//
// A rank's (tile, rank) pairs are the tiles of its rectangle, so the lists
// are built from the rectangles by two stable counting passes instead of
// emitting the pairs and sorting them on the tile bits:
//   rows     the ranks covering tile row y, for every y, in rank order, with
//            each rank's column span beside it: the counts per (row, block
//            of kBinBlock ranks) come from k_reorder; k_bin_rowtot scans each
//            row's counts, k_bin_plan the row totals; k_bin_rows places;
//   columns  each row's sequence is cut into chunks of bin_chunk(gx) items;
//            k_bin_count counts the items per (row, column, chunk);
//            k_bin_rowscan scans each row's counts in (column, chunk) order,
//            after the pairs of the rows above, which gives every tile's
//            start and every chunk's offset in each of its tiles; k_bin_place
//            writes the list entries.
// Both placements take 256 items at a time, one per thread, in order.  A
// warp's offset in bucket x is the bucket's running offset plus the items of
// earlier warps covering x (per-warp difference arrays); inside a warp the
// (item, bucket) pairs are dealt 32 per round in item order, and a pair's
// rank among the round's pairs of the same bucket (match_any) is added to a
// per-bucket counter.  Every list is therefore in rank order, the result a
// stable sort of the pairs by tile would give, and no step depends on timing
// or waits on another block.
#include <climits>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kBinThreads = 256;  // 8 warps
constexpr int kBinWarps = kBinThreads / 32;

__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

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
    const uint32_t inc = warp_inclusive_sum(s, lane);
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
      const uint32_t u = warp_inclusive_sum(lane < kWarps ? sm[lane] : 0u, lane);
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

// the sum of every thread's x over a block of NT threads (all threads get it)
template <int NT>
__device__ uint32_t block_sum(uint32_t x, uint32_t* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) s += sm[k];
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

// Shared memory of a span placement (about 41 KB).
struct SpanSmem {
  int cnt[kBinWarps][kMaxTileAxis + 1];  // per warp: difference array, counts, then offsets per bucket
  uint32_t run[kMaxTileAxis];            // per bucket: the running offset
  uint32_t ex[kBinWarps][32];            // per warp: exclusive prefix of the lanes' span widths
  int lo[kBinWarps][32];                 // per warp: the lanes' first buckets
  uint32_t v0[kBinWarps][32], v1[kBinWarps][32];  // per warp: the lanes' payloads
};

// Stable placement of 256 items, one per thread in thread order: an item with
// a <= b covers buckets a..b, and its copy for bucket x goes to
// out0 / out1[S.run[x] + the items of lower threads covering x].  S.run must
// hold the buckets' offsets and is advanced past the items.  Every thread of
// the block calls it.
__device__ void place_spans(SpanSmem& S, int nbk, int a, int b, uint32_t v0, uint32_t v1,
                            uint32_t* __restrict__ out0, uint32_t* __restrict__ out1, size_t cap) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* c = S.cnt[w];
  for (int x = lane; x <= nbk; x += 32) c[x] = 0;
  __syncwarp();
  const bool has = a <= b;
  if (has) {
    atomicAdd(&c[a], 1);
    atomicAdd(&c[b + 1], -1);
  }
  __syncwarp();
  uint32_t carry = 0;  // the warp's items per bucket: running sum of the difference array
  for (int x0 = 0; x0 < nbk; x0 += 32) {
    const int x = x0 + lane;
    const uint32_t v = warp_inclusive_sum(x < nbk ? (uint32_t)c[x] : 0u, lane);
    if (x < nbk) c[x] = (int)(carry + v);
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nbk; x += kBinThreads) {  // warp k starts after warps 0..k-1
    uint32_t base = S.run[x];
#pragma unroll
    for (int k = 0; k < kBinWarps; ++k) {
      const uint32_t n = (uint32_t)S.cnt[k][x];
      S.cnt[k][x] = (int)base;
      base += n;
    }
    S.run[x] = base;
  }
  __syncthreads();
  // the warp's (item, bucket) pairs in item order, 32 per round
  const uint32_t wid = has ? (uint32_t)(b - a + 1) : 0u;
  const uint32_t inc = warp_inclusive_sum(wid, lane);
  const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
  S.ex[w][lane] = inc - wid;
  S.lo[w][lane] = a;
  S.v0[w][lane] = v0;
  S.v1[w][lane] = v1;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  // four rounds at a time: their item searches are independent, so they run
  // side by side; the counters are then read and advanced round by round
  for (uint32_t p0 = 0; p0 < total; p0 += 128) {
    int jq[4], xq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t p = p0 + 32 * q + lane;
      int j = 0;  // the item of pair p: the last lane j with ex[j] <= p
#pragma unroll
      for (int s = 16; s > 0; s >>= 1)
        if (S.ex[w][j + s] <= p) j += s;
      jq[q] = j;
      xq[q] = S.lo[w][j] + (int)(p - S.ex[w][j]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (p0 + 32 * q >= total) break;  // the same for every lane
      const bool act = p0 + 32 * q + lane < total;
      const int j = jq[q], x = xq[q];
      const uint32_t m = __match_any_sync(0xffffffffu, act ? x : -1 - lane);
      if (act) {
        const uint32_t pos = (uint32_t)c[x] + (uint32_t)__popc(m & lt);
        if (pos < cap) {
          out0[pos] = S.v0[w][j];
          if (out1) out1[pos] = S.v1[w][j];
        }
      }
      __syncwarp();  // every lane has read its bucket's counter
      if (act && (m >> lane) == 1u) c[x] += __popc(m);
      __syncwarp();
    }
  }
  __syncthreads();  // S is rewritten by the next call
}

// Each row's block counts scanned in place (exclusive, within the row); the
// row's total goes to rs[y] for k_bin_plan.
__global__ void __launch_bounds__(kBinThreads) k_bin_rowtot(uint32_t* __restrict__ row_cnt, int nb, int gy,
                                                            uint32_t* __restrict__ plan) {
  __shared__ uint32_t sm[32];
  const int y = blockIdx.x;
  const uint32_t t = block_scan_inplace<kBinThreads>(row_cnt + (size_t)y * nb, (size_t)nb, 0u, sm);
  if (threadIdx.x == 0) plan[y] = t;
}

// One block of 1024 threads (gy <= 1024, one row per thread): row starts from
// the row totals, chunks per row and their starts, and the capacity check.
__global__ void __launch_bounds__(1024) k_bin_plan(int gy, uint32_t ch, size_t tab_words, int gx,
                                                  uint32_t* __restrict__ plan, uint32_t* header, int h_need,
                                                  int h_pairs, size_t cap) {
  __shared__ uint32_t sm[32];
  BinPlan P(plan, gy);
  const int y = threadIdx.x, lane = y & 31, w = y >> 5;
  const uint32_t m = y < gy ? P.rs[y] : 0u;  // the row's total
  const uint32_t c = (uint32_t)(((uint64_t)m + ch - 1) / ch);
  const uint32_t nch = y < gy ? (c > 1u ? c : 1u) : 0u;
  // exclusive prefixes of (m, nch) over the rows
  const uint32_t im = warp_inclusive_sum(m, lane), ic = warp_inclusive_sum(nch, lane);
  if (lane == 31) sm[w] = im;
  __syncthreads();
  const uint32_t wm = w == 0 ? warp_inclusive_sum(sm[lane], lane) : 0u;
  __syncthreads();
  if (w == 0) sm[lane] = wm;
  __syncthreads();
  const uint32_t rs = (w ? sm[w - 1] : 0u) + im - m, M = sm[31];
  __syncthreads();
  if (lane == 31) sm[w] = ic;
  __syncthreads();
  const uint32_t wc = w == 0 ? warp_inclusive_sum(sm[lane], lane) : 0u;
  __syncthreads();
  if (w == 0) sm[lane] = wc;
  __syncthreads();
  const uint32_t cb = (w ? sm[w - 1] : 0u) + ic - nch, C = sm[31];
  if (y < gy) {
    P.rs[y] = rs;
    P.cb[y] = cb;
    P.pairs[y] = 0u;
  }
  if (y == 0) {
    P.rs[gy] = M;
    P.cb[gy] = C;
    const uint32_t need = header[h_need];
    const bool ok = need <= cap && (size_t)C * (size_t)gx <= tab_words;
    header[h_pairs] = ok ? need : 0u;
    if (!ok) atomicCAS(&header[H_STATUS], 0u, (uint32_t)GS3_ERR_CAPACITY);
    *P.ok = ok ? 1u : 0u;
  }
}

// The row sequence: the block's 256 ranks over their rows, each copy with the
// rank's column span (x0 | x1 << 16) beside it; row y's offset for this block
// is the row's start plus the row's counts of the blocks before.
__global__ void __launch_bounds__(kBinThreads) k_bin_rows(int n, const SplatRec* __restrict__ rrec,
                                                          const uint32_t* __restrict__ row_cnt, int nb, int gy,
                                                          const uint32_t* __restrict__ plan,
                                                          uint32_t* __restrict__ rowseq, uint32_t* __restrict__ rowspan,
                                                          size_t cap) {
  __shared__ SpanSmem S;
  if (plan[3 * gy + 2] == 0u) return;
  for (int y = threadIdx.x; y < gy; y += kBinThreads) S.run[y] = plan[y] + row_cnt[(size_t)y * nb + blockIdx.x];
  const int r = blockIdx.x * kBinThreads + threadIdx.x;
  int a = 0, b = -1;
  uint32_t span = 0;
  if (r < n) {
    const int4 q = rrec[r].r;
    if (q.x >= 0) {
      a = q.y;
      b = q.w;
      span = (uint32_t)q.x | ((uint32_t)q.z << 16);
    }
  }
  __syncthreads();
  place_spans(S, gy, a, b, (uint32_t)r, span, rowseq, rowspan, cap);
}

// Counts per (row, column, chunk): a difference array over the columns of
// the chunk's spans, then its running sum, at tab[cb[y] gx + x nch + k]
// (row y's counts in (column, chunk) order); adds the chunk's list entries
// to the row's pairs.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const uint32_t* __restrict__ rowspan,
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
      const uint32_t sp = rowspan[i];
      const int x0 = (int)(sp & 0xFFFFu), x1 = (int)(sp >> 16);
      atomicAdd(&d[x0], 1);
      atomicAdd(&d[x1 + 1], -1);
      width += (uint32_t)(x1 - x0 + 1);
    }
    const uint32_t total = block_sum<kBinThreads>(width, sm);  // also orders the difference array's updates
    if (threadIdx.x == 0 && total) atomicAdd(P.pairs + y, total);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      uint32_t* out = tab + (size_t)c0 * gx + k;
      uint32_t run = 0;
      for (int x0 = 0; x0 < gx; x0 += 32) {
        const int x = x0 + lane;
        const uint32_t v = warp_inclusive_sum(x < gx ? (uint32_t)d[x] : 0u, lane);
        if (x < gx) out[(size_t)x * nch] = run + v;
        run += __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();  // d is cleared for the next chunk
  }
}

// One block per row: the row's counts scanned in (column, chunk) order after
// the list entries of the rows above; tile (y, x) starts at the scanned count
// of its first chunk.  The last row also writes the end of the last tile.
__global__ void __launch_bounds__(1024) k_bin_rowscan(uint32_t* __restrict__ tab, const uint32_t* __restrict__ plan,
                                                      int gx, int gy, uint32_t* __restrict__ tile_start) {
  __shared__ uint32_t sm[32];
  const int y = blockIdx.x;
  const uint32_t* cb = plan + gy + 1;
  const uint32_t* pairs = plan + 2 * gy + 2;
  uint32_t* ts = tile_start + (size_t)y * gx;
  if (plan[3 * gy + 2] == 0u) {  // over capacity: every list empty
    for (int x = threadIdx.x; x < gx; x += blockDim.x) ts[x] = 0u;
    if (y == gy - 1 && threadIdx.x == 0) tile_start[(size_t)gx * gy] = 0u;
    return;
  }
  uint32_t above = 0;
  for (int t = threadIdx.x; t < y; t += blockDim.x) above += pairs[t];
  above = block_sum<1024>(above, sm);
  const uint32_t c0 = cb[y], nch = cb[y + 1] - c0;
  uint32_t* seg = tab + (size_t)c0 * gx;
  const uint32_t end = block_scan_inplace<1024>(seg, (size_t)nch * gx, above, sm);
  for (int x = threadIdx.x; x < gx; x += blockDim.x) ts[x] = seg[(size_t)x * nch];
  if (y == gy - 1 && threadIdx.x == 0) tile_start[(size_t)gx * gy] = end;
}

// The list entries: each chunk in steps of 256 items over their columns,
// starting at the chunk's offsets in its tiles.  With dist (the light
// splat), each entry's distance goes beside it: the depth sort's key of rank
// r is the FP32 bit pattern of r's light distance.
__global__ void __launch_bounds__(kBinThreads) k_bin_place(const uint32_t* __restrict__ rowseq,
                                                           const uint32_t* __restrict__ rowspan,
                                                           const uint32_t* __restrict__ plan,
                                                           const uint32_t* __restrict__ tab, int gx, int gy,
                                                           uint32_t ch, const uint32_t* __restrict__ rank_key,
                                                           uint32_t* __restrict__ list, uint32_t* __restrict__ dist,
                                                           size_t cap) {
  __shared__ SpanSmem S;
  const uint32_t* rs = plan;
  const uint32_t* cb = plan + gy + 1;
  if (plan[3 * gy + 2] == 0u) return;
  const uint32_t C = cb[gy];
  for (uint32_t kg = blockIdx.x; kg < C; kg += gridDim.x) {
    const int y = chunk_row(cb, gy, kg);
    const uint32_t c0 = cb[y], nch = cb[y + 1] - c0, k = kg - c0;
    const uint32_t i0 = rs[y] + k * ch, i1 = min(rs[y + 1], i0 + ch);
    for (int x = threadIdx.x; x < gx; x += kBinThreads) S.run[x] = tab[(size_t)c0 * gx + (size_t)x * nch + k];
    __syncthreads();
    for (uint32_t sub = i0; sub < i1; sub += kBinThreads) {
      const uint32_t i = sub + threadIdx.x;
      int a = 0, b = -1;
      uint32_t r = 0, key = 0;
      if (i < i1) {
        r = rowseq[i];
        const uint32_t sp = rowspan[i];
        a = (int)(sp & 0xFFFFu);
        b = (int)(sp >> 16);
        if (dist) key = rank_key[r];
      }
      place_spans(S, gx, a, b, r, key, list, dist, cap);
    }
    __syncthreads();  // S.run is rewritten for the next chunk
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
  // the lists go where the composites and the backward read them, and for
  // the light splat each entry's distance where the occluder bounds read it;
  // the row sequence and spans use buffers that are free until then
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  uint32_t* list = at<uint32_t>(ws, b.tv[fin]);
  uint32_t* dist = sp ? at<uint32_t>(ws, b.tk[1 - fin]) : nullptr;
  uint32_t* rowseq = at<uint32_t>(ws, b.tk[fin]);
  uint32_t* rowspan = at<uint32_t>(ws, b.tv[1 - fin]);
  uint32_t* row_cnt = at<uint32_t>(ws, b.row_cnt);
  uint32_t* plan = at<uint32_t>(ws, b.bin_plan);
  uint32_t* tab = at<uint32_t>(ws, b.bin_tab);
  const uint32_t ch = bin_chunk(gx);
  k_bin_rowtot<<<gy, kBinThreads, 0, s>>>(row_cnt, nb, gy, plan);
  k_bin_plan<<<1, 1024, 0, s>>>(gy, ch, bin_tab_words(cap, gx, gy), gx, plan, header, h_need, h_pairs, cap);
  k_bin_rows<<<nb, kBinThreads, 0, s>>>(n, at<SplatRec>(ws, b.rrec), row_cnt, nb, gy, plan, rowseq, rowspan, cap);
  const size_t chunks = cap / ch + (size_t)gy + 1;
  int grid = device_sm_count() * 5;
  if ((size_t)grid > chunks) grid = (int)chunks;
  k_bin_count<<<grid, kBinThreads, 0, s>>>(rowspan, plan, gx, gy, ch, tab);
  k_bin_rowscan<<<gy, 1024, 0, s>>>(tab, plan, gx, gy, at<uint32_t>(ws, b.tile_start));
  k_bin_place<<<grid, kBinThreads, 0, s>>>(rowseq, rowspan, plan, tab, gx, gy, ch, at<uint32_t>(ws, b.sk[1]), list,
                                           dist, cap);
  count_launch(6);
}

}  // namespace gs3
