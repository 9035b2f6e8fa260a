// K6, K7: shadow splatting (Sec. 4.2, Fig. 3) and K9: camera compositing
// (Sec. 3, Eq. 2) with the deferred per-pixel combination (Sec. 4).
//
// Both composites stream a 16x16 tile's depth-ordered list through shared
// memory as tile-relative entries (splat_eval.cuh): the shadow composite
// over segments of the list with eight rays per lane, the camera composite
// with one 128-thread block per tile (two pixels per thread, batches of 256
// records).
#include "gs3_internal.cuh"
#include "splat_eval.cuh"

namespace gs3 {
namespace {

// ---------------------------------------------------------------------------
// K6: shadow composite.
// For every shadow ray m (light pixel) and every list entry j that passes the
// alpha test, T_m(j) = prod (1 - alpha_k,m) over passing k with
// d_k < d_j - bias.  The list is ordered by distance, so the occluders of j
// form a prefix of the tile's list; its end K(j) is precomputed per entry
// (k_bound_starts, k_bound_rest, from the distances the binning writes beside
// the list) and is non-decreasing in j.
//
// Work is split into segments of a tile's list: segment s holds receivers
// [R_s, R_s+1) (kSegLen entries; the last takes the rest) and needs the
// occluders [C_s, C_s+1) on top of the product A(C_s) that every ray carries
// into it, with C_s = K(R_s).  One warp takes one segment at a time from a
// ticket counter, in segment-major order (every tile's first segment, then
// every tile's second, ...), and:
//   1. computes each of its 256 rays' product Q over its occluder range (a
//      ray drops out once the product can no longer stay above the stop);
//   2. takes A(C_s) from the segment before it (published by that warp; a
//      bounded wait) and publishes A(C_s+1) = A(C_s) Q for the next one;
//   3. walks its receivers in order with the products P = A(C_s) q, q the
//      running product of the range's occluders, summing (beta P, beta) per
//      receiver into the (tile, Gaussian) partials.
// Step 1 runs before the wait, so the segments of a long list run side by
// side and only the cheap step 2 is chained.  When A(C_s) is already
// published as the warp starts, step 1 skips the rays that are stopped.
//
// Ray stop: a ray takes occluders only while its product P = A(C_s) q stays
// >= kShadowStop; the occluder that takes P below it is the ray's last, and
// P stays frozen for the rest of that segment's receivers.  A(C_s+1) of a ray
// that stopped is published as 0 (the receivers of later segments see 0; an
// exact product there is below kShadowStop as well).  The publication and
// the walk agree on where a ray stops: both multiply the same factors in the
// same order and compare round(A(C_s) q) with the stop, which is monotone in
// q.  Thread layout as in the splat evaluation: lane l owns column l & 15,
// rows (l >> 4) + 2 i, i = 0..7, which is ray 32 i + l of the tile.
// ---------------------------------------------------------------------------
constexpr int kSegWarps = 4;        // independent warps per block
constexpr int kRecv = 32;           // receivers staged at a time
constexpr int kOccWin = 32;         // occluder window
constexpr int kRedGroup = 16;       // receivers whose per-lane sums are reduced together
constexpr int kPx = 8;              // rays per lane
constexpr int kSegSpin = 1 << 20;   // polls of a predecessor's publication before giving up


struct ShadowParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const SplatRec* rrec;
  const uint32_t* off;
  const uint32_t* kbound;
  const uint32_t* tile_order;  // tiles by decreasing segment count
  const uint32_t* lvl_off;     // [kSegLevels + 1]: first work item of each segment level
  uint32_t* ticket;            // [3] work counters of K6a, K6b and K6c (zeroed per frame)
  float* pub_a;                // [item][256]: A(C_s+1) published by item
  uint32_t* pub_flag;          // [item]: 0 not yet, 1 published, 2 published and every ray stopped
  uint8_t* pass_mask;  // per list entry: halves with a passing pixel, 0x3 rows 0-7, 0xC rows 8-15
  float2* partial;
  float* light_final;     // per light pixel: the product where the ray ended
  uint32_t* light_stop;   // per light pixel: 1 + index of the occluder that stopped it, or kNoStop
  uint32_t* status;
  uint8_t* live_rank;  // per light rank: 1 if an entry of it lies in a segment with an open ray (K6b)
  uint8_t* den_found;  // per light rank: 1 once K6c found a passing pixel of a Gaussian with no such entry
  int W, H, gx;
  float amax;
};

struct ShadowSmem {  // one warp's
  float ain[kPx * 32];     // A(C_s) of the segment's rays (ray 32 i + lane)
  uint32_t xlim[kPx * 32]; // 1 + the occluder after which a ray stopped in this segment, or 0
  float4 r0[kRecv], r1[kRecv];
  uint32_t rk[kRecv], rslot[kRecv];
  float4 o0[kOccWin], o1[kOccWin];
  float2 red[kRedGroup][33];  // per receiver of the group, per lane: (num, den); padded row
};

// one list entry, staged: make_entry's record plus the halves its box and
// ellipse both reach (in e1.w)
__device__ __forceinline__ void stage_entry(const ShadowParams& p, uint32_t idx, float ox, float oy, float4& e0,
                                            float4& e1) {
  make_entry(p.rrec[p.list[idx]], ox, oy, e0, e1);
  e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* a) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* a, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// A receiver's four rays of one half: den += beta and num += beta a_i at the
// rays where it passes (power2 >= thr), beta = 2^power2.  Predicated, no branch.
template <bool WITH_NUM, int H>
__device__ __forceinline__ void recv_half(const float (&ly)[kPx], const float (&a)[kPx], float y, float c, float v,
                                          float sx, float thr, float& num, float& den) {
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    const int i = 4 * H + qq;
    const float dy = ly[i] - y;
    const float pw = fmaf(dy, fmaf(c, dy, v), sx);
    if (WITH_NUM)
      asm("{\n\t.reg .pred p;\n\t.reg .f32 b;\n\t"
          "setp.ge.f32 p, %2, %3;\n\t"
          "@p ex2.approx.ftz.f32 b, %2;\n\t"
          "@p add.rn.f32 %1, %1, b;\n\t"
          "@p fma.rn.f32 %0, b, %4, %0;\n\t}"
          : "+f"(num), "+f"(den) : "f"(pw), "f"(thr), "f"(a[i]));
    else
      asm("{\n\t.reg .pred p;\n\t.reg .f32 b;\n\t"
          "setp.ge.f32 p, %1, %2;\n\t"
          "@p ex2.approx.ftz.f32 b, %1;\n\t"
          "@p add.rn.f32 %0, %0, b;\n\t}"
          : "+f"(den) : "f"(pw), "f"(thr));
  }
}

// An occluder on four rays of one half, each still taking occluders
// (A q >= stop): q *= max(omin, 1 - gamma 2^power2) where it passes, then
// P = A q.  Returns bit qq set for the rays whose P fell below the stop here.
template <int I>
__device__ __forceinline__ uint32_t occ_ray(const float (&ly)[kPx], uint32_t ain, float (&q)[kPx], float (&P)[kPx],
                                            float y, float c, float v, float sx, float thr, float ngamma,
                                            float omin) {
  const float dy = ly[I] - y;
  const float pw = fmaf(dy, fmaf(c, dy, v), sx);
  uint32_t x;
  // ain: shared-memory address of the lane's A(C_s) of ray 0; ray I at + 128 I
  asm("{\n\t.reg .pred a, p, c;\n\t.reg .f32 b, f, e;\n\t"
      "setp.ge.f32 a, %1, %7;\n\t"           // still taking occluders
      "setp.ge.and.f32 p, %3, %4, a;\n\t"    // and this one passes
      "@p ex2.approx.ftz.f32 b, %3;\n\t"
      "@p ld.shared.f32 e, [%8+%9];\n\t"
      "@p fma.rn.f32 f, %5, b, 0f3F800000;\n\t"
      "@p max.f32 f, f, %6;\n\t"
      "@p mul.rn.f32 %0, %0, f;\n\t"
      "@p mul.rn.f32 %1, e, %0;\n\t"
      "setp.lt.and.f32 c, %1, %7, p;\n\t"    // its last one
      "selp.u32 %2, 1, 0, c;\n\t}"
      : "+f"(q[I]), "+f"(P[I]), "=r"(x)
      : "f"(pw), "f"(thr), "f"(ngamma), "f"(omin), "f"(kShadowStop), "r"(ain), "n"(128 * I));
  return x << I;
}

template <int H>
__device__ __forceinline__ uint32_t occ_half(const float (&ly)[kPx], uint32_t ain, float (&q)[kPx], float (&P)[kPx],
                                             float y, float c, float v, float sx, float thr, float ngamma,
                                             float omin) {
  return occ_ray<4 * H + 0>(ly, ain, q, P, y, c, v, sx, thr, ngamma, omin) |
         occ_ray<4 * H + 1>(ly, ain, q, P, y, c, v, sx, thr, ngamma, omin) |
         occ_ray<4 * H + 2>(ly, ain, q, P, y, c, v, sx, thr, ngamma, omin) |
         occ_ray<4 * H + 3>(ly, ain, q, P, y, c, v, sx, thr, ngamma, omin);
}

// halves (0x3, 0xC) with a ray whose product is still >= the stop
__device__ __forceinline__ uint32_t live_halves(const float (&P)[kPx]) {
  bool h0 = false, h1 = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h0 |= P[i] >= kShadowStop;
    h1 |= P[4 + i] >= kShadowStop;
  }
  return (__any_sync(0xffffffffu, h0) ? 0x3u : 0u) | (__any_sync(0xffffffffu, h1) ? 0xCu : 0u);
}

// The per-warp state of one segment (item) of the shadow composite.
struct SegState {
  int lane, tx, ty, s;
  float lx, ox, oy, omin;
  uint32_t C1;
  uint32_t k, wb, we;  // next occluder; staged occluder window [wb, we)
  uint32_t live;       // halves with a ray still taking occluders
  size_t pix0;         // the lane's first pixel
};

// Walks occluders up to kend (exclusive), staging windows of the range as it
// goes; a ray whose product falls below the stop records where it ended.
__device__ __forceinline__ void walk_to(const ShadowParams& p, ShadowSmem& S, SegState& st, uint32_t kend,
                                        const float (&ly)[kPx], uint32_t ain, float (&q)[kPx], float (&P)[kPx]) {
  while (st.live && st.k < kend) {
    if (st.k == st.we) {
      __syncwarp();
      st.wb = st.k;
      st.we = min(st.k + (uint32_t)kOccWin, st.C1);
      for (uint32_t t = st.lane; t < st.we - st.wb; t += 32)
        stage_entry(p, st.wb + t, st.ox, st.oy, S.o0[t], S.o1[t]);
      __syncwarp();
    }
    const uint32_t stop_at = min(kend, st.we);
    for (; st.k < stop_at; ++st.k) {
      const int t = (int)(st.k - st.wb);
      const float4 o1 = S.o1[t];
      const uint32_t bits = __float_as_uint(o1.w) & st.live;
      if (!bits) continue;
      const float4 o0 = S.o0[t];
      const float dx = st.lx - o0.x;
      const float sx = (o0.z * dx) * dx, v = o1.x * dx;
      uint32_t crossed = 0u;
      if (bits & 0x3u) crossed = occ_half<0>(ly, ain, q, P, o0.y, o0.w, v, sx, o1.y, -o1.z, st.omin);
      if (bits & 0xCu) crossed |= occ_half<1>(ly, ain, q, P, o0.y, o0.w, v, sx, o1.y, -o1.z, st.omin);
      if (crossed) {  // rare: the ray's last occluder (its product stays frozen from here)
#pragma unroll
        for (int i = 0; i < kPx; ++i)
          if (crossed & (1u << i)) S.xlim[32 * i + st.lane] = st.k + 1;
      }
    }
    st.live = live_halves(P);
  }
  if (!st.live) st.k = max(st.k, kend);
}

// Stages receivers [rb, rb + rc) of the segment into shared memory.
__device__ __forceinline__ void stage_receivers(const ShadowParams& p, ShadowSmem& S, const SegState& st, uint32_t rb,
                                                int rc) {
  __syncwarp();  // the previous batch is consumed
  for (int t = st.lane; t < rc; t += 32) {
    const uint32_t rank = p.list[rb + t];
    const SplatRec qr = p.rrec[rank];
    float4 e0, e1;
    make_entry(qr, st.ox, st.oy, e0, e1);
    e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));
    S.r0[t] = e0;
    S.r1[t] = e1;
    S.rk[t] = p.kbound[rb + t];
    S.rslot[t] = p.off[rank] + (uint32_t)((st.ty - qr.r.y) * (qr.r.z - qr.r.x + 1) + (st.tx - qr.r.x));
    p.live_rank[rank] = 1;
  }
  __syncwarp();
}

// Receiver jj of the batch at rb: its per-lane (num, den) to a row, its pass
// halves to pass_mask; every kRedGroup receivers (and at the batch's end)
// lane t < 16 adds num of receiver j0 + t over the 32 lanes, lane 16 + t its
// den, in lane order, into the (tile, Gaussian) partial.
__device__ __forceinline__ void finish_receiver(const ShadowParams& p, ShadowSmem& S, int lane, uint32_t rb, int jj,
                                                int rc, float num, float den0, float den1) {
  const uint32_t bits = (__any_sync(0xffffffffu, den0 > 0.f) ? 0x3u : 0u) |
                        (__any_sync(0xffffffffu, den1 > 0.f) ? 0xCu : 0u);
  S.red[jj % kRedGroup][lane] = make_float2(num, den0 + den1);
  if (lane == 0) p.pass_mask[rb + jj] = (uint8_t)bits;
  if (jj % kRedGroup == kRedGroup - 1 || jj == rc - 1) {
    __syncwarp();
    const int j0 = jj - jj % kRedGroup;
    const int t = lane & 15, c = lane >> 4;
    if (j0 + t <= jj) {
      const float* row = reinterpret_cast<const float*>(S.red[t]) + c;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int l = 0; l < 32; l += 4) {
        a0 += row[2 * l]; a1 += row[2 * l + 2]; a2 += row[2 * l + 4]; a3 += row[2 * l + 6];
      }
      reinterpret_cast<float*>(p.partial)[2 * (size_t)S.rslot[j0 + t] + c] = (a0 + a1) + (a2 + a3);
    }
    __syncwarp();  // the group's rows are free again
  }
}

// A(C_s) of the lane's rays: 1 / 0 (in / outside the image) for a tile's
// first segment, else the predecessor's publication (read from L2: it was
// written on another SM); flag 2 publishes that every ray stopped.
__device__ __forceinline__ void load_entering(const ShadowParams& p, int s, uint32_t wpred, uint32_t flag, int lane,
                                              int rows_in, float (&A)[kPx]) {
#pragma unroll
  for (int i = 0; i < kPx; ++i)
    A[i] = s == 0 ? (i < rows_in ? 1.f : 0.f)
                  : (flag == 2u ? 0.f : __ldcg(p.pub_a + (size_t)wpred * 256 + 32 * i + lane));
}

__device__ __forceinline__ bool all_stopped(const float (&A)[kPx]) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < kPx; ++i) any |= A[i] >= kShadowStop;
  return !__any_sync(0xffffffffu, any);
}

// den + 2^pw where pw >= thr (predicated, no branch)
__device__ __forceinline__ float recv_den(float pw, float thr, float den) {
  asm("{\n\t.reg .pred p;\n\t.reg .f32 b;\n\t"
      "setp.ge.f32 p, %1, %2;\n\t"
      "@p ex2.approx.ftz.f32 b, %1;\n\t"
      "@p add.rn.f32 %0, %0, b;\n\t}"
      : "+f"(den) : "f"(pw), "f"(thr));
  return den;
}

// The segment a work item names: its level s (segment index) and tile, the
// levels being prefixes of the tile order.
struct SegItem {
  int s, tile, tx, ty, rows_in;
  uint32_t R0, R1, C0, C1, wpred;
  bool last;
};

__device__ __forceinline__ SegItem seg_item(const ShadowParams& p, uint32_t w, int lane) {
  SegItem it;
  int lo = 0, hi = kSegLevels;  // largest s with lvl_off[s] <= w
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p.lvl_off[mid] <= w) lo = mid; else hi = mid;
  }
  it.s = lo;
  const uint32_t pos = w - p.lvl_off[lo];
  it.tile = (int)p.tile_order[pos];
  it.tx = it.tile % p.gx;
  it.ty = it.tile / p.gx;
  const uint32_t b = p.tile_start[it.tile], e = p.tile_start[it.tile + 1];
  it.last = (uint32_t)lo == seg_count(e - b) - 1;
  it.R0 = b + (uint32_t)lo * kSegLen;
  it.R1 = it.last ? e : it.R0 + kSegLen;
  it.C0 = e > b ? p.kbound[it.R0] : b;
  it.C1 = e > b ? (it.last ? p.kbound[e - 1] : p.kbound[it.R1]) : b;
  it.wpred = lo > 0 ? p.lvl_off[lo - 1] + pos : 0u;
  // ray i of the lane is row (lane >> 4) + 2 i: rows below the image hold no ray
  const int lxi = lane & 15, lyi = lane >> 4;
  it.rows_in = it.tx * kTile + lxi < p.W ? min(kPx, (p.H - it.ty * kTile - lyi + 1) / 2) : 0;
  return it;
}

// The next work item of the warp (a ticket), or false past the last.
__device__ __forceinline__ bool next_item(uint32_t* ticket, uint32_t total, int lane, uint32_t& w) {
  uint32_t t = 0;
  if (lane == 0) t = atomicAdd(ticket, 1u);
  w = __shfl_sync(0xffffffffu, t, 0);
  return w < total;
}

// K6a: A(C_s+1) of every segment but a tile's last, chained from A(C_s).
// Step 1 (the range's products Q) runs before the chain is known, so the
// segments of a list run side by side and only the combination is chained.
__device__ __forceinline__ void chain_item(const ShadowParams& p, uint32_t w, ShadowSmem& S, int lane) {
  const int lxi = lane & 15, lyi = lane >> 4;
  const float lx = lxi + 0.5f, omin = 1.f - p.amax;
  const uint32_t ain = (uint32_t)__cvta_generic_to_shared(&S.ain[lane]);

    const SegItem it = seg_item(p, w, lane);
    if (it.last) return;  // nothing follows it
    const float ox = (float)(it.tx * kTile), oy = (float)(it.ty * kTile);
    float ly[kPx];
#pragma unroll
    for (int i = 0; i < kPx; ++i) ly[i] = i < it.rows_in ? lyi + 2 * i + 0.5f : 1.0e6f;
    // A(C_s): known now for the first segment, or when the predecessor
    // published already; until then A = 1 stands in (A <= 1)
    uint32_t flag = 1u;
    if (it.s > 0 && lane == 0) flag = ld_acquire(p.pub_flag + it.wpred);
    flag = __shfl_sync(0xffffffffu, flag, 0);
    __syncwarp();  // orders every lane's reads after lane 0's acquire
    bool known = flag != 0u;
    float A[kPx];
    if (known) {
      load_entering(p, it.s, it.wpred, flag, lane, it.rows_in, A);
    } else {
#pragma unroll
      for (int i = 0; i < kPx; ++i) A[i] = i < it.rows_in ? 1.f : 0.f;
    }
    const bool dead = known && all_stopped(A);
    // the range's products Q; a ray drops out once A Q < stop (it stops
    // either way); the product so far is the same whichever A stood in
    float Q[kPx], PQ[kPx];
#pragma unroll
    for (int i = 0; i < kPx; ++i) {
      Q[i] = 1.f;
      PQ[i] = A[i] >= kShadowStop ? A[i] : 0.f;
    }
    if (!dead) {
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kPx; ++i) S.ain[32 * i + lane] = A[i];
      uint32_t live = live_halves(PQ);
      for (uint32_t wb = it.C0; wb < it.C1 && live; wb += kOccWin) {
        if (!known) {  // the predecessor may have published meanwhile
          uint32_t fl = 0u;
          if (lane == 0) fl = ld_acquire(p.pub_flag + it.wpred);
          fl = __shfl_sync(0xffffffffu, fl, 0);
          __syncwarp();
          if (fl != 0u) {
            known = true;
            load_entering(p, it.s, it.wpred, fl, lane, it.rows_in, A);
#pragma unroll
            for (int i = 0; i < kPx; ++i) {
              S.ain[32 * i + lane] = A[i];
              PQ[i] = A[i] >= kShadowStop ? A[i] * Q[i] : 0.f;
            }
            live = live_halves(PQ);
            if (!live) break;
          }
        }
        const int wc = (int)min((uint32_t)kOccWin, it.C1 - wb);
        __syncwarp();
        for (int t = lane; t < wc; t += 32) stage_entry(p, wb + t, ox, oy, S.o0[t], S.o1[t]);
        __syncwarp();
        for (int t = 0; t < wc; ++t) {
          const float4 o1 = S.o1[t];
          const uint32_t bits = __float_as_uint(o1.w) & live;
          if (!bits) continue;
          const float4 o0 = S.o0[t];
          const float dx = lx - o0.x;
          const float sx = (o0.z * dx) * dx, v = o1.x * dx;
          if (bits & 0x3u) occ_half<0>(ly, ain, Q, PQ, o0.y, o0.w, v, sx, o1.y, -o1.z, omin);
          if (bits & 0xCu) occ_half<1>(ly, ain, Q, PQ, o0.y, o0.w, v, sx, o1.y, -o1.z, omin);
        }
        live = live_halves(PQ);
      }
    }
    // A(C_s) from the predecessor (bounded wait), then A(C_s+1) for the successor
    if (!known) {
      uint32_t fl = 0u;
      if (lane == 0) {
        int spins = 0;
        while ((fl = ld_acquire(p.pub_flag + it.wpred)) == 0u) {
          if (++spins > kSegSpin) {
            atomicCAS(p.status, 0u, (uint32_t)GS3_ERR_TIMEOUT);
            fl = 2u;  // give up: the frame is reported invalid, the warp finishes
            break;
          }
          __nanosleep(64);
        }
      }
      fl = __shfl_sync(0xffffffffu, fl, 0);
      __syncwarp();
      load_entering(p, it.s, it.wpred, fl, lane, it.rows_in, A);
    }
    const bool dead_in = all_stopped(A);
    bool any = false;
#pragma unroll
    for (int i = 0; i < kPx; ++i) {
      float a = 0.f;
      if (A[i] >= kShadowStop) {
        a = A[i] * Q[i];
        if (!(a >= kShadowStop)) a = 0.f;  // the ray stops in this range
      }
      any |= a != 0.f;
      if (!dead_in) p.pub_a[(size_t)w * 256 + 32 * i + lane] = a;
    }
    const bool any_out = __any_sync(0xffffffffu, any);
    __threadfence();  // every lane's products before the flag
    __syncwarp();
    if (lane == 0) st_release(p.pub_flag + w, any_out ? 1u : 2u);
  }

// The work items of a batch of frames: the tickets run over every frame's
// items in turn; locate() maps a ticket to its frame and the frame's item.
__device__ __forceinline__ uint32_t batch_items(const ShadowParams* reqs, int nreq) {
  uint32_t t = 0;
  for (int r = 0; r < nreq; ++r) t += reqs[r].lvl_off[kSegLevels];
  return t;
}
__device__ __forceinline__ int locate(const ShadowParams* reqs, int nreq, uint32_t& w) {
  int r = 0;
  for (; r < nreq - 1; ++r) {
    const uint32_t t = reqs[r].lvl_off[kSegLevels];
    if (w < t) break;
    w -= t;
  }
  return r;
}

// One frame (p) or a batch of nreq frames (reqs, in device memory; p is the
// first, whose tickets the batch shares).
template <bool BATCH>
__global__ void __launch_bounds__(kSegWarps * 32, 4) k_shadow_chain(const ShadowParams p, const ShadowParams* reqs,
                                                                    int nreq) {
  __shared__ ShadowSmem smem[kSegWarps];
  ShadowSmem& S = smem[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint32_t total = BATCH ? batch_items(reqs, nreq) : p.lvl_off[kSegLevels];
  uint32_t w;
  while (next_item(p.ticket, total, lane, w)) {
    if (BATCH) {
      const int r = locate(reqs, nreq, w);
      chain_item(reqs[r], w, S, lane);
    } else {
      chain_item(p, w, S, lane);
    }
  }
}

// The light tile of the pixel nearest a splat's centre (k_dead_probe's
// pixel), or all ones off the image.
__device__ __forceinline__ uint32_t probe_tile(const SplatRec& q, int W, int H, int gx) {
  const float cx = q.a.x + q.b.w, cy = q.a.y + q.c.x;
  if (!(cx >= 0.f && cy >= 0.f && cx < (float)W && cy < (float)H)) return 0xFFFFFFFFu;
  return (uint32_t)(((int)cy / kTile) * gx + (int)cx / kTile);
}

// K6c: the receivers of the segments every ray of which stopped before the
// segment (A(C_s) = 0 throughout, as K6a published).  The products are 0,
// so a receiver needs only its beta sum over the tile, which depends on no
// other entry.  A warp stages up to kDeadBatch receivers, lists their
// (receiver, half) units (the halves their box and ellipse reach), and each
// lane walks the 16 x 8 pixels of one unit at a time, with the power
// arithmetic of the ray layout (pixel centres x + 0.5, y + 0.5); the two
// halves of a receiver are then added in a fixed order.
// A Gaussian none of whose entries lies in a segment with an open ray (K6b
// marked those) has a zero numerator everywhere, so its shadow value is 0 if
// any of its pixels passes and 1 otherwise: the beta sum only has to be
// known to be positive.  Once that is known (den_found: k_dead_probe found
// its pixel nearest the centre passing, or one of its units here found a
// passing pixel), its entries are skipped (partial (0, 0), no pass halves)
// except the one of the probe tile, which is evaluated in full, so the sum
// stays positive.  Which other entries are skipped depends on timing; T
// does not, and the backward takes nothing from such a Gaussian (its
// products and T are 0).
constexpr int kDeadBatch = 128;
constexpr int kDeadWarps = 4;

struct DeadSmem {  // one warp's
  float4 e0[kDeadBatch], e1[kDeadBatch];
  float den[2][kDeadBatch];
  uint32_t slot[kDeadBatch];      // the receiver's partial slot
  uint32_t rank[kDeadBatch];      // its depth rank, bit 31 set if K6b saw it
  uint16_t unit[2 * kDeadBatch];  // receiver (bits 0-7) and half (bit 8) of each unit
};

// The beta sum of one receiver entry over the 16 x 8 pixels of half h of an
// interior tile, column by column.
__device__ __forceinline__ float dead_half(const float4 e0, const float4 e1, int h) {
  float dy[8];
  const float y0 = 8.f * h + 0.5f;
#pragma unroll
  for (int y = 0; y < 8; ++y) dy[y] = (y0 + (float)y) - e0.y;
  float den = 0.f, fx = 0.5f;
#pragma unroll 1
  for (int x = 0; x < kTile; ++x) {
    const float dx = fx - e0.x;
    fx += 1.f;
    const float sx = (e0.z * dx) * dx, v = e1.x * dx;
#pragma unroll
    for (int y = 0; y < 8; ++y) den = recv_den(fmaf(dy[y], fmaf(e0.w, dy[y], v), sx), e1.y, den);
  }
  return den;
}

// the same over the pixels of half h that lie inside the image (edge tiles)
__device__ __forceinline__ float dead_half_edge(const float4 e0, const float4 e1, int h, int ncol, int nrow) {
  float den = 0.f, fx = 0.5f;
  const int y1 = min(8 * h + 8, nrow);
  for (int x = 0; x < ncol; ++x, fx += 1.f) {
    const float dx = fx - e0.x;
    const float sx = (e0.z * dx) * dx, v = e1.x * dx;
    float fy = 8.f * h + 0.5f;
    for (int y = 8 * h; y < y1; ++y, fy += 1.f) {
      const float dy = fy - e0.y;
      den = recv_den(fmaf(dy, fmaf(e0.w, dy, v), sx), e1.y, den);
    }
  }
  return den;
}

__device__ __forceinline__ void dead_item(const ShadowParams& p, uint32_t w, DeadSmem& D, int lane) {

    int lo = 0, hi = kSegLevels;  // the item's level: largest s with lvl_off[s] <= w
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (p.lvl_off[mid] <= w) lo = mid; else hi = mid;
    }
    if (lo == 0) return;  // a tile's first segment starts with every ray open
    const uint32_t pos = w - p.lvl_off[lo];
    if (__ldcg(p.pub_flag + p.lvl_off[lo - 1] + pos) != 2u) return;  // not stopped: K6b's
    const int tile = (int)p.tile_order[pos];
    const int tx = tile % p.gx, ty = tile / p.gx;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
    const bool last = (uint32_t)lo == seg_count(e - b) - 1;
    const uint32_t R0 = b + (uint32_t)lo * kSegLen, R1 = last ? e : R0 + kSegLen;
    const int ncol = min(kTile, p.W - tx * kTile), nrow = min(kTile, p.H - ty * kTile);
    const bool interior = ncol == kTile && nrow == kTile;
    for (uint32_t rb = R0; rb < R1; rb += kDeadBatch) {
      const int rc = (int)min((uint32_t)kDeadBatch, R1 - rb);
      // stage the receivers; list the units of half 0, then of half 1
      __syncwarp();
      int n0 = 0, n1 = 0;
      uint32_t box[kDeadBatch / 32];
#pragma unroll
      for (int c = 0; c < kDeadBatch / 32; ++c) {
        const int t = 32 * c + lane;
        box[c] = 0u;
        if (t < rc) {
          const uint32_t rank = p.list[rb + t];
          const SplatRec q = p.rrec[rank];
          const bool live = p.live_rank[rank] != 0;
          float4 e0, e1;
          make_entry(q, ox, oy, e0, e1);
          // skipped: a Gaussian with no open-ray entry whose den is known positive,
          // except in its probe tile (whose entry keeps den > 0 in the sum)
          const bool skip = !live && __ldcg(p.den_found + rank) != 0 &&
                            probe_tile(q, p.W, p.H, p.gx) != (uint32_t)(ty * p.gx + tx);
          box[c] = skip ? 0u : __float_as_uint(e1.w) & ellipse_halves(e0, e1);
          D.e0[t] = e0;
          D.e1[t] = e1;
          D.slot[t] = p.off[rank] + (uint32_t)((ty - q.r.y) * (q.r.z - q.r.x + 1) + (tx - q.r.x));
          D.rank[t] = rank | (live ? 0x80000000u : 0u);
        }
        n0 += __popc(__ballot_sync(0xffffffffu, (box[c] & 0x3u) != 0u));
        n1 += __popc(__ballot_sync(0xffffffffu, (box[c] & 0xCu) != 0u));
      }
      int b0 = 0, b1 = n0;  // next unit slot of each half
#pragma unroll
      for (int c = 0; c < kDeadBatch / 32; ++c) {
        const int t = 32 * c + lane;
        const uint32_t m0 = __ballot_sync(0xffffffffu, (box[c] & 0x3u) != 0u);
        const uint32_t m1 = __ballot_sync(0xffffffffu, (box[c] & 0xCu) != 0u);
        const uint32_t below = (1u << lane) - 1u;
        if (box[c] & 0x3u) D.unit[b0 + __popc(m0 & below)] = (uint16_t)t;
        if (box[c] & 0xCu) D.unit[b1 + __popc(m1 & below)] = (uint16_t)(t | 0x100);
        b0 += __popc(m0);
        b1 += __popc(m1);
        if (t < rc) D.den[0][t] = D.den[1][t] = 0.f;
      }
      __syncwarp();
      const int nu = n0 + n1;
      for (int u = lane; u < nu; u += 32) {
        const int code = D.unit[u];
        const int t = code & 0xFF, h = code >> 8;
        const float4 e0 = D.e0[t], e1 = D.e1[t];
        D.den[h][t] = interior ? dead_half(e0, e1, h) : dead_half_edge(e0, e1, h, ncol, nrow);
      }
      __syncwarp();
      for (int t = lane; t < rc; t += 32) {
        const float d0 = D.den[0][t], d1 = D.den[1][t];
        const uint32_t rk = D.rank[t];
        p.partial[D.slot[t]] = make_float2(0.f, d0 + d1);
        p.pass_mask[rb + t] = (uint8_t)((d0 > 0.f ? 0x3u : 0u) | (d1 > 0.f ? 0xCu : 0u));
        if (d0 + d1 > 0.f && !(rk >> 31)) __stcg(p.den_found + rk, (uint8_t)1);
      }
    }
  }

// Before K6c: a Gaussian none of whose entries K6b saw has its pixel nearest
// the splat centre tested with K6c's exact arithmetic (the entry of that
// tile, the pixel's power against the threshold); if it passes, den > 0 is
// known and K6c can skip every entry of the Gaussian.  Only a pixel that K6c
// itself would evaluate counts: inside the image, in a tile of the
// Gaussian's rectangle, in a half its box and ellipse reach.
__global__ void k_dead_probe(const ShadowParams p, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || p.live_rank[r]) return;
  const SplatRec q = p.rrec[r];
  if (q.r.x < 0) return;  // not in the light view
  const float cx = q.a.x + q.b.w, cy = q.a.y + q.c.x;
  if (!(cx >= 0.f && cy >= 0.f && cx < (float)p.W && cy < (float)p.H)) return;
  const int px = (int)cx, py = (int)cy;
  const int tx = px / kTile, ty = py / kTile;
  if (tx < q.r.x || tx > q.r.z || ty < q.r.y || ty > q.r.w) return;
  float4 e0, e1;
  make_entry(q, (float)(tx * kTile), (float)(ty * kTile), e0, e1);
  const int x = px - tx * kTile, y = py - ty * kTile, h = y >> 3;
  // K6c evaluates the half only if the entry's box and ellipse reach it
  if (!(__float_as_uint(e1.w) & ellipse_halves(e0, e1) & (3u << (2 * h)))) return;
  const float dx = (0.5f + (float)x) - e0.x;
  const float sx = (e0.z * dx) * dx, v = e1.x * dx;
  const float dy = ((8.f * h + 0.5f) + (float)(y & 7)) - e0.y;
  const float pw = fmaf(dy, fmaf(e0.w, dy, v), sx);
  if (pw >= e1.y) p.den_found[r] = 1;
}

template <bool BATCH>
__global__ void __launch_bounds__(kDeadWarps * 32, 7) k_shadow_dead(const ShadowParams p, const ShadowParams* reqs,
                                                                    int nreq) {
  __shared__ DeadSmem smem[kDeadWarps];
  DeadSmem& D = smem[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint32_t total = BATCH ? batch_items(reqs, nreq) : p.lvl_off[kSegLevels];
  uint32_t w;
  while (next_item(p.ticket + 2, total, lane, w)) {
    if (BATCH) {
      const int r = locate(reqs, nreq, w);
      dead_item(reqs[r], w, D, lane);
    } else {
      dead_item(p, w, D, lane);
    }
  }
}

// K6b: the receivers of every segment, with the products P = A(C_s) q, q the
// running product of the range's occluders; A(C_s) comes from K6a.
__device__ __forceinline__ void live_item(const ShadowParams& p, uint32_t w, ShadowSmem& S, int lane) {
  SegState st;
  st.lane = lane;
  const int lxi = lane & 15, lyi = lane >> 4;
  st.lx = lxi + 0.5f;
  st.omin = 1.f - p.amax;
  const uint32_t ain = (uint32_t)__cvta_generic_to_shared(&S.ain[lane]);

    const SegItem it = seg_item(p, w, lane);
    st.s = it.s;
    st.tx = it.tx;
    st.ty = it.ty;
    st.ox = (float)(it.tx * kTile);
    st.oy = (float)(it.ty * kTile);
    st.C1 = it.C1;
    float ly[kPx];
#pragma unroll
    for (int i = 0; i < kPx; ++i) ly[i] = i < it.rows_in ? lyi + 2 * i + 0.5f : 1.0e6f;
    // A(C_s) and A(C_s+1), as K6a published them
    uint32_t fl_in = it.s == 0 ? 1u : __ldcg(p.pub_flag + it.wpred);
    uint32_t fl_out = it.last ? 1u : __ldcg(p.pub_flag + w);
    float P[kPx];
    load_entering(p, it.s, it.wpred, fl_in, lane, it.rows_in, P);
    const bool dead = all_stopped(P);
    if (dead) return;  // K6c takes it
    // rays the publication has stop in this range (they must reach their stop)
    bool pending = false;
    float q[kPx];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kPx; ++i) {
      q[i] = 1.f;
      S.ain[32 * i + lane] = P[i];
      S.xlim[32 * i + lane] = 0u;
      if (P[i] >= kShadowStop && !it.last) {
        const float out = fl_out == 2u ? 0.f : __ldcg(p.pub_a + (size_t)w * 256 + 32 * i + lane);
        pending |= out == 0.f;
      }
      if (!(P[i] >= kShadowStop)) P[i] = 0.f;
    }
    __syncwarp();
    st.live = live_halves(P);
    st.k = st.wb = st.we = it.C0;
    st.pix0 = (size_t)(it.ty * kTile + lyi) * p.W + it.tx * kTile + lxi;
    // one pseudo-receiver past the last: the rest of the range, for rays that
    // stop in it after the last receiver
    const bool tail = __any_sync(0xffffffffu, pending);
    for (uint32_t rb = it.R0; rb < it.R1 || (tail && rb == it.R1); rb += kRecv) {
      const int rc = (int)min((uint32_t)kRecv, it.R1 - min(rb, it.R1));
      if (rc > 0) stage_receivers(p, S, st, rb, rc);
      const int steps = rc + (tail && rb + kRecv >= it.R1 ? 1 : 0);
      for (int jj = 0; jj < steps; ++jj) {
        const bool real = jj < rc;
        if (st.live) walk_to(p, S, st, real ? S.rk[jj] : st.C1, ly, ain, q, P);
        if (!real) break;
        const float4 r1 = S.r1[jj];
        const uint32_t box = __float_as_uint(r1.w);
        float den0 = 0.f, den1 = 0.f, num = 0.f;
        if (box) {
          const float4 r0 = S.r0[jj];
          const float dx = st.lx - r0.x;
          const float sx = (r0.z * dx) * dx, v = r1.x * dx;
          if (box & 0x3u) recv_half<true, 0>(ly, P, r0.y, r0.w, v, sx, r1.y, num, den0);
          if (box & 0xCu) recv_half<true, 1>(ly, P, r0.y, r0.w, v, sx, r1.y, num, den1);
        }
        finish_receiver(p, S, lane, rb, jj, rc, num, den0, den1);
      }
    }
    // where each ray ended (the backward starts from it): rays that stopped in
    // this segment, and those that ran through every segment without
    // stopping, written by the tile's last segment
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kPx; ++i) {
      const uint32_t lim = S.xlim[32 * i + lane];
      if (lim != 0u || (it.last && i < it.rows_in && P[i] >= kShadowStop)) {
        p.light_final[st.pix0 + (size_t)2 * i * p.W] = P[i];
        p.light_stop[st.pix0 + (size_t)2 * i * p.W] = lim != 0u ? lim : kNoStop;
      }
    }
  }

template <bool BATCH>
__global__ void __launch_bounds__(kSegWarps * 32, 4) k_shadow(const ShadowParams p, const ShadowParams* reqs, int nreq) {
  __shared__ ShadowSmem smem[kSegWarps];
  ShadowSmem& S = smem[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint32_t total = BATCH ? batch_items(reqs, nreq) : p.lvl_off[kSegLevels];
  uint32_t w;
  while (next_item(p.ticket + 1, total, lane, w)) {
    if (BATCH) {
      const int r = locate(reqs, nreq, w);
      live_item(reqs[r], w, S, lane);
    } else {
      live_item(p, w, S, lane);
    }
  }
}

// K(i) of entry i of a light list: the first index of i's tile list (from b)
// whose distance is >= d_i - bias, the end of i's occluder prefix.
__device__ __forceinline__ uint32_t occ_bound(const float* __restrict__ dl, uint32_t b, uint32_t i, float bias) {
  const float thr = __fsub_rn(dl[i], bias);
  uint32_t lo = b, hi = i;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (dl[mid] < thr) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The level s of work item w and the item's tile position (lvl_off holds
// each level's first item).
__device__ __forceinline__ int item_level(const uint32_t* lvl_off, uint32_t w) {
  int lo = 0, hi = kSegLevels;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (lvl_off[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// K at the entries the segment plan reads (every segment's first entry and
// every tile's last), one thread per segment, before K6a.
__global__ void __launch_bounds__(256) k_bound_starts(const ShadowParams p, const float* __restrict__ dl,
                                                      uint32_t* __restrict__ kb, float bias) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= p.lvl_off[kSegLevels]) return;
  const int s = item_level(p.lvl_off, w);
  const int tile = (int)p.tile_order[w - p.lvl_off[s]];
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  if (e <= b) return;
  const uint32_t r0 = b + (uint32_t)s * kSegLen;
  kb[r0] = occ_bound(dl, b, r0, bias);
  if ((uint32_t)s == seg_count(e - b) - 1 && e - 1 > r0) kb[e - 1] = occ_bound(dl, b, e - 1, bias);
}

// After K6a: K of every other entry of a segment with an open ray (K6b reads
// it per receiver), one warp per segment.  In a segment every ray enters
// stopped no kernel takes an occluder or needs the exact bound: its entries
// get the segment's first bound C_s (<= K(j)); the backward, which reads
// them, takes no occluder at or past a ray's stop, and every ray stopped
// before C_s, so any bound in [C_s, K(j)] gives it the same result.
__global__ void __launch_bounds__(256) k_bound_rest(const ShadowParams p, const float* __restrict__ dl,
                                                    uint32_t* __restrict__ kb, float bias) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= p.lvl_off[kSegLevels]) return;
  const int s = item_level(p.lvl_off, w);
  const uint32_t pos = w - p.lvl_off[s];
  const int tile = (int)p.tile_order[pos];
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  if (e <= b) return;
  const bool last = (uint32_t)s == seg_count(e - b) - 1;
  const uint32_t r0 = b + (uint32_t)s * kSegLen, r1 = last ? e : r0 + kSegLen;
  const bool open = s == 0 || __ldcg(p.pub_flag + p.lvl_off[s - 1] + pos) != 2u;
  const uint32_t c0 = kb[r0];
  for (uint32_t j = r0 + 1 + lane; j < r1; j += 32) {
    if (j == e - 1) continue;  // k_bound_starts's
    kb[j] = open ? occ_bound(dl, b, j, bias) : c0;
  }
}

// K7: per Gaussian, sum its (tile) partials; T = num / den, or 1 when the
// Gaussian meets no shadow ray.  Eight lanes per Gaussian rank (four per
// warp): lane s adds partials s, s + 8, ... in order, then three shuffle
// levels combine the eight sums in a fixed order.
__global__ void __launch_bounds__(256) k_shadow_reduce(int n, const uint32_t* __restrict__ off,
                                                       const uint32_t* __restrict__ cnt,
                                                       const float2* __restrict__ partial,
                                                       const uint32_t* __restrict__ order,
                                                       const uint32_t* header, float* __restrict__ T,
                                                       float* __restrict__ den_out) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int sub = threadIdx.x & 7;
  const bool valid = r < n;
  const uint32_t P = header[H_PAIRS_LIGHT];
  float num = 0.f, den = 0.f;
  if (valid) {
    const uint32_t o = off[r], c = cnt[r];
    if (o + c <= P) {
      for (uint32_t i = sub; i < c; i += 8) {
        const float2 v = partial[o + i];
        num += v.x;
        den += v.y;
      }
    }
  }
#pragma unroll
  for (int sh = 4; sh > 0; sh >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, sh);
    den += __shfl_xor_sync(0xffffffffu, den, sh);
  }
  if (valid && sub == 0) {
    T[order[r]] = den > 0.f ? num / den : 1.f;
    den_out[order[r]] = den;
  }
}

__global__ void k_fill(float* x, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// ---------------------------------------------------------------------------
// K9: camera composite of seven channels (shading rgb, refined shadow,
// residual rgb) front to back; a ray stops before the transmittance would
// fall below t_stop; the block leaves a batch loop once all rays stopped.
// Output: shading * shadow + residual per pixel.
// ---------------------------------------------------------------------------
constexpr int kCamThreads = 128;  // two pixels per thread
constexpr int kCamRec = 256;      // records staged per batch

struct CamParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const uint32_t* tile_order;  // block b renders tile tile_order[b] (longest list first)
  const SplatRec* rrec;
  const float4* ccol;
  float* out;
  float* final_t;
  uint32_t* n_contrib;
  float4* pix_aux;
  int W, H, gx;
  float amax, tstop;
};

struct CamSmem {
  float4 E0[kCamRec], E1[kCamRec], C0[kCamRec], C1[kCamRec];
};

// Block blk of a frame: tile tile_order[blk] (longest list first).  128
// threads, two pixels each: warp w covers quadrant w (the 8x8 block at
// (8 (w & 1), 8 (w >> 1))), lane l column l & 7 and rows l >> 3 and
// (l >> 3) + 4 of it, so the two pixels share the entry's dx terms and a
// warp skips an entry whose box and ellipse miss its quadrant.  Records are
// staged as shadow-splat entries (centre relative to the tile, conic times
// log2 e): the alpha is gamma 2^power2, the power's arithmetic that of the
// backward (power2_at).
__device__ __forceinline__ void camera_tile(const CamParams& p, int blk, CamSmem& M) {
  const int tile = (int)p.tile_order[blk];
  const int tx = tile % p.gx, ty = tile / p.gx;
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t wq = 1u << w;
  const int cx = 8 * (w & 1) + (lane & 7), cy0 = 8 * (w >> 1) + (lane >> 3);
  const int px = tx * kTile + cx, py[2] = {ty * kTile + cy0, ty * kTile + cy0 + 4};
  const float lx = cx + 0.5f, ly0 = cy0 + 0.5f, ly1 = cy0 + 4.5f;
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  float T[2] = {1.f, 1.f}, acc[2][7];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[k][c] = 0.f;
  bool done[2] = {!(px < p.W && py[0] < p.H), !(px < p.W && py[1] < p.H)};
  uint32_t consumed[2] = {0u, 0u};
  for (uint32_t rb = b; rb < e; rb += kCamRec) {
    if (__syncthreads_count(done[0] && done[1]) == kCamThreads) break;
    const int rc = (int)min((uint32_t)kCamRec, e - rb);
    for (int k = t; k < rc; k += kCamThreads) {
      const uint32_t rank = p.list[rb + k];
      float4 e0, e1;
      make_entry(p.rrec[rank], ox, oy, e0, e1);
      e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));
      M.E0[k] = e0;
      M.E1[k] = e1;
      M.C0[k] = p.ccol[2 * rank];
      M.C1[k] = p.ccol[2 * rank + 1];
    }
    __syncthreads();
    if (!(done[0] && done[1])) {
      // one pixel's step: false once its ray stopped here
      auto take = [&](int k, int jj, float pw, float g) {
        const float alpha = fminf(p.amax, g * ex2(pw));
        const float Tn = T[k] * (1.f - alpha);
        if (Tn < p.tstop) {
          done[k] = true;
          consumed[k] = rb - b + jj;
          return;
        }
        const float wt = alpha * T[k];
        const float4 c0 = M.C0[jj], c1 = M.C1[jj];
        acc[k][0] += wt * c0.x; acc[k][1] += wt * c0.y; acc[k][2] += wt * c0.z;
        acc[k][3] += wt * c0.w;
        acc[k][4] += wt * c1.x; acc[k][5] += wt * c1.y; acc[k][6] += wt * c1.z;
        T[k] = Tn;
      };
      // two records' powers are formed ahead of the updates (the same
      // arithmetic, in the same order, as one record at a time)
      for (int jj = 0; jj < rc; jj += 2) {
        const float4 ea = M.E1[jj];
        const bool two = jj + 1 < rc;
        const float4 eb = two ? M.E1[jj + 1] : ea;
        const bool ha = (__float_as_uint(ea.w) & wq) != 0u, hb = two && (__float_as_uint(eb.w) & wq) != 0u;
        float pa0 = 0.f, pa1 = 0.f, pb0 = 0.f, pb1 = 0.f;
        if (ha) powers2(M.E0[jj], ea.x, lx, ly0, ly1, pa0, pa1);
        if (hb) powers2(M.E0[jj + 1], eb.x, lx, ly0, ly1, pb0, pb1);
        if (ha) {
          if (!done[0] && pa0 >= ea.y) take(0, jj, pa0, ea.z);
          if (!done[1] && pa1 >= ea.y) take(1, jj, pa1, ea.z);
        }
        if (hb) {
          if (!done[0] && pb0 >= eb.y) take(0, jj + 1, pb0, eb.z);
          if (!done[1] && pb1 >= eb.y) take(1, jj + 1, pb1, eb.z);
        }
        if (done[0] && done[1]) break;
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (!done[k]) consumed[k] = rb - b + rc;
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (px < p.W && py[k] < p.H) {
      const size_t pix = (size_t)py[k] * p.W + px;
      const float* a = acc[k];
      p.out[3 * pix + 0] = a[0] * a[3] + a[4];
      p.out[3 * pix + 1] = a[1] * a[3] + a[5];
      p.out[3 * pix + 2] = a[2] * a[3] + a[6];
      p.final_t[pix] = T[k];
      p.n_contrib[pix] = consumed[k];
      p.pix_aux[2 * pix] = make_float4(a[0], a[1], a[2], a[3]);
      p.pix_aux[2 * pix + 1] = make_float4(a[4], a[5], a[6], 0.f);
    }
  }
}

// One frame (p), or a batch of nreq frames (reqs in device memory) whose
// tiles follow one another: frame r owns blocks [tile_prefix[r], tile_prefix[r + 1]).
template <bool BATCH>
__global__ void __launch_bounds__(kCamThreads) k_camera(const CamParams p, const CamParams* reqs, const uint32_t* tile_prefix,
                                                int nreq) {
  __shared__ CamSmem M;
  if (BATCH) {
    int r = 0;
    while (r < nreq - 1 && blockIdx.x >= tile_prefix[r + 1]) ++r;
    camera_tile(reqs[r], (int)(blockIdx.x - tile_prefix[r]), M);
  } else {
    camera_tile(p, (int)blockIdx.x, M);
  }
}

// ---------------------------------------------------------------------------
// K9 for an environment light (Sec. 4.5): the camera composite of nl <= 8
// lights in one pass.  The camera splat (alphas, order, stops) does not
// depend on the light, so every light's shading S_l and refined shadow Sh_l
// are composited on the same weights, each into its own accumulators, in the
// order camera_tile uses (each light's sums equal that light's own frame's);
// the residual R, which does not see the light, is composited once.
// out (+)= sum_l w_l (S_l Sh_l + R).
// ---------------------------------------------------------------------------
constexpr int kEnvRec = 128;  // records staged per batch

struct EnvCamParams {
  CamParams c;           // the first light's workspace: camera splat, residual colours, final T
  const float4* envcol;  // [rank][nl]: (shade_l rgb, T'_l)
  float w[kMaxBatch];
  int nl;
  int accumulate;  // add to out (a later group of lights)
};

struct EnvSmem {
  float4 E0[kEnvRec], E1[kEnvRec], R[kEnvRec];
  float4 C[kEnvRec][kMaxBatch];
};

// The thread layout and entry arithmetic of camera_tile, with 4 accumulators
// per light and pixel plus 3 for R.
__global__ void __launch_bounds__(kCamThreads) k_camera_env(const EnvCamParams e) {
  __shared__ EnvSmem M;
  const CamParams& p = e.c;
  const int nl = e.nl;
  const int tile = (int)p.tile_order[blockIdx.x];
  const int tx = tile % p.gx, ty = tile / p.gx;
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t wq = 1u << w;
  const int cx = 8 * (w & 1) + (lane & 7), cy0 = 8 * (w >> 1) + (lane >> 3);
  const int px = tx * kTile + cx, py[2] = {ty * kTile + cy0, ty * kTile + cy0 + 4};
  const float lx = cx + 0.5f, ly0 = cy0 + 0.5f, ly1 = cy0 + 4.5f;
  const uint32_t b = p.tile_start[tile], end = p.tile_start[tile + 1];
  float T[2] = {1.f, 1.f}, R[2][3], S[2][kMaxBatch][3], Sh[2][kMaxBatch];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    R[k][0] = R[k][1] = R[k][2] = 0.f;
#pragma unroll
    for (int l = 0; l < kMaxBatch; ++l) S[k][l][0] = S[k][l][1] = S[k][l][2] = Sh[k][l] = 0.f;
  }
  bool done[2] = {!(px < p.W && py[0] < p.H), !(px < p.W && py[1] < p.H)};
  uint32_t consumed[2] = {0u, 0u};
  for (uint32_t rb = b; rb < end; rb += kEnvRec) {
    if (__syncthreads_count(done[0] && done[1]) == kCamThreads) break;
    const int rc = (int)min((uint32_t)kEnvRec, end - rb);
    if (t < rc) {
      const uint32_t rank = p.list[rb + t];
      float4 e0, e1;
      make_entry(p.rrec[rank], ox, oy, e0, e1);
      e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));
      M.E0[t] = e0;
      M.E1[t] = e1;
      M.R[t] = p.ccol[2 * rank + 1];
      const float4* src = e.envcol + (size_t)rank * nl;
#pragma unroll
      for (int l = 0; l < kMaxBatch; ++l)
        if (l < nl) M.C[t][l] = src[l];
    }
    __syncthreads();
    if (!(done[0] && done[1])) {
      auto take = [&](int k, int jj, float pw, float g) {
        const float alpha = fminf(p.amax, g * ex2(pw));
        const float Tn = T[k] * (1.f - alpha);
        if (Tn < p.tstop) {
          done[k] = true;
          consumed[k] = rb - b + jj;
          return;
        }
        const float wt = alpha * T[k];
#pragma unroll
        for (int l = 0; l < kMaxBatch; ++l) {
          if (l < nl) {
            const float4 c = M.C[jj][l];
            S[k][l][0] += wt * c.x; S[k][l][1] += wt * c.y; S[k][l][2] += wt * c.z;
            Sh[k][l] += wt * c.w;
          }
        }
        const float4 r = M.R[jj];
        R[k][0] += wt * r.x; R[k][1] += wt * r.y; R[k][2] += wt * r.z;
        T[k] = Tn;
      };
      for (int jj = 0; jj < rc; ++jj) {
        const float4 e1 = M.E1[jj];
        if (!(__float_as_uint(e1.w) & wq)) continue;  // warp-uniform
        float p0, p1;
        powers2(M.E0[jj], e1.x, lx, ly0, ly1, p0, p1);
        if (!done[0] && p0 >= e1.y) take(0, jj, p0, e1.z);
        if (!done[1] && p1 >= e1.y) take(1, jj, p1, e1.z);
        if (done[0] && done[1]) break;
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (!done[k]) consumed[k] = rb - b + rc;
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (!(px < p.W && py[k] < p.H)) continue;
    const size_t pix = (size_t)py[k] * p.W + px;
    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
#pragma unroll
    for (int l = 0; l < kMaxBatch; ++l) {
      if (l < nl) {
        // the image light l's own frame gives, then its weight
        const float i0 = S[k][l][0] * Sh[k][l] + R[k][0], i1 = S[k][l][1] * Sh[k][l] + R[k][1],
                    i2 = S[k][l][2] * Sh[k][l] + R[k][2];
        o0 = fmaf(e.w[l], i0, o0);
        o1 = fmaf(e.w[l], i1, o1);
        o2 = fmaf(e.w[l], i2, o2);
      }
    }
    if (e.accumulate) {
      o0 += p.out[3 * pix + 0];
      o1 += p.out[3 * pix + 1];
      o2 += p.out[3 * pix + 2];
    }
    p.out[3 * pix + 0] = o0;
    p.out[3 * pix + 1] = o1;
    p.out[3 * pix + 2] = o2;
    p.final_t[pix] = T[k];
    p.n_contrib[pix] = consumed[k];
  }
}

// Launch order of a splat's tiles: longest list first, so that the last
// blocks to start are the short ones and the final partial wave stays short
// (a longest-processing-time-first schedule).  One block: a counting sort on
// a key of the list length (1024 buckets, the largest first), placed by
// shared-memory atomics.  The key is the length in steps of 8 (longer lists
// share the top bucket), or with seg_len > 0 the tile's number of shadow
// segments, seg_count(length); then lvl_off[s] (s = 0..1024) also receives
// the first work item of segment level s: the number of segments of levels
// below s, level s holding every tile with more than s segments (a prefix of
// the order).  The order within a bucket may vary from run to run; no result
// depends on it.
__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ tile_start, int ntiles,
                                                     uint32_t* __restrict__ order, uint32_t seg_len,
                                                     uint32_t* __restrict__ lvl_off) {
  constexpr int kBuckets = 1024;
  __shared__ uint32_t cnt[kBuckets];
  __shared__ uint32_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  auto bucket = [&](int i) {
    const uint32_t len = tile_start[i + 1] - tile_start[i];
    const uint32_t key = seg_len ? seg_count(len) : min(len >> 3, (uint32_t)(kBuckets - 1));
    return (uint32_t)(kBuckets - 1) - key;  // largest key first
  };
  // exclusive scan of one value per thread over the block
  auto block_scan = [&](uint32_t c) -> uint32_t {
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;
    }
    __syncthreads();
    const uint32_t r = (warp ? wsum[warp - 1] : 0u) + x - c;
    __syncthreads();  // wsum is free for the next scan
    return r;
  };
  cnt[t] = 0u;
  __syncthreads();
  for (int i = t; i < ntiles; i += blockDim.x) atomicAdd(&cnt[bucket(i)], 1u);
  __syncthreads();
  const uint32_t before = block_scan(cnt[t]);  // tiles in buckets < t: key > 1023 - t
  __syncthreads();
  cnt[t] = before;
  __syncthreads();
  if (lvl_off) {
    // level s holds the tiles with more than s segments: cnt[1023 - s] of them
    const uint32_t c = t < kBuckets - 1 ? cnt[kBuckets - 1 - t] : 0u;
    const uint32_t off = block_scan(c);
    lvl_off[t] = off;
    if (t == kBuckets - 1) lvl_off[kBuckets] = off + c;
  }
  __syncthreads();
  for (int i = t; i < ntiles; i += blockDim.x) order[atomicAdd(&cnt[bucket(i)], 1u)] = (uint32_t)i;
}

}  // namespace

void launch_tile_order(const FrameArgs& f, int splat, cudaStream_t s) {
  const Workspace& L = *f.L;
  uint32_t* order = at<uint32_t>(f.ws, L.tile_order[splat]);
  k_tile_order<<<1, 1024, 0, s>>>(at<uint32_t>(f.ws, L.sp[splat].tile_start), L.ntiles, order, 0u, nullptr);
  count_launch();
}

size_t shadow_seg_items(int ntiles, size_t cap) { return (size_t)ntiles + cap / kSegLen + 1; }

namespace {

// The shadow composite's parameters of a prepared frame.
ShadowParams shadow_params(const FrameArgs& f) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  uint32_t* lvl = at<uint32_t>(ws, f.L->seg_lvl);
  uint32_t* header = at<uint32_t>(ws, f.L->header);
  ShadowParams p;
  p.tile_order = at<uint32_t>(ws, f.L->tile_order[1]);
  p.lvl_off = lvl;
  p.ticket = lvl + kSegLevels + 1;
  p.pub_a = at<float>(ws, f.L->seg_pub);
  p.pub_flag = at<uint32_t>(ws, f.L->seg_flag);
  p.list = at<uint32_t>(ws, b.tv[fin]);
  p.tile_start = at<uint32_t>(ws, b.tile_start);
  p.rrec = at<SplatRec>(ws, b.rrec);
  p.off = at<uint32_t>(ws, b.off);
  p.kbound = at<uint32_t>(ws, b.tv[1 - fin]);
  p.pass_mask = at<uint8_t>(ws, b.tk[1 - fin]);  // over the distances, once the occluder bounds are done
  p.partial = at<float2>(ws, f.L->partial);
  p.light_final = at<float>(ws, f.L->light_final);
  p.light_stop = at<uint32_t>(ws, f.L->light_stop);
  p.status = header + H_STATUS;
  p.live_rank = at<uint8_t>(ws, f.L->rank_flags);
  p.den_found = p.live_rank + f.L->n;
  p.W = f.L->width; p.H = f.L->height; p.gx = f.L->gx;
  p.amax = f.opts.alpha_max;
  return p;
}

CamParams camera_params(const FrameArgs& f, float* out_rgb) {
  const SplatBufs& b = f.L->sp[0];
  unsigned char* ws = f.ws;
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  CamParams p;
  p.list = at<uint32_t>(ws, b.tv[fin]);
  p.tile_start = at<uint32_t>(ws, b.tile_start);
  p.rrec = at<SplatRec>(ws, b.rrec);
  p.ccol = at<float4>(ws, f.L->ccol);
  p.out = out_rgb;
  p.final_t = at<float>(ws, f.L->final_t);
  p.n_contrib = at<uint32_t>(ws, f.L->n_contrib);
  p.pix_aux = at<float4>(ws, f.L->pix_aux);
  p.W = f.L->width; p.H = f.L->height; p.gx = f.L->gx;
  p.amax = f.opts.alpha_max; p.tstop = f.opts.t_stop;
  p.tile_order = at<uint32_t>(ws, f.L->tile_order[0]);  // from the camera binning stage
  return p;
}

// Blocks per SM of the persistent segment kernels (per device, looked up once).
struct SegOccupancy {
  int chain, live, dead;
};
SegOccupancy seg_occupancy() {
  static DeviceOnce once;
  static SegOccupancy occ[kMaxDevices];
  once.run([] {
    int d = 0;
    cudaGetDevice(&d);
    bool ok = true;
    for (const void* k : {(const void*)k_shadow<false>, (const void*)k_shadow<true>, (const void*)k_shadow_chain<false>,
                          (const void*)k_shadow_chain<true>})
      ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
    if (d >= 0 && d < kMaxDevices) {
      SegOccupancy& o = occ[d];
      ok = ok &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.chain, k_shadow_chain<true>, kSegWarps * 32, 0) ==
               cudaSuccess &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.live, k_shadow<true>, kSegWarps * 32, 0) == cudaSuccess &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.dead, k_shadow_dead<true>, kDeadWarps * 32, 0) ==
               cudaSuccess;
    }
    return ok;
  });
  int d = 0;
  cudaGetDevice(&d);
  SegOccupancy o{1, 1, 1};
  if (d >= 0 && d < kMaxDevices) o = occ[d];
  if (o.chain < 1) o.chain = 1;
  if (o.live < 1) o.live = 1;
  if (o.dead < 1) o.dead = 1;
  return o;
}

// Layout of a batch's parameter block (device, and its pinned host staging).
struct BatchLayout {
  static constexpr size_t shadow = 0;
  static constexpr size_t camera = ((sizeof(ShadowParams) * kMaxBatch + 255) / 256) * 256;
  static constexpr size_t prefix = camera + ((sizeof(CamParams) * kMaxBatch + 255) / 256) * 256;
  static constexpr size_t total = prefix + 4 * (kMaxBatch + 1);
};

}  // namespace

size_t batch_param_bytes() { return BatchLayout::total; }

void prepare_shadow_composite(const FrameArgs& f, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  // the distance of every list entry (written by the binning) and the occluder bounds
  float* dl = at<float>(ws, b.tk[1 - fin]);
  uint32_t* kb = at<uint32_t>(ws, b.tv[1 - fin]);
  // the light tiles by segment count, and the work items of each segment level
  uint32_t* lvl = at<uint32_t>(ws, f.L->seg_lvl);
  cudaMemsetAsync(lvl + kSegLevels + 1, 0, 12, s);  // the tickets
  cudaMemsetAsync(at<uint32_t>(ws, f.L->seg_flag), 0, 4 * shadow_seg_items(f.L->ntiles, f.L->cap), s);
  cudaMemsetAsync(ws + f.L->rank_flags, 0, 2 * (size_t)f.L->n, s);
  k_tile_order<<<1, 1024, 0, s>>>(at<uint32_t>(ws, b.tile_start), f.L->ntiles, at<uint32_t>(ws, f.L->tile_order[1]),
                                  kSegLen, lvl);
  // the occluder bounds the segment plan reads; the rest follow K6a
  const size_t items = shadow_seg_items(f.L->ntiles, f.L->cap);
  k_bound_starts<<<(int)((items + 255) / 256), 256, 0, s>>>(shadow_params(f), dl, kb, f.opts.shadow_bias);
  count_launch(2);
}

// the occluder bounds of the open segments' other entries (after K6a)
void launch_bound_rest(const FrameArgs& f, const ShadowParams& p, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  const size_t items = shadow_seg_items(f.L->ntiles, f.L->cap);
  k_bound_rest<<<(int)((items * 32 + 255) / 256), 256, 0, s>>>(p, at<float>(f.ws, b.tk[1 - fin]),
                                                               at<uint32_t>(f.ws, b.tv[1 - fin]), f.opts.shadow_bias);
  count_launch();
}

void launch_shadow_composite(const FrameArgs& f, cudaStream_t s) {
  prepare_shadow_composite(f, s);
  const ShadowParams p = shadow_params(f);
  const SegOccupancy o = seg_occupancy();
  const int nsm = device_sm_count();
  // persistent warps: every resident warp slot takes segments from a ticket
  k_shadow_chain<false><<<nsm * o.chain, kSegWarps * 32, 0, s>>>(p, nullptr, 1);
  launch_bound_rest(f, p, s);
  k_shadow<false><<<nsm * o.live, kSegWarps * 32, 0, s>>>(p, nullptr, 1);
  k_dead_probe<<<(f.L->n + 255) / 256, 256, 0, s>>>(p, f.L->n);
  k_shadow_dead<false><<<nsm * o.dead, kDeadWarps * 32, 0, s>>>(p, nullptr, 1);
  count_launch(4);
}

// Self-test of the chain's bounded waits: the segment plan of a frame whose
// light binning ran, then K6a with its ticket starting at the second segment
// level, so that no first segment ever publishes and every second segment's
// wait runs out (each then publishes its rays as stopped).
__global__ void k_skip_first_level(const uint32_t* lvl_off, uint32_t* ticket) {
  if (threadIdx.x == 0) ticket[0] = lvl_off[1];
}

void launch_shadow_chain_selftest(const FrameArgs& f, cudaStream_t s) {
  prepare_shadow_composite(f, s);
  const ShadowParams p = shadow_params(f);
  k_skip_first_level<<<1, 32, 0, s>>>(p.lvl_off, p.ticket);
  const SegOccupancy o = seg_occupancy();
  k_shadow_chain<false><<<device_sm_count() * o.chain, kSegWarps * 32, 0, s>>>(p, nullptr, 1);
  count_launch(2);
}

void launch_shadow_composite_batch(const FrameArgs* const* f, int n, unsigned char* dev, unsigned char* host,
                                   cudaStream_t s) {
  ShadowParams* hp = reinterpret_cast<ShadowParams*>(host + BatchLayout::shadow);
  for (int r = 0; r < n; ++r) hp[r] = shadow_params(*f[r]);
  cudaMemcpyAsync(dev + BatchLayout::shadow, hp, sizeof(ShadowParams) * n, cudaMemcpyHostToDevice, s);
  const ShadowParams* dp = reinterpret_cast<const ShadowParams*>(dev + BatchLayout::shadow);
  // the batch shares the first frame's tickets; every frame's flags were zeroed when it was prepared
  const SegOccupancy o = seg_occupancy();
  const int nsm = device_sm_count();
  k_shadow_chain<true><<<nsm * o.chain, kSegWarps * 32, 0, s>>>(hp[0], dp, n);
  for (int r = 0; r < n; ++r) launch_bound_rest(*f[r], hp[r], s);
  k_shadow<true><<<nsm * o.live, kSegWarps * 32, 0, s>>>(hp[0], dp, n);
  for (int r = 0; r < n; ++r) k_dead_probe<<<(f[r]->L->n + 255) / 256, 256, 0, s>>>(hp[r], f[r]->L->n);
  k_shadow_dead<true><<<nsm * o.dead, kDeadWarps * 32, 0, s>>>(hp[0], dp, n);
  count_launch(2 + n + 1);
}

void launch_shadow_reduce(const FrameArgs& f, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int n = f.sc.n;
  k_shadow_reduce<<<(n * 8 + 255) / 256, 256, 0, s>>>(
      n, at<uint32_t>(ws, b.off), at<uint32_t>(ws, b.cnt), at<float2>(ws, f.L->partial),
      at<uint32_t>(ws, b.sv[1]), at<uint32_t>(ws, f.L->header), at<float>(ws, f.L->T),
      at<float>(ws, f.L->shadow_den));
  count_launch();
}

void launch_fill_shadow_one(const FrameArgs& f, cudaStream_t s) {
  const int n = f.sc.n;
  k_fill<<<(n + 255) / 256, 256, 0, s>>>(at<float>(f.ws, f.L->T), n, 1.f);
  k_fill<<<(n + 255) / 256, 256, 0, s>>>(at<float>(f.ws, f.L->shadow_den), n, 0.f);
  count_launch();
  count_launch();
}

void launch_camera_composite(const FrameArgs& f, float* out_rgb, cudaStream_t s) {
  k_camera<false><<<f.L->ntiles, kCamThreads, 0, s>>>(camera_params(f, out_rgb), nullptr, nullptr, 1);
  count_launch();
}

void launch_camera_env(const FrameArgs& f0, const float4* envcol, int nl, const float* w, bool accumulate,
                       float* out_rgb, cudaStream_t s) {
  EnvCamParams e;
  e.c = camera_params(f0, out_rgb);
  e.envcol = envcol;
  e.nl = nl;
  for (int l = 0; l < kMaxBatch; ++l) e.w[l] = l < nl ? w[l] : 0.f;
  e.accumulate = accumulate ? 1 : 0;
  k_camera_env<<<f0.L->ntiles, kCamThreads, 0, s>>>(e);
  count_launch();
}

void launch_camera_composite_batch(const FrameArgs* const* f, float* const* out, int n, unsigned char* dev,
                                   unsigned char* host, cudaStream_t s) {
  CamParams* hp = reinterpret_cast<CamParams*>(host + BatchLayout::camera);
  uint32_t* pre = reinterpret_cast<uint32_t*>(host + BatchLayout::prefix);
  pre[0] = 0;
  for (int r = 0; r < n; ++r) {
    hp[r] = camera_params(*f[r], out[r]);
    pre[r + 1] = pre[r] + (uint32_t)f[r]->L->ntiles;
  }
  cudaMemcpyAsync(dev + BatchLayout::camera, hp, sizeof(CamParams) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dev + BatchLayout::prefix, pre, 4 * (n + 1), cudaMemcpyHostToDevice, s);
  k_camera<true><<<pre[n], kCamThreads, 0, s>>>(hp[0], reinterpret_cast<const CamParams*>(dev + BatchLayout::camera),
                                         reinterpret_cast<const uint32_t*>(dev + BatchLayout::prefix), n);
  count_launch();
}

}  // namespace gs3
