// K6, K7: shadow splatting (Sec. 4.2, Fig. 3) and K9: camera compositing
// (Sec. 3, Eq. 2) with the deferred per-pixel combination (Sec. 4).
//
// Both composites stream a 16x16 tile's depth-ordered list through shared
// memory: the shadow composite with one warp per tile (eight rays per lane),
// the camera composite with one 256-thread block per tile (one pixel per
// thread, batches of 256 records).
#include "gs3_internal.cuh"
#include "splat_eval.cuh"

namespace gs3 {
namespace {

// Pixel of thread t inside its 16x16 tile: warp w covers the 8x4 block at
// (8 (w & 1), 4 (w >> 1)); lane l is pixel (l & 7, l >> 3) of that block.
__device__ __forceinline__ int tile_px(int t) { return ((t >> 5) & 1) * 8 + (t & 7); }
__device__ __forceinline__ int tile_py(int t) { return ((t >> 5) >> 1) * 4 + ((t & 31) >> 3); }

// Bit w set when the splat's alpha >= alpha_min box can reach warp w's 8x4
// pixel block of tile (tx, ty); a warp whose bit is clear has no passing
// pixel and skips the splat.
__device__ __forceinline__ uint32_t warp_mask(const SplatRec& q, int tx, int ty) {
  const float hx = q.c.y, hy = q.c.z;
  if (!(hx >= 0.f)) return 0u;
  const float u = q.a.x + q.b.w, v = q.a.y + q.c.x;
  uint32_t m = 0u;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const float x0 = tx * kTile + (w & 1) * 8 + 0.5f, y0 = ty * kTile + (w >> 1) * 4 + 0.5f;
    const bool hit = (u + hx >= x0) && (u - hx <= x0 + 7.f) && (v + hy >= y0) && (v - hy <= y0 + 3.f);
    m |= hit ? (1u << w) : 0u;
  }
  return m;
}

// power of a splat at a pixel centre; the centre is (a.x + b.w, a.y + c.x),
// high part subtracted first so the offset keeps its precision.
__device__ __forceinline__ float splat_power(const float4 a, const float4 b, float vlo, float fx, float fy) {
  const float dx = (fx - a.x) - b.w, dy = (fy - a.y) - vlo;
  return -0.5f * (b.x * dx * dx + b.z * dy * dy) - b.y * dx * dy;
}

// ---------------------------------------------------------------------------
// K6: shadow composite.
// For every shadow ray m (light pixel) and every list entry j that passes the
// alpha test, T_m(j) = prod (1 - alpha_k,m) over passing k with
// d_k < d_j - bias.  The list is ordered by distance, so the occluders of j
// form a prefix of the tile's list; its end K(j) is precomputed per entry
// (k_occluder_bound) and is non-decreasing in j.
//
// One warp per 16x16 tile, eight pixels per lane: lane l owns column l & 15,
// rows (l >> 4) + 2 i, i = 0..7 (i < 4: the tile's top half).  The warp walks
// the tile's list once: receivers are staged kRecv at a time, the occluders
// they need through a window of up to kOccWin records, and each lane keeps
// its eight rays' products A over the consumed occluders.  Records hold the
// splat centre relative to the tile origin (pixel offsets are one exact
// subtraction) and the pre-scaled conic.  A receiver is evaluated only in
// the halves of the tile (8 rows each) that both its alpha >= alpha_min box
// and its ellipse reach.  Per receiver each lane sums (beta A, beta) over its
// eight rays into a shared-memory row; every kRedGroup receivers the warp
// adds the rows' 32 lane sums per receiver, in lane order, into the
// (tile, Gaussian) partials (no shuffle chain per receiver).  The halves
// where a receiver passed are recorded at once (two votes, as quadrant bits
// 0x3 / 0xC); an occluder is evaluated only in the halves where it passed as
// a receiver (same power test) and where some ray has not stopped.  A ray
// stops taking occluders once its product is below kShadowStop; once all
// 256 rays stopped, the warp walks the rest of the list as receivers only.
// ---------------------------------------------------------------------------
constexpr int kRecv = 64;
constexpr int kOccWin = 128;
constexpr int kRedGroup = 16;  // receivers whose per-lane sums are reduced together
constexpr int kShadowThreads = 32;
constexpr int kPx = 8;  // pixels per lane

struct ShadowParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const SplatRec* rrec;
  const uint32_t* off;
  const uint32_t* kbound;
  const uint32_t* tile_order;  // block b renders tile tile_order[b]
  uint8_t* pass_mask;  // per list entry: halves with a passing pixel, 0x3 rows 0-7, 0xC rows 8-15
  float2* partial;
  float* light_final;     // per light pixel: the product where the ray ended
  uint32_t* light_stop;   // per light pixel: 1 + index of the occluder that stopped it, or kNoStop
  int W, H, gx;
  float amax;
};

struct ShadowSmem {
  float4 r0[kRecv], r1[kRecv];
  uint32_t rk[kRecv], rslot[kRecv];
  uint32_t rpass[kRecv];  // halves in which the receiver passed
  float4 o0[kOccWin], o1[kOccWin];
  float2 red[kRedGroup][33];  // per receiver of the group, per lane: (num, den); padded row
};

// Halves of a tile (0x3: rows 0-7, 0xC: rows 8-15, as quadrant bits) where
// the entry's alpha >= alpha_min ellipse can hold a pixel centre.  With
// q = -power2 = al dx^2 + be dx dy + ga dy^2 (positive definite), a pixel
// passes where q <= -thr.  The minimum of q over a half's rectangle of pixel
// centres is 0 if the splat centre lies inside, else it lies on an edge: on
// x = X the minimiser is dy = -be X / (2 ga) clamped to the edge, on y = Y
// dx = -be Y / (2 al).  The margin, 1e-4 of a bound on the terms' size, is far
// above the FP32 rounding of either side, so a half with a passing pixel is
// never dropped; only the work is culled, not the result.
__device__ __forceinline__ uint32_t ellipse_halves(const float4 e0, const float4 e1) {
  const float al = -e0.z, ga = -e0.w, be = -e1.x, lim = -e1.y;
  const float X0 = 0.5f - e0.x, X1 = 15.5f - e0.x;
  const float mx = fmaxf(X0 * X0, X1 * X1);
  auto q = [&](float dx, float dy) { return fmaf(dx, fmaf(al, dx, be * dy), ga * dy * dy); };
  uint32_t m = 0u;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float Y0 = 8.f * h + 0.5f - e0.y, Y1 = 8.f * h + 7.5f - e0.y;
    float best = 0.f;
    if (!(X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f)) {
      const float kx = -be / (2.f * ga), ky = -be / (2.f * al);
      best = fminf(fminf(q(X0, fminf(fmaxf(kx * X0, Y0), Y1)), q(X1, fminf(fmaxf(kx * X1, Y0), Y1))),
                   fminf(q(fminf(fmaxf(ky * Y0, X0), X1), Y0), q(fminf(fmaxf(ky * Y1, X0), X1), Y1)));
    }
    const float size = 2.f * (al * mx + ga * fmaxf(Y0 * Y0, Y1 * Y1));
    if (best <= lim + 1e-4f * (1.f + size)) m |= 3u << (2 * h);
  }
  return m;
}

__global__ void __launch_bounds__(kShadowThreads, 18) k_shadow(ShadowParams p) {
  __shared__ ShadowSmem S;
  const int tile = (int)p.tile_order[blockIdx.x];
  const int tx = tile % p.gx, ty = tile / p.gx;
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const int lane = threadIdx.x;
  const int lxi = lane & 15, lyi = lane >> 4;
  const bool inx = tx * kTile + lxi < p.W;
  const float lx = lxi + 0.5f;
  // A pixel outside the image is moved far from every splat: its power is
  // then far below any threshold and it never passes.  It starts stopped.
  const float kFar = 1.0e6f;
  float ly[kPx], A[kPx];
  uint32_t lim[kPx];
  bool any_in = false;
#pragma unroll
  for (int i = 0; i < kPx; ++i) {
    const bool in = inx && ty * kTile + lyi + 2 * i < p.H;
    ly[i] = in ? lyi + 2 * i + 0.5f : kFar;
    A[i] = in ? 1.f : 0.f;
    lim[i] = kNoStop;
    any_in |= in;
  }
  const float omin = 1.f - p.amax;
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  bool dead = !__any_sync(0xffffffffu, any_in);  // all 256 rays stopped
  uint32_t live = dead ? 0u : 0xFu;  // halves (0x3, 0xC) with a ray that has not stopped
  uint32_t k = b;

  // one occluder (list index kk, window slot i) on the lane's rays
  auto occlude8 = [&](int i, uint32_t kk, uint32_t rb) {
    const float4 o1 = S.o1[i];
    const uint32_t bits = (kk >= rb ? S.rpass[kk - rb] : __float_as_uint(o1.w)) & live;
    if (!bits) return;
    const float4 o0 = S.o0[i];
    const float dx = lx - o0.x;
    const float sx = (o0.z * dx) * dx, v = o1.x * dx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(bits & (3u << (2 * h)))) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i8 = 4 * h + q;
        const float dy = ly[i8] - o0.y;
        const float pw = fmaf(dy, fmaf(o0.w, dy, v), sx);
        if (pw >= o1.y && A[i8] >= kShadowStop) {
          A[i8] *= fmaxf(omin, fmaf(-o1.z, ex2(pw), 1.f));
          if (A[i8] < kShadowStop) lim[i8] = kk + 1;
        }
      }
    }
  };
  // refreshes the live halves after an occluder run; false once every ray stopped
  auto still_alive = [&]() {
    bool al[2] = {false, false};
#pragma unroll
    for (int i = 0; i < kPx; ++i) al[i >> 2] |= A[i] >= kShadowStop;
    live = (__any_sync(0xffffffffu, al[0]) ? 0x3u : 0u) | (__any_sync(0xffffffffu, al[1]) ? 0xCu : 0u);
    return live != 0u;
  };

  // Sums of the receivers of group [j0, jl]: lane t < 16 adds num of receiver
  // j0 + t over the 32 lanes, lane 16 + t its den, in lane order.
  auto reduce_group = [&](int jl) {
    const int j0 = jl - jl % kRedGroup;
    const int t = lane & 15, c = lane >> 4;
    if (j0 + t <= jl) {
      const float* row = reinterpret_cast<const float*>(S.red[t]) + c;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int l = 0; l < 32; l += 4) {
        a0 += row[2 * l]; a1 += row[2 * l + 2]; a2 += row[2 * l + 4]; a3 += row[2 * l + 6];
      }
      reinterpret_cast<float*>(p.partial)[2 * (size_t)S.rslot[j0 + t] + c] = (a0 + a1) + (a2 + a3);
    }
    __syncwarp();  // the group's rows are free again
  };

  // receiver jj of the staged batch: the lane's (beta A, beta) sums over its
  // eight rays, and the halves where it passed somewhere in the tile
  auto eval_receiver = [&](int jj, float& num, float& den) -> uint32_t {
    const float4 r1 = S.r1[jj];
    const uint32_t box = __float_as_uint(r1.w);
    num = 0.f;
    den = 0.f;
    if (!box) return 0u;  // its ellipse reaches no pixel centre of the tile
    const float4 r0 = S.r0[jj];
    const float dx = lx - r0.x;
    const float sx = (r0.z * dx) * dx, v = r1.x * dx;
    bool hit[2] = {false, false};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(box & (3u << (2 * h)))) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i8 = 4 * h + q;
        const float dy = ly[i8] - r0.y;
        const float pw = fmaf(dy, fmaf(r0.w, dy, v), sx);
        if (pw >= r1.y) {
          const float beta = ex2(pw);
          num = fmaf(beta, A[i8], num);
          den += beta;
          hit[h] = true;
        }
      }
    }
    return (__any_sync(0xffffffffu, hit[0]) ? 0x3u : 0u) | (__any_sync(0xffffffffu, hit[1]) ? 0xCu : 0u);
  };

  for (uint32_t rb = b; rb < e; rb += kRecv) {
    const int rc = (int)min((uint32_t)kRecv, e - rb);
    __syncwarp();  // the previous batch is consumed
    for (int t = lane; t < rc; t += kShadowThreads) {
      const uint32_t rank = p.list[rb + t];
      const SplatRec q = p.rrec[rank];
      float4 e0, e1;
      make_entry(q, ox, oy, e0, e1);
      // a half must be reached by the alpha box (one of its quadrants) and by the ellipse
      e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));
      S.r0[t] = e0;
      S.r1[t] = e1;
      if (!dead) S.rk[t] = p.kbound[rb + t];
      S.rslot[t] = p.off[rank] + (uint32_t)((ty - q.r.y) * (q.r.z - q.r.x + 1) + (tx - q.r.x));
    }
    __syncwarp();
    if (dead) {
      // every ray stopped: no occluders, no windows, no pass lookups by
      // occluders; the receivers only
      for (int jj = 0; jj < rc; ++jj) {
        float num, den;
        const uint32_t bits = eval_receiver(jj, num, den);
        S.red[jj % kRedGroup][lane] = make_float2(num, den);
        if (lane == 0) p.pass_mask[rb + jj] = (uint8_t)bits;
        if (jj % kRedGroup == kRedGroup - 1 || jj == rc - 1) {
          __syncwarp();
          reduce_group(jj);
        }
      }
      continue;
    }
    const uint32_t klast = S.rk[rc - 1];
    int jj = 0;
    while (jj < rc) {
      // once every ray stopped the rest of the batch's occluders form one
      // window that nobody loads
      const uint32_t kt = dead ? klast : min(klast, k + (uint32_t)kOccWin);
      if (!dead) {
        // an occluder of an earlier batch carries the halves where it passed
        // as a receiver; one of this batch is looked up when it is used
        for (uint32_t i = lane; i < kt - k; i += kShadowThreads) {
          make_entry(p.rrec[p.list[k + i]], ox, oy, S.o0[i], S.o1[i]);
          if (k + i < rb) S.o1[i].w = __uint_as_float((uint32_t)p.pass_mask[k + i]);
        }
      }
      __syncwarp();
      const uint32_t ow = k;
      for (; jj < rc; ++jj) {
        const uint32_t kend = S.rk[jj];
        if (kend > kt) break;
        if (dead) {
          k = max(k, kend);
        } else if (k < kend) {
          for (; k < kend; ++k) occlude8((int)(k - ow), k, rb);
          dead = !still_alive();
        }
        // receiver jj: sum (beta A, beta) over the tile's 256 rays
        float num, den;
        const uint32_t bits = eval_receiver(jj, num, den);
        S.red[jj % kRedGroup][lane] = make_float2(num, den);
        if (lane == 0) {
          p.pass_mask[rb + jj] = (uint8_t)bits;
          S.rpass[jj] = bits;
        }
        __syncwarp();  // rpass is read by later occluders; red by reduce_group
        if (jj % kRedGroup == kRedGroup - 1 || jj == rc - 1) reduce_group(jj);
      }
      if (dead) {  // the next receiver needs occluders past this window
        k = max(k, kt);
      } else if (k < kt) {
        for (; k < kt; ++k) occlude8((int)(k - ow), k, rb);
        dead = !still_alive();
      }
      __syncwarp();  // the window is consumed
    }
  }
  // the product where each ray ended and where it stopped (the backward starts from them)
  if (inx) {
#pragma unroll
    for (int i = 0; i < kPx; ++i) {
      const int y = ty * kTile + lyi + 2 * i;
      if (y < p.H) {
        const size_t pix = (size_t)y * p.W + tx * kTile + lxi;
        p.light_final[pix] = A[i];
        p.light_stop[pix] = lim[i];
      }
    }
  }
}

// The distance of every list entry, from the depth sort's keys: the key of
// depth rank r is the FP32 bit pattern of rank r's light distance (the
// record's a.w), so this reads 4 bytes per entry instead of a record.
__global__ void __launch_bounds__(256) k_gather_depth(const uint32_t* __restrict__ list,
                                                      const uint32_t* __restrict__ rank_key,
                                                      const uint32_t* header, float* __restrict__ dl,
                                                      uint32_t limit) {
  const uint32_t P = min(header[H_PAIRS_LIGHT], limit);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    dl[i] = __uint_as_float(rank_key[list[i]]);
}

// K(i) for every entry i of the light lists: the first index of i's tile
// segment whose distance is >= d_i - bias (the end of i's occluder prefix).
__global__ void __launch_bounds__(256) k_occluder_bound(const uint32_t* __restrict__ keys,
                                                        const uint32_t* __restrict__ tile_start,
                                                        const float* __restrict__ dl, const uint32_t* header,
                                                        float bias, uint32_t* __restrict__ kb, uint32_t limit) {
  const uint32_t P = min(header[H_PAIRS_LIGHT], limit);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float thr = __fsub_rn(dl[i], bias);
    uint32_t lo = tile_start[keys[i]], hi = i;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (dl[mid] < thr) lo = mid + 1; else hi = mid;
    }
    kb[i] = lo;
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

__global__ void __launch_bounds__(256) k_camera(CamParams p) {
  __shared__ float4 Ga[256], Gb[256], Gc[256], C0[256], C1[256];
  __shared__ uint32_t Gmask[256];
  const int tile = (int)p.tile_order[blockIdx.x];
  const int tx = tile % p.gx, ty = tile / p.gx;
  const int t = threadIdx.x;
  const uint32_t wbit = 1u << (t >> 5);
  const int px = tx * kTile + tile_px(t), py = ty * kTile + tile_py(t);
  const bool inside = px < p.W && py < p.H;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  float T = 1.f, S0 = 0.f, S1 = 0.f, S2 = 0.f, Sh = 0.f, R0 = 0.f, R1 = 0.f, R2 = 0.f;
  bool done = !inside;
  uint32_t consumed = 0;
  for (uint32_t rb = b; rb < e; rb += 256) {
    if (__syncthreads_count(done) == 256) break;
    const int rc = (int)min(256u, e - rb);
    if (t < rc) {
      const uint32_t rank = p.list[rb + t];
      const SplatRec q = p.rrec[rank];
      Ga[t] = q.a;
      Gb[t] = q.b;
      Gc[t] = q.c;
      Gmask[t] = warp_mask(q, tx, ty);
      C0[t] = p.ccol[2 * rank];
      C1[t] = p.ccol[2 * rank + 1];
    }
    __syncthreads();
    if (!done) {
      // two records' alphas are formed ahead of the serial update of T (the
      // same arithmetic, in the same order, as one record at a time)
      auto alpha_of = [&](int jj, float& alpha) -> bool {
        if (!(Gmask[jj] & wbit)) return false;
        const float4 ga = Ga[jj], gc = Gc[jj];
        const float pw = splat_power(ga, Gb[jj], gc.x, fx, fy);
        if (!(pw >= gc.w)) return false;
        alpha = fminf(p.amax, ga.z * __expf(pw));
        return true;
      };
      auto take = [&](int jj, float alpha) -> bool {
        const float Tn = T * (1.f - alpha);
        if (Tn < p.tstop) {
          done = true;
          consumed = rb - b + jj;
          return false;
        }
        const float w = alpha * T;
        const float4 c0 = C0[jj], c1 = C1[jj];
        S0 += w * c0.x; S1 += w * c0.y; S2 += w * c0.z;
        Sh += w * c0.w;
        R0 += w * c1.x; R1 += w * c1.y; R2 += w * c1.z;
        T = Tn;
        return true;
      };
      for (int jj = 0; jj < rc; jj += 2) {
        float a0 = 0.f, a1 = 0.f;
        const bool p0 = alpha_of(jj, a0);
        const bool p1 = jj + 1 < rc && alpha_of(jj + 1, a1);
        if (p0 && !take(jj, a0)) break;
        if (p1 && !take(jj + 1, a1)) break;
      }
      if (!done) consumed = rb - b + rc;
    }
  }
  if (inside) {
    const size_t pix = (size_t)py * p.W + px;
    p.out[3 * pix + 0] = S0 * Sh + R0;
    p.out[3 * pix + 1] = S1 * Sh + R1;
    p.out[3 * pix + 2] = S2 * Sh + R2;
    p.final_t[pix] = T;
    p.n_contrib[pix] = consumed;
    p.pix_aux[2 * pix] = make_float4(S0, S1, S2, Sh);
    p.pix_aux[2 * pix + 1] = make_float4(R0, R1, R2, 0.f);
  }
}

// Launch order of a splat's tiles: longest list first, so that the last
// blocks to start are the short ones and the final partial wave stays short
// (a longest-processing-time-first schedule).  One block: a counting sort on
// the list length in steps of 8 (1024 buckets; longer lists share the first),
// placed by shared-memory atomics.  The order within a bucket may vary from
// run to run; no result depends on it, since every tile writes only its own
// outputs.
__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ tile_start, int ntiles,
                                                     uint32_t* __restrict__ order) {
  constexpr int kBuckets = 1024;
  __shared__ uint32_t cnt[kBuckets];
  __shared__ uint32_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  auto bucket = [&](int i) {
    const uint32_t len = tile_start[i + 1] - tile_start[i];
    return (uint32_t)(kBuckets - 1) - min(len >> 3, (uint32_t)(kBuckets - 1));  // longest first
  };
  cnt[t] = 0u;
  __syncthreads();
  for (int i = t; i < ntiles; i += blockDim.x) atomicAdd(&cnt[bucket(i)], 1u);
  __syncthreads();
  // exclusive scan of the 1024 bucket counts (thread t owns bucket t)
  const uint32_t c = cnt[t];
  uint32_t x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  cnt[t] = (warp ? wsum[warp - 1] : 0u) + x - c;
  __syncthreads();
  for (int i = t; i < ntiles; i += blockDim.x) order[atomicAdd(&cnt[bucket(i)], 1u)] = (uint32_t)i;
}

}  // namespace

void launch_tile_order(const FrameArgs& f, int splat, cudaStream_t s) {
  const Workspace& L = *f.L;
  uint32_t* order = at<uint32_t>(f.ws, L.tile_order[splat]);
  k_tile_order<<<1, 1024, 0, s>>>(at<uint32_t>(f.ws, L.sp[splat].tile_start), L.ntiles, order);
  count_launch();
}

void launch_shadow_composite(const FrameArgs& f, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  // the non-final tile-sort buffers are free after the sort: depth per entry, occluder bound
  float* dl = at<float>(ws, b.tk[1 - fin]);
  uint32_t* kb = at<uint32_t>(ws, b.tv[1 - fin]);
  const uint32_t* header = at<uint32_t>(ws, f.L->header);
  int blocks = (int)((f.L->cap + 255) / 256);
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  // the depth sort's four passes leave the keys in rank order in sk[1]
  k_gather_depth<<<blocks, 256, 0, s>>>(at<uint32_t>(ws, b.tv[fin]), at<uint32_t>(ws, b.sk[1]), header, dl,
                                        (uint32_t)f.L->cap);
  k_occluder_bound<<<blocks, 256, 0, s>>>(at<uint32_t>(ws, b.tk[fin]), at<uint32_t>(ws, b.tile_start), dl, header,
                                          f.opts.shadow_bias, kb, (uint32_t)f.L->cap);
  count_launch(2);
  launch_tile_order(f, 1, s);
  ShadowParams p;
  p.tile_order = at<uint32_t>(ws, f.L->tile_order[1]);
  p.list = at<uint32_t>(ws, b.tv[fin]);
  p.tile_start = at<uint32_t>(ws, b.tile_start);
  p.rrec = at<SplatRec>(ws, b.rrec);
  p.off = at<uint32_t>(ws, b.off);
  p.kbound = kb;
  p.pass_mask = reinterpret_cast<uint8_t*>(dl);  // the depths are consumed by k_occluder_bound
  p.partial = at<float2>(ws, f.L->partial);
  p.light_final = at<float>(ws, f.L->light_final);
  p.light_stop = at<uint32_t>(ws, f.L->light_stop);
  p.W = f.L->width; p.H = f.L->height; p.gx = f.L->gx;
  p.amax = f.opts.alpha_max;
  static DeviceOnce once;
  once.run([] {
    return cudaFuncSetAttribute(k_shadow, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
  });
  k_shadow<<<f.L->ntiles, kShadowThreads, 0, s>>>(p);
  count_launch();
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
  k_camera<<<f.L->ntiles, 256, 0, s>>>(p);
  count_launch();
}

}  // namespace gs3
