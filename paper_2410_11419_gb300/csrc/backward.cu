// Backward of the frame (differentiation form): gradients of a loss with
// respect to every scene parameter and MLP weight, given dL/d(image).
//
// Reverse order of the forward, reading the forward's workspace:
//   K9b  camera composite, back to front per pixel from the stored final
//        transmittance, recovering T by division (per-tile recomputation; no
//        per-pixel lists are stored)                          (Eq. 2, Sec. 4)
//   K8b  Psi and Phi: forward recomputed per 32-row tile, backward through
//        the layers, weight gradients as per-block partials summed in a fixed
//        order                                                  (Sec. 4.2, 4.3)
//   K6b  shadow splat: per shadow ray, back to front from the stored final
//        occluder product; receivers j add (dL/dT_j / den_j) beta T_m(j) to a
//        suffix sum S; an occluder k gets dL/dalpha = -S / (1 - alpha)  (Sec. 4.2)
//   K1b  per Gaussian: both EWA projections and the shading back to the
//        parameters                                       (Eq. 1-5, Sec. 3, 4.1)
// Per-Gaussian accumulators are summed with float atomics (after warp
// reductions); the result is deterministic up to the order of those atomics.
#include "gs3_internal.cuh"
#include "splat_eval.cuh"

namespace gs3 {
namespace {

constexpr int kGeom = 8;    // du, dv, dA, dB, dC, dgamma
constexpr int kColor = 8;   // dshade rgb, dT', dres rgb
constexpr int kMlpIn = 24;  // Phi: dmu 3, dwi 3, dl 6; Psi: dmu 3, dwo 3, dl 6

struct BwdBufs {
  float* cam_geom;    // [N][8]
  float* light_geom;  // [N][8]
  float* color;       // [N][8]
  float* dT;          // [N]
  float* mlp_in;      // [N][24]
};

__host__ __device__ size_t mlp_params(const MlpDev& m) {
  size_t s = 0;
  int din = m.in_dim;
  for (int l = 0; l <= m.n_hidden; ++l) {
    const int dout = l == m.n_hidden ? m.out_dim : m.width;
    s += (size_t)dout * din + dout;
    din = dout;
  }
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct BwdPlan {
  size_t cam_geom, light_geom, color, dT, mlp_in, wred[2], mlp_scratch, total;
};

BwdPlan plan_bwd(int n, const MlpDev& phi, const MlpDev& psi) {
  BwdPlan p;
  size_t c = 0;
  auto take = [&](size_t b) { size_t o = c; c = align256(c + b); return o; };
  p.cam_geom = take(4ull * kGeom * n);
  p.light_geom = take(4ull * kGeom * n);
  p.color = take(4ull * kColor * n);
  p.dT = take(4ull * n);
  p.mlp_in = take(4ull * kMlpIn * n);
  p.wred[0] = take(4ull * mlp_params(phi));
  p.wred[1] = take(4ull * mlp_params(psi));
  const size_t sa = mlp_bwd_scratch_bytes(n, phi), sb = mlp_bwd_scratch_bytes(n, psi);
  p.mlp_scratch = take(sa > sb ? sa : sb);  // Phi and Psi use it in turn
  p.total = c;
  return p;
}

// pixel offset, power and alpha of a splat record at a pixel centre
struct Eval {
  float dx, dy, beta, alpha;
  bool pass, clamped;
};
// A camera-splat entry (make_entry, tile-relative) at the tile pixel centre
// (lx, ly), with the forward composite's arithmetic (power2_at): pass,
// beta = 2^power2, alpha = min(amax, gamma beta); (dx, dy) = pixel - centre.
__device__ __forceinline__ Eval eval_entry(const float4 e0, const float4 e1, float lx, float ly, float amax) {
  Eval r;
  r.dx = lx - e0.x;
  r.dy = ly - e0.y;
  const float pw = power2_at(e0, e1.x, lx, ly);
  r.pass = pw >= e1.y;
  r.beta = r.pass ? ex2(pw) : 0.f;
  const float ga = e1.z * r.beta;
  r.clamped = ga >= amax;
  r.alpha = fminf(amax, ga);
  return r;
}

// dL/dpower -> (du, dv, dA, dB, dC)
__device__ __forceinline__ void power_grad(const SplatRec& q, const Eval& e, float dpow, float* g) {
  const float A = q.b.x, B = q.b.y, C = q.b.z;
  g[0] = (A * e.dx + B * e.dy) * dpow;
  g[1] = (C * e.dy + B * e.dx) * dpow;
  g[2] = -0.5f * e.dx * e.dx * dpow;
  g[3] = -e.dx * e.dy * dpow;
  g[4] = -0.5f * e.dy * e.dy * dpow;
}

// ---------------------------------------------------------------------------
// K9b: camera composite backward
// ---------------------------------------------------------------------------
struct CamBwdParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const uint32_t* tile_order;  // the forward's launch order of the camera tiles
  const SplatRec* rrec;
  const float4* ccol;
  const uint32_t* order;
  const float* final_t;
  const uint32_t* n_contrib;
  const float4* pix_aux;
  const float* dimg;
  float* cam_geom;
  float* color;
  int W, H, gx;
  float amax;
};

// Sums v[0..15] over the warp with one transposing butterfly (16 shuffles):
// each level sends the half of the remaining values that the partner lane
// keeps.  Lane L ends with the total of value
// 8 ((L >> 4) & 1) + 4 ((L >> 3) & 1) + 2 ((L >> 2) & 1) + ((L >> 1) & 1).
__device__ __forceinline__ float warp_sum16(const float (&v)[16], int lane) {
  float a8[8], a4[4], a2[2];
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0, h2 = (lane & 2) != 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a8[i] = (h16 ? v[8 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, h16 ? v[i] : v[8 + i], 16);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    a4[i] = (h8 ? a8[4 + i] : a8[i]) + __shfl_xor_sync(0xffffffffu, h8 ? a8[i] : a8[4 + i], 8);
#pragma unroll
  for (int i = 0; i < 2; ++i)
    a2[i] = (h4 ? a4[2 + i] : a4[i]) + __shfl_xor_sync(0xffffffffu, h4 ? a4[i] : a4[2 + i], 4);
  float x = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? a2[0] : a2[1], 2);
  return x + __shfl_xor_sync(0xffffffffu, x, 1);
}

__global__ void __launch_bounds__(256) k_camera_bwd(CamBwdParams p) {
  __shared__ SplatRec R[256];
  __shared__ float4 E0[256], E1[256], C0[256], C1[256];
  __shared__ uint32_t G[256];
  __shared__ int s_max;
  const int tile = (int)p.tile_order[blockIdx.x], tx = tile % p.gx, ty = tile / p.gx, t = threadIdx.x;
  // warps 2q and 2q + 1 take quadrant q of the tile (the 8x8 block at
  // (8 (q & 1), 8 (q >> 1))), so a warp skips an entry whose alpha box misses it
  const int q4 = t >> 6, qi = t & 63;
  const uint32_t qbit = 1u << q4;
  const int cx = 8 * (q4 & 1) + (qi & 7), cy = 8 * (q4 >> 1) + (qi >> 3);
  const int px = tx * kTile + cx, py = ty * kTile + cy;
  const bool inside = px < p.W && py < p.H;
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const float lx = (float)cx + 0.5f, ly = (float)cy + 0.5f;
  const uint32_t b = p.tile_start[tile];
  const size_t pix = (size_t)py * p.W + px;
  uint32_t nc = 0;
  float T = 1.f, g7[7] = {0, 0, 0, 0, 0, 0, 0};
  if (inside) {
    nc = p.n_contrib[pix];
    T = p.final_t[pix];
    const float4 s = p.pix_aux[2 * pix], r = p.pix_aux[2 * pix + 1];
    const float gr = p.dimg[3 * pix], gg = p.dimg[3 * pix + 1], gb = p.dimg[3 * pix + 2];
    g7[0] = gr * s.w; g7[1] = gg * s.w; g7[2] = gb * s.w;
    g7[3] = gr * s.x + gg * s.y + gb * s.z;
    g7[4] = gr; g7[5] = gg; g7[6] = gb;
    (void)r;
  }
  if (t == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, (int)nc);
  __syncthreads();
  const uint32_t end = min(b + (uint32_t)s_max, p.tile_start[tile + 1]);
  float B7[7] = {0, 0, 0, 0, 0, 0, 0};
  for (uint32_t hi = end; hi > b; ) {
    const uint32_t lo = hi > b + 256 ? hi - 256 : b;
    const int cnt = (int)(hi - lo);
    __syncthreads();
    if (t < cnt) {
      const uint32_t rank = p.list[lo + t];
      const SplatRec q = p.rrec[rank];
      R[t] = q;
      float4 e0, e1;
      make_entry(q, ox, oy, e0, e1);
      e1.w = __uint_as_float(__float_as_uint(e1.w) & ellipse_halves(e0, e1));  // as the forward culls
      E0[t] = e0;
      E1[t] = e1;
      C0[t] = p.ccol[2 * rank];
      C1[t] = p.ccol[2 * rank + 1];
      G[t] = p.order[rank];
    }
    __syncthreads();
    for (int jj = cnt - 1; jj >= 0; --jj) {
      if (!(__float_as_uint(E1[jj].w) & qbit)) continue;  // warp-uniform: the forward skipped it here too
      const uint32_t i = lo + jj;
      const bool active = inside && (i - b) < nc;
      float gv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) gv[k] = 0.f;
      bool contrib = false;
      if (active) {
        const SplatRec q = R[jj];
        const Eval ev = eval_entry(E0[jj], E1[jj], lx, ly, p.amax);
        if (ev.pass) {
          contrib = true;
          T = T / (1.f - ev.alpha);
          const float w = ev.alpha * T;
          const float c[7] = {C0[jj].x, C0[jj].y, C0[jj].z, C0[jj].w, C1[jj].x, C1[jj].y, C1[jj].z};
          float dalpha = 0.f;
          const float inv = 1.f / (1.f - ev.alpha);
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            gv[6 + k] = w * g7[k];
            dalpha += g7[k] * (c[k] * T - B7[k] * inv);
            B7[k] += w * c[k];
          }
          if (!ev.clamped) {
            gv[5] = dalpha * ev.beta;
            power_grad(q, ev, dalpha * ev.alpha, gv);
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        // geometry terms 0-5 and colour terms 6-12 in one butterfly; lane pair
        // (2 k', 2 k' + 1) holds term k', and the even lane adds it
        const int lane = t & 31;
        const float v = warp_sum16(gv, lane);
        const int k = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        if ((lane & 1) == 0 && k < 13 && v != 0.f) {
          const uint32_t g = G[jj];
          if (k < 6) atomicAdd(p.cam_geom + (size_t)kGeom * g + k, v);
          else atomicAdd(p.color + (size_t)kColor * g + (k - 6), v);
        }
      }
    }
    hi = lo;
  }
}

__global__ void k_copy_strided(const float* src, int stride, int off, float* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[(size_t)stride * i + off];
}

// ---------------------------------------------------------------------------
// K6b: shadow splat backward.
// Reverse sweep of the forward's two-cursor pass over each light tile, with
// the forward's thread layout (one warp per tile, eight rays per lane), its
// entries and alpha decisions (splat_eval.cuh).  Per ray m the lane restarts
// from the product A_m where the forward's ray ended and the limit below
// which it took occluders (both stored by the forward; a ray that stopped
// keeps its frozen product past the limit, so occluders at or past it are
// skipped), and a suffix sum S_m = sum coef_j beta_jm T_m(j) over the
// receivers already visited (coef_j = dL/dT_j / den_j):
//   occluder k (passing, taken):  A /= (1 - alpha_k),  dL/dalpha_k = -S / (1 - alpha_k)
//   receiver j (passing):  dL/dbeta_j = coef_j (A - T_j),  S += coef_j beta_j A
// with A = T_m(j) when receiver j is reached.  Occluders are undone before
// the receiver whose prefix end K(j) they reach, so S holds exactly the
// receivers with K(j) > k.  An entry is evaluated only in the halves of the
// tile where it passed in the forward (the pass halves it stored).
// With dL/dpower = w at a pixel (dx, dy) from the splat centre, the centre
// and conic gradients are linear in (w, w dy, w dy^2) for a fixed dx, and
// a lane's eight pixels share dx: each lane sums those three moments and
// forms (du, dv, dA, dB, dC) once per entry; the warp then sums them and
// dgamma over its 256 rays through shared-memory rows, four entries at a
// time, and adds them to the Gaussian's accumulators.
// ---------------------------------------------------------------------------
struct ShadowBwdParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const SplatRec* rrec;
  const uint32_t* order;
  const uint32_t* kbound;
  const uint32_t* tile_order;  // the forward's launch order of the light tiles
  const uint8_t* pass_mask;
  const float* light_final;    // the product where each ray ended
  const uint32_t* light_stop;  // each ray took the occluders below this list index
  const float* dT;   // by index
  const float* den;  // by index
  const float* T;    // by index
  const uint32_t* lvl_off;   // the forward's segment plan: first work item of each segment level
  const uint32_t* pub_flag;  // per item: 2 when every ray entered the next segment stopped
  float* light_geom;
  int W, H, gx;
  float amax;
};

// The first entry of the tile at launch position pos whose segment every ray
// enters stopped (the forward's K6a published A = 0 for all rays into it),
// or e.  Such segments form a suffix of the list.
__device__ __forceinline__ uint32_t stopped_from(const ShadowBwdParams& p, uint32_t pos, uint32_t b, uint32_t e,
                                                 int lane) {
  const uint32_t nseg = seg_count(e - b);
  for (uint32_t s0 = 1; s0 < nseg; s0 += 32) {
    const uint32_t s = s0 + (uint32_t)lane;
    const bool dead = s < nseg && __ldcg(p.pub_flag + p.lvl_off[s - 1] + pos) == 2u;
    const uint32_t m = __ballot_sync(0xffffffffu, dead);
    if (m) return b + (s0 + (uint32_t)(__ffs(m) - 1)) * kSegLen;
  }
  return e;
}

constexpr int kBRecv = 64;
constexpr int kBOcc = 128;
constexpr int kGradGroup = 4;  // entries whose per-lane gradients are reduced together
constexpr int kBThreads = 32;
constexpr int kBPx = 8;  // rays per lane: column lane & 15, rows (lane >> 4) + 2 i
constexpr float kLn2 = 0.6931471805599453f;

struct ShadowBwdSmem {
  float4 r0[kBRecv], r1[kBRecv];
  uint32_t rk[kBRecv], rg[kBRecv];
  float rc[kBRecv], rt[kBRecv];
  float4 o0[kBOcc], o1[kBOcc];
  uint32_t og[kBOcc];
  float gr[kGradGroup][6][33];  // per entry of the group, per gradient term, per lane (padded row)
  uint32_t gg[kGradGroup];      // the entries' Gaussians
};

// The lane's (du, dv, dA, dB, dC) from its moments m0 = sum w, m1 = sum w dy,
// m2 = sum w dy^2 at column offset dx, in g[0..4]: the power (log2 units) is
// a dx^2 + r dx dy + c dy^2 (e0.z = a, e0.w = c), with the conic
// (A, B, C) = -(2 a, r, 2 c) ln 2 and d/du = A dx + B dy, d/dv = C dy + B dx,
// d/dA = -dx^2 / 2, d/dB = -dx dy, d/dC = -dy^2 / 2 (natural units).
__device__ __forceinline__ void moments_to_grad(const float4 e0, float r, float dx, float m0, float m1, float m2,
                                                float (&g)[8]) {
  g[0] = -(2.f * e0.z * dx * m0 + r * m1) * kLn2;
  g[1] = -(2.f * e0.w * m1 + r * dx * m0) * kLn2;
  g[2] = -0.5f * dx * dx * m0;
  g[3] = -dx * m1;
  g[4] = -0.5f * m2;
}

__global__ void __launch_bounds__(kBThreads, 18) k_shadow_bwd(ShadowBwdParams p) {
  __shared__ ShadowBwdSmem S;
  const int tile = (int)p.tile_order[blockIdx.x], tx = tile % p.gx, ty = tile / p.gx;
  const int lane = threadIdx.x;
  const int lxi = lane & 15, lyi = lane >> 4;
  const bool inx = tx * kTile + lxi < p.W;
  const float lx = lxi + 0.5f;
  const float kFar = 1.0e6f;  // off-image pixels never pass (same rule as the forward)
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const float omin = 1.f - p.amax;
  const uint32_t b = p.tile_start[tile], e_all = p.tile_start[tile + 1];
  if (b == e_all) return;
  // receivers from the first stopped segment on are k_shadow_bwd_stopped's;
  // this warp sweeps the open segments back to front
  const uint32_t e = stopped_from(p, blockIdx.x, b, e_all, lane);
  float ly[kBPx], A[kBPx], Sm[kBPx];
  uint32_t lim[kBPx];
  uint32_t lmax = 0u;
#pragma unroll
  for (int i = 0; i < kBPx; ++i) {
    const int y = ty * kTile + lyi + 2 * i;
    const bool in = inx && y < p.H;
    const size_t pix = (size_t)y * p.W + tx * kTile + lxi;
    ly[i] = in ? lyi + 2 * i + 0.5f : kFar;
    A[i] = in ? p.light_final[pix] : 1.f;
    lim[i] = in ? p.light_stop[pix] : 0u;  // an off-image ray took nothing
    Sm[i] = 0.f;
    lmax = max(lmax, lim[i]);
  }
  // occluders at or past every ray's limit were taken by none
  const uint32_t wlim = __reduce_max_sync(0xffffffffu, lmax);
  // occluders the forward walked end at K of the last entry, or, before a
  // stopped segment, at its first bound C (every ray stopped below it)
  uint32_t kc = min(e < e_all ? p.kbound[e] : p.kbound[e - 1], max(wlim, b));

  // An entry's gradient terms, per lane, go to a shared-memory row; every
  // kGradGroup entries lane 6 e + c (< 24) adds term c of entry e over the
  // 32 lanes, in lane order, and adds the total to the Gaussian's
  // accumulator.  No shuffle chain per entry.
  int ng = 0;
  auto reduce_grads = [&]() {
    const int ge = lane / 6, gc = lane % 6;
    if (ge < ng) {
      const float* row = S.gr[ge][gc];
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int l = 0; l < 32; l += 4) {
        a0 += row[l]; a1 += row[l + 1]; a2 += row[l + 2]; a3 += row[l + 3];
      }
      const float v = (a0 + a1) + (a2 + a3);
      if (v != 0.f) atomicAdd(p.light_geom + (size_t)kGeom * S.gg[ge] + gc, v);
    }
    __syncwarp();  // the rows are free again
    ng = 0;
  };
  auto push_grad = [&](uint32_t g, const float (&v)[8]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) S.gr[ng][c][lane] = v[c];
    if (lane == 0) S.gg[ng] = g;
    __syncwarp();
    if (++ng == kGradGroup) reduce_grads();
  };

  // undo occluder kk (window slot i) on the lane's rays; accumulate its gradient
  auto occlude_bwd = [&](int i, uint32_t kk) {
    const float4 o1 = S.o1[i];
    const uint32_t bits = __float_as_uint(o1.w);
    if (!bits) return;
    const float4 o0 = S.o0[i];
    const float dx = lx - o0.x;
    const float sx = (o0.z * dx) * dx, v = o1.x * dx;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, dg = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(bits & (3u << (2 * h)))) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i8 = 4 * h + q;
        const float dy = ly[i8] - o0.y;
        const float pw = fmaf(dy, fmaf(o0.w, dy, v), sx);
        if (pw >= o1.y && kk < lim[i8]) {
          const float beta = ex2(pw), ga = o1.z * beta;
          const float f = fmaxf(omin, fmaf(-o1.z, beta, 1.f));
          const float inv = __frcp_rn(f);
          A[i8] *= inv;
          if (ga < p.amax) {  // alpha = gamma beta (not clamped)
            const float dalpha = -Sm[i8] * inv;
            dg = fmaf(dalpha, beta, dg);  // d/dgamma
            const float w = dalpha * ga, wdy = w * dy;
            m0 += w;
            m1 += wdy;
            m2 = fmaf(wdy, dy, m2);
          }
        }
      }
    }
    float g[8];
    moments_to_grad(o0, o1.x, dx, m0, m1, m2, g);
    g[5] = dg;
    g[6] = g[7] = 0.f;
    push_grad(S.og[i], g);
  };
  // load the occluder window [kt, kc)
  auto load_window = [&](uint32_t kt) {
    __syncwarp();
    for (uint32_t i = lane; i < kc - kt; i += kBThreads) {
      const uint32_t rank = p.list[kt + i];
      make_entry(p.rrec[rank], ox, oy, S.o0[i], S.o1[i]);
      S.o1[i].w = __uint_as_float((uint32_t)p.pass_mask[kt + i]);
      S.og[i] = p.order[rank];
    }
    __syncwarp();
  };

  for (uint32_t re = e; re > b;) {
    const uint32_t rs = re > b + kBRecv ? re - kBRecv : b;
    const int rc = (int)(re - rs);
    __syncwarp();
    for (int t = lane; t < rc; t += kBThreads) {
      const uint32_t rank = p.list[rs + t];
      const uint32_t g = p.order[rank];
      make_entry(p.rrec[rank], ox, oy, S.r0[t], S.r1[t]);
      S.r1[t].w = __uint_as_float((uint32_t)p.pass_mask[rs + t]);
      S.rk[t] = p.kbound[rs + t];
      S.rg[t] = g;
      const float den = p.den[g];
      S.rc[t] = den > 0.f ? p.dT[g] / den : 0.f;
      S.rt[t] = p.T[g];
    }
    __syncwarp();
    int jj = rc - 1;
    while (jj >= 0) {
      const uint32_t kfirst = S.rk[0];
      const uint32_t kt = kc > kfirst + kBOcc ? kc - kBOcc : min(kfirst, kc);
      load_window(kt);
      for (; jj >= 0; --jj) {
        const uint32_t kend = S.rk[jj];
        if (kend < kt) break;
        for (; kc > kend; --kc) occlude_bwd((int)(kc - 1 - kt), kc - 1);
        const float4 r1 = S.r1[jj];
        const uint32_t bits = __float_as_uint(r1.w);
        if (!bits) continue;
        const float4 r0 = S.r0[jj];
        const float dx = lx - r0.x;
        const float sx = (r0.z * dx) * dx, v = r1.x * dx;
        const float coef = S.rc[jj], Tj = S.rt[jj];
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!(bits & (3u << (2 * h)))) continue;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i8 = 4 * h + q;
            const float dy = ly[i8] - r0.y;
            const float pw = fmaf(dy, fmaf(r0.w, dy, v), sx);
            if (pw >= r1.y) {
              const float cb = coef * ex2(pw);
              Sm[i8] = fmaf(cb, A[i8], Sm[i8]);
              const float w = cb * (A[i8] - Tj), wdy = w * dy;
              m0 += w;
              m1 += wdy;
              m2 = fmaf(wdy, dy, m2);
            }
          }
        }
        float g[8];
        moments_to_grad(r0, r1.x, dx, m0, m1, m2, g);
        g[5] = g[6] = g[7] = 0.f;
        push_grad(S.rg[jj], g);
      }
      for (; kc > kt; --kc) occlude_bwd((int)(kc - 1 - kt), kc - 1);
    }
    re = rs;
  }
  // occluders below every receiver's prefix end: S holds all receivers
  while (kc > b) {
    const uint32_t kt = kc > b + kBOcc ? kc - kBOcc : b;
    load_window(kt);
    for (; kc > kt; --kc) occlude_bwd((int)(kc - 1 - kt), kc - 1);
  }
  if (ng) reduce_grads();
}


// K6b for the receivers of the segments every ray enters stopped: the
// forward's products there are 0 (its K6a publishes A = 0 into them), so
// receiver j's beta at ray m carries dL/dbeta = coef_j (0 - T_j) and no
// occluder of these segments is taken.  The receivers are independent: a
// warp takes one such segment, its lanes one (receiver, half) unit at a time
// (the halves the forward found passing), walk the unit's 16 x 8 pixels with
// the forward's power arithmetic, and turn the per-column moments of
// w = dL/dpower into the centre and conic gradients, added to the Gaussian's
// accumulators.  A receiver with T_j = 0 (no pixel of it sees light) adds
// nothing and is skipped.
constexpr int kStopWarps = 4;
__global__ void __launch_bounds__(kStopWarps * 32) k_shadow_bwd_stopped(ShadowBwdParams p) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = blockIdx.x * kStopWarps + (threadIdx.x >> 5);
  if (w >= p.lvl_off[kSegLevels]) return;
  int lo = 0, hi = kSegLevels;  // the item's level: largest s with lvl_off[s] <= w
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p.lvl_off[mid] <= w) lo = mid; else hi = mid;
  }
  if (lo == 0) return;  // a tile's first segment starts with every ray open
  const uint32_t pos = w - p.lvl_off[lo];
  if (__ldcg(p.pub_flag + p.lvl_off[lo - 1] + pos) != 2u) return;
  const int tile = (int)p.tile_order[pos];
  const int tx = tile % p.gx, ty = tile / p.gx;
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  const bool last = (uint32_t)lo == seg_count(e - b) - 1;
  const uint32_t r0 = b + (uint32_t)lo * kSegLen, r1 = last ? e : r0 + kSegLen;
  const int ncol = min(kTile, p.W - tx * kTile), nrow = min(kTile, p.H - ty * kTile);
  // units (receiver, half), two per receiver, taken by the lanes in turn
  for (uint32_t u = lane; u < 2u * (r1 - r0); u += 32) {
    const uint32_t j = r0 + (u >> 1);
    const int h = (int)(u & 1u);
    const uint32_t bits = p.pass_mask[j];
    if (!(bits & (3u << (2 * h)))) continue;
    const uint32_t rank = p.list[j];
    const uint32_t g = p.order[rank];
    const float den = p.den[g], Tj = p.T[g];
    const float coef = den > 0.f ? p.dT[g] / den : 0.f;
    const float cw = -coef * Tj;  // w = dL/dpower = coef beta (0 - T_j)
    if (cw == 0.f) continue;
    float4 e0, e1;
    make_entry(p.rrec[rank], ox, oy, e0, e1);
    float gsum[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int y1 = min(8 * h + 8, nrow);
    for (int x = 0; x < ncol; ++x) {
      const float lx = (float)x + 0.5f;
      const float dx = lx - e0.x;
      const float sx = (e0.z * dx) * dx, v = e1.x * dx;
      float m0 = 0.f, m1 = 0.f, m2 = 0.f;
      for (int y = 8 * h; y < y1; ++y) {
        const float dy = ((float)y + 0.5f) - e0.y;
        const float pw = fmaf(dy, fmaf(e0.w, dy, v), sx);
        if (pw >= e1.y) {
          const float wv = cw * ex2(pw), wdy = wv * dy;
          m0 += wv;
          m1 += wdy;
          m2 = fmaf(wdy, dy, m2);
        }
      }
      float gc[8];
      moments_to_grad(e0, e1.x, dx, m0, m1, m2, gc);
#pragma unroll
      for (int c = 0; c < 5; ++c) gsum[c] += gc[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (gsum[c] != 0.f) atomicAdd(p.light_geom + (size_t)kGeom * g + c, gsum[c]);
  }
}

// ---------------------------------------------------------------------------
// K1b: per-Gaussian backward of both projections and the shading
// ---------------------------------------------------------------------------
struct M3 {
  float m[9];
};

__device__ __forceinline__ void quat_rot(const float4 qr, float Rm[9], float qn[4], float& len) {
  len = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
  const float w = qr.x / len, x = qr.y / len, y = qr.z / len, z = qr.w / len;
  qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
  Rm[0] = 1.f - 2.f * (y * y + z * z); Rm[1] = 2.f * (x * y - w * z);       Rm[2] = 2.f * (x * z + w * y);
  Rm[3] = 2.f * (x * y + w * z);       Rm[4] = 1.f - 2.f * (x * x + z * z); Rm[5] = 2.f * (y * z - w * x);
  Rm[6] = 2.f * (x * z - w * y);       Rm[7] = 2.f * (y * z + w * x);       Rm[8] = 1.f - 2.f * (x * x + y * y);
}

// dL/dR (row-major) of R(q / |q|) -> dL/dq
__device__ __forceinline__ float4 quat_bwd(const float G[9], const float qn[4], float len) {
  const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  float dw = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  float dx = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.f * x * G[8]);
  float dy = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.f * y * G[8]);
  float dz = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
  const float dot = w * dw + x * dx + y * dy + z * dz;
  return make_float4((dw - w * dot) / len, (dx - x * dot) / len, (dy - y * dot) / len, (dz - z * dot) / len);
}

struct ViewB {
  float R[9], t[3];
  float fx, fy, lowpass;
  float ortho;  // > 0: orthographic view with this many pixels per world unit
};

// one EWA projection's backward; adds to dmu, ds and dR (of R(q))
__device__ void proj_bwd(const float4 m, const float4 s, const float Rq[9], const ViewB& v, const float* gg,
                         float dmu[3], float ds[3], float dRq[9]) {
  const float* R = v.R;
  const float x = R[0] * m.x + R[1] * m.y + R[2] * m.z + v.t[0];
  const float y = R[3] * m.x + R[4] * m.y + R[5] * m.z + v.t[1];
  const float z = R[6] * m.x + R[7] * m.y + R[8] * m.z + v.t[2];
  const bool ortho = v.ortho > 0.f;
  const float iz = 1.f / z, iz2 = iz * iz;
  const float sv[3] = {s.x, s.y, s.z};
  float M[9], Sg[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * sv[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Sg[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
  // J = [[fx / z, 0, -fx x / z^2], [0, fy / z, -fy y / z^2]], or [[s, 0, 0], [0, s, 0]]
  const float J00 = ortho ? v.ortho : v.fx * iz, J02 = ortho ? 0.f : -v.fx * x * iz2;
  const float J11 = ortho ? v.ortho : v.fy * iz, J12 = ortho ? 0.f : -v.fy * y * iz2;
  float T[6];
  for (int k = 0; k < 3; ++k) {
    T[k] = J00 * R[k] + J02 * R[6 + k];
    T[3 + k] = J11 * R[3 + k] + J12 * R[6 + k];
  }
  float TS[6];  // T Sigma
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 3; ++k)
      TS[3 * i + k] = T[3 * i] * Sg[k] + T[3 * i + 1] * Sg[3 + k] + T[3 * i + 2] * Sg[6 + k];
  const float a = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + v.lowpass;
  const float b = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
  const float c = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + v.lowpass;
  const float det = a * c - b * b, id = 1.f / det;
  const float CA = c * id, CB = -b * id, CC = a * id;
  // d/d(a, b, c) = -C Gs C with Gs = [[dA, dB/2], [dB/2, dC]]
  const float gA = gg[2], gB = 0.5f * gg[3], gC = gg[4];
  const float X00 = CA * gA + CB * gB, X01 = CA * gB + CB * gC;
  const float X10 = CB * gA + CC * gB, X11 = CB * gB + CC * gC;
  const float D00 = -(X00 * CA + X01 * CB), D01 = -(X00 * CB + X01 * CC), D11 = -(X10 * CB + X11 * CC);
  // G2 (symmetric) = [[D00, D01], [D01, D11]];  dT = 2 G2 T Sigma;  dSigma = T^T G2 T
  float dT[6];
  for (int k = 0; k < 3; ++k) {
    dT[k] = 2.f * (D00 * TS[k] + D01 * TS[3 + k]);
    dT[3 + k] = 2.f * (D01 * TS[k] + D11 * TS[3 + k]);
  }
  float dS[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      dS[3 * i + j] = T[i] * (D00 * T[j] + D01 * T[3 + j]) + T[3 + i] * (D01 * T[j] + D11 * T[3 + j]);
  // dM = 2 dSigma M;  M = Rq diag(s)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const float dM = 2.f * (dS[3 * i] * M[j] + dS[3 * i + 1] * M[3 + j] + dS[3 * i + 2] * M[6 + j]);
      dRq[3 * i + j] += dM * sv[j];
      ds[j] += dM * Rq[3 * i + j];
    }
  // T = J R:  dJ = dT R^T
  const float dJ00 = dT[0] * R[0] + dT[1] * R[1] + dT[2] * R[2];
  const float dJ02 = dT[0] * R[6] + dT[1] * R[7] + dT[2] * R[8];
  const float dJ11 = dT[3] * R[3] + dT[4] * R[4] + dT[5] * R[5];
  const float dJ12 = dT[3] * R[6] + dT[4] * R[7] + dT[5] * R[8];
  const float du = gg[0], dv = gg[1];
  if (ortho) {  // u = s x + cx, v = s y + cy; J constant
    const float dx = du * v.ortho, dy = dv * v.ortho;
    dmu[0] += R[0] * dx + R[3] * dy;
    dmu[1] += R[1] * dx + R[4] * dy;
    dmu[2] += R[2] * dx + R[5] * dy;
    return;
  }
  const float dx = du * v.fx * iz + dJ02 * (-v.fx * iz2);
  const float dy = dv * v.fy * iz + dJ12 * (-v.fy * iz2);
  const float dz = du * (-v.fx * x * iz2) + dv * (-v.fy * y * iz2) + dJ00 * (-v.fx * iz2) +
                   dJ02 * (2.f * v.fx * x * iz2 * iz) + dJ11 * (-v.fy * iz2) + dJ12 * (2.f * v.fy * y * iz2 * iz);
  dmu[0] += R[0] * dx + R[3] * dy + R[6] * dz;
  dmu[1] += R[1] * dx + R[4] * dy + R[7] * dz;
  dmu[2] += R[2] * dx + R[5] * dy + R[8] * dz;
}

struct PrepBwdParams {
  SceneDev sc;
  ViewB cam, light;  // the light view's R, t and scale come from the forward's header
  const float* header_view;  // R (9), t (3) at H_LIGHT_VIEW, scale at H_LIGHT_ORTHO
  float4 lh;                 // homogeneous light (light_h)
  float cam_pos[3], intensity;
  int ablate;
  int falloff;
  const float* cam_geom;
  const float* light_geom;
  const float* color;
  const float* mlp_in;
  gs3_grads out;
};

// One Gaussian of K1b.  With a shared lobe basis the frame and deviation
// gradients of lobe j go to the block's accumulators sacc[8 j + 0..6]
// (rotation 4, sigma 3) instead of per-Gaussian outputs.
__device__ __forceinline__ void prep_bwd_one(const PrepBwdParams& p, int g, float* sacc) {
  const int n = p.sc.n;
  const float4 m = p.sc.mean_op[g], s = p.sc.scale[g];
  const float gamma = 1.f / (1.f + expf(-m.w));
  const float* gc = p.cam_geom + (size_t)kGeom * g;
  const float* gl = p.light_geom + (size_t)kGeom * g;
  float dmu[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dRq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  float Rq[9], qn[4], qlen;
  quat_rot(p.sc.rot[g], Rq, qn, qlen);
  ViewB lv = p.light;
#pragma unroll
  for (int i = 0; i < 12; ++i) (i < 9 ? lv.R[i] : lv.t[i - 9]) = p.header_view[H_LIGHT_VIEW + i];
  lv.ortho = p.header_view[H_LIGHT_ORTHO];
  proj_bwd(m, s, Rq, p.cam, gc, dmu, ds, dRq);
  proj_bwd(m, s, Rq, lv, gl, dmu, ds, dRq);
  const float4 dq = quat_bwd(dRq, qn, qlen);
  const float dgamma = gc[5] + gl[5];
  const float dlogit = dgamma * gamma * (1.f - gamma);

  // ---- shading backward (Eq. 2-5) ----
  const float* dcol = p.color + (size_t)kColor * g;
  const float lx = p.lh.x - p.lh.w * m.x, ly = p.lh.y - p.lh.w * m.y, lz = p.lh.z - p.lh.w * m.z;
  const float d2 = lx * lx + ly * ly + lz * lz, dl = sqrtf(d2);
  const float wi[3] = {lx / dl, ly / dl, lz / dl};
  const float vx = p.cam_pos[0] - m.x, vy = p.cam_pos[1] - m.y, vz = p.cam_pos[2] - m.z;
  const float dvn = sqrtf(vx * vx + vy * vy + vz * vz);
  const float wo[3] = {vx / dvn, vy / dvn, vz / dvn};
  float Rs[9], qs[4], qslen;
  quat_rot(p.sc.shade_rot[g], Rs, qs, qslen);
  float wil[3], wol[3];
  for (int i = 0; i < 3; ++i) {
    wil[i] = Rs[3 * i] * wi[0] + Rs[3 * i + 1] * wi[1] + Rs[3 * i + 2] * wi[2];
    wol[i] = Rs[3 * i] * wo[0] + Rs[3 * i + 1] * wo[1] + Rs[3 * i + 2] * wo[2];
  }
  const float off = 0.01f * (1.f - 0.36787944117144233f);
  const float xz = wil[2];
  const float fd = ((xz > 0.f ? xz : 0.01f * expm1f(xz)) + off) / ((1.f + off) * 3.14159265358979323846f);
  const float dfd_dx = (xz > 0.f ? 1.f : 0.01f * expf(xz)) / ((1.f + off) * 3.14159265358979323846f);
  float hs[3] = {wil[0] + wol[0], wil[1] + wol[1], wil[2] + wol[2]};
  const float hn = sqrtf(hs[0] * hs[0] + hs[1] * hs[1] + hs[2] * hs[2]);
  // the Lambertian-only stage has no lobes: no specular term and no lobe gradients
  const bool have_h = hn * hn >= 1e-24f && !(p.ablate & GS3_ABLATE_SPECULAR);
  float h[3] = {0, 0, 0};
  if (have_h) { h[0] = hs[0] / hn; h[1] = hs[1] / hn; h[2] = hs[2] / hn; }
  const bool falloff = p.falloff && p.lh.w != 0.f;  // a directional light's E is constant
  const float E = falloff ? p.intensity / d2 : p.intensity;
  const float4 rd = p.sc.albedo_d[g], rsp = p.sc.albedo_s[g];
  const float rdv[3] = {rd.x, rd.y, rd.z}, rsv[3] = {rsp.x, rsp.y, rsp.z};
  // f_s (recomputed) and the lobe gradients
  float fs[3] = {0, 0, 0};
  const int K = p.sc.k;
  float dfs[3];
  for (int c = 0; c < 3; ++c) dfs[c] = dcol[c] * E * rsv[c];
  float dh[3] = {0, 0, 0};
  if (have_h) {
    for (int j = 0; j < K; ++j) {
      const size_t li = (size_t)j * n + g;
      float Rl[9], ql[4], qllen;
      const size_t ls = p.sc.lobe_shared ? (size_t)j : li;
      quat_rot(p.sc.lobe_rot[ls], Rl, ql, qllen);
      const float4 sig = p.sc.lobe_sigma[ls];
      const float4 amp = p.sc.lobe_amp[li];
      const float hx = Rl[0] * h[0] + Rl[3] * h[1] + Rl[6] * h[2];
      const float hy = Rl[1] * h[0] + Rl[4] * h[1] + Rl[7] * h[2];
      const float hz = Rl[2] * h[0] + Rl[5] * h[1] + Rl[8] * h[2];
      const float sxy = sqrtf(hx * hx + hy * hy);
      const float theta = atan2f(sxy, hz);
      float Pq = 0.f, e2 = 0.f, G;
      const float iz = 1.f / sig.z;
      if (sxy > 1e-20f) {
        Pq = (hx / sig.x) * (hx / sig.x) + (hy / sig.y) * (hy / sig.y);
        e2 = theta * theta / (sxy * sxy) * Pq * iz * iz;
      } else if (hz < 0.f) {
        e2 = (3.14159265358979323846f / sig.x) * (3.14159265358979323846f / sig.x) * iz * iz;
      }
      G = expf(-0.5f * e2) * iz;
      fs[0] += amp.x * G; fs[1] += amp.y * G; fs[2] += amp.z * G;
      const float dG = dfs[0] * amp.x + dfs[1] * amp.y + dfs[2] * amp.z;
      p.out.lobe_amp[4 * li + 0] = dfs[0] * G;
      p.out.lobe_amp[4 * li + 1] = dfs[1] * G;
      p.out.lobe_amp[4 * li + 2] = dfs[2] * G;
      p.out.lobe_amp[4 * li + 3] = 0.f;
      float dsx = 0.f, dsy = 0.f, dsz = dG * G * (e2 - 1.f) * iz;
      float dhl[3] = {0.f, 0.f, 0.f};
      if (sxy > 1e-20f) {
        const float de2 = dG * (-0.5f * G);
        const float dF = de2 * iz * iz;
        const float is2 = 1.f / (sxy * sxy);
        dsx = dF * theta * theta * is2 * (-2.f * hx * hx / (sig.x * sig.x * sig.x));
        dsy = dF * theta * theta * is2 * (-2.f * hy * hy / (sig.y * sig.y * sig.y));
        const float r2 = sxy * sxy + hz * hz;
        const float th_s = hz / r2, th_z = -sxy / r2;
        const float dF_dsxy = 2.f * theta * th_s * Pq * is2 - 2.f * theta * theta * Pq * is2 / sxy;
        dhl[0] = dF * (dF_dsxy * hx / sxy + theta * theta * is2 * 2.f * hx / (sig.x * sig.x));
        dhl[1] = dF * (dF_dsxy * hy / sxy + theta * theta * is2 * 2.f * hy / (sig.y * sig.y));
        dhl[2] = dF * 2.f * theta * th_z * Pq * is2;
      }
      if (!p.sc.lobe_shared) {
        p.out.lobe_sigma[4 * li + 0] = dsx;
        p.out.lobe_sigma[4 * li + 1] = dsy;
        p.out.lobe_sigma[4 * li + 2] = dsz;
        p.out.lobe_sigma[4 * li + 3] = 0.f;
      }
      // hl = Rl^T h: dh += Rl dhl; dRl[k][i] += h_k dhl_i
      float dRl[9];
      for (int k = 0; k < 3; ++k) {
        dh[k] += Rl[3 * k] * dhl[0] + Rl[3 * k + 1] * dhl[1] + Rl[3 * k + 2] * dhl[2];
        for (int i = 0; i < 3; ++i) dRl[3 * k + i] = h[k] * dhl[i];
      }
      const float4 dql = quat_bwd(dRl, ql, qllen);
      if (p.sc.lobe_shared) {
        float* a = sacc + 8 * j;
        atomicAdd(a + 0, dql.x); atomicAdd(a + 1, dql.y); atomicAdd(a + 2, dql.z); atomicAdd(a + 3, dql.w);
        atomicAdd(a + 4, dsx); atomicAdd(a + 5, dsy); atomicAdd(a + 6, dsz);
      } else {
        reinterpret_cast<float4*>(p.out.lobe_rot)[li] = dql;
      }
    }
  } else {
    for (int j = 0; j < K; ++j) {
      const size_t li = (size_t)j * n + g;
      reinterpret_cast<float4*>(p.out.lobe_amp)[li] = make_float4(0, 0, 0, 0);
      if (!p.sc.lobe_shared) {
        reinterpret_cast<float4*>(p.out.lobe_sigma)[li] = make_float4(0, 0, 0, 0);
        reinterpret_cast<float4*>(p.out.lobe_rot)[li] = make_float4(0, 0, 0, 0);
      }
    }
  }
  float dE = 0.f, dfd = 0.f;
  float drd[3], drs[3];
  for (int c = 0; c < 3; ++c) {
    drd[c] = dcol[c] * E * fd;
    drs[c] = dcol[c] * E * fs[c];
    dE += dcol[c] * (rdv[c] * fd + rsv[c] * fs[c]);
    dfd += dcol[c] * E * rdv[c];
  }
  reinterpret_cast<float4*>(p.out.albedo_d)[g] = make_float4(drd[0], drd[1], drd[2], 0.f);
  reinterpret_cast<float4*>(p.out.albedo_s)[g] = make_float4(drs[0], drs[1], drs[2], 0.f);
  // h = hs / |hs|
  float dwil[3] = {0, 0, 0}, dwol[3] = {0, 0, 0};
  if (have_h) {
    const float hd = h[0] * dh[0] + h[1] * dh[1] + h[2] * dh[2];
    for (int i = 0; i < 3; ++i) {
      const float dhs = (dh[i] - h[i] * hd) / hn;
      dwil[i] = dhs;
      dwol[i] = dhs;
    }
  }
  dwil[2] += dfd * dfd_dx;
  // local = Rs w
  float dRs[9];
  float dwi[3], dwo[3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) dRs[3 * i + k] = dwil[i] * wi[k] + dwol[i] * wo[k];
  for (int k = 0; k < 3; ++k) {
    dwi[k] = Rs[k] * dwil[0] + Rs[3 + k] * dwil[1] + Rs[6 + k] * dwil[2];
    dwo[k] = Rs[k] * dwol[0] + Rs[3 + k] * dwol[1] + Rs[6 + k] * dwol[2];
  }
  const float4 dqs = quat_bwd(dRs, qs, qslen);
  // MLP inputs
  const float* mi = p.mlp_in + (size_t)kMlpIn * g;
  for (int k = 0; k < 3; ++k) {
    dmu[k] += mi[k] + mi[12 + k];
    dwi[k] += mi[3 + k];
    dwo[k] += mi[15 + k];
  }
  // w_i = (L.xyz - L.w mu)/|.|, w_o = (pC - mu)/|.|, E = I / |pL - mu|^2 (point light)
  const float wid = wi[0] * dwi[0] + wi[1] * dwi[1] + wi[2] * dwi[2];
  const float wod = wo[0] * dwo[0] + wo[1] * dwo[1] + wo[2] * dwo[2];
  const float dd2 = falloff ? -dE * E / d2 : 0.f;
  const float lvv[3] = {lx, ly, lz};
  for (int k = 0; k < 3; ++k) {
    dmu[k] -= p.lh.w * (dwi[k] - wi[k] * wid) / dl;
    dmu[k] -= (dwo[k] - wo[k] * wod) / dvn;
    dmu[k] -= 2.f * lvv[k] * dd2;
  }
  reinterpret_cast<float4*>(p.out.mean_op)[g] = make_float4(dmu[0], dmu[1], dmu[2], dlogit);
  reinterpret_cast<float4*>(p.out.scale)[g] = make_float4(ds[0], ds[1], ds[2], 0.f);
  reinterpret_cast<float4*>(p.out.rot)[g] = dq;
  reinterpret_cast<float4*>(p.out.shade_rot)[g] = dqs;
  reinterpret_cast<float4*>(p.out.latent)[g] =
      make_float4(mi[6] + mi[18], mi[7] + mi[19], mi[8] + mi[20], mi[9] + mi[21]);
  reinterpret_cast<float4*>(p.out.latent)[n + g] = make_float4(mi[10] + mi[22], mi[11] + mi[23], 0.f, 0.f);
}

__global__ void __launch_bounds__(128) k_prep_bwd(PrepBwdParams p) {
  __shared__ float sacc[8 * kMaxLobes];
  const bool shared = p.sc.lobe_shared != 0;
  if (shared) {
    for (int i = threadIdx.x; i < 8 * p.sc.k; i += blockDim.x) sacc[i] = 0.f;
    __syncthreads();
  }
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < p.sc.n) prep_bwd_one(p, g, sacc);
  if (shared) {  // the block's sums of the shared basis gradients
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * p.sc.k; i += blockDim.x) {
      const int j = i >> 3, c = i & 7;
      if (c < 4) atomicAdd(p.out.lobe_rot + 4 * j + c, sacc[i]);
      else if (c < 7) atomicAdd(p.out.lobe_sigma + 4 * j + (c - 4), sacc[i]);
    }
  }
}

// scatter the reduced MLP parameter gradients into the (weights, biases) layout
__global__ void k_split_params(const float* red, int in_dim, int width, int nh, int out_dim, float* dw, float* db) {
  // red holds, per layer: W (out x in) then b (out)
  size_t ro = 0, wo = 0, bo = 0;
  int din = in_dim;
  for (int l = 0; l <= nh; ++l) {
    const int dout = l == nh ? out_dim : width;
    const size_t nw = (size_t)dout * din;
    for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x)
      dw[wo + i] = red[ro + i];
    for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)dout; i += gridDim.x * blockDim.x)
      db[bo + i] = red[ro + nw + i];
    ro += nw + dout;
    wo += nw;
    bo += dout;
    din = dout;
  }
}

}  // namespace

size_t backward_workspace_bytes(int n, const MlpDev& phi, const MlpDev& psi) {
  return plan_bwd(n, phi, psi).total;
}

gs3_status run_backward(const FrameArgs& f, const float* dimg, void* bws, size_t bws_bytes,
                        const gs3_grads& out, cudaStream_t s, SideStream* side) {
  const int n = f.sc.n;
  const BwdPlan bp = plan_bwd(n, f.sc.phi, f.sc.psi);
  if (bws_bytes < bp.total) return GS3_ERR_INVALID_ARG;
  unsigned char* B = static_cast<unsigned char*>(bws);
  float* cam_geom = reinterpret_cast<float*>(B + bp.cam_geom);
  float* light_geom = reinterpret_cast<float*>(B + bp.light_geom);
  float* color = reinterpret_cast<float*>(B + bp.color);
  float* dT = reinterpret_cast<float*>(B + bp.dT);
  float* mlp_in = reinterpret_cast<float*>(B + bp.mlp_in);
  cudaMemsetAsync(B, 0, bp.mlp_scratch, s);  // per-Gaussian accumulators start at zero
  unsigned char* ws = f.ws;
  const Workspace& L = *f.L;
  const int fin = (L.ntiles <= 256 ? 1 : 2) & 1;
  // K9b
  {
    CamBwdParams p;
    p.list = at<uint32_t>(ws, L.sp[0].tv[fin]);
    p.tile_start = at<uint32_t>(ws, L.sp[0].tile_start);
    p.tile_order = at<uint32_t>(ws, L.tile_order[0]);
    p.rrec = at<SplatRec>(ws, L.sp[0].rrec);
    p.ccol = at<float4>(ws, L.ccol);
    p.order = at<uint32_t>(ws, L.sp[0].sv[1]);
    p.final_t = at<float>(ws, L.final_t);
    p.n_contrib = at<uint32_t>(ws, L.n_contrib);
    p.pix_aux = at<float4>(ws, L.pix_aux);
    p.dimg = dimg;
    p.cam_geom = cam_geom;
    p.color = color;
    p.W = L.width; p.H = L.height; p.gx = L.gx;
    p.amax = f.opts.alpha_max;
    k_camera_bwd<<<L.ntiles, 256, 0, s>>>(p);
    count_launch();
  }
  // K8b: one network's backward, then its weight gradients in fixed block order
  auto mlp_bwd = [&](int which, cudaStream_t st) {
    const MlpDev& m = which == 0 ? f.sc.phi : f.sc.psi;
    float* wred = reinterpret_cast<float*>(B + bp.wred[which]);
    const bool identity = (f.opts.ablate & (which == 0 ? GS3_ABLATE_PHI : GS3_ABLATE_PSI)) != 0;
    float* dw = which == 0 ? out.phi_w : out.psi_w;
    float* db = which == 0 ? out.phi_b : out.psi_b;
    const size_t np = mlp_params(m);
    if (identity) {
      cudaMemsetAsync(wred, 0, 4 * np, st);
      if (which == 0) {  // T' = T: the gradient passes straight through
        k_copy_strided<<<(n + 255) / 256, 256, 0, st>>>(color, kColor, 3, dT, n);
        count_launch();
      }
    } else {
      MlpArgs a;
      a.net = m;
      a.n = n;
      a.which = which;
      a.mean_op = f.sc.mean_op;
      a.latent = f.sc.latent;
      a.T = at<float>(ws, L.T);
      const float4 lh = light_h(f.light);
      a.light_pos[0] = lh.x; a.light_pos[1] = lh.y; a.light_pos[2] = lh.z; a.light_w = lh.w;
      for (int i = 0; i < 3; ++i) a.cam_pos[i] = f.cam.pos[i];
      a.color = color;
      a.dT = dT;
      a.mlp_in = mlp_in;
      a.status = at<uint32_t>(ws, L.header) + H_STATUS;
      run_mlp_backward(a, B + bp.mlp_scratch, wred, st);
    }
    k_split_params<<<64, 256, 0, st>>>(wred, m.in_dim, m.width, m.n_hidden, m.out_dim, dw, db);
    count_launch();
  };
  // Phi first: the shadow backward takes its dL/dT.  Then Psi, which the
  // shadow backward does not need, runs on the side stream beside it (the
  // networks share the MLP scratch, so they run in turn), with the receivers
  // of the stopped segments; the one-warp-per-tile sweep leaves most SMs idle
  // towards its end.
  mlp_bwd(0, s);
  cudaStream_t ss = s;
  if (side) {
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->s, side->fork, 0);
    ss = side->s;
  }
  // K6b
  if (!(f.opts.ablate & GS3_ABLATE_SHADOW_SPLAT)) {
    ShadowBwdParams p;
    p.list = at<uint32_t>(ws, L.sp[1].tv[fin]);
    p.tile_start = at<uint32_t>(ws, L.sp[1].tile_start);
    p.rrec = at<SplatRec>(ws, L.sp[1].rrec);
    p.order = at<uint32_t>(ws, L.sp[1].sv[1]);
    p.kbound = at<uint32_t>(ws, L.sp[1].tv[1 - fin]);
    p.pass_mask = reinterpret_cast<const uint8_t*>(at<float>(ws, L.sp[1].tk[1 - fin]));
    p.tile_order = at<uint32_t>(ws, L.tile_order[1]);
    p.light_final = at<float>(ws, L.light_final);
    p.light_stop = at<uint32_t>(ws, L.light_stop);
    p.dT = dT;
    p.den = at<float>(ws, L.shadow_den);
    p.T = at<float>(ws, L.T);
    p.lvl_off = at<uint32_t>(ws, L.seg_lvl);
    p.pub_flag = at<uint32_t>(ws, L.seg_flag);
    p.light_geom = light_geom;
    p.W = L.width; p.H = L.height; p.gx = L.gx;
    p.amax = f.opts.alpha_max;
    static DeviceOnce once;
    once.run([] {
      return cudaFuncSetAttribute(k_shadow_bwd, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
    });
    k_shadow_bwd<<<L.ntiles, kBThreads, 0, s>>>(p);
    const size_t items = shadow_seg_items(L.ntiles, L.cap);
    k_shadow_bwd_stopped<<<(int)((items + kStopWarps - 1) / kStopWarps), kStopWarps * 32, 0, ss>>>(p);
    count_launch(2);
  }
  mlp_bwd(1, ss);
  if (side) {
    cudaEventRecord(side->join, ss);
    cudaStreamWaitEvent(s, side->join, 0);
  }
  // K1b
  {
    PrepBwdParams p;
    p.sc = f.sc;
    p.header_view = reinterpret_cast<const float*>(at<uint32_t>(ws, L.header));
    for (int i = 0; i < 9; ++i) p.cam.R[i] = f.cam.R[i];
    for (int i = 0; i < 3; ++i) p.cam.t[i] = f.cam.t[i];
    p.cam.fx = f.cam.fx; p.cam.fy = f.cam.fy; p.cam.lowpass = f.opts.lowpass;
    p.cam.ortho = 0.f;
    p.light = p.cam;  // rotation, translation and scale are read from the header
    p.lh = light_h(f.light);
    p.ablate = f.opts.ablate;
    for (int i = 0; i < 3; ++i) p.cam_pos[i] = f.cam.pos[i];
    p.intensity = f.light.intensity;
    p.falloff = f.opts.falloff;
    p.cam_geom = cam_geom;
    p.light_geom = light_geom;
    p.color = color;
    p.mlp_in = mlp_in;
    p.out = out;
    if (f.sc.lobe_shared && f.sc.k > 0) {  // accumulated with atomics
      cudaMemsetAsync(out.lobe_rot, 0, 16ull * f.sc.k, s);
      cudaMemsetAsync(out.lobe_sigma, 0, 16ull * f.sc.k, s);
    }
    k_prep_bwd<<<(n + 127) / 128, 128, 0, s>>>(p);
    count_launch();
  }
  return GS3_OK;
}

}  // namespace gs3
