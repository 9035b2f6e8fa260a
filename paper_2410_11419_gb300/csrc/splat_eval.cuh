// Shadow-splat evaluation shared by the forward composite (composite.cu) and
// its backward (backward.cu), so both take every alpha decision with the
// same arithmetic: the power at pixel (lx, ly) of a tile is
// fma(dy, fma(c, dy, r dx), (a dx) dx) with dx = lx - ux, dy = ly - vy,
// whatever the thread layout.  Quadrant w of a 16x16 tile is the 8x8 block
// at (8 (w & 1), 8 (w >> 1)).
#pragma once
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

// Bit w set when the splat's alpha >= alpha_min box can reach quadrant w
// (tile-relative centre (ux, vy), half extents hx, hy).
__device__ __forceinline__ uint32_t warp_mask8(float ux, float vy, float hx, float hy) {
  if (!(hx >= 0.f)) return 0u;
  uint32_t m = 0u;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const float x0 = (w & 1) * 8 + 0.5f, y0 = (w >> 1) * 8 + 0.5f;
    const bool hit = (ux + hx >= x0) && (ux - hx <= x0 + 7.f) && (vy + hy >= y0) && (vy - hy <= y0 + 7.f);
    m |= hit ? (1u << w) : 0u;
  }
  return m;
}

// Entries carry the conic pre-multiplied by log2(e), so beta = 2^power2 with
//   power2 = a dx^2 + r dx dy + c dy^2 = dx (a dx) + dy (c dy + r dx),
//   a = -A/2 log2e, r = -B log2e, c = -C/2 log2e, (dx, dy) = pixel - centre.
// e0 = (ux, vy, a, c): centre relative to the tile origin (ox, oy);
// e1 = (r, pthr log2e, gamma, quadrant bits of the alpha box).
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void make_entry(const SplatRec& q, float ox, float oy, float4& e0, float4& e1) {
  const float ux = (q.a.x - ox) + q.b.w, vy = (q.a.y - oy) + q.c.x;
  const uint32_t m = warp_mask8(ux, vy, q.c.y, q.c.z);
  e0 = make_float4(ux, vy, -0.5f * kLog2e * q.b.x, -0.5f * kLog2e * q.b.z);
  e1 = make_float4(-kLog2e * q.b.y, kLog2e * q.c.w, q.a.z, __uint_as_float(m));
}

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

// power2 at the thread's two pixels (lx, ly0), (lx, ly1): the dx terms are shared
__device__ __forceinline__ void powers2(const float4 e0, float r, float lx, float ly0, float ly1, float& p0,
                                        float& p1) {
  const float dx = lx - e0.x;
  const float sx = (e0.z * dx) * dx, v = r * dx;
  const float dy0 = ly0 - e0.y, dy1 = ly1 - e0.y;
  p0 = fmaf(dy0, fmaf(e0.w, dy0, v), sx);
  p1 = fmaf(dy1, fmaf(e0.w, dy1, v), sx);
}

// The same power2 at one pixel (lx, ly) of the tile: the camera composite
// and its backward evaluate an entry with this arithmetic (powers2 is its
// two-pixel form), so both take every alpha decision alike.
__device__ __forceinline__ float power2_at(const float4 e0, float r, float lx, float ly) {
  const float dx = lx - e0.x;
  const float sx = (e0.z * dx) * dx, v = r * dx;
  const float dy = ly - e0.y;
  return fmaf(dy, fmaf(e0.w, dy, v), sx);
}

// A shadow ray stops taking occluders once its product A falls below
// kShadowStop: the occluder that takes A below it is the last one applied,
// and A stays frozen after it.  Every receiver behind the stop would see an
// exact product in [0, kShadowStop) and sees the frozen one, also in
// [0, kShadowStop), so each T_m(j) and every beta-weighted average of them
// moves by less than kShadowStop.  Without the stop, FP32 products underflow
// on deep rays (thousands of passing entries through an object), and the
// backward, which rebuilds A from the ray's final product, would rebuild 0
// for every receiver of such a ray.  A frozen A is at least
// kShadowStop (1 - alpha_max), far from the denormals.
constexpr float kShadowStop = 0x1p-40f;
constexpr uint32_t kNoStop = 0xFFFFFFFFu;  // the ray never stopped

}  // namespace
}  // namespace gs3
