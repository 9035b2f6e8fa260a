// K1: per-Gaussian preparation, fused for both splats.
//
// One thread per spatial Gaussian reads its structure-of-arrays parameters
// (coalesced float4 loads) and writes
//   - the camera splat record and FP32 view-depth key          (Sec. 3, Eq. 1)
//   - the light splat record and FP32 light-distance key       (Sec. 4.2)
//   - the shading colour E (rho_d f_d + rho_s f_s)             (Sec. 4.1, Eq. 2-5)
//
// Keys, rectangles and culling follow the fixed FP32 recipe (explicit
// round-to-nearest intrinsics, no contraction into FMA, correctly rounded
// division and square root) so that the tile lists are reproducible bit for
// bit by any IEEE implementation of the same recipe.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

#define M_(a, b) __fmul_rn((a), (b))
#define A_(a, b) __fadd_rn((a), (b))
#define S_(a, b) __fsub_rn((a), (b))
#define D_(a, b) __fdiv_rn((a), (b))
#define Q_(a) __fsqrt_rn(a)

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return A_(A_(M_(a0, b0), M_(a1, b1)), M_(a2, b2));
}

// Light camera: at the light, looking at the target, +z up (+y if parallel).
__device__ void light_view_rn(const float pL[3], const float tg[3], float R[9], float t[3]) {
  float fx = S_(tg[0], pL[0]), fy = S_(tg[1], pL[1]), fz = S_(tg[2], pL[2]);
  float n = Q_(dot3_rn(fx, fy, fz, fx, fy, fz));
  fx = D_(fx, n); fy = D_(fy, n); fz = D_(fz, n);
  float ux = 0.f, uy = 0.f, uz = 1.f;
  if (fabsf(fz) > 0.999f) { uy = 1.f; uz = 0.f; }
  float rx = S_(M_(fy, uz), M_(fz, uy));
  float ry = S_(M_(fz, ux), M_(fx, uz));
  float rz = S_(M_(fx, uy), M_(fy, ux));
  float rn = Q_(dot3_rn(rx, ry, rz, rx, ry, rz));
  rx = D_(rx, rn); ry = D_(ry, rn); rz = D_(rz, rn);
  float dx = S_(M_(fy, rz), M_(fz, ry));
  float dy = S_(M_(fz, rx), M_(fx, rz));
  float dz = S_(M_(fx, ry), M_(fy, rx));
  R[0] = rx; R[1] = ry; R[2] = rz;
  R[3] = dx; R[4] = dy; R[5] = dz;
  R[6] = fx; R[7] = fy; R[8] = fz;
  for (int i = 0; i < 3; ++i) t[i] = -dot3_rn(R[3 * i], R[3 * i + 1], R[3 * i + 2], pL[0], pL[1], pL[2]);
}

// Light view of either kind (Sec. 4.2 point, Sec. 4.5 directional): a
// directional light looks along -dir from the eye target + dir (4 extent)
// with pixel scale s = (min(W, H) / 2) / extent; returns s (0 for a point).
__device__ float light_view_any_rn(const gs3_light& L, const float tg[3], int W, int H, float R[9], float t[3]) {
  if (L.type != GS3_LIGHT_DIRECTIONAL) {
    light_view_rn(L.pos, tg, R, t);
    return 0.f;
  }
  const float reach = M_(4.f, L.extent);
  const float e[3] = {A_(tg[0], M_(L.dir[0], reach)), A_(tg[1], M_(L.dir[1], reach)), A_(tg[2], M_(L.dir[2], reach))};
  light_view_rn(e, tg, R, t);
  return D_(M_(0.5f, (float)(W < H ? W : H)), L.extent);
}

struct View {
  float R[9], t[3];
  float fx, fy, cx, cy;
  int W, H;
  float ortho;  // > 0: orthographic with this many pixels per world unit
};

__device__ void accurate_geometry(const float4 m, const float Rq[9], const float sv[3], const View& v,
                                  float lowpass, float gamma, float amin, SplatRec& rec);

// FP32 recipe: returns false when culled; fills the record otherwise.
__device__ bool project_rn(const float4 m, const float4 s, const float4 q, const View& v,
                           const gs3_render_opts& o, int gx, int gy, const float* pL, float gamma,
                           float nl_amin, SplatRec& rec) {
  const float* R = v.R;
  float tx = A_(dot3_rn(R[0], R[1], R[2], m.x, m.y, m.z), v.t[0]);
  float ty = A_(dot3_rn(R[3], R[4], R[5], m.x, m.y, m.z), v.t[1]);
  float tz = A_(dot3_rn(R[6], R[7], R[8], m.x, m.y, m.z), v.t[2]);
  if (!(tz > o.near_z)) return false;
  const bool ortho = v.ortho > 0.f;
  float xz = 0.f, yz = 0.f, u, vv;
  if (ortho) {  // u = s x + cx, v = s y + cy
    const float limx = M_(o.frustum, D_(M_(0.5f, (float)v.W), v.ortho));
    const float limy = M_(o.frustum, D_(M_(0.5f, (float)v.H), v.ortho));
    if (tx < -limx || tx > limx || ty < -limy || ty > limy) return false;
    u = A_(M_(v.ortho, tx), v.cx);
    vv = A_(M_(v.ortho, ty), v.cy);
  } else {
    xz = D_(tx, tz);
    yz = D_(ty, tz);
    const float limx = M_(o.frustum, D_(M_(0.5f, (float)v.W), v.fx));
    const float limy = M_(o.frustum, D_(M_(0.5f, (float)v.H), v.fy));
    if (xz < -limx || xz > limx || yz < -limy || yz > limy) return false;
    u = A_(M_(v.fx, xz), v.cx);
    vv = A_(M_(v.fy, yz), v.cy);
  }

  float n2 = A_(A_(A_(M_(q.x, q.x), M_(q.y, q.y)), M_(q.z, q.z)), M_(q.w, q.w));
  if (!(n2 > 0.f)) return false;
  float qn = Q_(n2);
  float w = D_(q.x, qn), x = D_(q.y, qn), y = D_(q.z, qn), z = D_(q.w, qn);
  float Rq[9];
  Rq[0] = S_(1.f, M_(2.f, A_(M_(y, y), M_(z, z))));
  Rq[1] = M_(2.f, S_(M_(x, y), M_(w, z)));
  Rq[2] = M_(2.f, A_(M_(x, z), M_(w, y)));
  Rq[3] = M_(2.f, A_(M_(x, y), M_(w, z)));
  Rq[4] = S_(1.f, M_(2.f, A_(M_(x, x), M_(z, z))));
  Rq[5] = M_(2.f, S_(M_(y, z), M_(w, x)));
  Rq[6] = M_(2.f, S_(M_(x, z), M_(w, y)));
  Rq[7] = M_(2.f, A_(M_(y, z), M_(w, x)));
  Rq[8] = S_(1.f, M_(2.f, A_(M_(x, x), M_(y, y))));
  const float sv[3] = {s.x, s.y, s.z};
  float Mm[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Mm[3 * i + j] = M_(Rq[3 * i + j], sv[j]);
  float Sg[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Sg[3 * i + j] = dot3_rn(Mm[3 * i], Mm[3 * i + 1], Mm[3 * i + 2], Mm[3 * j], Mm[3 * j + 1], Mm[3 * j + 2]);
  float T0[3], T1[3];
  if (ortho) {  // J = [[s, 0, 0], [0, s, 0]]
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = M_(v.ortho, R[k]);
      T1[k] = M_(v.ortho, R[3 + k]);
    }
  } else {
    float j00 = D_(v.fx, tz), j02 = -D_(M_(v.fx, xz), tz);
    float j11 = D_(v.fy, tz), j12 = -D_(M_(v.fy, yz), tz);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = A_(M_(j00, R[k]), M_(j02, R[6 + k]));
      T1[k] = A_(M_(j11, R[3 + k]), M_(j12, R[6 + k]));
    }
  }
  float U0[3], U1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U0[k] = dot3_rn(T0[0], T0[1], T0[2], Sg[k], Sg[3 + k], Sg[6 + k]);
    U1[k] = dot3_rn(T1[0], T1[1], T1[2], Sg[k], Sg[3 + k], Sg[6 + k]);
  }
  float a = A_(dot3_rn(U0[0], U0[1], U0[2], T0[0], T0[1], T0[2]), o.lowpass);
  float b = dot3_rn(U0[0], U0[1], U0[2], T1[0], T1[1], T1[2]);
  float c = A_(dot3_rn(U1[0], U1[1], U1[2], T1[0], T1[1], T1[2]), o.lowpass);
  float det = S_(M_(a, c), M_(b, b));
  if (!(det > 0.f)) return false;
  float mid = M_(0.5f, A_(a, c));
  float disc = S_(M_(mid, mid), det);
  float lam = A_(mid, Q_(fmaxf(0.1f, disc)));
  float r = ceilf(M_(3.f, Q_(lam)));
  const float ts = (float)kTile;
  float fx0 = floorf(D_(S_(u, r), ts)), fx1 = floorf(D_(A_(u, r), ts));
  float fy0 = floorf(D_(S_(vv, r), ts)), fy1 = floorf(D_(A_(vv, r), ts));
  // Cut the square to the box holding every pixel with alpha >= alpha_min:
  // ln(gamma) <= min(0, logit), so r2 = 2 (min(0, logit) - ln alpha_min) bounds
  // 2 ln(gamma / alpha_min) without a transcendental of per-Gaussian data.
  const float r2 = M_(2.f, A_(fminf(0.f, m.w), nl_amin));
  if (!(r2 > 0.f)) return false;  // gamma < alpha_min: no pixel passes
  const float hx = Q_(M_(r2, a)), hy = Q_(M_(r2, c));
  fx0 = fmaxf(fx0, floorf(D_(S_(u, hx), ts)));
  fx1 = fminf(fx1, floorf(D_(A_(u, hx), ts)));
  fy0 = fmaxf(fy0, floorf(D_(S_(vv, hy), ts)));
  fy1 = fminf(fy1, floorf(D_(A_(vv, hy), ts)));
  if (fx1 < 0.f || fx0 > (float)(gx - 1) || fy1 < 0.f || fy0 > (float)(gy - 1)) return false;
  rec.r = make_int4((int)fmaxf(fx0, 0.f), (int)fmaxf(fy0, 0.f), (int)fminf(fx1, (float)(gx - 1)),
                    (int)fminf(fy1, (float)(gy - 1)));
  float depth;
  if (pL && !ortho) {
    float dx = S_(m.x, pL[0]), dy = S_(m.y, pL[1]), dz = S_(m.z, pL[2]);
    depth = Q_(dot3_rn(dx, dy, dz, dx, dy, dz));
  } else {
    depth = tz;
  }
  accurate_geometry(m, Rq, sv, v, o.lowpass, gamma, o.alpha_min, rec);
  rec.a.w = depth;
  return true;
}

// Compositing geometry (not key-relevant), accurate to a few FP32 ulps:
//  - screen position in FP64, stored as a (hi, lo) float pair so that the
//    pixel offset dx = (x - u_hi) - u_lo keeps its precision at 1000-pixel
//    coordinates;
//  - 2-D covariance as P P^T + lowpass I with P = J W R S (2x3), its
//    determinant by the Lagrange identity |P0|^2 |P1|^2 - (P0.P1)^2 =
//    |P0 x P1|^2 (minors with an FMA-compensated difference), so elongated
//    splats do not lose the determinant to cancellation.
__device__ __forceinline__ float minor_fma(float a, float b, float c, float d) {  // a d - b c
  const float w = b * c;
  const float e = fmaf(-b, c, w);
  const float f = fmaf(a, d, -w);
  return f + e;
}

__device__ void accurate_geometry(const float4 m, const float Rq[9], const float sv[3], const View& v,
                                  float lowpass, float gamma, float amin, SplatRec& rec) {
  const float* R = v.R;
  const double tx = (double)R[0] * m.x + (double)R[1] * m.y + (double)R[2] * m.z + (double)v.t[0];
  const double ty = (double)R[3] * m.x + (double)R[4] * m.y + (double)R[5] * m.z + (double)v.t[1];
  const double tz = (double)R[6] * m.x + (double)R[7] * m.y + (double)R[8] * m.z + (double)v.t[2];
  const bool ortho = v.ortho > 0.f;
  const double itz = 1.0 / tz;
  const double u = ortho ? (double)v.ortho * tx + (double)v.cx : (double)v.fx * (tx * itz) + (double)v.cx;
  const double vv = ortho ? (double)v.ortho * ty + (double)v.cy : (double)v.fy * (ty * itz) + (double)v.cy;
  const float uh = (float)u, vh = (float)vv;
  const float ul = (float)(u - (double)uh), vl = (float)(vv - (double)vh);
  float T0[3], T1[3];
  if (ortho) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = v.ortho * R[k];
      T1[k] = v.ortho * R[3 + k];
    }
  } else {
    const float fz = (float)tz, xz = (float)(tx * itz), yz = (float)(ty * itz);
    const float j00 = v.fx / fz, j02 = -v.fx * xz / fz;
    const float j11 = v.fy / fz, j12 = -v.fy * yz / fz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = fmaf(j00, R[k], j02 * R[6 + k]);
      T1[k] = fmaf(j11, R[3 + k], j12 * R[6 + k]);
    }
  }
  float P0[3], P1[3];  // P = T (R_q S)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float c0 = Rq[j] * sv[j], c1 = Rq[3 + j] * sv[j], c2 = Rq[6 + j] * sv[j];
    P0[j] = fmaf(T0[0], c0, fmaf(T0[1], c1, T0[2] * c2));
    P1[j] = fmaf(T1[0], c0, fmaf(T1[1], c1, T1[2] * c2));
  }
  const float a0 = fmaf(P0[0], P0[0], fmaf(P0[1], P0[1], P0[2] * P0[2]));
  const float c0 = fmaf(P1[0], P1[0], fmaf(P1[1], P1[1], P1[2] * P1[2]));
  const float b = fmaf(P0[0], P1[0], fmaf(P0[1], P1[1], P0[2] * P1[2]));
  const float m0 = minor_fma(P0[1], P0[2], P1[1], P1[2]);
  const float m1 = minor_fma(P0[2], P0[0], P1[2], P1[0]);
  const float m2 = minor_fma(P0[0], P0[1], P1[0], P1[1]);
  const float det = fmaf(m0, m0, fmaf(m1, m1, m2 * m2)) + lowpass * (a0 + c0) + lowpass * lowpass;
  const float a = a0 + lowpass, c = c0 + lowpass;
  rec.a = make_float4(uh, vh, gamma, 0.f);
  rec.b = make_float4(c / det, -b / det, a / det, ul);
  // alpha >= amin  <=>  power >= ln(amin / gamma)  <=>  d^T conic d <= r2 = 2 ln(gamma / amin);
  // that ellipse lies inside |dx| <= sqrt(r2 a), |dy| <= sqrt(r2 c) (Sigma_2D = [[a, b], [b, c]]).
  // The box is widened by 0.1 % + 0.01 px so rounding never drops a passing pixel.
  const float pthr = logf(amin / gamma);
  const float r2 = -2.f * pthr;
  float hx = -1.f, hy = -1.f;
  if (r2 > 0.f) {
    hx = sqrtf(r2 * a) * 1.001f + 0.01f;
    hy = sqrtf(r2 * c) * 1.001f + 0.01f;
  }
  rec.c = make_float4(vl, hx, hy, pthr);
}

__device__ __forceinline__ void quat_mat(float4 q, float Rm[9]) {
  float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  float w = q.x * n, x = q.y * n, y = q.z * n, z = q.w * n;
  Rm[0] = 1.f - 2.f * (y * y + z * z); Rm[1] = 2.f * (x * y - w * z);       Rm[2] = 2.f * (x * z + w * y);
  Rm[3] = 2.f * (x * y + w * z);       Rm[4] = 1.f - 2.f * (x * x + z * z); Rm[5] = 2.f * (y * z - w * x);
  Rm[6] = 2.f * (x * z - w * y);       Rm[7] = 2.f * (y * z + w * x);       Rm[8] = 1.f - 2.f * (x * x + y * y);
}

// Eq. 3 (ELU alpha = 0.01, eps = 0.01)
__device__ __forceinline__ float diffuse(float x) {
  const float off = 0.01f * (1.f - 0.36787944117144233f);
  float elu = x > 0.f ? x : 0.01f * expm1f(x);
  return (elu + off) / ((1.f + off) * 3.14159265358979323846f);
}

// Eq. 5 in the theta/sin(theta) form: theta^2 q^2 = (theta/|hxy|)^2 ((hx/sx)^2 + (hy/sy)^2)
__device__ __forceinline__ float angular_gaussian(float hx, float hy, float hz, float4 sig) {
  float sxy = sqrtf(hx * hx + hy * hy);
  float theta = atan2f(sxy, hz);
  float e2;
  if (sxy > 1e-30f) {
    float ratio = theta / sxy;
    float px = hx / sig.x, py = hy / sig.y;
    e2 = ratio * ratio * (px * px + py * py);
  } else {
    e2 = hz < 0.f ? (3.14159265358979323846f / sig.x) * (3.14159265358979323846f / sig.x) : 0.f;
  }
  float iz = 1.f / sig.z;
  return __expf(-0.5f * e2 * iz * iz) * iz;
}

struct PrepParams {
  SceneDev sc;
  View cam;
  gs3_light light;
  float4 lh;  // homogeneous light (light_h)
  float nl_amin;  // -ln(alpha_min) as FP32, from double precision on the host
  float cam_pos[3];
  float intensity;
  gs3_render_opts o;
  int gx, gy;
  int sp0;  // first splat projected: 0 camera and light, 1 light only
  uint32_t* key[2];
  SplatRec* rec[2];
  int4* rect[2];
  float4* shade;
  uint32_t* header;
};

__global__ void __launch_bounds__(256) k_prep(PrepParams p) {
  __shared__ float sR[9], st[3], sortho;
  if (threadIdx.x == 0) {
    sortho = light_view_any_rn(p.light, p.o.target, p.cam.W, p.cam.H, sR, st);
    if (blockIdx.x == 0) {
      float* hv = reinterpret_cast<float*>(p.header + H_LIGHT_VIEW);
      for (int i = 0; i < 9; ++i) hv[i] = sR[i];
      for (int i = 0; i < 3; ++i) hv[9 + i] = st[i];
      reinterpret_cast<float*>(p.header)[H_LIGHT_ORTHO] = sortho;
    }
  }
  __syncthreads();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.sc.n) return;
  const int n = p.sc.n;
  const float4 m = p.sc.mean_op[g];
  const float4 s = p.sc.scale[g];
  const float4 q = p.sc.rot[g];
  const float gamma = 1.f / (1.f + expf(-m.w));

  View lv = p.cam;
#pragma unroll
  for (int i = 0; i < 9; ++i) lv.R[i] = sR[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) lv.t[i] = st[i];
  lv.ortho = sortho;

#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    if (sp < p.sp0) continue;
    SplatRec rec;
    bool vis = project_rn(m, s, q, sp ? lv : p.cam, p.o, p.gx, p.gy, sp ? p.light.pos : nullptr, gamma,
                          p.nl_amin, rec);
    if (!vis) {
      rec.a = make_float4(0.f, 0.f, 0.f, 0.f);
      rec.b = make_float4(0.f, 0.f, 0.f, 0.f);
      rec.c = make_float4(0.f, 0.f, 0.f, 0.f);
      rec.r = make_int4(-1, -1, -2, -2);
    }
    rec.a.z = gamma;
    p.key[sp][g] = vis ? __float_as_uint(rec.a.w) : 0xFFFFFFFFu;
    p.rec[sp][g] = rec;
    p.rect[sp][g] = rec.r;
  }

  // ---- shading colour (Sec. 4.1); omega_i = normalize(L.xyz - L.w mu) ----
  float lx = p.lh.x - p.lh.w * m.x, ly = p.lh.y - p.lh.w * m.y, lz = p.lh.z - p.lh.w * m.z;
  float d2 = lx * lx + ly * ly + lz * lz;
  float il = rsqrtf(d2);
  float wi[3] = {lx * il, ly * il, lz * il};
  float vx = p.cam_pos[0] - m.x, vy = p.cam_pos[1] - m.y, vz = p.cam_pos[2] - m.z;
  float iv = rsqrtf(vx * vx + vy * vy + vz * vz);
  float wo[3] = {vx * iv, vy * iv, vz * iv};
  float Rs[9];
  quat_mat(p.sc.shade_rot[g], Rs);
  float wil[3], wol[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    wil[i] = Rs[3 * i] * wi[0] + Rs[3 * i + 1] * wi[1] + Rs[3 * i + 2] * wi[2];
    wol[i] = Rs[3 * i] * wo[0] + Rs[3 * i + 1] * wo[1] + Rs[3 * i + 2] * wo[2];
  }
  const float fd = diffuse(wil[2]);
  float fs[3] = {0.f, 0.f, 0.f};
  float hx = wil[0] + wol[0], hy = wil[1] + wol[1], hz = wil[2] + wol[2];
  float hn2 = hx * hx + hy * hy + hz * hz;
  if (hn2 >= 1e-24f && !(p.o.ablate & GS3_ABLATE_SPECULAR)) {
    float ih = rsqrtf(hn2);
    hx *= ih; hy *= ih; hz *= ih;
    for (int j = 0; j < p.sc.k; ++j) {
      const size_t li = (size_t)j * n + g;
      const size_t ls = p.sc.lobe_shared ? (size_t)j : li;  // frame and deviations of lobe j
      float Rl[9];
      quat_mat(p.sc.lobe_rot[ls], Rl);
      // components of h' in the lobe frame: columns of Rl are the lobe axes
      float ax = Rl[0] * hx + Rl[3] * hy + Rl[6] * hz;
      float ay = Rl[1] * hx + Rl[4] * hy + Rl[7] * hz;
      float az = Rl[2] * hx + Rl[5] * hy + Rl[8] * hz;
      float G = angular_gaussian(ax, ay, az, p.sc.lobe_sigma[ls]);
      float4 amp = p.sc.lobe_amp[li];
      fs[0] += amp.x * G; fs[1] += amp.y * G; fs[2] += amp.z * G;
    }
  }
  // a directional light's irradiance does not fall off (Sec. 4.5)
  const float E = (p.o.falloff && p.lh.w != 0.f) ? p.intensity / d2 : p.intensity;
  const float4 rd = p.sc.albedo_d[g], rs = p.sc.albedo_s[g];
  p.shade[g] = make_float4(E * (rd.x * fd + rs.x * fs[0]), E * (rd.y * fd + rs.y * fs[1]),
                           E * (rd.z * fd + rs.z * fs[2]), 0.f);
}

}  // namespace

void launch_prep(const FrameArgs& f, cudaStream_t s, bool light_only) {
  PrepParams p;
  p.sp0 = light_only ? 1 : 0;
  p.sc = f.sc;
  for (int i = 0; i < 9; ++i) p.cam.R[i] = f.cam.R[i];
  for (int i = 0; i < 3; ++i) { p.cam.t[i] = f.cam.t[i]; p.cam_pos[i] = f.cam.pos[i]; }
  p.cam.ortho = 0.f;
  p.light = f.light;
  p.lh = light_h(f.light);
  p.nl_amin = (float)(-log((double)f.opts.alpha_min));
  p.cam.fx = f.cam.fx; p.cam.fy = f.cam.fy; p.cam.cx = f.cam.cx; p.cam.cy = f.cam.cy;
  p.cam.W = f.cam.width; p.cam.H = f.cam.height;
  p.intensity = f.light.intensity;
  p.o = f.opts;
  p.gx = f.L->gx; p.gy = f.L->gy;
  for (int sp = 0; sp < 2; ++sp) {
    p.key[sp] = at<uint32_t>(f.ws, f.L->sp[sp].key);
    p.rec[sp] = at<SplatRec>(f.ws, f.L->sp[sp].rec);
    p.rect[sp] = at<int4>(f.ws, f.L->sp[sp].rect);
  }
  p.shade = at<float4>(f.ws, f.L->shade);
  p.header = at<uint32_t>(f.ws, f.L->header);
  const int n = f.sc.n;
  k_prep<<<(n + 255) / 256, 256, 0, s>>>(p);
  count_launch();
}

}  // namespace gs3
