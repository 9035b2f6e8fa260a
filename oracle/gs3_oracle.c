/*
 * gs3_oracle.c -- plain FP64 CPU restatement of the GS^3 per-frame render
 * (Bi et al., "GS^3: Efficient Relighting with Triple Gaussian Splatting").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA library is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or constant generator with
 * the CUDA path; the two meet only in the seeded inputs.
 *
 * What it computes, step by step, in the paper's order:
 *   O1  spatial Gaussian parameters: Sigma = R S S^T R^T, opacity      (Eq. 1)
 *   O2  light / view directions, local frame via the shading quaternion (Sec. 4.1)
 *   O3  modified Lambertian f_d                                         (Eq. 3)
 *   O4  angular Gaussian lobes f_s = sum_j alpha_j G_ang,j(h')          (Eq. 4, Eq. 5)
 *   O5  shading colour  E * (rho_d f_d + rho_s f_s)                     (Eq. 2)
 *   O6  EWA projection to the camera and to the light camera            (Sec. 3)
 *   O7  tile footprints and (tile, depth) keys                          (Sec. 3, Sec. 4.2)
 *   O8  per-tile order: ascending (depth bits, Gaussian index)
 *   O10 shadow splatting: biased cumulative opacity per light-pixel,
 *       beta-weighted average per Gaussian                               (Sec. 4.2, Fig. 3)
 *   O11 shadow refinement MLP Phi with 4-band positional encoding       (Sec. 4.2)
 *   O12 residual MLP Psi                                                 (Sec. 4.3)
 *   O9  camera alpha compositing of shading / shadow / residual and the
 *       per-pixel combination  shading * shadow + residual              (Eq. 2, Sec. 4)
 *
 * Readings where the paper is silent (listed in the design notes):
 *   - keys, rectangles and culling follow a fixed FP32 recipe (IEEE
 *     round-to-nearest, no contraction: build with -ffp-contract=off,
 *     correctly rounded sqrt and division, no transcendental), so that the
 *     tile lists can be compared bit for bit; everything else is FP64;
 *   - EWA follows the base splatting method's conventions: +0.3 px^2
 *     low-pass, radius ceil(3 sqrt(lambda_max)), 16x16 tiles, near plane 0.2,
 *     frustum cull at 1.3x the half-tangent;
 *   - alpha = min(0.99, gamma*beta), skipped below 1/255, camera rays stop
 *     before T would fall below 1e-4; shadow rays never stop early;
 *   - shadow bias: occluder k shadows receiver j on a ray only if
 *     d_k < d_j - 0.015 (FP32 subtraction and comparison of the FP32 light
 *     distances); a Gaussian with no shadow-ray intersection gets T = 1;
 *   - n' = e_z of the shading frame; lobe frames live in the shading frame;
 *   - point-light irradiance E = I / |p_L - mu|^2 (switchable);
 *   - positional encoding [v, sin(2^k pi v), cos(2^k pi v)], k = 0..3;
 *   - the light camera looks at the scene centre with the scene camera's
 *     intrinsics and resolution.
 *
 * Decision-ambiguous cases: an FP32 implementation may take the other side of
 * a threshold test whose FP64 operand lies within a relative margin of its
 * cutoff.  The oracle records every such case and turns it into an explicit
 * bound on the change of each affected output; the parity tests add that
 * bound to their tolerance.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <time.h>

#define GO_PI 3.14159265358979323846

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by oracle.py through ctypes).                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int in_dim, width, n_hidden, out_dim, act; /* act: 0 relu, 1 leaky relu 0.01 */
    const float *w;                            /* layer weights (out,in) row-major, concatenated */
    const float *b;                            /* biases, concatenated */
} go_mlp;

/* lobe_shared = 0: every spatial Gaussian has its own K lobes (lobe-major
 * [j n + g] arrays).  lobe_shared = 1: a basis of K angular Gaussians (frame,
 * sigma) shared by all spatial Gaussians, lobe_rot / lobe_sigma hold K
 * entries, and each spatial Gaussian keeps its weights lobe_amp[j n + g]
 * (the shared basis of Sec. 4.1). */
typedef struct {
    int n, k;
    const float *mean_op, *scale, *rot, *shade_rot, *albedo_d, *albedo_s, *latent;
    const float *lobe_rot, *lobe_sigma, *lobe_amp;
    go_mlp phi, psi;
    int lobe_shared;
} go_scene;

typedef struct {
    float R[9], t[3], pos[3];
    float fx, fy, cx, cy;
    int width, height;
} go_camera;

/* type 0: point light at pos (Sec. 4.2); type 1: directional light from the
 * scene towards dir (Sec. 4.5), orthographic light view of half-width
 * extent (world units) centred at the options' target. */
typedef struct {
    float pos[3];
    float intensity;
    int type;
    float dir[3];
    float extent;
} go_light;

typedef struct {
    float near_z, lowpass, frustum, shadow_bias, alpha_min, alpha_max, t_stop;
    float target[3];
    int falloff, tile, ablate; /* ablate bits: 1 no shadow splat, 2 no Phi, 4 no Psi,
                                  8 Lambertian only (no lobes: the first training stage, Sec. 4.4) */
    int threads;
    double margin_alpha, margin_tstop;
    int crop[4]; /* x0, y0, x1, y1 (exclusive) pixel window of both composites; all 0 = full */
    /* Testing the bounds of decision-ambiguous cases.  A decision is named by
     * the code (kind << 60) | (pixel << 32) | list position, with kind 0 the
     * alpha test of a shadow-ray entry, 1 the alpha test of a camera-ray
     * entry, 2 the camera ray's stop test after an entry; pixel = y W + x and
     * the position is the entry's index in that splat's sorted list.
     *   flip:       nflip codes, ascending: these ambiguous decisions are taken
     *               on their other side (as an FP32 evaluation may take them)
     *   record_amb: 1 = list every ambiguous decision in the frame's amb */
    const int64_t *flip;
    int nflip;
    int record_amb;
} go_opts;

enum { AMB_SHADOW_ALPHA = 0, AMB_CAMERA_ALPHA = 1, AMB_CAMERA_STOP = 2 };

static int64_t amb_code(int kind, size_t pixel, size_t pos)
{
    return ((int64_t)kind << 60) | ((int64_t)pixel << 32) | (int64_t)pos;
}

/* true when the options ask for decision `code` to be flipped */
static int flipped(const go_opts *o, int64_t code)
{
    int lo = 0, hi = o->nflip;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (o->flip[mid] < code) lo = mid + 1; else hi = mid;
    }
    return lo < o->nflip && o->flip[lo] == code;
}

typedef struct {
    int n, width, height, gx, gy, ntiles;
    float light_R[9], light_t[3];
    float light_ortho; /* orthographic light view: pixels per world unit (0: perspective) */
    /* per splat s = 0 camera, 1 light */
    uint32_t *key[2];      /* FP32 depth (camera) / distance (light) bits, 0xFFFFFFFF if culled */
    int32_t *rect[2];      /* x0, y0, x1, y1 tile rectangle (inclusive); x0 = -1 if culled */
    float *uv_f32[2];      /* FP32 recipe screen position */
    double *uv[2];         /* FP64 screen position */
    double *conic[2];      /* FP64 inverse 2-D covariance (A, B, C) */
    double *opacity;       /* gamma */
    uint32_t P[2];
    uint32_t *tile_start[2]; /* ntiles + 1 */
    uint32_t *list[2];       /* Gaussian index per entry */
    double *shade;         /* N x 3 */
    double *T;             /* shadow value before refinement */
    double *T_bound;       /* bound on |dT| from ambiguous decisions */
    double *Tp;            /* refined shadow value T' */
    double *Tp_bound;
    double *res;           /* N x 3 residual */
    double *img;           /* H x W x 3 */
    double *img_bound;     /* H x W x 3, absolute bound from ambiguous decisions */
    double *final_T;       /* H x W */
    int32_t *n_contrib;    /* H x W: entries consumed before the ray stopped */
    double *S, *Sh, *Rimg; /* composited shading (3), shadow (1), residual (3) images */
    int64_t shadow_evals, shadow_pass, camera_evals;
    int64_t amb_shadow, amb_camera;
    int64_t camera_pass; /* (pixel, Gaussian) pairs composited by the camera rays */
    double t_prep, t_bin, t_shadow, t_mlp, t_camera; /* wall seconds per stage */
    int64_t *amb;  /* with record_amb: the codes of every ambiguous decision (unordered) */
    int64_t namb, amb_cap;
    /* between the stages of go_begin / go_shadow_rows / go_finish */
    double *sacc;       /* N x 4: shadow-ray sums num, den, bnum, bden over the rows done so far */
    double *wi, *wo;    /* N x 3: unit directions to the light and to the camera (O2) */
} go_frame;

/* appends an ambiguous decision to the frame's record (any thread) */
static void record_amb(go_frame *f, const go_opts *o, int64_t code)
{
    if (!o->record_amb) return;
#ifdef _OPENMP
#pragma omp critical(go_amb_record)
#endif
    {
        if (f->namb == f->amb_cap) {
            f->amb_cap = f->amb_cap ? 2 * f->amb_cap : 1024;
            f->amb = realloc(f->amb, sizeof(int64_t) * (size_t)f->amb_cap);
        }
        f->amb[f->namb++] = code;
    }
}

/* pixel window of the composites (the whole image unless a crop is set) */
static void window(const go_opts *o, int W, int H, int *x0, int *y0, int *x1, int *y1)
{
    *x0 = 0; *y0 = 0; *x1 = W; *y1 = H;
    if (o->crop[2] > o->crop[0] && o->crop[3] > o->crop[1]) {
        *x0 = o->crop[0] < 0 ? 0 : o->crop[0];
        *y0 = o->crop[1] < 0 ? 0 : o->crop[1];
        *x1 = o->crop[2] > W ? W : o->crop[2];
        *y1 = o->crop[3] > H ? H : o->crop[3];
    }
}

/* ------------------------------------------------------------------------ */
/* FP32 key recipe.  Every operation below is one IEEE binary32 operation;   */
/* the file is compiled with -ffp-contract=off so no multiply-add is fused.  */
/* ------------------------------------------------------------------------ */
typedef struct { float x, y, z; } f3;

static f3 f3_normalize(f3 v)
{
    float n2 = v.x * v.x + v.y * v.y + v.z * v.z; /* ((xx + yy) + zz) */
    float n = sqrtf(n2);
    f3 r = {v.x / n, v.y / n, v.z / n};
    return r;
}

static f3 f3_cross(f3 a, f3 b)
{
    f3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}

/* Light camera (reading of Sec. 4.2): centred at the light, looking at the scene
 * centre, world +z up unless nearly parallel (+y then). Rows of R: right, down, forward. */
void go_light_view(const float pL[3], const float target[3], float R[9], float t[3])
{
    f3 e = {pL[0], pL[1], pL[2]};
    f3 f = f3_normalize((f3){target[0] - e.x, target[1] - e.y, target[2] - e.z});
    f3 up = (fabsf(f.z) > 0.999f) ? (f3){0.0f, 1.0f, 0.0f} : (f3){0.0f, 0.0f, 1.0f};
    f3 r = f3_normalize(f3_cross(f, up));
    f3 d = f3_cross(f, r);
    R[0] = r.x; R[1] = r.y; R[2] = r.z;
    R[3] = d.x; R[4] = d.y; R[5] = d.z;
    R[6] = f.x; R[7] = f.y; R[8] = f.z;
    for (int i = 0; i < 3; ++i)
        t[i] = -(R[3 * i] * e.x + R[3 * i + 1] * e.y + R[3 * i + 2] * e.z);
}

/* Light view of either kind.  Directional (Sec. 4.5): the perspective
 * shadow camera is replaced by an orthographic one looking along -dir at the
 * target from the eye e = target + dir (4 extent), with pixel scale
 * s = (min(W, H) / 2) / extent (so the view's half-width is extent) and the
 * depth along the view axis as the sorting distance.  FP32, one rounding per
 * operation.  Returns s (0 for a point light). */
float go_light_view_any(const go_light *L, const float target[3], int W, int H, float R[9], float t[3])
{
    if (L->type != 1) {
        go_light_view(L->pos, target, R, t);
        return 0.0f;
    }
    float reach = 4.0f * L->extent;
    float e[3] = {target[0] + L->dir[0] * reach, target[1] + L->dir[1] * reach, target[2] + L->dir[2] * reach};
    go_light_view(e, target, R, t);
    float half = 0.5f * (float)(W < H ? W : H);
    return half / L->extent;
}

typedef struct { uint32_t key; int x0, y0, x1, y1; float u, v; } keyrec;

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* One Gaussian through the FP32 recipe.  Returns 0 when culled. */
/* -ln(alpha_min) as FP32, the one transcendental of the rectangle rule,
 * taken once per frame from the FP32 option in double precision */
static float neg_log_amin(const go_opts *o) { return (float)(-log((double)o->alpha_min)); }

static int key_recipe(const float m[4], const float s[3], const float q[4],
                      const float R[9], const float t[3], float fx, float fy, float cx, float cy,
                      int W, int H, const go_opts *o, const float *pL, float ortho, keyrec *out)
{
    const float nl_amin = neg_log_amin(o);
    out->key = 0xFFFFFFFFu; out->x0 = -1; out->y0 = -1; out->x1 = -2; out->y1 = -2;
    out->u = 0.0f; out->v = 0.0f;
    float tx = R[0] * m[0] + R[1] * m[1] + R[2] * m[2] + t[0];
    float ty = R[3] * m[0] + R[4] * m[1] + R[5] * m[2] + t[1];
    float tz = R[6] * m[0] + R[7] * m[1] + R[8] * m[2] + t[2];
    if (!(tz > o->near_z)) return 0;
    float xz = 0.0f, yz = 0.0f, u, v;
    if (ortho > 0.0f) { /* orthographic: u = s x + cx, v = s y + cy */
        float limx = o->frustum * ((0.5f * (float)W) / ortho);
        float limy = o->frustum * ((0.5f * (float)H) / ortho);
        if (tx < -limx || tx > limx || ty < -limy || ty > limy) return 0;
        u = ortho * tx + cx;
        v = ortho * ty + cy;
    } else {
        xz = tx / tz;
        yz = ty / tz;
        float limx = o->frustum * ((0.5f * (float)W) / fx);
        float limy = o->frustum * ((0.5f * (float)H) / fy);
        if (xz < -limx || xz > limx || yz < -limy || yz > limy) return 0;
        u = fx * xz + cx;
        v = fy * yz + cy;
    }

    float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > 0.0f)) return 0;
    float qn = sqrtf(n2);
    float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (y * y + z * z);
    Rq[1] = 2.0f * (x * y - w * z);
    Rq[2] = 2.0f * (x * z + w * y);
    Rq[3] = 2.0f * (x * y + w * z);
    Rq[4] = 1.0f - 2.0f * (x * x + z * z);
    Rq[5] = 2.0f * (y * z - w * x);
    Rq[6] = 2.0f * (x * z - w * y);
    Rq[7] = 2.0f * (y * z + w * x);
    Rq[8] = 1.0f - 2.0f * (x * x + y * y);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];
    float Sg[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Sg[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
    float T0[3], T1[3];
    if (ortho > 0.0f) { /* J = [[s, 0, 0], [0, s, 0]] */
        for (int k = 0; k < 3; ++k) {
            T0[k] = ortho * R[k];
            T1[k] = ortho * R[3 + k];
        }
    } else {
        float j00 = fx / tz, j02 = -((fx * xz) / tz);
        float j11 = fy / tz, j12 = -((fy * yz) / tz);
        for (int k = 0; k < 3; ++k) {
            T0[k] = j00 * R[k] + j02 * R[6 + k];
            T1[k] = j11 * R[3 + k] + j12 * R[6 + k];
        }
    }
    float U0[3], U1[3];
    for (int k = 0; k < 3; ++k) {
        U0[k] = T0[0] * Sg[k] + T0[1] * Sg[3 + k] + T0[2] * Sg[6 + k];
        U1[k] = T1[0] * Sg[k] + T1[1] * Sg[3 + k] + T1[2] * Sg[6 + k];
    }
    float a = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + o->lowpass;
    float b = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    float c = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + o->lowpass;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return 0;
    float mid = 0.5f * (a + c);
    float disc = mid * mid - det;
    float lam = mid + sqrtf(fmaxf(0.1f, disc));
    float r = ceilf(3.0f * sqrtf(lam));
    float ts = (float)o->tile;
    int gx = (W + o->tile - 1) / o->tile, gy = (H + o->tile - 1) / o->tile;
    float fx0 = floorf((u - r) / ts), fx1 = floorf((u + r) / ts);
    float fy0 = floorf((v - r) / ts), fy1 = floorf((v + r) / ts);
    /* Tiles no pixel can reach with alpha >= alpha_min are dropped: that
     * region is the ellipse d^T Sigma^-1 d <= 2 ln(gamma / alpha_min), inside
     * the box |dx| <= sqrt(r2 Sigma_xx), |dy| <= sqrt(r2 Sigma_yy) for any
     * r2 >= 2 ln(gamma / alpha_min).  With ln(gamma) = ln sigmoid(l) <= min(0, l),
     * r2 = 2 (min(0, l) - ln alpha_min) is such a bound without a
     * transcendental of per-Gaussian data; r2 <= 0 means no pixel can pass. */
    float r2 = 2.0f * (fminf(0.0f, m[3]) + nl_amin);
    if (!(r2 > 0.0f)) return 0;
    float hx = sqrtf(r2 * a), hy = sqrtf(r2 * c);
    fx0 = fmaxf(fx0, floorf((u - hx) / ts));
    fx1 = fminf(fx1, floorf((u + hx) / ts));
    fy0 = fmaxf(fy0, floorf((v - hy) / ts));
    fy1 = fminf(fy1, floorf((v + hy) / ts));
    if (fx1 < 0.0f || fx0 > (float)(gx - 1) || fy1 < 0.0f || fy0 > (float)(gy - 1)) return 0;
    out->x0 = (int)fmaxf(fx0, 0.0f);
    out->x1 = (int)fminf(fx1, (float)(gx - 1));
    out->y0 = (int)fmaxf(fy0, 0.0f);
    out->y1 = (int)fminf(fy1, (float)(gy - 1));
    out->u = u; out->v = v;
    if (pL && !(ortho > 0.0f)) {
        float dx = m[0] - pL[0], dy = m[1] - pL[1], dz = m[2] - pL[2];
        out->key = f32_bits(sqrtf(dx * dx + dy * dy + dz * dz));
    } else {
        out->key = f32_bits(tz); /* camera depth, or depth along an orthographic light view */
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* FP64 maths                                                                */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } d3;
static d3 d3_sub(d3 a, d3 b) { return (d3){a.x - b.x, a.y - b.y, a.z - b.z}; }
static double d3_dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 d3_scale(d3 a, double s) { return (d3){a.x * s, a.y * s, a.z * s}; }
static d3 d3_unit(d3 a) { return d3_scale(a, 1.0 / sqrt(d3_dot(a, a))); }

/* Rotation matrix of the normalised quaternion (w, x, y, z), row-major. */
static void quat_to_mat(const float qf[4], double Rm[9])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    Rm[0] = 1 - 2 * (y * y + z * z); Rm[1] = 2 * (x * y - w * z);     Rm[2] = 2 * (x * z + w * y);
    Rm[3] = 2 * (x * y + w * z);     Rm[4] = 1 - 2 * (x * x + z * z); Rm[5] = 2 * (y * z - w * x);
    Rm[6] = 2 * (x * z - w * y);     Rm[7] = 2 * (y * z + w * x);     Rm[8] = 1 - 2 * (x * x + y * y);
}

static d3 mat_mul(const double Rm[9], d3 v)
{
    return (d3){Rm[0] * v.x + Rm[1] * v.y + Rm[2] * v.z,
                Rm[3] * v.x + Rm[4] * v.y + Rm[5] * v.z,
                Rm[6] * v.x + Rm[7] * v.y + Rm[8] * v.z};
}

static d3 mat_tmul(const double Rm[9], d3 v) /* R^T v */
{
    return (d3){Rm[0] * v.x + Rm[3] * v.y + Rm[6] * v.z,
                Rm[1] * v.x + Rm[4] * v.y + Rm[7] * v.z,
                Rm[2] * v.x + Rm[5] * v.y + Rm[8] * v.z};
}

/* Eq. 3: modified Lambertian with ELU (alpha = 0.01) and epsilon = 0.01. */
double go_diffuse(double x)
{
    const double eps = 0.01;
    double elu = x > 0.0 ? x : 0.01 * (exp(x) - 1.0);
    double off = eps * (1.0 - exp(-1.0));
    return (elu + off) / ((1.0 + off) * GO_PI);
}

/* Eq. 5: angular Gaussian at the half vector h (shading frame), lobe frame
 * given by quaternion q (inside the shading frame), deviations sig[0..2]. */
double go_angular_gaussian(const double h[3], const float q[4], const double sig[3])
{
    double Rl[9];
    quat_to_mat(q, Rl);
    /* lobe axes x, y, z are the columns of Rl */
    d3 hv = {h[0], h[1], h[2]};
    d3 hl = mat_tmul(Rl, hv);
    double hz = hl.z;
    if (hz > 1.0) hz = 1.0;
    if (hz < -1.0) hz = -1.0;
    double theta = acos(hz);
    double sxy = sqrt(hl.x * hl.x + hl.y * hl.y);
    double sx = 1.0, sy = 0.0;
    if (sxy > 0.0) { sx = hl.x / sxy; sy = hl.y / sxy; }
    double q2 = (sx / sig[0]) * (sx / sig[0]) + (sy / sig[1]) * (sy / sig[1]);
    double e = theta * sqrt(q2) / sig[2];
    return exp(-0.5 * e * e) / sig[2];
}

/* Eq. 2 with Eq. 3-5 for Gaussian g: writes colour rgb and the unit directions. */
static void shade_one(const go_scene *sc, int g, const go_camera *cam, const go_light *L,
                      const go_opts *o, double rgb[3], d3 *wi_out, d3 *wo_out)
{
    d3 mu = {sc->mean_op[4 * g], sc->mean_op[4 * g + 1], sc->mean_op[4 * g + 2]};
    d3 pc = {cam->pos[0], cam->pos[1], cam->pos[2]};
    int directional = L->type == 1;
    d3 tol = directional ? (d3){L->dir[0], L->dir[1], L->dir[2]}
                         : d3_sub((d3){L->pos[0], L->pos[1], L->pos[2]}, mu);
    double dist2 = d3_dot(tol, tol);
    d3 wi = d3_unit(tol);
    d3 wo = d3_unit(d3_sub(pc, mu));
    *wi_out = wi; *wo_out = wo;
    double Rs[9];
    quat_to_mat(sc->shade_rot + 4 * g, Rs);
    d3 wil = mat_mul(Rs, wi), wol = mat_mul(Rs, wo);
    double fd = go_diffuse(wil.z); /* n' = e_z */
    double fs[3] = {0, 0, 0};
    d3 hs = {wil.x + wol.x, wil.y + wol.y, wil.z + wol.z};
    double hn = sqrt(d3_dot(hs, hs));
    if (hn >= 1e-12 && !(o->ablate & 8)) {
        double h[3] = {hs.x / hn, hs.y / hn, hs.z / hn};
        for (int j = 0; j < sc->k; ++j) {
            size_t li = (size_t)j * sc->n + g;
            size_t ls = sc->lobe_shared ? (size_t)j : li; /* the lobe's frame and deviations */
            double sig[3] = {sc->lobe_sigma[4 * ls], sc->lobe_sigma[4 * ls + 1], sc->lobe_sigma[4 * ls + 2]};
            double G = go_angular_gaussian(h, sc->lobe_rot + 4 * ls, sig);
            for (int c = 0; c < 3; ++c) fs[c] += sc->lobe_amp[4 * li + c] * G;
        }
    }
    /* a directional light's irradiance does not fall off (Sec. 4.5) */
    double E = (o->falloff && !directional) ? L->intensity / dist2 : L->intensity;
    for (int c = 0; c < 3; ++c)
        rgb[c] = E * (sc->albedo_d[4 * g + c] * fd + sc->albedo_s[4 * g + c] * fs[c]);
}

/* FP64 EWA projection (same conventions as the FP32 recipe, no culling). */
static void project_f64(const float mf[3], const float sf[3], const float qf[4],
                        const float Rf[9], const float tf[3], double fx, double fy, double cx,
                        double cy, double lowpass, double ortho, double uv[2], double conic[3])
{
    double R[9], t[3], m[3] = {mf[0], mf[1], mf[2]}, s[3] = {sf[0], sf[1], sf[2]};
    for (int i = 0; i < 9; ++i) R[i] = Rf[i];
    for (int i = 0; i < 3; ++i) t[i] = tf[i];
    double tx = R[0] * m[0] + R[1] * m[1] + R[2] * m[2] + t[0];
    double ty = R[3] * m[0] + R[4] * m[1] + R[5] * m[2] + t[1];
    double tz = R[6] * m[0] + R[7] * m[1] + R[8] * m[2] + t[2];
    if (ortho > 0.0) {
        uv[0] = ortho * tx + cx;
        uv[1] = ortho * ty + cy;
    } else {
        uv[0] = fx * tx / tz + cx;
        uv[1] = fy * ty / tz + cy;
    }
    double Rq[9];
    quat_to_mat(qf, Rq);
    double Sg[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += Rq[3 * i + k] * s[k] * s[k] * Rq[3 * j + k];
            Sg[3 * i + j] = acc;
        }
    double J[6] = {fx / tz, 0.0, -fx * tx / (tz * tz), 0.0, fy / tz, -fy * ty / (tz * tz)};
    if (ortho > 0.0) {
        J[0] = ortho; J[2] = 0.0;
        J[4] = ortho; J[5] = 0.0;
    }
    double T[6];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k)
            T[3 * i + k] = J[3 * i] * R[k] + J[3 * i + 1] * R[3 + k] + J[3 * i + 2] * R[6 + k];
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += T[3 * i + a] * Sg[3 * a + b] * T[3 * j + b];
            C2[2 * i + j] = acc;
        }
    double a = C2[0] + lowpass, b = C2[1], c = C2[3] + lowpass;
    double det = a * c - b * b;
    conic[0] = c / det;
    conic[1] = -b / det;
    conic[2] = a / det;
}

/* 4-band positional encoding: [v, sin(2^k pi v), cos(2^k pi v)], k = 0..3. */
static int pos_enc(d3 v, double *out)
{
    double a[3] = {v.x, v.y, v.z};
    int o = 0;
    for (int c = 0; c < 3; ++c) out[o++] = a[c];
    for (int k = 0; k < 4; ++k) {
        double f = ldexp(GO_PI, k);
        for (int c = 0; c < 3; ++c) out[o++] = sin(f * a[c]);
        for (int c = 0; c < 3; ++c) out[o++] = cos(f * a[c]);
    }
    return o; /* 27 */
}

/* MLP: hidden layers with ReLU / leaky ReLU, sigmoid output (Sec. 4.2, 4.3). */
void go_mlp_eval(const go_mlp *m, int rows, const double *x, double *y)
{
    int maxw = m->width > m->in_dim ? m->width : m->in_dim;
    if (m->out_dim > maxw) maxw = m->out_dim;
    double *h0 = malloc(sizeof(double) * maxw), *h1 = malloc(sizeof(double) * maxw);
    for (int r = 0; r < rows; ++r) {
        int din = m->in_dim;
        memcpy(h0, x + (size_t)r * m->in_dim, sizeof(double) * din);
        size_t wo = 0, bo = 0;
        for (int l = 0; l <= m->n_hidden; ++l) {
            int dout = (l == m->n_hidden) ? m->out_dim : m->width;
            for (int i = 0; i < dout; ++i) {
                double acc = m->b[bo + i];
                for (int j = 0; j < din; ++j) acc += (double)m->w[wo + (size_t)i * din + j] * h0[j];
                if (l < m->n_hidden) {
                    if (acc < 0.0) acc = (m->act == 1) ? 0.01 * acc : 0.0;
                } else {
                    acc = 1.0 / (1.0 + exp(-acc));
                }
                h1[i] = acc;
            }
            wo += (size_t)dout * din;
            bo += dout;
            din = dout;
            double *tmp = h0; h0 = h1; h1 = tmp;
        }
        memcpy(y + (size_t)r * m->out_dim, h0, sizeof(double) * m->out_dim);
    }
    free(h0);
    free(h1);
}

static void phi_input(const go_scene *sc, int g, double T, d3 wi, double *x)
{
    int o = 0;
    x[o++] = T;
    o += pos_enc(wi, x + o);
    d3 mu = {sc->mean_op[4 * g], sc->mean_op[4 * g + 1], sc->mean_op[4 * g + 2]};
    o += pos_enc(mu, x + o);
    for (int i = 0; i < 4; ++i) x[o++] = sc->latent[4 * g + i];
    for (int i = 0; i < 2; ++i) x[o++] = sc->latent[4 * ((size_t)sc->n + g) + i];
}

static void psi_input(const go_scene *sc, int g, d3 wo, double *x)
{
    int o = 0;
    o += pos_enc(wo, x + o);
    d3 mu = {sc->mean_op[4 * g], sc->mean_op[4 * g + 1], sc->mean_op[4 * g + 2]};
    o += pos_enc(mu, x + o);
    for (int i = 0; i < 4; ++i) x[o++] = sc->latent[4 * g + i];
    for (int i = 0; i < 2; ++i) x[o++] = sc->latent[4 * ((size_t)sc->n + g) + i];
}

/* ------------------------------------------------------------------------ */
/* Tile lists (O7, O8)                                                       */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t tile, key, idx; } entry;

static int entry_cmp(const void *pa, const void *pb)
{
    const entry *a = pa, *b = pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static void build_lists(go_frame *f, int s)
{
    size_t P = 0;
    for (int g = 0; g < f->n; ++g) {
        const int32_t *r = f->rect[s] + 4 * g;
        if (r[0] < 0) continue;
        P += (size_t)(r[2] - r[0] + 1) * (size_t)(r[3] - r[1] + 1);
    }
    entry *e = malloc(sizeof(entry) * (P ? P : 1));
    size_t p = 0;
    for (int g = 0; g < f->n; ++g) {
        const int32_t *r = f->rect[s] + 4 * g;
        if (r[0] < 0) continue;
        for (int ty = r[1]; ty <= r[3]; ++ty)
            for (int tx = r[0]; tx <= r[2]; ++tx) {
                e[p].tile = (uint32_t)(ty * f->gx + tx);
                e[p].key = f->key[s][g];
                e[p].idx = (uint32_t)g;
                ++p;
            }
    }
    qsort(e, P, sizeof(entry), entry_cmp);
    f->P[s] = (uint32_t)P;
    f->list[s] = malloc(sizeof(uint32_t) * (P ? P : 1));
    f->tile_start[s] = calloc((size_t)f->ntiles + 1, sizeof(uint32_t));
    for (size_t i = 0; i < P; ++i) {
        f->list[s][i] = e[i].idx;
        f->tile_start[s][e[i].tile + 1]++;
    }
    for (int t = 0; t < f->ntiles; ++t) f->tile_start[s][t + 1] += f->tile_start[s][t];
    free(e);
}

/* ------------------------------------------------------------------------ */
/* Shadow splatting (Sec. 4.2, Fig. 3)                                        */
/* ------------------------------------------------------------------------ */
static float key_to_float(uint32_t k) { float f; memcpy(&f, &k, 4); return f; }

/* O10 for the shadow rays of light-view rows [y0, y1) (inside the crop
 * window): adds each Gaussian's sums of beta T_m and beta (and of their
 * bounds) to f->sacc */
static void shadow_rows(go_frame *f, const go_opts *o, int y0, int y1)
{
    int n = f->n, W = f->width, H = f->height, ts = o->tile;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *acc = calloc((size_t)nthr * n * 4, sizeof(double)); /* num, den, bnum, bden */
    int64_t evals = 0, passes = 0, ambs = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(+ : evals, passes, ambs)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *num = acc + (size_t)tid * n * 4, *den = num + n, *bnum = den + n, *bden = bnum + n;
        size_t cap = 1024;
        double *al = malloc(sizeof(double) * cap), *be = malloc(sizeof(double) * cap);
        double *A = malloc(sizeof(double) * (cap + 1)), *Q = malloc(sizeof(double) * (cap + 1));
        float *d = malloc(sizeof(float) * cap);
        uint32_t *gi = malloc(sizeof(uint32_t) * cap);
        int *amb = malloc(sizeof(int) * cap);
        int *pass = malloc(sizeof(int) * cap);
        int wx0, wy0, wx1, wy1;
        window(o, W, H, &wx0, &wy0, &wx1, &wy1);
        if (wy0 < y0) wy0 = y0;
        if (wy1 > y1) wy1 = y1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int py = wy0; py < wy1; ++py) {
            for (int px = wx0; px < wx1; ++px) {
                int t = (py / ts) * f->gx + (px / ts);
                uint32_t b = f->tile_start[1][t], e = f->tile_start[1][t + 1];
                size_t L = e - b;
                if (L > cap) {
                    cap = L;
                    al = realloc(al, sizeof(double) * cap); be = realloc(be, sizeof(double) * cap);
                    A = realloc(A, sizeof(double) * (cap + 1)); d = realloc(d, sizeof(float) * cap);
                    Q = realloc(Q, sizeof(double) * (cap + 1));
                    gi = realloc(gi, sizeof(uint32_t) * cap); amb = realloc(amb, sizeof(int) * cap);
                    pass = realloc(pass, sizeof(int) * cap);
                }
                double cxp = px + 0.5, cyp = py + 0.5;
                /* alpha of every list entry on this shadow ray, in list order */
                for (size_t i = 0; i < L; ++i) {
                    uint32_t g = f->list[1][b + i];
                    double dx = cxp - f->uv[1][2 * g], dy = cyp - f->uv[1][2 * g + 1];
                    const double *C = f->conic[1] + 3 * g;
                    double power = -0.5 * (C[0] * dx * dx + C[2] * dy * dy) - C[1] * dx * dy;
                    double beta = exp(power);
                    double a = f->opacity[g] * beta;
                    if (a > o->alpha_max) a = o->alpha_max;
                    al[i] = a; be[i] = beta; gi[i] = g;
                    d[i] = key_to_float(f->key[1][g]);
                    /* the conic is positive definite, so the power is never positive:
                     * no test on its sign (Eq. 2 has none) */
                    pass[i] = a >= o->alpha_min;
                    amb[i] = fabs(a - o->alpha_min) <= o->margin_alpha * o->alpha_min;
                    if (amb[i]) {
                        ambs++;
                        const int64_t code = amb_code(AMB_SHADOW_ALPHA, (size_t)py * W + px, b + i);
                        record_amb(f, o, code);
                        if (o->nflip && flipped(o, code)) pass[i] = !pass[i];
                    }
                    evals++;
                    passes += pass[i];
                }
                /* A[i] = product of (1 - alpha_k) over passing k < i (Eq. 2);
                 * Q[i] = product of 1 / (1 - alpha_k) over ambiguous k < i: whichever
                 * subset of those an FP32 evaluation takes the other way (a removed
                 * factor divides A by 1 - alpha, an added one multiplies it by
                 * 1 - alpha), A[i] moves by at most A[i] (Q[i] - 1) */
                A[0] = 1.0;
                Q[0] = 1.0;
                for (size_t i = 0; i < L; ++i) {
                    A[i + 1] = A[i] * (pass[i] ? 1.0 - al[i] : 1.0);
                    Q[i + 1] = Q[i] * (amb[i] ? 1.0 / (1.0 - al[i]) : 1.0);
                }
                /* receiver j gets T_m(j) = A[K], K = #entries with d_k < d_j - bias */
                size_t K = 0;
                for (size_t j = 0; j < L; ++j) {
                    if (!pass[j] && !amb[j]) continue;
                    float thr = d[j] - o->shadow_bias;
                    while (K < L && d[K] < thr) ++K;
                    double Tm = A[K];
                    if (pass[j]) {
                        num[gi[j]] += be[j] * Tm;
                        den[gi[j]] += be[j];
                        /* occluder side: straddling decisions in front of it */
                        if (Q[K] > 1.0) bnum[gi[j]] += be[j] * Tm * (Q[K] - 1.0);
                    }
                    if (amb[j]) { /* receiver side: its own term may appear or vanish */
                        bnum[gi[j]] += be[j] * Tm * Q[K];
                        bden[gi[j]] += be[j];
                    }
                }
            }
        }
        free(al); free(be); free(A); free(Q); free(d); free(gi); free(amb); free(pass);
    }
    f->shadow_evals += evals;
    f->shadow_pass += passes;
    f->amb_shadow += ambs;
    for (int g = 0; g < n; ++g) {
        for (int t = 0; t < nthr; ++t) {
            double *a = acc + (size_t)t * n * 4;
            for (int q = 0; q < 4; ++q) f->sacc[4 * (size_t)g + q] += a[(size_t)q * n + g];
        }
    }
    free(acc);
}

/* O10: T = sum beta T_m / sum beta per Gaussian (1 when no shadow ray meets
 * it), and the bound of its straddling decisions */
static void shadow_average(go_frame *f)
{
    int n = f->n;
    for (int g = 0; g < n; ++g) {
        const double *a = f->sacc + 4 * (size_t)g;
        double num = a[0], den = a[1], bnum = a[2], bden = a[3];
        f->T[g] = den > 0.0 ? num / den : 1.0;
        if (bnum == 0.0 && bden == 0.0) {
            f->T_bound[g] = 0.0;
        } else if (den - bden > 0.0) {
            f->T_bound[g] = (bnum + f->T[g] * bden) / (den - bden);
            if (f->T_bound[g] > 1.0) f->T_bound[g] = 1.0;
        } else {
            f->T_bound[g] = 1.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Camera compositing (Eq. 2) and the deferred combination (Sec. 4)          */
/* ------------------------------------------------------------------------ */
static void camera_composite(go_frame *f, const go_opts *o)
{
    int W = f->width, H = f->height, ts = o->tile;
    int64_t evals = 0, ambs = 0, cpass = 0;
    int wx0, wy0, wx1, wy1;
    window(o, W, H, &wx0, &wy0, &wx1, &wy1);
    for (size_t p = 0; p < (size_t)W * H; ++p) { /* outside the window: empty */
        f->final_T[p] = 1.0; f->n_contrib[p] = 0; f->Sh[p] = 0.0;
        for (int c = 0; c < 3; ++c) {
            f->S[3 * p + c] = 0.0; f->Rimg[3 * p + c] = 0.0; f->img[3 * p + c] = 0.0;
            f->img_bound[3 * p + c] = 0.0;
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : evals, ambs, cpass)
#endif
    for (int py = wy0; py < wy1; ++py) {
        for (int px = wx0; px < wx1; ++px) {
            int t = (py / ts) * f->gx + (px / ts);
            uint32_t b = f->tile_start[0][t], e = f->tile_start[0][t + 1];
            double cxp = px + 0.5, cyp = py + 0.5;
            double T = 1.0, S[3] = {0, 0, 0}, Sh = 0.0, R[3] = {0, 0, 0};
            double bS[3] = {0, 0, 0}, bSh = 0.0, bR[3] = {0, 0, 0};
            /* P = product of 1 / (1 - alpha) over the earlier ambiguous alpha tests:
             * whichever subset of them an FP32 evaluation takes the other way, the
             * transmittance T' it carries lies in [T / P, T P] */
            double P = 1.0;
            double cmax[7] = {0, 0, 0, 0, 0, 0, 0};
            for (uint32_t i = b; i < e; ++i) {
                uint32_t g = f->list[0][i];
                for (int c = 0; c < 3; ++c) {
                    if (fabs(f->shade[3 * g + c]) > cmax[c]) cmax[c] = fabs(f->shade[3 * g + c]);
                    if (fabs(f->res[3 * g + c]) > cmax[4 + c]) cmax[4 + c] = fabs(f->res[3 * g + c]);
                }
                if (fabs(f->Tp[g]) > cmax[3]) cmax[3] = fabs(f->Tp[g]);
            }
            int32_t consumed = 0;
            for (uint32_t i = b; i < e; ++i) {
                uint32_t g = f->list[0][i];
                consumed = (int32_t)(i - b + 1);
                double dx = cxp - f->uv[0][2 * g], dy = cyp - f->uv[0][2 * g + 1];
                const double *C = f->conic[0] + 3 * g;
                double power = -0.5 * (C[0] * dx * dx + C[2] * dy * dy) - C[1] * dx * dy;
                evals++;
                double a = f->opacity[g] * exp(power); /* power <= 0: the conic is positive definite */
                if (a > o->alpha_max) a = o->alpha_max;
                int amb = fabs(a - o->alpha_min) <= o->margin_alpha * o->alpha_min;
                int take = a >= o->alpha_min;
                if (amb) {
                    /* its own term may appear or vanish, at a transmittance up to T P */
                    ambs++;
                    double w = a * T * P;
                    for (int c = 0; c < 3; ++c) {
                        bS[c] += w * fabs(f->shade[3 * g + c]);
                        bR[c] += w * fabs(f->res[3 * g + c]);
                    }
                    bSh += w * fabs(f->Tp[g]);
                    P /= 1.0 - a;
                    const int64_t code = amb_code(AMB_CAMERA_ALPHA, (size_t)py * W + px, i);
                    record_amb(f, o, code);
                    if (o->nflip && flipped(o, code)) take = !take;
                }
                if (!take) continue;
                double Tn = T * (1.0 - a);
                int stop = Tn < o->t_stop;
                /* the stop test straddles when Tn lies within the margin of t_stop, or
                 * when earlier straddling alpha tests can carry it across */
                if (Tn * P >= o->t_stop * (1.0 - o->margin_tstop) && Tn <= P * o->t_stop * (1.0 + o->margin_tstop)) {
                    /* the ray may stop here or go on: everything from here on, at most
                     * the remaining transmittance T P times the largest colour */
                    ambs++;
                    for (int c = 0; c < 3; ++c) { bS[c] += T * P * cmax[c]; bR[c] += T * P * cmax[4 + c]; }
                    bSh += T * P * cmax[3];
                    const int64_t code = amb_code(AMB_CAMERA_STOP, (size_t)py * W + px, i);
                    record_amb(f, o, code);
                    if (o->nflip && flipped(o, code)) stop = !stop;
                }
                if (stop) { consumed = (int32_t)(i - b); break; }
                cpass++;
                double w = a * T;
                for (int c = 0; c < 3; ++c) {
                    S[c] += w * f->shade[3 * g + c];
                    R[c] += w * f->res[3 * g + c];
                    if (P > 1.0) { /* the same term at a transmittance in [T / P, T P] */
                        bS[c] += (P - 1.0) * w * fabs(f->shade[3 * g + c]);
                        bR[c] += (P - 1.0) * w * fabs(f->res[3 * g + c]);
                    }
                }
                Sh += w * f->Tp[g];
                if (P > 1.0) bSh += (P - 1.0) * w * fabs(f->Tp[g]);
                bSh += P * w * f->Tp_bound[g]; /* propagated shadow-value bound */
                T = Tn;
            }
            size_t p = (size_t)py * W + px;
            f->final_T[p] = T;
            f->n_contrib[p] = consumed;
            f->Sh[p] = Sh;
            for (int c = 0; c < 3; ++c) {
                f->S[3 * p + c] = S[c];
                f->Rimg[3 * p + c] = R[c];
                f->img[3 * p + c] = S[c] * Sh + R[c];
                f->img_bound[3 * p + c] = bS[c] * fabs(Sh) + fabs(S[c]) * bSh + bS[c] * bSh + bR[c];
            }
        }
    }
    f->camera_evals = evals;
    f->amb_camera = ambs;
    f->camera_pass = cpass;
}

/* ------------------------------------------------------------------------ */
/* Whole frame                                                               */
/* ------------------------------------------------------------------------ */
/* Stages of one frame, for callers that time them apart (the whole frame is
 * go_render; the same arithmetic in the same order):
 *   go_begin        O1-O8: parameters, directions, shading, both projections,
 *                   keys and per-tile lists
 *   go_shadow_rows  O10 for the shadow rays of light-view rows [y0, y1); every
 *                   row once, in any number of calls
 *   go_finish       O10's per-Gaussian average, O11-O12 (Phi, Psi), O9 (the
 *                   camera composite and the deferred combination) */
go_frame *go_begin(const go_scene *sc, const go_camera *cam, const go_light *L, const go_opts *o)
{
#ifdef _OPENMP
    if (o->threads > 0) omp_set_num_threads(o->threads);
#endif
    go_frame *f = calloc(1, sizeof(go_frame));
    int n = sc->n;
    f->n = n; f->width = cam->width; f->height = cam->height;
    f->gx = (cam->width + o->tile - 1) / o->tile;
    f->gy = (cam->height + o->tile - 1) / o->tile;
    f->ntiles = f->gx * f->gy;
    f->light_ortho = go_light_view_any(L, o->target, cam->width, cam->height, f->light_R, f->light_t);
    for (int s = 0; s < 2; ++s) {
        f->key[s] = malloc(sizeof(uint32_t) * n);
        f->rect[s] = malloc(sizeof(int32_t) * 4 * n);
        f->uv_f32[s] = malloc(sizeof(float) * 2 * n);
        f->uv[s] = malloc(sizeof(double) * 2 * n);
        f->conic[s] = malloc(sizeof(double) * 3 * n);
    }
    f->opacity = malloc(sizeof(double) * n);
    f->shade = malloc(sizeof(double) * 3 * n);
    f->T = malloc(sizeof(double) * n);
    f->T_bound = calloc(n, sizeof(double));
    f->Tp = malloc(sizeof(double) * n);
    f->Tp_bound = calloc(n, sizeof(double));
    f->res = malloc(sizeof(double) * 3 * n);
    size_t np = (size_t)cam->width * cam->height;
    f->img = malloc(sizeof(double) * 3 * np);
    f->img_bound = malloc(sizeof(double) * 3 * np);
    f->final_T = malloc(sizeof(double) * np);
    f->n_contrib = malloc(sizeof(int32_t) * np);
    f->S = malloc(sizeof(double) * 3 * np);
    f->Sh = malloc(sizeof(double) * np);
    f->Rimg = malloc(sizeof(double) * 3 * np);
    f->sacc = calloc((size_t)n * 4, sizeof(double));

    double t0 = now_s();
    d3 *wi = malloc(sizeof(d3) * n), *wo = malloc(sizeof(d3) * n);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int g = 0; g < n; ++g) {
        const float *m = sc->mean_op + 4 * g, *s = sc->scale + 4 * g, *q = sc->rot + 4 * g;
        f->opacity[g] = 1.0 / (1.0 + exp(-(double)m[3]));
        for (int sp = 0; sp < 2; ++sp) {
            keyrec kr;
            const float *R = sp ? f->light_R : cam->R, *t = sp ? f->light_t : cam->t;
            const float ortho = sp ? f->light_ortho : 0.0f;
            int vis = key_recipe(m, s, q, R, t, cam->fx, cam->fy, cam->cx, cam->cy, cam->width,
                                 cam->height, o, sp ? L->pos : NULL, ortho, &kr);
            f->key[sp][g] = kr.key;
            f->rect[sp][4 * g] = vis ? kr.x0 : -1;
            f->rect[sp][4 * g + 1] = vis ? kr.y0 : -1;
            f->rect[sp][4 * g + 2] = vis ? kr.x1 : -2;
            f->rect[sp][4 * g + 3] = vis ? kr.y1 : -2;
            f->uv_f32[sp][2 * g] = kr.u;
            f->uv_f32[sp][2 * g + 1] = kr.v;
            project_f64(m, s, q, R, t, cam->fx, cam->fy, cam->cx, cam->cy, o->lowpass, ortho,
                        f->uv[sp] + 2 * g, f->conic[sp] + 3 * g);
        }
        shade_one(sc, g, cam, L, o, f->shade + 3 * g, wi + g, wo + g);
    }
    f->wi = (double *)wi;
    f->wo = (double *)wo;
    double t1 = now_s();
    build_lists(f, 0);
    build_lists(f, 1);
    double t2 = now_s();
    f->t_prep = t1 - t0;
    f->t_bin = t2 - t1;
    return f;
}

void go_shadow_rows(go_frame *f, const go_opts *o, int y0, int y1)
{
#ifdef _OPENMP
    if (o->threads > 0) omp_set_num_threads(o->threads);
#endif
    if (o->ablate & 1) return;
    double t0 = now_s();
    shadow_rows(f, o, y0, y1);
    f->t_shadow += now_s() - t0;
}

void go_finish(go_frame *f, const go_scene *sc, const go_opts *o)
{
#ifdef _OPENMP
    if (o->threads > 0) omp_set_num_threads(o->threads);
#endif
    int n = f->n;
    const d3 *wi = (const d3 *)f->wi, *wo = (const d3 *)f->wo;
    double t2 = now_s();
    if (o->ablate & 1) {
        for (int g = 0; g < n; ++g) f->T[g] = 1.0;
    } else {
        shadow_average(f);
    }
    double t3 = now_s();
    /* Phi and Psi per Gaussian (Sec. 4.2, 4.3) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int g = 0; g < n; ++g) {
        double x[64], y[4];
        if (o->ablate & 2) {
            f->Tp[g] = f->T[g];
            f->Tp_bound[g] = f->T_bound[g];
        } else {
            phi_input(sc, g, f->T[g], wi[g], x);
            go_mlp_eval(&sc->phi, 1, x, y);
            f->Tp[g] = y[0];
            if (f->T_bound[g] > 0.0) { /* propagate the shadow bound through Phi */
                double lo = 0.0, hi = 0.0;
                x[0] = f->T[g] - f->T_bound[g];
                go_mlp_eval(&sc->phi, 1, x, &lo);
                x[0] = f->T[g] + f->T_bound[g];
                go_mlp_eval(&sc->phi, 1, x, &hi);
                double bnd = fabs(lo - y[0]) > fabs(hi - y[0]) ? fabs(lo - y[0]) : fabs(hi - y[0]);
                f->Tp_bound[g] = 2.0 * bnd;
            }
        }
        if (o->ablate & 4) {
            f->res[3 * g] = f->res[3 * g + 1] = f->res[3 * g + 2] = 0.0;
        } else {
            psi_input(sc, g, wo[g], x);
            go_mlp_eval(&sc->psi, 1, x, y);
            for (int c = 0; c < 3; ++c) f->res[3 * g + c] = y[c];
        }
    }
    double t4 = now_s();
    camera_composite(f, o);
    double t5 = now_s();
    f->t_shadow += t3 - t2;
    f->t_mlp = t4 - t3;
    f->t_camera = t5 - t4;
}

go_frame *go_render(const go_scene *sc, const go_camera *cam, const go_light *L, const go_opts *o)
{
    go_frame *f = go_begin(sc, cam, L, o);
    go_shadow_rows(f, o, 0, f->height);
    go_finish(f, sc, o);
    return f;
}

void go_frame_free(go_frame *f)
{
    if (!f) return;
    for (int s = 0; s < 2; ++s) {
        free(f->key[s]); free(f->rect[s]); free(f->uv_f32[s]); free(f->uv[s]);
        free(f->conic[s]); free(f->tile_start[s]); free(f->list[s]);
    }
    free(f->opacity); free(f->shade); free(f->T); free(f->T_bound); free(f->Tp);
    free(f->Tp_bound); free(f->res); free(f->img); free(f->img_bound); free(f->final_T);
    free(f->n_contrib); free(f->S); free(f->Sh); free(f->Rimg); free(f->amb);
    free(f->sacc); free(f->wi); free(f->wo);
    free(f);
}

/* Threads the oracle's parallel loops use. */
int go_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Shading of one Gaussian (for closed-form pins). */
void go_shade(const go_scene *sc, int g, const go_camera *cam, const go_light *L,
              const go_opts *o, double rgb[3])
{
    d3 wi, wo;
    shade_one(sc, g, cam, L, o, rgb, &wi, &wo);
}

/* FP32 recipe of one Gaussian (for pins on the key recipe). */
int go_key_recipe(const float m[4], const float s[3], const float q[4], const float R[9],
                  const float t[3], float fx, float fy, float cx, float cy, int W, int H,
                  const go_opts *o, const float *pL, float ortho, uint32_t *key, int32_t rect[4],
                  float uv[2])
{
    keyrec kr;
    int vis = key_recipe(m, s, q, R, t, fx, fy, cx, cy, W, H, o, pL, ortho, &kr);
    *key = kr.key;
    rect[0] = kr.x0; rect[1] = kr.y0; rect[2] = kr.x1; rect[3] = kr.y1;
    uv[0] = kr.u; uv[1] = kr.v;
    return vis;
}

/* FP64 projection of one Gaussian (for pins). */
void go_project(const float m[3], const float s[3], const float q[4], const float R[9],
                const float t[3], double fx, double fy, double cx, double cy, double lowpass,
                double ortho, double uv[2], double conic[3])
{
    project_f64(m, s, q, R, t, fx, fy, cx, cy, lowpass, ortho, uv, conic);
}

/* Positional encoding of one 3-vector (for pins). */
int go_pos_enc(const double v[3], double out[27])
{
    d3 a = {v[0], v[1], v[2]};
    return pos_enc(a, out);
}
