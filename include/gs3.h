/*
 * gs3.h -- C ABI of the GB300 (sm_103a) GS^3 triple-splatting renderer.
 *
 * GS^3 (Bi et al., SIGGRAPH Asia 2024) renders a relit image of a set of
 * spatial Gaussians for one camera and one point light (Sec. 4, Sec. 4.5):
 *   1. colour every Gaussian with a Lambertian plus a mixture of angular
 *      Gaussian lobes (Sec. 4.1, Eq. 2-5);
 *   2. splat all Gaussians toward the light and alpha-composite every shadow
 *      ray front to back to get one shadow value per Gaussian (Sec. 4.2,
 *      Fig. 3), refined by the MLP Phi;
 *   3. colour every Gaussian with the residual MLP Psi (Sec. 4.3);
 *   4. splat shading, shadow and residual toward the camera (Sec. 3, Eq. 2)
 *      and combine them per pixel: shading * shadow + residual (Sec. 4).
 *
 * Conventions for every entry point:
 *   - Pointers documented as "device" are CUDA device pointers on the current
 *     device; "host" pointers are ordinary CPU memory.
 *   - The library never frees caller memory and never keeps a caller pointer
 *     beyond the call, except the scene parameter pointers captured by
 *     gs3_create_scene, which must stay valid until gs3_destroy_scene.
 *   - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t
 *     passed as void*; NULL is the legacy default stream) and is asynchronous
 *     unless stated otherwise.
 *   - Errors are returned as gs3_status; no exception or abort crosses the
 *     ABI.  gs3_last_error() gives a thread-local message for the last error.
 *   - Errors found on the device (key capacity exceeded, a bounded wait that
 *     ran out) are written to a status word in the workspace and read back by
 *     gs3_workspace_read_header after the stream has been synchronised.
 */
#ifndef GS3_H
#define GS3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS3_OK = 0,
    GS3_ERR_INVALID_ARG = 1, /* a size, pointer or option is out of range */
    GS3_ERR_OOM = 2,         /* a scene-owned allocation failed */
    GS3_ERR_CAPACITY = 3,    /* more (tile, Gaussian) pairs than key_capacity */
    GS3_ERR_CUDA = 4,        /* a CUDA runtime call failed (message in gs3_last_error) */
    GS3_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    GS3_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} gs3_status;

enum { GS3_ACT_RELU = 0, GS3_ACT_LEAKY_RELU = 1 };         /* hidden-layer activation */
/* MLP operand precision of the hidden layers (the output layer and the
 * sigmoid stay FP32).  BF16 and FP8 run on the tensor cores with FP32
 * accumulation.  FP8 E4M3 uses per-tensor scales: each weight matrix is
 * scaled by max|W| / 448, each hidden layer's input by twice its largest
 * magnitude over a calibration pass that gs3_create_scene runs (FP32, on a
 * strided sample of up to 16384 Gaussians for 8 fixed directions); inputs
 * beyond the calibrated range saturate at 448.  BF16 and FP8 need hidden
 * widths of 32, 64 or 128 (gs3_create_scene: GS3_ERR_UNSUPPORTED otherwise).
 * BF16 layers start their FP32 accumulators at the bias. */
enum { GS3_MLP_FP32 = 0, GS3_MLP_BF16 = 1, GS3_MLP_FP8_E4M3 = 2 };
/* Ablations (render modes): no shadow splat (T = 1), no Phi (T' = T), no Psi
 * (residual 0), Lambertian only (no angular-Gaussian lobes: the first stage
 * of the two-stage training of Sec. 4.4). */
enum { GS3_ABLATE_SHADOW_SPLAT = 1, GS3_ABLATE_PHI = 2, GS3_ABLATE_PSI = 4, GS3_ABLATE_SPECULAR = 8 };

/* Fully connected network in_dim -> [width] x n_hidden -> out_dim with a
 * sigmoid output (Sec. 4.2: Phi, Sec. 4.3: Psi).
 *   w: device, float32, every layer's (out, in) row-major matrix, concatenated
 *   b: device, float32, every layer's bias, concatenated
 * Supported: in_dim = 61 (Phi) / 60 (Psi), out_dim = 1 (Phi) / 3 (Psi),
 * 1 <= n_hidden <= 4, width in {16, 32, 64, 128}. */
typedef struct {
    int32_t in_dim, width, n_hidden, out_dim, act;
    const float *w;
    const float *b;
} gs3_mlp_desc;

/* Scene parameters: structure of arrays, every array float4-padded, device,
 * float32, borrowed (the caller keeps them alive until gs3_destroy_scene).
 *   mean_op[N]    (x, y, z, opacity logit); opacity = sigmoid(logit)   Eq. 1-2
 *   scale[N]      (sx, sy, sz, -) positive; Sigma = R S S^T R^T        Eq. 1
 *   rot[N]        (w, x, y, z) quaternion of R (normalised inside)     Eq. 1
 *   shade_rot[N]  (w, x, y, z) world -> shading frame [t, b, n]; the normal
 *                 n' is the frame's z axis                             Sec. 4.1
 *   albedo_d[N], albedo_s[N]  (rgb, -) rho_d, rho_s                    Eq. 2
 *   latent[2N]    latent[g] = (l0..l3), latent[N+g] = (l4, l5, -, -)   Sec. 4.2
 *   lobe_rot[K*N]   (w, x, y, z) lobe frame [x, y, z] in the shading frame,
 *                   lobe-major: lobe j of Gaussian g at j*N + g          Eq. 5
 *   lobe_sigma[K*N] (sigma_x, sigma_y, sigma_z, -)                       Eq. 5
 *   lobe_amp[K*N]   (alpha_j rgb, -) lobe weights                        Eq. 4
 * 1 <= N, 0 <= K <= 16. */
typedef struct {
    int32_t n, k;
    const float *mean_op, *scale, *rot, *shade_rot, *albedo_d, *albedo_s, *latent;
    const float *lobe_rot, *lobe_sigma, *lobe_amp;
    gs3_mlp_desc phi, psi;
    int32_t mlp_dtype; /* GS3_MLP_FP32, GS3_MLP_BF16 or GS3_MLP_FP8_E4M3 */
    int32_t lobe_shared; /* 1: lobe_rot and lobe_sigma are one basis of K angular Gaussians
                            shared by every spatial Gaussian (K entries each, Sec. 4.1);
                            lobe_amp stays per Gaussian.  0: K lobes per Gaussian. */
} gs3_scene_desc;

/* Pinhole camera, host struct.  R: world -> camera rotation rows (x right,
 * y down, z forward); t: translation (p_cam = R p + t); pos: camera centre
 * in world space; fx, fy, cx, cy in pixels; pixel (x, y) has its centre at
 * (x + 0.5, y + 0.5).  The shadow splat's light camera uses the same
 * intrinsics and resolution (Sec. 4.2). */
typedef struct {
    float R[9], t[3], pos[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} gs3_camera;

/* Light, host struct.
 *   GS3_LIGHT_POINT (Sec. 4.2): at pos; irradiance intensity / d^2 when
 *     opts.falloff is set, else intensity; perspective shadow splat from pos.
 *   GS3_LIGHT_DIRECTIONAL (Sec. 4.5): from the scene towards dir (normalised
 *     inside); irradiance intensity (no fall-off); orthographic shadow splat
 *     along -dir over a view of half-width `extent` world units centred at
 *     opts.target (pixel scale min(W, H) / (2 extent)), its eye at
 *     target + dir * 4 extent; Gaussians are sorted by depth along the axis.
 * Zero-initialised type, dir and extent give a point light. */
enum { GS3_LIGHT_POINT = 0, GS3_LIGHT_DIRECTIONAL = 1 };
typedef struct {
    float pos[3];
    float intensity;
    int32_t type;
    float dir[3];
    float extent;
} gs3_light;

/* Render options, host struct; gs3_default_opts fills the paper's values:
 *   shadow_bias 0.015 (Sec. 4.2), alpha_min 1/255, alpha_max 0.99,
 *   t_stop 1e-4, near_z 0.2, lowpass 0.3 px^2, frustum 1.3, tile 16,
 *   target (0,0,0) = point the light camera looks at, falloff 1 (irradiance
 *   I / d^2), ablate 0 (bits GS3_ABLATE_*). */
typedef struct {
    float near_z, lowpass, frustum, shadow_bias, alpha_min, alpha_max, t_stop;
    float target[3];
    int32_t falloff, tile, ablate;
} gs3_render_opts;

typedef struct gs3_scene gs3_scene;

/* Device status word and pair counts at the start of every workspace. */
typedef struct {
    uint32_t status;      /* GS3_OK, or the first device-side error */
    uint32_t pairs_cam;   /* (tile, Gaussian) pairs of the camera splat */
    uint32_t pairs_light; /* (tile, Gaussian) pairs of the shadow splat */
    uint32_t pairs_cam_needed, pairs_light_needed; /* before clamping to the capacity */
    uint32_t reserved[3];
    float light_R[9], light_t[3]; /* light camera used by the shadow splat */
    float light_ortho;            /* its pixels per world unit if orthographic, else 0 */
} gs3_ws_header;

/* Byte offsets of the named intermediate buffers inside a workspace (for
 * inspection and tests).  Per-splat arrays are indexed [0] camera, [1] light. */
typedef struct {
    size_t total;
    size_t header;
    size_t key[2];        /* uint32[N] FP32 depth / light-distance bits by Gaussian */
    size_t order[2];      /* uint32[N] Gaussian index of depth rank r */
    size_t tile_start[2]; /* uint32[tiles + 1] per-tile range into the sorted list */
    size_t list[2];       /* uint32[capacity] sorted list: depth rank per entry */
    size_t rect[2];       /* int4[N] tile rectangle x0, y0, x1, y1 by Gaussian (x0 < 0: culled) */
    size_t shade;         /* float4[N] shading colour rgb by Gaussian */
    size_t shadow;        /* float[N] shadow value T by Gaussian */
    size_t shadow_refined;/* float[N] T' = Phi(...) by Gaussian */
    size_t residual;      /* float4[N] Psi(...) rgb by Gaussian */
    size_t final_t;       /* float[H*W] transmittance left after the camera ray */
    size_t n_contrib;     /* uint32[H*W] list entries consumed by the camera ray */
    size_t light_final;   /* float[H*W] occluder product where each shadow ray ended */
    size_t light_stop;    /* uint32[H*W] 1 + light-list index of the occluder after which the
                             shadow ray's product fell below 2^-40 and took no more
                             occluders, or 0xFFFFFFFF when it never did */
} gs3_ws_layout;

/* Fill `o` with the paper's defaults (see gs3_render_opts). */
void gs3_default_opts(gs3_render_opts *o);

/* Validate `desc` and create a scene.  The scene borrows the parameter and
 * weight pointers and owns derived buffers (packed / BF16 MLP weights).
 * Errors: INVALID_ARG (sizes, NULL pointers, unsupported MLP shape), OOM. */
gs3_status gs3_create_scene(const gs3_scene_desc *desc, gs3_scene **out);

/* The per-tensor scales of an FP8 scene's MLP (which = 0: Phi, 1: Psi):
 * out[2l] = sx_l (input of hidden layer l), out[2l + 1] = sw_l (its weights),
 * so that layer l computes (sum_k q(x_k / sx_l) q(w_jk / sw_l)) sx_l sw_l + b_j
 * with q = round to E4M3, saturating.  out: host, cap >= 2 n_hidden floats.
 * Synchronous.  GS3_ERR_UNSUPPORTED unless the scene is GS3_MLP_FP8_E4M3. */
gs3_status gs3_scene_mlp_scales(const gs3_scene *scene, int32_t which, float *out, int32_t cap);

/* Release a scene; waits for nothing (the caller synchronises first). */
gs3_status gs3_destroy_scene(gs3_scene *scene);

/* Bytes of workspace one render of an n-Gaussian scene at width x height
 * needs when at most key_capacity (tile, Gaussian) pairs per splat fit. */
size_t gs3_workspace_size(int32_t n, int32_t width, int32_t height, size_t key_capacity);

/* Offsets of the workspace buffers for the same arguments. */
gs3_status gs3_workspace_layout(int32_t n, int32_t width, int32_t height, size_t key_capacity,
                                gs3_ws_layout *out);

/* Render one relit frame (Sec. 4, Sec. 4.5): shading, shadow splat, Phi, Psi,
 * camera splat and the per-pixel combination.
 *   out_rgb:   device, float32 [height][width][3], caller-owned, overwritten
 *   workspace: device, >= gs3_workspace_size(n, w, h, key_capacity) bytes,
 *              256-byte aligned, caller-owned; holds every intermediate and
 *              the status header.  Calls that overlap on the GPU must use
 *              different workspaces.
 *   stream:    cudaStream_t (void*)
 * Asynchronous.  Host-detectable errors (INVALID_ARG, CUDA launch errors) are
 * returned; a capacity overflow is reported in the workspace header (status
 * GS3_ERR_CAPACITY, the image is then undefined) and is read with
 * gs3_workspace_read_header after the work completes. */
gs3_status gs3_render(gs3_scene *scene, const gs3_camera *camera, const gs3_light *light,
                      const gs3_render_opts *opts, float *out_rgb, void *workspace,
                      size_t workspace_bytes, size_t key_capacity, void *stream);

/* Stage bits of gs3_render_stages (in pipeline order). */
enum {
    GS3_STAGE_PREP = 1,             /* K1: shading colour, both projections, keys */
    GS3_STAGE_CAMERA_BIN = 2,       /* camera splat: depth sort, per-tile lists and ranges, tile launch order */
    GS3_STAGE_LIGHT_BIN = 4,        /* light splat: the same toward the light */
    GS3_STAGE_SHADOW_COMPOSITE = 8, /* shadow rays: biased transmittance, partial sums (Sec. 4.2) */
    GS3_STAGE_SHADOW_REDUCE = 16,   /* per-Gaussian beta-weighted average (Sec. 4.2) */
    GS3_STAGE_MLP = 32,             /* Phi and Psi (Sec. 4.2, 4.3) */
    GS3_STAGE_CAMERA = 64,          /* camera composite and combination (Eq. 2, Sec. 4) */
    GS3_STAGE_ALL = 127
};

/* Run only the selected stages of gs3_render on `workspace`, in pipeline
 * order.  Each stage reads what the earlier stages left in the same
 * workspace, so a frame split into several calls (same scene, camera, light,
 * options and workspace, stages in order, header reset by the call that
 * includes GS3_STAGE_PREP) equals one gs3_render.  Used to time stages with
 * events recorded on `stream` between the calls.
 * A moving camera under a fixed light: the shadow values T (Sec. 4.2) depend
 * on the scene, the light, the image size and the options, not on the
 * camera.  After one full frame on a workspace, GS3_STAGE_PREP |
 * GS3_STAGE_CAMERA_BIN | GS3_STAGE_MLP | GS3_STAGE_CAMERA with another camera
 * (same scene, light, size, options and workspace) equals gs3_render of that
 * view bit for bit, without the light splat.  The header's light pair counts
 * then read 0.  Errors as gs3_render. */
gs3_status gs3_render_stages(gs3_scene *scene, const gs3_camera *camera, const gs3_light *light,
                             const gs3_render_opts *opts, float *out_rgb, void *workspace,
                             size_t workspace_bytes, size_t key_capacity, uint32_t stages,
                             void *stream);

/* Environment light (Sec. 4.5): out_rgb = sum_l weights[l] * (the image
 * gs3_render gives for lights[l]), the lights directional (or point), all
 * rendered as one batched frame.  The camera splat, Psi and the camera
 * composite's weights do not depend on the light and run once; per group of
 * up to 8 lights, the lights' shadow splats run beside one another on
 * sub-streams, Phi runs once over 8 N rows, and one camera composite adds the
 * group's sum_l w_l (S_l Sh_l + R).  Each light's shadow values and refined
 * shadow equal those of its own gs3_render.
 *   lights, weights: host arrays of `count` entries, 1 <= count <= 4096
 *   out_rgb:         device float32 [height][width][3], overwritten
 *   workspace:       device, 256-byte aligned, at least
 *                    gs3_environment_workspace_size(n, width, height, count,
 *                    key_capacity) bytes, caller-owned; its header (start of
 *                    the workspace) then holds the first non-OK status, the
 *                    camera's pair counts and the largest light pair counts
 * Asynchronous on `stream` (sub-streams of the scene, made on the first call,
 * join it).  Calls on one scene from several threads are serialised while
 * they enqueue.  Errors: as gs3_render; GS3_ERR_INVALID_ARG for count out of
 * range or a workspace smaller than the size below. */
size_t gs3_environment_workspace_size(int32_t n, int32_t width, int32_t height, int32_t count,
                                      size_t key_capacity);
gs3_status gs3_render_environment(gs3_scene *scene, const gs3_camera *camera, const gs3_light *lights,
                                  const float *weights, int32_t count, const gs3_render_opts *opts,
                                  float *out_rgb, void *workspace, size_t workspace_bytes,
                                  size_t key_capacity, void *stream);

/* Copy the workspace header to `out` (host) and synchronise `stream`. */
gs3_status gs3_workspace_read_header(const void *workspace, gs3_ws_header *out, void *stream);

/* ---- Backward (differentiation form) -------------------------------------
 * Gradients of a scalar loss L with respect to every parameter, given
 * dL/d(image).  Device float32 arrays in the layouts of gs3_scene_desc
 * (float4-padded, the pad lanes are written as 0), caller-owned, overwritten:
 *   mean_op[N]: (dL/dmu, dL/d opacity logit); scale, rot, shade_rot,
 *   albedo_d, albedo_s [N]; latent [2N]; lobe_rot, lobe_sigma, lobe_amp [K N];
 *   phi_w, phi_b, psi_w, psi_b: packed like the scene's MLP weights. */
typedef struct {
    float *mean_op, *scale, *rot, *shade_rot, *albedo_d, *albedo_s, *latent;
    float *lobe_rot, *lobe_sigma, *lobe_amp;
    float *phi_w, *phi_b, *psi_w, *psi_b;
} gs3_grads;

/* Bytes of the extra backward workspace for a scene. */
size_t gs3_backward_workspace_size(const gs3_scene *scene);

/* Backward of gs3_render (Sec. 4, Eq. 2-5 and the Phi / Psi MLPs): reverse
 * camera composite (per-tile recomputation from the stored final
 * transmittance), MLP backward, reverse shadow sweep from each ray's stored
 * final occluder product, then both projections and the shading.
 *   dL_drgb:   device float32 [height][width][3]
 *   workspace: the workspace of a gs3_render of the same scene, camera,
 *              light and options, unchanged since (it holds the forward state)
 *   bwd_ws:    device, >= gs3_backward_workspace_size bytes, caller-owned
 * The MLP gradients are those of the scene's FP32 networks evaluated at the
 * forward's inputs (their GEMMs on the tensor cores in three-pass TF32,
 * about FP32 accuracy); for a BF16 or FP8 scene the rest of the backward
 * uses the forward's reduced-precision T' and residual, so the rounding of
 * the MLP operands passes straight through.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
gs3_status gs3_render_backward(gs3_scene *scene, const gs3_camera *camera, const gs3_light *light,
                               const gs3_render_opts *opts, const float *dL_drgb, void *workspace,
                               size_t workspace_bytes, size_t key_capacity, void *bwd_ws,
                               size_t bwd_bytes, const gs3_grads *grads, void *stream);

/* Loss of Sec. 4.4 and its image gradient:
 *   L = (1 - lambda) mean|I - I*| + lambda (1 - SSIM(I, I*)),
 * SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
 * zero padding, averaged over pixels and channels (lambda = 0.2 in the paper).
 *   img, target: device float32 [height][width][3]
 *   loss_out:    device float32 [1]
 *   dL_dimg:     device float32 [height][width][3], overwritten
 *   scratch:     device, >= gs3_loss_scratch_size(width, height) bytes
 * Asynchronous; deterministic (fixed-order reductions). */
size_t gs3_loss_scratch_size(int32_t width, int32_t height);
gs3_status gs3_loss_l1_dssim(const float *img, const float *target, int32_t width, int32_t height,
                             float lambda, float *loss_out, float *dL_dimg, void *scratch,
                             size_t scratch_bytes, void *stream);

/* One Adam step (Kingma and Ba; the optimiser of Sec. 4.4) on n parameters,
 * in place:  m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *            p = max(lower_bound, p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)).
 *   param, m, v: device float32 [n], updated;  grad: device float32 [n]
 *   step: t >= 1 (bias correction);  lower_bound: -INFINITY for none
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
gs3_status gs3_adam_step(float *param, const float *grad, float *m, float *v, size_t n, float lr,
                         float beta1, float beta2, float eps, int32_t step, float lower_bound, void *stream);

/* ---- Continuous-batching server -----------------------------------------
 * Serving form of gs3_render (no counterpart in the paper, which renders one
 * frame at a time): a worker thread keeps a queue of (scene, camera, light)
 * requests and max_inflight slots.  A free slot takes up to max_batch
 * requests from the head of the queue whose workspaces fit in the HBM budget
 * and renders them as one batch: each frame's shading, projections and
 * binning on its own sub-stream, then the shadow composite's persistent
 * segment kernels and the camera composite over every frame of the batch in
 * single launches.  Requests that arrive while batches are on the GPU join
 * the next free slot's batch; the slots' batches overlap on the device.  Each
 * frame equals the same frame rendered alone by gs3_render, bit for bit.  The
 * workspace capacity is estimated per (scene, resolution) from the pair
 * counts seen so far; a request that overflows it is re-admitted once with
 * the exact count.  Latency is measured from gs3_server_submit to the
 * completion of the request's batch on the GPU. */
enum { GS3_REQ_QUEUED = 0, GS3_REQ_RUNNING = 1, GS3_REQ_DONE = 2, GS3_REQ_FAILED = 3 };

typedef struct {
    size_t hbm_budget;             /* bytes of workspace admitted requests may hold together */
    int32_t max_inflight;          /* in-flight slots (streams), 1..64 */
    int32_t device;                /* CUDA device of every scene added */
    int32_t inject_alloc_failures; /* testing: fail this many workspace allocations (0 in use) */
    float initial_pairs;           /* first-request capacity guess: pairs per Gaussian at 800x800,
                                      scaled with the pixel count (0: 64) */
    int32_t max_batch;             /* requests rendered together by one slot, 1..8 (0: 1: every
                                      request alone on its slot's streams) */
    int32_t light_cache;           /* 0..4096: shadow values kept for this many (scene, light,
                                      image size, options) keys (0: none).  A request alone on its
                                      slot whose key is kept copies them into its workspace and runs
                                      only the camera-side stages (gs3_render_stages); its image
                                      still equals its gs3_render bit for bit.  When all keys are
                                      taken, the least recently used one that no admitted request
                                      reads is dropped.  Each key holds 4 n bytes of device memory
                                      outside the budget. */
} gs3_server_opts;

typedef struct {
    uint64_t completed, failed, retries, queued, in_flight, max_in_flight;
    uint64_t bytes_in_use, peak_bytes_in_use;
    double device_span_ms; /* CUDA-event time from the first admitted batch's start to the
                              last completed batch's end since the last reset */
    uint64_t batches;      /* batches launched */
    uint64_t max_batch;    /* the most requests one batch held */
    uint64_t light_reuse;  /* requests rendered from kept shadow values (light_cache) */
} gs3_server_counters;

typedef struct gs3_server gs3_server;

/* Create a server and start its worker thread.  Errors: INVALID_ARG, CUDA. */
gs3_status gs3_server_create(const gs3_server_opts *opts, gs3_server **out);

/* Register a scene (borrowed; it must outlive the server).  Not thread-safe
 * against concurrent gs3_destroy_scene of the same scene. */
gs3_status gs3_server_add_scene(gs3_server *server, gs3_scene *scene, int32_t *scene_id);

/* Queue one frame.  camera, light, opts: host structs, copied.  out_rgb:
 * device float32 [height][width][3], caller-owned, written when the request
 * completes.  The server's streams do not wait for work queued on other
 * streams: nothing may still be writing out_rgb when it is submitted (the
 * caller synchronises first), and it must stay allocated until the request
 * completes.  Returns at once with a ticket.  Errors: INVALID_ARG. */
gs3_status gs3_server_submit(gs3_server *server, int32_t scene_id, const gs3_camera *camera,
                             const gs3_light *light, const gs3_render_opts *opts, float *out_rgb,
                             uint64_t *ticket);

/* Non-blocking state (GS3_REQ_*) and latency of a ticket.  A finished ticket
 * is forgotten after this call reports it; the return value is the request's
 * own status (GS3_OK unless it failed: OOM when its workspace could not be
 * allocated or can never fit the budget, CAPACITY, CUDA). */
gs3_status gs3_server_poll(gs3_server *server, uint64_t ticket, int32_t *state, double *latency_ms);

/* Block until the ticket finishes or timeout_s passes (GS3_ERR_TIMEOUT);
 * returns the request's status and forgets the ticket. */
gs3_status gs3_server_wait(gs3_server *server, uint64_t ticket, double timeout_s, double *latency_ms);

/* Counters of the server since creation. */
gs3_status gs3_server_stats(gs3_server *server, gs3_server_counters *out);

/* Zero the counters and the device time span (call while the server is idle). */
gs3_status gs3_server_reset_counters(gs3_server *server);

/* Stop the worker, wait for in-flight work, release streams and memory.
 * Queued requests that were never admitted are dropped. */
gs3_status gs3_server_destroy(gs3_server *server);

/* ---- Depth sort without allocation --------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory at all: a renderer embedded in a host
 * application that owns the GPU's memory budget, or a real-time loop that
 * must never risk an allocation stall or an out-of-memory failure in the
 * middle of a frame.  It is the per-splat depth sort of gs3_render (stable
 * ascending order of 32-bit keys, the FP32 depth or light-distance bits) with
 * its scratch in a file-scope device array of GS3_STATIC_SORT_MAX_KEYS keys
 * (about 12.3 MB), which every GPU that loads the library holds until exit.
 *   keys:      device, uint32[n], read only
 *   order_out: device, uint32[n], caller-owned; receives the permutation
 *              order_out[r] = position of the r-th smallest key (ties in
 *              input order), the same as the workspace `order` of gs3_render
 *   n:         0 <= n <= GS3_STATIC_SORT_MAX_KEYS; larger n returns
 *              GS3_ERR_INVALID_ARG (message in gs3_last_error) and launches
 *              nothing
 * Calls no cudaMalloc, cudaFree or other allocating routine.  The first call
 * on a device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it with the id of the device's CUDA
 * context.  After a cudaDeviceReset the module may load elsewhere in the new
 * context: the first call there sees another context id and looks the
 * address up again.  Make the first call on a device, and the first after a
 * reset, before any stream capture.  Every call on a device shares the one
 * array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Nothing in the array needs to start at zero:
 * each pass overwrites all scratch it reads. */
#define GS3_STATIC_SORT_MAX_KEYS 1048576u
gs3_status gs3_depth_order_static(const uint32_t *keys, uint32_t n, uint32_t *order_out, void *stream);

/* ---- Self-test of the bounded device waits ------------------------------
 * Not an operation of the paper: a check that a device-side wait which can
 * never end gives up instead of holding the GPU.  Runs one pass of the
 * look-back radix sort that gs3_render's depth sorts use (each block waits
 * for the digit counts of the blocks before it; here with blocks of 4096
 * keys) over n zero keys in scratch it
 * allocates and frees, with the block tickets starting at 1, so the waits
 * reach ticket 0's words, which no block writes.  Each such wait gives up
 * after its poll bound (well under a second) and the pass records
 * GS3_ERR_TIMEOUT, then finishes; the context stays usable.
 *   n:          4096 < n <= 1048576 (at least two blocks of 4096 keys)
 *   status_out: host, one uint32: the pass's status word, GS3_ERR_TIMEOUT
 *               when the bounded wait works
 * Synchronous (synchronises the device).  GS3_ERR_INVALID_ARG for n out of
 * range or a null status_out; GS3_ERR_OOM or GS3_ERR_CUDA (message in
 * gs3_last_error) when the scratch allocation or a CUDA call fails. */
gs3_status gs3_selftest_wait_timeout(uint32_t n, uint32_t *status_out);

/* ---- Measured ALU peaks --------------------------------------------------
 * Not an operation of the paper: the denominators of the roofline of the
 * ALU-bound composites, whose every (pixel, splat) test is FP32 fused
 * multiply-adds, a compare and one MUFU ex2.  Times two micro-kernels that
 * fill every SM (64 warps each, eight independent dependency chains per
 * thread) with CUDA events on the legacy default stream: FP32 FMA (2 FLOP
 * each) and ex2.approx, and reports the best of `repeats` launches after one
 * warm-up launch of each.
 *   ffma_tflops: host, FP32 FMA throughput in TFLOP/s
 *   ex2_gops:    host, ex2 throughput in G operations/s
 * The figures hold for the SM clock during the call.  Synchronous (allocates
 * and frees a small output buffer).  Errors: INVALID_ARG (null output,
 * repeats outside [1, 100]), CUDA. */
gs3_status gs3_measure_alu_peak(int32_t repeats, double *ffma_tflops, double *ex2_gops);

/* Not an operation of the paper either: a check that the shadow composite's
 * chain of segment products gives up instead of holding the GPU when a
 * predecessor never publishes.  Runs the frame's shading, projections and
 * light binning (the checks and workspace of gs3_render_stages), then the
 * chain kernel with its work tickets starting past every tile's first
 * segment, so that the waits of every second segment can never end: each
 * gives up after its poll bound (well under a second), records
 * GS3_ERR_TIMEOUT and publishes its rays as stopped.
 *   status_out: host, one uint32: the workspace's status word afterwards,
 *               GS3_ERR_TIMEOUT when the bounded waits work (a frame whose
 *               light tiles all hold one segment has nothing to wait for)
 * Synchronous (synchronises the device); the context stays usable.  Errors:
 * as gs3_render_stages, INVALID_ARG for a null status_out or a shadow-splat
 * ablation, CUDA. */
gs3_status gs3_selftest_shadow_wait(gs3_scene *scene, const gs3_camera *camera, const gs3_light *light,
                                    const gs3_render_opts *opts, void *workspace, size_t workspace_bytes,
                                    size_t key_capacity, uint32_t *status_out);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices); a host-side counter for launch accounting. */
uint64_t gs3_kernel_launches(void);

/* Message of the last error on the calling thread ("" if none). */
const char *gs3_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GS3_H */
