// C ABI of libgs3 (declared in include/gs3.h): validation, workspace layout
// and the stream-ordered launch sequence of one frame.
#include <atomic>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>

#include "gs3_internal.cuh"


namespace gs3 {

std::atomic<uint64_t> g_launches{0};

namespace {
thread_local std::string g_last_error;
}  // namespace

gs3_status fail(gs3_status st, const char* msg) {
  g_last_error = msg;
  return st;
}

gs3_status cuda_fail(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_last_error = buf;
  return GS3_ERR_CUDA;
}

// Why a light cannot be rendered, or null.
const char* light_problem(const gs3_light& l, const gs3_render_opts& o) {
  if (l.type == GS3_LIGHT_POINT) {
    const float tl[3] = {o.target[0] - l.pos[0], o.target[1] - l.pos[1], o.target[2] - l.pos[2]};
    if (!(tl[0] * tl[0] + tl[1] * tl[1] + tl[2] * tl[2] >= 1e-12f))
      return "gs3_render: light coincides with the light-camera target";
    return nullptr;
  }
  if (l.type != GS3_LIGHT_DIRECTIONAL) return "gs3_render: light type must be GS3_LIGHT_POINT or GS3_LIGHT_DIRECTIONAL";
  if (!(l.dir[0] * l.dir[0] + l.dir[1] * l.dir[1] + l.dir[2] * l.dir[2] >= 1e-12f))
    return "gs3_render: directional light needs a non-zero direction";
  if (!(l.extent > 0.f) || !(l.extent < 1e30f)) return "gs3_render: directional light needs extent > 0";
  return nullptr;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Planner {
  size_t cur = 0;
  size_t take(size_t bytes) {
    size_t o = cur;
    cur = align256(cur + (bytes ? bytes : 1));
    return o;
  }
};

bool mlp_ok(const gs3_mlp_desc& m, int in_dim, int out_dim) {
  if (m.in_dim != in_dim || m.out_dim != out_dim) return false;
  if (m.n_hidden < 1 || m.n_hidden > 4) return false;
  if (m.width != 16 && m.width != 32 && m.width != 64 && m.width != 128) return false;
  if (m.act != GS3_ACT_RELU && m.act != GS3_ACT_LEAKY_RELU) return false;
  return m.w && m.b;
}

}  // namespace

void set_last_error(const char* msg) { g_last_error = msg; }

// True unless the driver reports that [ptr, ptr + bytes) leaves the device
// allocation containing ptr (memory from sub-allocators such as torch's
// caching allocator is checked against its whole segment).
bool device_range_ok(const void* ptr, size_t bytes) {
  typedef int (*range_fn)(unsigned long long*, size_t*, unsigned long long);
  static const range_fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<range_fn>(f);
    return (range_fn) nullptr;
  }();
  if (!fn || !ptr) return true;
  unsigned long long base = 0;
  size_t size = 0;
  if (fn(&base, &size, reinterpret_cast<unsigned long long>(ptr)) != 0) return false;  // not device memory
  const unsigned long long p = reinterpret_cast<unsigned long long>(ptr);
  return p >= base && p - base + bytes <= size;
}

int device_sm_count() {
  static std::atomic<int> cached[kMaxDevices];
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0) return 1;
  if (d < kMaxDevices) {
    const int c = cached[d].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v < 1) return 1;
  if (d < kMaxDevices) cached[d].store(v, std::memory_order_relaxed);
  return v;
}

Workspace plan_workspace(int n, int width, int height, size_t cap) {
  Workspace L;
  L.n = n;
  L.width = width;
  L.height = height;
  L.gx = (width + kTile - 1) / kTile;
  L.gy = (height + kTile - 1) / kTile;
  L.ntiles = L.gx * L.gy;
  L.cap = cap;
  L.nb_n = (int)((n + kDepthSortItems - 1) / kDepthSortItems);
  L.nb_rows = (int)((n + kBinBlock - 1) / kBinBlock);
  const size_t N = (size_t)n;
  const size_t scan_words = scan_scratch_words(N);  // the scan of the tile counts
  Planner P;
  L.header = P.take(256);
  for (int s = 0; s < 2; ++s) {
    SplatBufs& b = L.sp[s];
    b.key = P.take(4 * N);
    b.sk[0] = P.take(4 * N);
    b.sk[1] = P.take(4 * N);
    b.sv[0] = P.take(4 * N);
    b.sv[1] = P.take(4 * N);
    b.order = b.sv[1];
    b.rank_of = P.take(4 * N);
    b.rect = P.take(16 * N);
    b.rec = P.take(sizeof(SplatRec) * N);
    b.rrec = P.take(sizeof(SplatRec) * N);
    b.cnt = P.take(4 * N);
    b.off = P.take(4 * N);
    b.tk[0] = P.take(4 * cap);
    b.tk[1] = P.take(4 * cap);
    b.tv[0] = P.take(4 * cap);
    b.tv[1] = P.take(4 * cap);
    b.tile_start = P.take(4 * ((size_t)L.ntiles + 1));
    b.scan_part = P.take(4 * scan_words);
    b.dlook = P.take(onesweep_bytes(L.nb_n, 4));
    b.row_cnt = P.take(4 * (size_t)L.gy * (size_t)L.nb_rows);
    b.bin_plan = P.take(4 * (3 * (size_t)L.gy + 3));
    b.bin_tab = P.take(4 * bin_tab_words(cap, L.gx, L.gy));
  }
  L.partial = P.take(8 * cap);
  L.tile_order[0] = P.take(4 * (size_t)L.ntiles);
  L.tile_order[1] = P.take(4 * (size_t)L.ntiles);
  const size_t items = shadow_seg_items(L.ntiles, cap);
  L.seg_lvl = P.take(4 * (1025 + 3));
  L.seg_flag = P.take(4 * items);
  L.seg_pub = P.take(4 * 256 * items);
  L.rank_flags = P.take(2 * N);
  L.shade = P.take(16 * N);
  L.T = P.take(4 * N);
  L.Tp = P.take(4 * N);
  L.res = P.take(16 * N);
  L.ccol = P.take(32 * N);
  L.final_t = P.take(4 * (size_t)width * height);
  L.n_contrib = P.take(4 * (size_t)width * height);
  L.pix_aux = P.take(32 * (size_t)width * height);
  L.light_final = P.take(4 * (size_t)width * height);
  L.light_stop = P.take(4 * (size_t)width * height);
  L.shadow_den = P.take(4 * N);
  L.total = P.cur;
  return L;
}

}  // namespace gs3

using namespace gs3;

extern "C" {

const char* gs3_last_error(void) { return g_last_error.c_str(); }

uint64_t gs3_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void gs3_default_opts(gs3_render_opts* o) {
  if (!o) return;
  o->near_z = 0.2f;
  o->lowpass = 0.3f;
  o->frustum = 1.3f;
  o->shadow_bias = 0.015f;
  o->alpha_min = 1.0f / 255.0f;
  o->alpha_max = 0.99f;
  o->t_stop = 1e-4f;
  o->target[0] = o->target[1] = o->target[2] = 0.f;
  o->falloff = 1;
  o->tile = kTile;
  o->ablate = 0;
}

gs3_status gs3_create_scene(const gs3_scene_desc* d, gs3_scene** out) {
  if (!d || !out) return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: null argument");
  *out = nullptr;
  if (d->n < 1) return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: n must be >= 1");
  if (d->k < 0 || d->k > kMaxLobes) return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: k must be in [0, 16]");
  if (!d->mean_op || !d->scale || !d->rot || !d->shade_rot || !d->albedo_d || !d->albedo_s || !d->latent)
    return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: null parameter array");
  if (d->k > 0 && (!d->lobe_rot || !d->lobe_sigma || !d->lobe_amp))
    return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: null lobe array");
  if (!mlp_ok(d->phi, 61, 1)) return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: unsupported Phi shape");
  if (!mlp_ok(d->psi, 60, 3)) return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: unsupported Psi shape");
  if (d->mlp_dtype != GS3_MLP_FP32 && d->mlp_dtype != GS3_MLP_BF16 && d->mlp_dtype != GS3_MLP_FP8_E4M3)
    return fail(GS3_ERR_INVALID_ARG,
                "gs3_create_scene: mlp_dtype must be GS3_MLP_FP32, GS3_MLP_BF16 or GS3_MLP_FP8_E4M3");
  gs3_scene* s = new (std::nothrow) gs3_scene;
  if (!s) return fail(GS3_ERR_OOM, "gs3_create_scene: host allocation failed");
  SceneDev& v = s->dev;
  v.n = d->n;
  v.k = d->k;
  auto f4 = [](const float* p) { return reinterpret_cast<const float4*>(p); };
  v.mean_op = f4(d->mean_op);
  v.scale = f4(d->scale);
  v.rot = f4(d->rot);
  v.shade_rot = f4(d->shade_rot);
  v.albedo_d = f4(d->albedo_d);
  v.albedo_s = f4(d->albedo_s);
  v.latent = f4(d->latent);
  v.lobe_rot = f4(d->lobe_rot);
  v.lobe_sigma = f4(d->lobe_sigma);
  v.lobe_amp = f4(d->lobe_amp);
  v.phi = {d->phi.in_dim, d->phi.width, d->phi.n_hidden, d->phi.out_dim, d->phi.act, d->phi.w, d->phi.b};
  v.psi = {d->psi.in_dim, d->psi.width, d->psi.n_hidden, d->psi.out_dim, d->psi.act, d->psi.w, d->psi.b};
  v.mlp_dtype = d->mlp_dtype;
  if (d->lobe_shared != 0 && d->lobe_shared != 1) {
    delete s;
    return fail(GS3_ERR_INVALID_ARG, "gs3_create_scene: lobe_shared must be 0 or 1");
  }
  v.lobe_shared = d->lobe_shared;
  if (d->mlp_dtype != GS3_MLP_FP32) {
    for (int w = 0; w < 2; ++w) {
      const MlpDev& m = w == 0 ? v.phi : v.psi;
      if (!mlp_tc_supported(m, d->mlp_dtype)) {
        gs3_destroy_scene(s);
        return fail(GS3_ERR_UNSUPPORTED, "gs3_create_scene: MLP shape not supported by the tensor-core path");
      }
      if (cudaMalloc(&s->tc_blob[w], mlp_tc_blob_bytes(m, d->mlp_dtype)) != cudaSuccess) {
        s->tc_blob[w] = nullptr;
        gs3_destroy_scene(s);
        return fail(GS3_ERR_OOM, "gs3_create_scene: tensor-core weight allocation failed");
      }
      pack_mlp_tc(m, d->mlp_dtype, v, w, s->tc_blob[w], 0);
    }
    cudaError_t e = cudaStreamSynchronize(0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      gs3_destroy_scene(s);
      return cuda_fail(e, "gs3_create_scene: tensor-core weight packing");
    }
  }
  *out = s;
  return GS3_OK;
}

gs3_status gs3_scene_mlp_scales(const gs3_scene* s, int32_t which, float* out, int32_t cap) {
  if (!s || !out || (which != 0 && which != 1)) return fail(GS3_ERR_INVALID_ARG, "gs3_scene_mlp_scales: bad argument");
  if (s->dev.mlp_dtype != GS3_MLP_FP8_E4M3)
    return fail(GS3_ERR_UNSUPPORTED, "gs3_scene_mlp_scales: the scene's MLPs are not FP8");
  const MlpDev& m = which == 0 ? s->dev.phi : s->dev.psi;
  if (cap < 2 * m.n_hidden) return fail(GS3_ERR_INVALID_ARG, "gs3_scene_mlp_scales: out holds fewer than 2 n_hidden");
  const cudaError_t e = cudaMemcpy(out, s->tc_blob[which] + mlp_tc_scale_offset(m, s->dev.mlp_dtype),
                                   sizeof(float) * 2 * m.n_hidden, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GS3_OK : cuda_fail(e, "gs3_scene_mlp_scales");
}

gs3_status gs3_destroy_scene(gs3_scene* s) {
  if (!s) return GS3_OK;
  if (s->env_ready) s->env_bs.destroy();
  for (int w = 0; w < 2; ++w)
    if (s->tc_blob[w]) cudaFree(s->tc_blob[w]);
  delete s;
  return GS3_OK;
}

size_t gs3_workspace_size(int32_t n, int32_t width, int32_t height, size_t key_capacity) {
  if (n < 1 || width < 1 || height < 1) return 0;
  return plan_workspace(n, width, height, key_capacity).total;
}

gs3_status gs3_workspace_layout(int32_t n, int32_t width, int32_t height, size_t key_capacity,
                                gs3_ws_layout* out) {
  if (!out || n < 1 || width < 1 || height < 1) return fail(GS3_ERR_INVALID_ARG, "gs3_workspace_layout: bad argument");
  Workspace L = plan_workspace(n, width, height, key_capacity);
  out->total = L.total;
  out->header = L.header;
  const int fin = (L.ntiles <= 256 ? 1 : 2) & 1;
  for (int s = 0; s < 2; ++s) {
    out->key[s] = L.sp[s].key;
    out->order[s] = L.sp[s].order;
    out->tile_start[s] = L.sp[s].tile_start;
    out->list[s] = L.sp[s].tv[fin];
    out->rect[s] = L.sp[s].rect;
  }
  out->shade = L.shade;
  out->shadow = L.T;
  out->shadow_refined = L.Tp;
  out->residual = L.res;
  out->final_t = L.final_t;
  out->n_contrib = L.n_contrib;
  out->light_final = L.light_final;
  out->light_stop = L.light_stop;
  return GS3_OK;
}

gs3_status gs3_render_stages(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                             const gs3_render_opts* opts, float* out_rgb, void* workspace, size_t ws_bytes,
                             size_t key_capacity, uint32_t stages, void* stream) {
  // a whole frame forks its light chain onto the calling thread's side stream
  SideStream* side = stages == GS3_STAGE_ALL ? thread_side_stream() : nullptr;
  return render_frame(scene, cam, light, opts, out_rgb, workspace, ws_bytes, key_capacity, stages,
                      reinterpret_cast<cudaStream_t>(stream), side);
}

}  // extern "C"

namespace gs3 {

bool SideStream::create() {
  if (s) return true;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { s = nullptr; return false; }
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
    destroy();
    return false;
  }
  return true;
}

void SideStream::destroy() {
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (s) cudaStreamDestroy(s);
  s = nullptr;
  fork = join = nullptr;
}

SideStream* thread_side_stream() {
  struct PerThread {
    SideStream dev[64];
    ~PerThread() {}  // streams live until the process ends (a thread may exit mid-use elsewhere)
  };
  thread_local PerThread t;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
  return t.dev[d].create() ? &t.dev[d] : nullptr;
}

gs3_status render_frame(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                        const gs3_render_opts* opts, float* out_rgb, void* workspace, size_t ws_bytes,
                        size_t key_capacity, uint32_t stages, cudaStream_t stream, SideStream* side) {
  if (!scene || !cam || !light || !opts || !out_rgb || !workspace)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: null argument");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: image size out of range");
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(GS3_ERR_INVALID_ARG, "gs3_render: focal length must be > 0");
  if (opts->tile != kTile) return fail(GS3_ERR_INVALID_ARG, "gs3_render: tile must be 16");
  if (key_capacity < 1 || key_capacity > 0x7FFFFFFFull)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: key_capacity must be in [1, 2^31)");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: workspace must be 256-byte aligned");
  const int ntiles = ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
  if (ntiles > 65536) return fail(GS3_ERR_INVALID_ARG, "gs3_render: more than 65536 tiles");
  if ((double)scene->dev.n * (double)ntiles >= 4294967295.0)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: n * tiles must stay below 2^32");
  {
    const char* why = light_problem(*light, *opts);
    if (why) return fail(GS3_ERR_INVALID_ARG, why);
  }
  Workspace L = plan_workspace(scene->dev.n, cam->width, cam->height, key_capacity);
  if (ws_bytes < L.total) return fail(GS3_ERR_INVALID_ARG, "gs3_render: workspace too small");
  if (!device_range_ok(workspace, L.total))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: workspace is not device memory of the stated size");
  if ((stages & GS3_STAGE_CAMERA) &&
      !device_range_ok(out_rgb, (size_t)cam->width * cam->height * 3 * sizeof(float)))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render: out_rgb is not device memory of width*height*3 floats");
  cudaStream_t s = stream;
  FrameArgs f;
  f.sc = scene->dev;
  f.cam = *cam;
  f.light = *light;
  f.opts = *opts;
  f.ws = static_cast<unsigned char*>(workspace);
  f.L = &L;
  cudaError_t e = cudaSuccess;
  const bool no_shadow = (opts->ablate & GS3_ABLATE_SHADOW_SPLAT) != 0;
  if (stages & GS3_STAGE_PREP) {
    e = cudaMemsetAsync(f.ws + L.header, 0, 4 * H_RESET_WORDS, s);
    if (e != cudaSuccess) return cuda_fail(e, "gs3_render: header reset");
    launch_prep(f, s);
  }
  // The light chain (light binning, shadow composite, shadow reduce) and the
  // camera binning use disjoint buffers: with a side stream they overlap.
  const bool fork = side && !no_shadow && (stages & GS3_STAGE_CAMERA_BIN) && (stages & GS3_STAGE_LIGHT_BIN);
  cudaStream_t sl = s;
  if (fork) {
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->s, side->fork, 0);
    sl = side->s;
  }
  if ((stages & GS3_STAGE_LIGHT_BIN) && !no_shadow) {
    launch_depth_sort(f, 1, sl);
    launch_binning(f, 1, sl);
  }
  if ((stages & GS3_STAGE_SHADOW_COMPOSITE) && !no_shadow) launch_shadow_composite(f, sl);
  if (stages & GS3_STAGE_SHADOW_REDUCE) {
    if (no_shadow) launch_fill_shadow_one(f, sl);
    else launch_shadow_reduce(f, sl);
  }
  if (stages & GS3_STAGE_CAMERA_BIN) {
    launch_depth_sort(f, 0, s);
    launch_binning(f, 0, s);
    launch_tile_order(f, 0, s);  // the camera composite's launch order
  }
  if (fork) {
    cudaEventRecord(side->join, sl);
    cudaStreamWaitEvent(s, side->join, 0);
  }
  if (stages & GS3_STAGE_MLP) {
    if (scene->dev.mlp_dtype != GS3_MLP_FP32) {
      launch_mlp(f, s, /*identity_only=*/true);
      const unsigned char* blobs[2] = {scene->tc_blob[0], scene->tc_blob[1]};
      launch_mlp_tc(f, blobs, s);
    } else {
      launch_mlp(f, s);
    }
  }
  if (stages & GS3_STAGE_CAMERA) launch_camera_composite(f, out_rgb, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gs3_render: launch");
  return GS3_OK;
}

bool BatchStreams::create(int n) {
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork2, cudaEventDisableTiming) != cudaSuccess)
    return false;
  if (cudaEventCreateWithFlags(&cam, cudaEventDisableTiming) != cudaSuccess) return false;
  for (int r = 0; r < n; ++r) {
    if (cudaStreamCreateWithFlags(&sub[r], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&join[r], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join2[r], cudaEventDisableTiming) != cudaSuccess)
      return false;
  }
  return true;
}

void BatchStreams::destroy() {
  for (int r = 0; r < 8; ++r) {
    if (sub[r]) cudaStreamDestroy(sub[r]);
    if (join[r]) cudaEventDestroy(join[r]);
    if (join2[r]) cudaEventDestroy(join2[r]);
    sub[r] = nullptr;
    join[r] = join2[r] = nullptr;
  }
  if (fork) cudaEventDestroy(fork);
  if (fork2) cudaEventDestroy(fork2);
  if (cam) cudaEventDestroy(cam);
  fork = fork2 = cam = nullptr;
}

// A batch of frames rendered together (the serving form; each frame has its
// own workspace and equals the same frame rendered alone, bit for bit):
//   1. per frame, on its own sub-stream: header reset, shading and both
//      projections (K1), the light binning and the shadow composite's
//      per-frame set-up (occluder bounds, segment plan), then the camera
//      binning, which runs beside step 2;
//   2. on `stream`: the shadow composite's three persistent segment kernels
//      over every segment of every frame, from shared tickets;
//   3. per frame, on its sub-stream again: the shadow reduce and the MLPs;
//   4. on `stream`: one camera composite over every frame's tiles.
gs3_status render_batch(const BatchFrame* frames, int n, cudaStream_t s, BatchStreams& bs,
                        unsigned char* param_dev, unsigned char* param_host) {
  if (n < 1 || n > kMaxBatch) return fail(GS3_ERR_INVALID_ARG, "render_batch: 1 <= n <= 8 frames");
  Workspace L[kMaxBatch];
  FrameArgs f[kMaxBatch];
  for (int r = 0; r < n; ++r) {
    const BatchFrame& b = frames[r];
    if (!b.scene || !b.out || !b.ws || b.opts.tile != kTile || b.cam.width < 1 || b.cam.height < 1 ||
        b.cam.width > 16384 || b.cam.height > 16384 || !(b.cam.fx > 0.f) || !(b.cam.fy > 0.f))
      return fail(GS3_ERR_INVALID_ARG, "render_batch: bad frame");
    if (light_problem(b.light, b.opts)) return fail(GS3_ERR_INVALID_ARG, light_problem(b.light, b.opts));
    L[r] = plan_workspace(b.scene->dev.n, b.cam.width, b.cam.height, b.cap);
    if (b.ws_bytes < L[r].total || reinterpret_cast<uintptr_t>(b.ws) % 256 != 0)
      return fail(GS3_ERR_INVALID_ARG, "render_batch: workspace too small or misaligned");
    f[r].sc = b.scene->dev;
    f[r].cam = b.cam;
    f[r].light = b.light;
    f[r].opts = b.opts;
    f[r].ws = static_cast<unsigned char*>(b.ws);
    f[r].L = &L[r];
  }
  (void)cudaGetLastError();  // only this call's launches are checked below
  // 1. per-frame stages beside one another: the light chain first (the batch's
  //    shadow composite waits for it), then the camera binning, which runs on
  //    beside the shadow composite
  cudaEventRecord(bs.fork, s);
  const FrameArgs* shadowed[kMaxBatch];
  int ns = 0;
  for (int r = 0; r < n; ++r) {
    cudaStream_t sr = bs.sub[r];
    cudaStreamWaitEvent(sr, bs.fork, 0);
    cudaMemsetAsync(f[r].ws + L[r].header, 0, 4 * H_RESET_WORDS, sr);
    launch_prep(f[r], sr);
    if (!(f[r].opts.ablate & GS3_ABLATE_SHADOW_SPLAT)) {
      launch_depth_sort(f[r], 1, sr);
      launch_binning(f[r], 1, sr);
      prepare_shadow_composite(f[r], sr);
      shadowed[ns++] = &f[r];
    }
    cudaEventRecord(bs.join[r], sr);
    launch_depth_sort(f[r], 0, sr);
    launch_binning(f[r], 0, sr);
    launch_tile_order(f[r], 0, sr);
  }
  for (int r = 0; r < n; ++r) cudaStreamWaitEvent(s, bs.join[r], 0);
  // 2. the shadow composite of the whole batch
  if (ns > 0) launch_shadow_composite_batch(shadowed, ns, param_dev, param_host, s);
  // 3. per frame (after its camera binning): shadow average and the MLPs
  cudaEventRecord(bs.fork2, s);
  for (int r = 0; r < n; ++r) {
    cudaStream_t sr = bs.sub[r];
    cudaStreamWaitEvent(sr, bs.fork2, 0);
    if (f[r].opts.ablate & GS3_ABLATE_SHADOW_SPLAT) launch_fill_shadow_one(f[r], sr);
    else launch_shadow_reduce(f[r], sr);
    const gs3_scene* sc = frames[r].scene;
    if (sc->dev.mlp_dtype != GS3_MLP_FP32) {
      launch_mlp(f[r], sr, /*identity_only=*/true);
      const unsigned char* blobs[2] = {sc->tc_blob[0], sc->tc_blob[1]};
      launch_mlp_tc(f[r], blobs, sr);
    } else {
      launch_mlp(f[r], sr);
    }
    cudaEventRecord(bs.join2[r], sr);
  }
  for (int r = 0; r < n; ++r) cudaStreamWaitEvent(s, bs.join2[r], 0);
  // 4. the camera composite of the whole batch
  const FrameArgs* all[kMaxBatch];
  float* outs[kMaxBatch];
  for (int r = 0; r < n; ++r) {
    all[r] = &f[r];
    outs[r] = frames[r].out;
  }
  launch_camera_composite_batch(all, outs, n, param_dev, param_host, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "render_batch: launch");
  return GS3_OK;
}

}  // namespace gs3

extern "C" {

gs3_status gs3_render(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                      const gs3_render_opts* opts, float* out_rgb, void* workspace, size_t ws_bytes,
                      size_t key_capacity, void* stream) {
  return gs3_render_stages(scene, cam, light, opts, out_rgb, workspace, ws_bytes, key_capacity,
                           GS3_STAGE_ALL, stream);
}

size_t gs3_backward_workspace_size(const gs3_scene* scene) {
  if (!scene) return 0;
  return backward_workspace_bytes(scene->dev.n, scene->dev.phi, scene->dev.psi);
}

// light camera of the frame, the same FP32 recipe as the forward kernel's

gs3_status gs3_render_backward(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                               const gs3_render_opts* opts, const float* dimg, void* workspace,
                               size_t ws_bytes, size_t key_capacity, void* bws, size_t bws_bytes,
                               const gs3_grads* grads, void* stream) {
  if (!scene || !cam || !light || !opts || !dimg || !workspace || !bws || !grads)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: null argument");
  if (cam->width < 1 || cam->height < 1 || opts->tile != kTile)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: bad camera or options");
  if (light_problem(*light, *opts)) return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: invalid light");
  Workspace L = plan_workspace(scene->dev.n, cam->width, cam->height, key_capacity);
  if (ws_bytes < L.total || !device_range_ok(workspace, L.total))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: workspace too small");
  if (!device_range_ok(dimg, (size_t)cam->width * cam->height * 3 * sizeof(float)))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: dL_drgb is not width*height*3 floats");
  const size_t need = backward_workspace_bytes(scene->dev.n, scene->dev.phi, scene->dev.psi);
  if (bws_bytes < need || !device_range_ok(bws, need))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_backward: backward workspace too small");
  FrameArgs f;
  f.sc = scene->dev;
  f.cam = *cam;
  f.light = *light;
  f.opts = *opts;
  f.ws = static_cast<unsigned char*>(workspace);
  f.L = &L;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  gs3_status st = run_backward(f, dimg, bws, bws_bytes, *grads, s, thread_side_stream());
  if (st != GS3_OK) return fail(st, "gs3_render_backward: bad workspace");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gs3_render_backward: launch");
  return GS3_OK;
}

gs3_status gs3_selftest_shadow_wait(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                                    const gs3_render_opts* opts, void* workspace, size_t ws_bytes,
                                    size_t key_capacity, uint32_t* status_out) {
  if (!status_out) return fail(GS3_ERR_INVALID_ARG, "gs3_selftest_shadow_wait: null status_out");
  if (opts && (opts->ablate & GS3_ABLATE_SHADOW_SPLAT))
    return fail(GS3_ERR_INVALID_ARG, "gs3_selftest_shadow_wait: needs the shadow splat");
  // shading, projections and the light binning, with the render's own checks
  gs3_status st = render_frame(scene, cam, light, opts, reinterpret_cast<float*>(workspace), workspace, ws_bytes,
                               key_capacity, GS3_STAGE_PREP | GS3_STAGE_LIGHT_BIN, 0, nullptr);
  if (st != GS3_OK) return st;
  Workspace L = plan_workspace(scene->dev.n, cam->width, cam->height, key_capacity);
  FrameArgs f;
  f.sc = scene->dev;
  f.cam = *cam;
  f.light = *light;
  f.opts = *opts;
  f.ws = static_cast<unsigned char*>(workspace);
  f.L = &L;
  launch_shadow_chain_selftest(f, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(status_out, static_cast<unsigned char*>(workspace) + L.header, 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GS3_OK : cuda_fail(e, "gs3_selftest_shadow_wait");
}

gs3_status gs3_adam_step(float* param, const float* grad, float* m, float* v, size_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, float lower_bound, void* stream) {
  if (!param || !grad || !m || !v || n == 0 || step < 1)
    return fail(GS3_ERR_INVALID_ARG, "gs3_adam_step: null array, n = 0 or step < 1");
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f) || !(lr >= 0.f))
    return fail(GS3_ERR_INVALID_ARG, "gs3_adam_step: betas must be in [0, 1), lr and eps >= 0");
  const size_t b = n * sizeof(float);
  if (!device_range_ok(param, b) || !device_range_ok(grad, b) || !device_range_ok(m, b) || !device_range_ok(v, b))
    return fail(GS3_ERR_INVALID_ARG, "gs3_adam_step: an array is shorter than n floats");
  launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, lower_bound, reinterpret_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GS3_OK : cuda_fail(e, "gs3_adam_step");
}

size_t gs3_loss_scratch_size(int32_t width, int32_t height) {
  if (width < 1 || height < 1) return 0;
  return loss_scratch_bytes(width, height);
}

gs3_status gs3_loss_l1_dssim(const float* img, const float* target, int32_t width, int32_t height, float lambda,
                             float* loss_out, float* dimg, void* scratch, size_t scratch_bytes, void* stream) {
  if (!img || !target || !loss_out || !dimg || !scratch || width < 1 || height < 1)
    return fail(GS3_ERR_INVALID_ARG, "gs3_loss_l1_dssim: bad argument");
  const size_t img_bytes = (size_t)width * height * 3 * sizeof(float);
  const size_t need = loss_scratch_bytes(width, height);
  if (scratch_bytes < need || !device_range_ok(scratch, need) || !device_range_ok(img, img_bytes) ||
      !device_range_ok(target, img_bytes) || !device_range_ok(dimg, img_bytes) ||
      !device_range_ok(loss_out, sizeof(float)))
    return fail(GS3_ERR_INVALID_ARG, "gs3_loss_l1_dssim: a buffer is smaller than stated");
  const gs3_status st = run_loss(img, target, width, height, lambda, loss_out, dimg, scratch,
                                 reinterpret_cast<cudaStream_t>(stream));
  if (st != GS3_OK) return fail(st, "gs3_loss_l1_dssim: launch failed");
  return GS3_OK;
}

gs3_status gs3_workspace_read_header(const void* workspace, gs3_ws_header* out, void* stream) {
  if (!workspace || !out) return fail(GS3_ERR_INVALID_ARG, "gs3_workspace_read_header: null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, workspace, sizeof(gs3_ws_header), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "gs3_workspace_read_header");
  return GS3_OK;
}

}  // extern "C"
