// Environment light (Sec. 4.5): a weighted sum of renders under sampled
// directional lights, rendered as one batched frame.
//
// Of a frame's stages only three depend on the light: the shading colour
// (K1's shading part), the shadow splat (light projection, binning,
// composite, reduce) and Phi.  The camera splat (projection, binning, tile
// order), Psi (a function of the view direction, Sec. 4.3) and the camera
// composite's alphas are the same for every light.  So for lights taken in
// groups of up to kMaxBatch:
//   1. per light, on its own sub-stream: header reset, shading and the light
//      projection, light binning, shadow composite and shadow average (the
//      lights' persistent composite kernels run beside one another);
//   2. once, on `stream`, beside step 1: the camera splat's binning and tile
//      order, then Psi;
//   3. on `stream`: Phi over the group's lights in one launch over nl N rows,
//      writing (S_l, T'_l) per camera rank and light;
//   4. one camera composite of the group's lights (k_camera_env), which adds
//      sum_l w_l (S_l Sh_l + R) into the image.
// Each light's shadow values and Phi outputs equal that light's single frame
// bit for bit, and so do its composited S_l and Sh_l.
#include <mutex>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

struct EnvHeaders {
  uint32_t* h[kMaxBatch];
};

// Folds the group's headers into the first workspace's environment words:
// the first non-OK status, the camera's pair counts, the largest light counts.
__global__ void k_env_merge(EnvHeaders hs, int nl, int first) {
  if (threadIdx.x != 0) return;
  uint32_t* env = hs.h[0] + H_ENV;
  if (first) {
    for (int k = 0; k < 5; ++k) env[k] = 0u;
    env[H_PAIRS_CAM] = hs.h[0][H_PAIRS_CAM];
    env[H_NEED_CAM] = hs.h[0][H_NEED_CAM];
  }
  for (int l = 0; l < nl; ++l) {
    if (env[H_STATUS] == 0u) env[H_STATUS] = hs.h[l][H_STATUS];
    env[H_PAIRS_LIGHT] = max(env[H_PAIRS_LIGHT], hs.h[l][H_PAIRS_LIGHT]);
    env[H_NEED_LIGHT] = max(env[H_NEED_LIGHT], hs.h[l][H_NEED_LIGHT]);
  }
}

__global__ void k_env_publish(uint32_t* header) {
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) header[k] = header[H_ENV + k];
}

constexpr int kMaxEnvLights = 4096;

}  // namespace

EnvPlan plan_environment(int n, int width, int height, int count, size_t cap) {
  EnvPlan E;
  E.L = plan_workspace(n, width, height, cap);
  E.stride = (E.L.total + 255) & ~size_t(255);
  E.slices = count < kMaxBatch ? count : kMaxBatch;
  E.envcol = E.stride * (size_t)E.slices;
  E.total = E.envcol + 16ull * (size_t)n * (size_t)E.slices;
  return E;
}

}  // namespace gs3

using namespace gs3;

extern "C" {

size_t gs3_environment_workspace_size(int32_t n, int32_t width, int32_t height, int32_t count,
                                      size_t key_capacity) {
  if (n < 1 || width < 1 || height < 1 || count < 1) return 0;
  return plan_environment(n, width, height, count, key_capacity).total;
}

gs3_status gs3_render_environment(gs3_scene* scene, const gs3_camera* cam, const gs3_light* lights,
                                  const float* weights, int32_t count, const gs3_render_opts* opts,
                                  float* out_rgb, void* workspace, size_t ws_bytes, size_t key_capacity,
                                  void* stream) {
  if (!scene || !cam || !opts || !out_rgb || !workspace)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: null argument");
  if (!lights || !weights || count < 1 || count > kMaxEnvLights)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: need 1 <= count <= 4096 lights and weights");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: image size out of range");
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: focal length must be > 0");
  if (opts->tile != kTile) return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: tile must be 16");
  if (key_capacity < 1 || key_capacity > 0x7FFFFFFFull)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: key_capacity must be in [1, 2^31)");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: workspace must be 256-byte aligned");
  const int ntiles = ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
  if (ntiles > 65536) return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: more than 65536 tiles");
  if ((double)scene->dev.n * (double)ntiles >= 4294967295.0)
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: n * tiles must stay below 2^32");
  for (int32_t l = 0; l < count; ++l) {
    const char* why = light_problem(lights[l], *opts);
    if (why) return fail(GS3_ERR_INVALID_ARG, why);
  }
  const EnvPlan E = plan_environment(scene->dev.n, cam->width, cam->height, count, key_capacity);
  if (ws_bytes < E.total || !device_range_ok(workspace, E.total))
    return fail(GS3_ERR_INVALID_ARG,
                "gs3_render_environment: workspace smaller than gs3_environment_workspace_size");
  if (!device_range_ok(out_rgb, (size_t)cam->width * cam->height * 3 * sizeof(float)))
    return fail(GS3_ERR_INVALID_ARG, "gs3_render_environment: out_rgb is not width*height*3 floats");

  std::lock_guard<std::mutex> lock(scene->env_mu);
  if (!scene->env_ready) {
    if (!scene->env_bs.create(kMaxBatch)) {
      scene->env_bs.destroy();
      return cuda_fail(cudaGetLastError(), "gs3_render_environment: stream creation");
    }
    scene->env_ready = true;
  }
  BatchStreams& bs = scene->env_bs;
  (void)cudaGetLastError();  // only this call's launches are checked below
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = static_cast<unsigned char*>(workspace);
  float4* envcol = at<float4>(base, E.envcol);
  FrameArgs f[kMaxBatch];
  for (int r = 0; r < E.slices; ++r) {
    f[r].sc = scene->dev;
    f[r].cam = *cam;
    f[r].opts = *opts;
    f[r].ws = base + (size_t)r * E.stride;
    f[r].L = &E.L;
  }
  const bool no_shadow = (opts->ablate & GS3_ABLATE_SHADOW_SPLAT) != 0;
  const bool tc = scene->dev.mlp_dtype != GS3_MLP_FP32;
  const unsigned char* blobs[2] = {scene->tc_blob[0], scene->tc_blob[1]};
  for (int32_t g0 = 0; g0 < count; g0 += kMaxBatch) {
    const int nl = count - g0 < kMaxBatch ? count - g0 : kMaxBatch;
    const bool first = g0 == 0;
    for (int r = 0; r < nl; ++r) f[r].light = lights[g0 + r];
    // 1. per light, on its sub-stream: shading, the light projection, binning,
    //    shadow composite and average
    cudaEventRecord(bs.fork, s);
    for (int r = 0; r < nl; ++r) {
      cudaStream_t sr = bs.sub[r];
      cudaStreamWaitEvent(sr, bs.fork, 0);
      cudaMemsetAsync(f[r].ws + E.L.header, 0, 4 * H_RESET_WORDS, sr);
      launch_prep(f[r], sr, /*light_only=*/!(first && r == 0));
      if (first && r == 0) cudaEventRecord(bs.cam, sr);  // the camera projection is done
      if (no_shadow) {
        launch_fill_shadow_one(f[r], sr);
      } else {
        launch_depth_sort(f[r], 1, sr);
        launch_binning(f[r], 1, sr);
        launch_shadow_composite(f[r], sr);
        launch_shadow_reduce(f[r], sr);
      }
      cudaEventRecord(bs.join[r], sr);
    }
    if (first) {
      // 2. once, on `stream` beside the light chains: the camera splat (after
      //    the first light's projections) and Psi
      cudaStreamWaitEvent(s, bs.cam, 0);
      launch_depth_sort(f[0], 0, s);
      launch_binning(f[0], 0, s);
      launch_tile_order(f[0], 0, s);
      launch_mlp(f[0], s, /*identity_only=*/tc, /*which_mask=*/2);
      if (tc) launch_mlp_tc(f[0], blobs, s, /*which_mask=*/2);
    }
    for (int r = 0; r < nl; ++r) cudaStreamWaitEvent(s, bs.join[r], 0);
    // 3. Phi over the group's lights; 4. their camera composite
    const FrameArgs* fl[kMaxBatch];
    for (int r = 0; r < nl; ++r) fl[r] = &f[r];
    if (tc && !(opts->ablate & GS3_ABLATE_PHI)) launch_phi_lights_tc(fl, nl, envcol, blobs[0], s);
    else launch_phi_lights(fl, nl, envcol, s);
    launch_camera_env(f[0], envcol, nl, weights + g0, !first, out_rgb, s);
    EnvHeaders hs;
    for (int r = 0; r < kMaxBatch; ++r) hs.h[r] = at<uint32_t>(f[r < nl ? r : 0].ws, E.L.header);
    k_env_merge<<<1, 32, 0, s>>>(hs, nl, first ? 1 : 0);
    count_launch();
  }
  k_env_publish<<<1, 32, 0, s>>>(at<uint32_t>(base, E.L.header));
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GS3_OK : cuda_fail(e, "gs3_render_environment: launch");
}

}  // extern "C"
