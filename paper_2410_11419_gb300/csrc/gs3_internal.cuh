// Internal declarations shared by the CUDA translation units of libgs3.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <stdint.h>

#include "gs3.h"

namespace gs3 {

constexpr int kTile = 16;             // screen tile edge (pixels)
constexpr int kTilePix = kTile * kTile;
constexpr int kSortThreads = 256;     // radix-sort block size
constexpr int kSortRounds = 16;       // items per thread per block tile
constexpr int kSortTileItems = kSortThreads * kSortRounds;  // 4096 items per block
constexpr int kTileSortRounds = 16;   // look-back sort of the wait self-test: items per thread per block
constexpr int kTileSortItems = kSortThreads * kTileSortRounds;
// Tile binning by counting (tile_bin.cu)
constexpr int kMaxTileAxis = 1024;    // tiles per image row or column (16384 pixels)
constexpr int kBinBlock = 256;        // depth ranks per block of the row counts
// items of a tile row's rank sequence per chunk of the column counts
inline uint32_t bin_chunk(int gx) { return 256u * (uint32_t)((gx + 127) / 128); }
// words of the (row, column, chunk) count table: at most cap / chunk + gy chunks
inline size_t bin_tab_words(size_t cap, int gx, int gy) {
  return (cap / bin_chunk(gx) + (size_t)gy + 1) * (size_t)gx;
}
constexpr int kDepthSortRounds = 4;   // the per-splat depth sort: 1024 keys per block
constexpr int kDepthSortItems = kSortThreads * kDepthSortRounds;
constexpr int kScanItems = 4096;      // items per block in the device-wide scan
constexpr int kMaxLobes = 16;

// Per-Gaussian splat record (one per splat, by Gaussian index or by rank).
//   a = (u_hi, v_hi, opacity, depth)  screen position (high part), gamma, FP32 sort depth
//   b = (A, B, C, u_lo)               conic: power = -0.5 (A dx^2 + C dy^2) - B dx dy
//   c = (v_lo, hx, hy, pthr)          v = v_hi + v_lo; half extents of the box holding
//                                     every pixel with alpha >= alpha_min; power threshold
//                                     ln(alpha_min / gamma) (alpha >= alpha_min <=> power >= pthr)
//   r = (x0, y0, x1, y1)              inclusive tile rectangle, x0 < 0 when culled
struct __align__(16) SplatRec {
  float4 a;
  float4 b;
  float4 c;
  int4 r;
};

struct SplatBufs {
  size_t key;           // u32[N] depth key by index
  size_t sk[2], sv[2];  // u32[N] depth-sort ping-pong
  size_t order;         // u32[N] index of rank r
  size_t rank_of;       // u32[N] rank of index g
  size_t rect;          // int4[N] rectangle by index (copy of rec.r, for inspection)
  size_t rec;           // SplatRec[N] by index
  size_t rrec;          // SplatRec[N] by rank
  size_t cnt;           // u32[N] tiles covered, by rank
  size_t off;           // u32[N] exclusive prefix of cnt
  size_t tk[2], tv[2];  // u32[cap] each: tv[fin] the tile lists, tk[fin] the row sequence, the rest scratch
  size_t tile_start;    // u32[ntiles + 1]
  size_t scan_part;     // u32 partial sums of the device-wide scan
  size_t dlook;         // depth sort's look-back region, onesweep_bytes(nb_n, 4)
  size_t row_cnt;       // u32[gy][nb_rows]: ranks per (tile row, block of kBinBlock ranks), then scanned
  size_t bin_plan;      // u32[3 gy + 3]: row starts, chunk starts, pairs per row, capacity flag
  size_t bin_tab;       // u32[bin_tab_words]: list entries per (row, column, chunk), then scanned per row
};

struct Workspace {
  size_t total = 0;
  size_t header = 0;
  SplatBufs sp[2];
  size_t partial = 0;  // float2[cap] shadow partials (num, den) per light entry
  size_t shade = 0;    // float4[N] shading colour by index
  size_t T = 0;        // float[N] shadow value by index
  size_t Tp = 0;       // float[N] refined shadow value by index
  size_t res = 0;      // float4[N] residual by index
  size_t ccol = 0;     // float4[2N] camera colours by camera rank: (shade, T'), (res, 0)
  size_t final_t = 0;  // float[HW]
  size_t n_contrib = 0;  // u32[HW]
  size_t pix_aux = 0;    // float4[2 HW]: (S rgb, Sh), (R rgb, 0) composited per camera pixel
  size_t light_final = 0;  // float[HW] occluder product where each shadow ray ended
  size_t light_stop = 0;   // u32[HW] 1 + list index of the occluder that stopped the ray, or all ones
  size_t shadow_den = 0;   // float[N] sum of beta per Gaussian (by index)
  size_t tile_order[2] = {0, 0};  // u32[ntiles] per splat: tiles by decreasing list length (launch order)
  size_t seg_lvl = 0;   // u32[1025 + 3]: shadow work items per segment level, then three ticket counters
  size_t seg_flag = 0;  // u32[items]: shadow segment publications (0 none, 1 done, 2 done and all stopped)
  size_t seg_pub = 0;   // float[items][256]: the products each shadow segment hands to the next
  size_t rank_flags = 0;  // u8[2N] by light rank: has an entry in a segment with an open ray; a dead unit passed
  int n = 0, width = 0, height = 0, gx = 0, gy = 0, ntiles = 0;
  size_t cap = 0;
  int nb_n = 0;     // radix blocks over N
  int nb_rows = 0;  // blocks of kBinBlock depth ranks
};

Workspace plan_workspace(int n, int width, int height, size_t cap);

// Error reporting of the C ABI: sets gs3_last_error's message, returns st /
// GS3_ERR_CUDA.
gs3_status fail(gs3_status st, const char* msg);
gs3_status cuda_fail(cudaError_t e, const char* where);
// why a light cannot be rendered with these options, or null
const char* light_problem(const gs3_light& l, const gs3_render_opts& o);

// Header word indices (u32) -- must match gs3_ws_header.
enum { H_STATUS = 0, H_PAIRS_CAM = 1, H_PAIRS_LIGHT = 2, H_NEED_CAM = 3, H_NEED_LIGHT = 4,
       H_LIGHT_VIEW = 8, H_LIGHT_ORTHO = 20,
       H_RESET_WORDS = 24,  // words a render resets; the rest survive across renders
       H_ENV = 24 };        // environment render: status, pairs cam/light, needed cam/light

// The light in homogeneous form (x, y, z, w): a point light (pos, 1) or a
// directional light (dir / |dir|, 0).  omega_i = normalize(L.xyz - L.w mu)
// covers both, and the inverse-square fall-off applies only when w = 1.
inline float4 light_h(const gs3_light& l) {
  if (l.type == GS3_LIGHT_DIRECTIONAL) {
    const float n = sqrtf(l.dir[0] * l.dir[0] + l.dir[1] * l.dir[1] + l.dir[2] * l.dir[2]);
    return make_float4(l.dir[0] / n, l.dir[1] / n, l.dir[2] / n, 0.f);
  }
  return make_float4(l.pos[0], l.pos[1], l.pos[2], 1.f);
}

struct MlpDev {
  int in_dim, width, n_hidden, out_dim, act;
  const float* w;
  const float* b;
};

struct SceneDev {
  int n, k;
  const float4 *mean_op, *scale, *rot, *shade_rot, *albedo_d, *albedo_s, *latent;
  const float4 *lobe_rot, *lobe_sigma, *lobe_amp;
  MlpDev phi, psi;
  int mlp_dtype;
  int lobe_shared;  // lobe_rot / lobe_sigma: K shared entries instead of K x N
};

// A side stream and fork/join events for running a frame's light chain
// (light binning, shadow composite, shadow reduce) beside its camera binning.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool create();
  void destroy();
};
// the calling thread's side stream on the current device (created on first use)
SideStream* thread_side_stream();
// the frame with an explicit side stream (null: everything on `stream`)
gs3_status render_frame(gs3_scene* scene, const gs3_camera* cam, const gs3_light* light,
                        const gs3_render_opts* opts, float* out_rgb, void* workspace, size_t ws_bytes,
                        size_t key_capacity, uint32_t stages, cudaStream_t stream, SideStream* side);

// One frame of a batch: its scene, view, light, options, output and workspace.
struct BatchFrame {
  gs3_scene* scene;
  gs3_camera cam;
  gs3_light light;
  gs3_render_opts opts;
  float* out;
  void* ws;
  size_t ws_bytes;
  size_t cap;
};
// Streams and events of a batch: a sub-stream per frame for the per-frame stages.
struct BatchStreams {
  cudaStream_t sub[8] = {};
  cudaEvent_t fork = nullptr, fork2 = nullptr, cam = nullptr, join[8] = {}, join2[8] = {};
  bool create(int n);
  void destroy();
};
// Renders n <= kMaxBatch frames together on `stream` (see render_batch in api.cu).
gs3_status render_batch(const BatchFrame* frames, int n, cudaStream_t stream, BatchStreams& bs,
                        unsigned char* param_dev, unsigned char* param_host);

// Workspace of an environment render: min(count, kMaxBatch) frame
// workspaces `stride` bytes apart (one per light of a group; the first also
// holds the camera splat), then the lights' camera colours envcol
// (float4[N][slices]).
struct EnvPlan {
  Workspace L;
  size_t stride = 0, envcol = 0, total = 0;
  int slices = 0;
};
EnvPlan plan_environment(int n, int width, int height, int count, size_t cap);

// ---- launchers (stream-ordered, no host synchronisation) ----
struct FrameArgs {
  SceneDev sc;
  gs3_camera cam;
  gs3_light light;
  gs3_render_opts opts;
  unsigned char* ws;
  const Workspace* L;
};

void launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                 int step, float lo, cudaStream_t s);
size_t loss_scratch_bytes(int W, int H);
gs3_status run_loss(const float* img, const float* tgt, int W, int H, float lambda, float* loss, float* dimg,
                    void* scratch, cudaStream_t s);
size_t backward_workspace_bytes(int n, const MlpDev& phi, const MlpDev& psi);
// MLP backward (mlp_bwd.cu): one network's parameter gradients into wred
// (its parameter order) and its input gradients into mlp_in / dT
struct MlpArgs {
  MlpDev net;
  int n, which;  // 0 Phi, 1 Psi
  const float4* mean_op;
  const float4* latent;
  const float* T;
  float light_pos[3], cam_pos[3];
  float light_w;       // homogeneous light (see light_h)
  const float* color;  // [N][8]: dT' at 3, dres at 4..6
  float* dT;           // Phi: d/d(input T)
  float* mlp_in;       // [N][24]
  uint32_t* status;    // device status word (GS3_ERR_TIMEOUT of a tensor-core GEMM's wait)
};
size_t mlp_bwd_scratch_bytes(int n, const MlpDev& m);
void run_mlp_backward(const MlpArgs& a, void* scratch, float* wred, cudaStream_t s);
// side: a second stream for the parts that can overlap (null: all on s)
gs3_status run_backward(const FrameArgs& f, const float* dimg, void* bws, size_t bws_bytes,
                        const gs3_grads& out, cudaStream_t s, SideStream* side = nullptr);

// shading and both projections (K1); light_only: the shadow splat's projection only
void launch_prep(const FrameArgs& f, cudaStream_t s, bool light_only = false);
void launch_depth_sort(const FrameArgs& f, int splat, cudaStream_t s);
void launch_binning(const FrameArgs& f, int splat, cudaStream_t s);
void launch_shadow_composite(const FrameArgs& f, cudaStream_t s);
// Batches of frames (up to kMaxBatch, each with its own workspace): the
// shadow composite's per-frame set-up (on each frame's stream), then its
// segment kernels and the camera composite over every frame of the batch in
// single launches.  dev / host: a batch parameter block, device memory and
// pinned host staging of batch_param_bytes() each, not reused until the
// batch's work completed.
constexpr int kMaxBatch = 8;
size_t batch_param_bytes();
void prepare_shadow_composite(const FrameArgs& f, cudaStream_t s);
void launch_shadow_chain_selftest(const FrameArgs& f, cudaStream_t s);
void launch_shadow_composite_batch(const FrameArgs* const* f, int n, unsigned char* dev, unsigned char* host,
                                   cudaStream_t s);
void launch_camera_composite_batch(const FrameArgs* const* f, float* const* out, int n, unsigned char* dev,
                                   unsigned char* host, cudaStream_t s);
// shadow composite work items (tile segments) a frame can have at most
size_t shadow_seg_items(int ntiles, size_t cap);
// A light tile's list is cut into segments of kSegLen entries, at most
// kSegLevels - 1 per tile (the last takes the rest); the shadow composite and
// its backward share the cut.
constexpr uint32_t kSegLen = 256;
constexpr int kSegLevels = 1024;
__host__ __device__ inline uint32_t seg_count(uint32_t len) {
  const uint32_t n = (len + kSegLen - 1) / kSegLen;
  return n < 1 ? 1u : (n > (uint32_t)(kSegLevels - 1) ? (uint32_t)(kSegLevels - 1) : n);
}
// a splat's tiles ordered longest list first (in length steps of 8), into L.tile_order[splat]
void launch_tile_order(const FrameArgs& f, int splat, cudaStream_t s);
void launch_shadow_reduce(const FrameArgs& f, cudaStream_t s);
// Phi and Psi of one frame; which_mask bit 0 Phi, bit 1 Psi; identity_only:
// only the networks an ablation replaces by the identity / zero
void launch_mlp(const FrameArgs& f, cudaStream_t s, bool identity_only = false, int which_mask = 3);
// Phi of nl <= kMaxBatch frames of one scene and camera (an environment
// light's directional lights; the camera ranks of f[0]) in one launch over
// nl N rows; (shade_l, T'_l) of camera rank r go to envcol[r nl + l]
void launch_phi_lights(const FrameArgs* const* f, int nl, float4* envcol, cudaStream_t s);
void launch_phi_lights_tc(const FrameArgs* const* f, int nl, float4* envcol, const unsigned char* blob,
                          cudaStream_t s);
// BF16 / FP8 tensor-core MLPs (mlp_tc.cu)
size_t mlp_tc_blob_bytes(const MlpDev& m, int dtype);
size_t mlp_tc_scale_offset(const MlpDev& m, int dtype);  // FP8: (sx, sw) per hidden layer
void pack_mlp_tc(const MlpDev& m, int dtype, const SceneDev& sc, int which, unsigned char* dst, cudaStream_t s);
bool mlp_tc_supported(const MlpDev& m, int dtype);
void launch_mlp_tc(const FrameArgs& f, const unsigned char* const blobs[2], cudaStream_t s, int which_mask = 3);
void launch_camera_composite(const FrameArgs& f, float* out_rgb, cudaStream_t s);
// camera composite of nl <= kMaxBatch lights over f0's camera splat:
// out (+)= sum_l w[l] (S_l Sh_l + R), (S_l, Sh_l) per camera rank from envcol
void launch_camera_env(const FrameArgs& f0, const float4* envcol, int nl, const float* w, bool accumulate,
                       float* out_rgb, cudaStream_t s);
void launch_fill_shadow_one(const FrameArgs& f, cudaStream_t s);

// exclusive scan of n u32 values (in place allowed: out may equal in);
// the total goes to *total if non-null
void device_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total,
                           uint32_t* scratch, cudaStream_t s);
size_t scan_scratch_words(size_t n);

// bytes of a look-back sort's region: u64[passes][256 * nblocks] look-back
// words, u32 tickets[passes], u32 totals[passes][256]
inline size_t onesweep_bytes(int nblocks, int passes) {
  return 8ull * passes * 256 * (size_t)nblocks + 4ull * (passes + passes * 256);
}

// stable LSD radix sort of n (key, value) pairs on the low 8 * passes key bits
// (vin null: values are the input positions); the result lands in (k1, v1)
// for an even number of passes, (k0, v0) for an odd one
void radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                      uint32_t* v1, uint32_t n, int passes, uint32_t* hist, uint32_t* scan_part,
                      cudaStream_t s);

// false when [ptr, ptr + bytes) provably leaves ptr's device allocation
bool device_range_ok(const void* ptr, size_t bytes);

// sets the message gs3_last_error returns on this thread
void set_last_error(const char* msg);

// Per-device one-time set-up (kernel attributes, constant tables): run() calls
// fn() at most once per CUDA device until it succeeds, with that device
// current, from any thread.  Devices beyond kMaxDevices run fn() every time.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
  std::mutex mu;
  std::atomic<bool> done[kMaxDevices];
  template <typename F>
  bool run(F&& fn) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return fn();
    if (done[d].load(std::memory_order_acquire)) return true;
    std::lock_guard<std::mutex> lock(mu);
    if (done[d].load(std::memory_order_relaxed)) return true;
    const bool ok = fn();
    if (ok) done[d].store(true, std::memory_order_release);
    return ok;
  }
};

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount),
// looked up once per device; grid caps are multiples of it.
int device_sm_count();

// host-side count of kernel launches (reported by gs3_kernel_launches)
extern std::atomic<uint64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

template <typename T>
__host__ __device__ inline T* at(unsigned char* ws, size_t off) {
  return reinterpret_cast<T*>(ws + off);
}

}  // namespace gs3

// The scene handle of the C ABI: borrowed parameters plus owned derived buffers.
struct gs3_scene {
  gs3::SceneDev dev;
  unsigned char* tc_blob[2] = {nullptr, nullptr};  // tensor-core weights and FP8 scales (owned)
  // environment renders: sub-streams made on first use; env_mu serialises the
  // calls' launch sequences on them
  std::mutex env_mu;
  gs3::BatchStreams env_bs;
  bool env_ready = false;
};
