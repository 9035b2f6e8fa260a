// Continuous-batching render server over device-resident scenes.
//
// A worker thread owns a FIFO of (scene, camera, light) requests and a set
// of in-flight slots.  A free slot takes up to max_batch requests from the
// head of the queue, as long as their workspaces fit in the HBM budget
// (bytes in use by admitted requests), and renders them as one batch: every
// frame's shading, projections and binning on its own sub-stream, then the
// shadow composite's persistent segment kernels and the camera composite
// over all the batch's frames in single launches (render_batch).  Requests
// that arrive while batches are on the GPU wait for the next free slot and
// join its batch; batches in different slots overlap on the device.
// Workspaces come from a stream-ordered memory pool and go back to it when
// the batch's completion event fires.  The workspace capacity
// (tile/Gaussian pairs) is estimated per (scene, resolution) from the largest
// count seen so far; a request that overflows is re-admitted once with the
// exact count its first run reported.
// With a light cache, the shadow values T of a completed frame are kept per
// (scene, light, image size, options): they depend on nothing else (not on
// the camera), so a later request alone on its slot with the same key copies
// them into its workspace and runs only the camera-side stages.  A kept entry
// becomes usable when the frame that filled it has completed without error;
// when the cache is full, the least recently used entry that no admitted
// frame reads makes room.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int scene = 0;
  gs3_camera cam{};
  gs3_light light{};
  gs3_render_opts opts{};
  float* out = nullptr;
  Clock::time_point t_submit;
  size_t forced_cap = 0;  // exact capacity for a re-admitted request
  int attempts = 0;
};

// One request of a batch and its workspace.
struct Member {
  Request req;
  gs3_ws_header* hdr = nullptr;  // pinned copy of the workspace header
  void* ws = nullptr;
  size_t bytes = 0;
  size_t cap = 0;
  std::string fill;   // the light-cache key this frame's shadow values fill, or empty
  std::string reuse;  // the light-cache key this frame copies its shadow values from, or empty
};

// Shadow values T (n floats) of one light-cache key.
struct LightEntry {
  float* T = nullptr;
  size_t n = 0;
  bool ready = false;  // the frame that filled it completed without error
  int users = 0;       // admitted frames copying from it that have not completed
  uint64_t last_use = 0;
};

// the stages that depend on the camera (gs3_render_stages)
constexpr uint32_t kCameraSide = GS3_STAGE_PREP | GS3_STAGE_CAMERA_BIN | GS3_STAGE_MLP | GS3_STAGE_CAMERA;

struct Slot {
  cudaStream_t stream = nullptr;
  SideStream side;     // a lone frame's light chain
  BatchStreams batch;  // a batch's per-frame sub-streams
  unsigned char* param_dev = nullptr;   // the batch's kernel parameters
  unsigned char* param_host = nullptr;  // and their pinned staging
  cudaEvent_t start = nullptr;
  cudaEvent_t done = nullptr;
  Member m[kMaxBatch];
  int n = 0;  // requests in the batch
  bool busy = false;
};

struct Result {
  int state = GS3_REQ_QUEUED;
  gs3_status status = GS3_OK;
  double latency_ms = 0.0;
};

}  // namespace
}  // namespace gs3

using namespace gs3;

struct gs3_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  size_t peak_in_use = 0;
  int inject_alloc_failures = 0;
  double initial_pairs = 64.0;
  cudaEvent_t epoch = nullptr;  // device time origin of the counters
  bool epoch_set = false;
  double span_lo = 1e300, span_hi = -1e300;
  std::vector<gs3_scene*> scenes;
  std::unordered_map<uint64_t, size_t> cap_hint;  // (scene, w, h) -> pairs
  std::deque<Request> queue;
  std::vector<Slot> slots;
  std::unordered_map<uint64_t, Result> results;
  uint64_t next_ticket = 1;
  uint64_t completed = 0, failed = 0, retries = 0;
  int max_inflight_seen = 0;
  int max_batch = 1;
  int max_batch_seen = 0;
  uint64_t batches = 0;
  int light_cache_max = 0;
  std::unordered_map<std::string, LightEntry> light_cache;
  uint64_t light_reuse = 0;
  uint64_t light_clock = 0;  // orders the entries' last uses
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  cudaMemPool_t pool = nullptr;
};

namespace gs3 {
namespace {

uint64_t hint_key(int scene, int w, int h) {
  return ((uint64_t)scene << 40) ^ ((uint64_t)w << 20) ^ (uint64_t)h;
}

// The light-cache key: scene, image size, light and options, byte for byte
// (padding bytes that differ can only cause a miss).
std::string light_key(const Request& r) {
  const int32_t v[3] = {r.scene, r.cam.width, r.cam.height};
  std::string k(sizeof v + sizeof(gs3_light) + sizeof(gs3_render_opts), '\0');
  std::memcpy(&k[0], v, sizeof v);
  std::memcpy(&k[sizeof v], &r.light, sizeof(gs3_light));
  std::memcpy(&k[sizeof v + sizeof(gs3_light)], &r.opts, sizeof(gs3_render_opts));
  return k;
}

// A frame that was to fill a light-cache entry has finished: the entry becomes
// usable if the frame succeeded, else it is dropped (its memory returned in
// stream order after the frame's copy).
void settle_fill(gs3_server* S, Slot& sl, Member& m, bool ok) {
  if (m.fill.empty()) return;
  auto it = S->light_cache.find(m.fill);
  if (it != S->light_cache.end()) {
    if (ok) {
      it->second.ready = true;
    } else {
      cudaFreeAsync(it->second.T, sl.stream);
      S->light_cache.erase(it);
    }
  }
  m.fill.clear();
}

// A frame that copied kept shadow values has finished (or was not launched).
void settle_reuse(gs3_server* S, Member& m) {
  if (m.reuse.empty()) return;
  auto it = S->light_cache.find(m.reuse);
  if (it != S->light_cache.end() && it->second.users > 0) --it->second.users;
  m.reuse.clear();
}

// Room for one more light-cache entry: below the limit, or after freeing the
// least recently used entry that is ready and that no admitted frame reads
// (its copies have completed, so its memory is idle).  False if none can go.
bool light_cache_room(gs3_server* S, cudaStream_t s) {
  if ((int)S->light_cache.size() < S->light_cache_max) return true;
  auto victim = S->light_cache.end();
  for (auto it = S->light_cache.begin(); it != S->light_cache.end(); ++it)
    if (it->second.ready && it->second.users == 0 &&
        (victim == S->light_cache.end() || it->second.last_use < victim->second.last_use))
      victim = it;
  if (victim == S->light_cache.end()) return false;
  cudaFreeAsync(victim->second.T, s);
  S->light_cache.erase(victim);
  return true;
}

size_t estimate_cap(gs3_server* S, const Request& r) {
  if (r.forced_cap) return r.forced_cap;
  auto it = S->cap_hint.find(hint_key(r.scene, r.cam.width, r.cam.height));
  if (it != S->cap_hint.end()) return it->second;
  // first request of this (scene, resolution): initial_pairs per Gaussian per splat
  // at 800 x 800, scaled with the pixel count, plus 4 per Gaussian
  const double n = (double)S->scenes[r.scene]->dev.n;
  const double px = (double)r.cam.width * r.cam.height / (800.0 * 800.0);
  double c = n * (4.0 + S->initial_pairs * px);
  if (c > 2.0e9) c = 2.0e9;
  return (size_t)c;
}

void finish(gs3_server* S, const Request& req, gs3_status st) {
  Result& res = S->results[req.ticket];
  res.state = st == GS3_OK ? GS3_REQ_DONE : GS3_REQ_FAILED;
  res.status = st;
  res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - req.t_submit).count();
  if (st == GS3_OK) ++S->completed; else ++S->failed;
}

void release(gs3_server* S, Slot& sl, Member& m) {
  if (m.ws) cudaFreeAsync(m.ws, sl.stream);
  m.ws = nullptr;
  S->in_use -= m.bytes;
  m.bytes = 0;
}

// Completions: called with the lock held.
bool poll_slots(gs3_server* S) {
  bool any = false;
  for (Slot& sl : S->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    any = true;
    bool timed = false;
    for (int i = 0; i < sl.n; ++i) {
      Member& m = sl.m[i];
      gs3_status st = GS3_OK;
      if (q != cudaSuccess) {
        st = GS3_ERR_CUDA;
      } else if (m.hdr->status == GS3_ERR_CAPACITY && m.req.attempts < 2) {
        // re-admit at the front with the exact pair count of this frame
        Request r = m.req;
        const size_t need = m.hdr->pairs_cam_needed > m.hdr->pairs_light_needed ? m.hdr->pairs_cam_needed
                                                                                : m.hdr->pairs_light_needed;
        r.forced_cap = need + need / 16 + 1024;
        ++S->retries;
        auto& hint = S->cap_hint[hint_key(r.scene, r.cam.width, r.cam.height)];
        if (r.forced_cap > hint) hint = r.forced_cap;
        settle_fill(S, sl, m, false);
        settle_reuse(S, m);
        release(S, sl, m);
        S->results[r.ticket].state = GS3_REQ_QUEUED;
        S->queue.push_front(r);
        continue;
      } else {
        st = (gs3_status)m.hdr->status;
        const size_t seen = m.hdr->pairs_cam > m.hdr->pairs_light ? m.hdr->pairs_cam : m.hdr->pairs_light;
        auto& hint = S->cap_hint[hint_key(m.req.scene, m.req.cam.width, m.req.cam.height)];
        const size_t want = seen + seen / 8 + 1024;  // 12.5 % head room over the largest count seen
        if (want > hint) hint = want;
      }
      if (st == GS3_OK && S->epoch_set && !timed) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, S->epoch, sl.start) == cudaSuccess &&
            cudaEventElapsedTime(&b, S->epoch, sl.done) == cudaSuccess) {
          if (a < S->span_lo) S->span_lo = a;
          if (b > S->span_hi) S->span_hi = b;
        }
        timed = true;
      }
      settle_fill(S, sl, m, st == GS3_OK);
      settle_reuse(S, m);
      finish(S, m.req, st);
      release(S, sl, m);
    }
    sl.n = 0;
    sl.busy = false;
  }
  return any;
}

// Admission: called with the lock held.  FIFO: the head waits for memory.  A
// free slot takes up to max_batch requests from the head of the queue.
bool admit(gs3_server* S) {
  bool any = false;
  while (!S->queue.empty()) {
    Slot* free_slot = nullptr;
    for (Slot& sl : S->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    if (!free_slot) break;
    Slot& sl = *free_slot;
    sl.n = 0;
    while (!S->queue.empty() && sl.n < S->max_batch) {
      const Request& head = S->queue.front();
      gs3_scene* sc = S->scenes[head.scene];
      const size_t cap = estimate_cap(S, head);
      const size_t bytes = gs3_workspace_size(sc->dev.n, head.cam.width, head.cam.height, cap) + 256;
      const bool fits_ever = bytes <= S->budget;
      if (fits_ever && S->in_use + bytes > S->budget) break;  // wait for memory
      Request req = head;
      req.attempts += 1;
      S->queue.pop_front();
      any = true;
      if (!fits_ever) {  // can never fit: fail it rather than block the queue
        finish(S, req, GS3_ERR_OOM);
        continue;
      }
      void* ws = nullptr;
      cudaError_t e = cudaSuccess;
      if (S->inject_alloc_failures > 0) {
        --S->inject_alloc_failures;
        e = cudaErrorMemoryAllocation;
      } else {
        e = cudaMallocFromPoolAsync(&ws, bytes, S->pool, sl.stream);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        finish(S, req, GS3_ERR_OOM);
        continue;
      }
      Member& m = sl.m[sl.n++];
      m.req = req;
      m.ws = ws;
      m.bytes = bytes;
      m.cap = cap;
      m.fill.clear();
      m.reuse.clear();
      S->in_use += bytes;
      if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
      S->results[req.ticket].state = GS3_REQ_RUNNING;
    }
    if (sl.n == 0) break;  // the head waits for memory
    sl.busy = true;
    if (!S->epoch_set) {
      cudaEventRecord(S->epoch, sl.stream);
      S->epoch_set = true;
    }
    cudaEventRecord(sl.start, sl.stream);
    gs3_status st = GS3_OK;
    void* aligned[kMaxBatch];
    for (int i = 0; i < sl.n; ++i)
      aligned[i] = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(sl.m[i].ws) + 255) & ~uintptr_t(255));
    if (sl.n == 1) {
      Member& m = sl.m[0];
      gs3_scene* sc = S->scenes[m.req.scene];
      const size_t n = (size_t)sc->dev.n;
      const LightEntry* kept = nullptr;
      if (S->light_cache_max > 0) {
        const std::string key = light_key(m.req);
        auto it = S->light_cache.find(key);
        if (it != S->light_cache.end()) {
          if (it->second.ready) {  // else its frame is still in flight: render in full
            kept = &it->second;
            ++it->second.users;
            it->second.last_use = ++S->light_clock;
            m.reuse = key;
          }
        } else if (light_cache_room(S, sl.stream)) {
          void* T = nullptr;
          if (cudaMallocFromPoolAsync(&T, 4 * n, S->pool, sl.stream) == cudaSuccess) {
            LightEntry e;
            e.T = static_cast<float*>(T);
            e.n = n;
            e.last_use = ++S->light_clock;
            S->light_cache.emplace(key, e);
            m.fill = key;
          } else {
            cudaGetLastError();
          }
        }
      }
      // the shadow values' place in this request's workspace
      unsigned char* Tws = static_cast<unsigned char*>(aligned[0]) +
                           plan_workspace(sc->dev.n, m.req.cam.width, m.req.cam.height, m.cap).T;
      if (kept) {
        cudaMemcpyAsync(Tws, kept->T, 4 * n, cudaMemcpyDeviceToDevice, sl.stream);
        st = render_frame(sc, &m.req.cam, &m.req.light, &m.req.opts, m.req.out, aligned[0], m.bytes - 256, m.cap,
                          kCameraSide, sl.stream, nullptr);
        if (st == GS3_OK) ++S->light_reuse;
      } else {
        st = render_frame(sc, &m.req.cam, &m.req.light, &m.req.opts, m.req.out, aligned[0], m.bytes - 256, m.cap,
                          GS3_STAGE_ALL, sl.stream, sl.side.s ? &sl.side : nullptr);
        if (st == GS3_OK && !m.fill.empty())
          cudaMemcpyAsync(S->light_cache[m.fill].T, Tws, 4 * n, cudaMemcpyDeviceToDevice, sl.stream);
      }
      if (st != GS3_OK) {
        settle_fill(S, sl, m, false);
        settle_reuse(S, m);
      }
    } else {
      BatchFrame fr[kMaxBatch];
      for (int i = 0; i < sl.n; ++i) {
        const Member& m = sl.m[i];
        fr[i] = BatchFrame{S->scenes[m.req.scene], m.req.cam, m.req.light, m.req.opts, m.req.out, aligned[i],
                           m.bytes - 256, m.cap};
      }
      st = render_batch(fr, sl.n, sl.stream, sl.batch, sl.param_dev, sl.param_host);
    }
    if (st == GS3_OK) {
      for (int i = 0; i < sl.n; ++i)
        cudaMemcpyAsync(sl.m[i].hdr, aligned[i], sizeof(gs3_ws_header), cudaMemcpyDeviceToHost, sl.stream);
      cudaEventRecord(sl.done, sl.stream);
      ++S->batches;
      if (sl.n > S->max_batch_seen) S->max_batch_seen = sl.n;
    } else {
      for (int i = 0; i < sl.n; ++i) {
        finish(S, sl.m[i].req, st);
        release(S, sl, sl.m[i]);
      }
      sl.n = 0;
      sl.busy = false;
    }
    int inflight = 0;
    for (Slot& s2 : S->slots) inflight += s2.busy ? s2.n : 0;
    if (inflight > S->max_inflight_seen) S->max_inflight_seen = inflight;
  }
  return any;
}

void worker_main(gs3_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    const bool a = poll_slots(S);
    const bool b = admit(S);
    if (a) S->cv_done.notify_all();
    bool busy = false;
    for (Slot& sl : S->slots) busy |= sl.busy;
    if (!a && !b) {
      if (busy) {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lock.lock();
      } else {
        S->cv_work.wait_for(lock, std::chrono::milliseconds(5));
      }
    }
  }
}

}  // namespace
}  // namespace gs3

extern "C" {

gs3_status gs3_server_create(const gs3_server_opts* o, gs3_server** out) {
  if (!o || !out || o->max_inflight < 1 || o->max_inflight > 64 || o->hbm_budget == 0) {
    set_last_error("gs3_server_create: bad options");
    return GS3_ERR_INVALID_ARG;
  }
  *out = nullptr;
  gs3_server* S = new (std::nothrow) gs3_server;
  if (!S) return GS3_ERR_OOM;
  if (o->max_batch < 0 || o->max_batch > kMaxBatch) {
    delete S;
    set_last_error("gs3_server_create: max_batch must be in [0, 8]");
    return GS3_ERR_INVALID_ARG;
  }
  if (o->light_cache < 0 || o->light_cache > 4096) {
    delete S;
    set_last_error("gs3_server_create: light_cache must be in [0, 4096]");
    return GS3_ERR_INVALID_ARG;
  }
  S->budget = o->hbm_budget;
  S->max_batch = o->max_batch > 0 ? o->max_batch : 1;
  S->light_cache_max = o->light_cache;
  S->inject_alloc_failures = o->inject_alloc_failures;
  if (o->initial_pairs > 0.f) S->initial_pairs = o->initial_pairs;
  S->device = o->device;
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete S;
    set_last_error("gs3_server_create: cudaSetDevice failed");
    return GS3_ERR_CUDA;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
    delete S;
    set_last_error("gs3_server_create: cudaMemPoolCreate failed");
    return GS3_ERR_CUDA;
  }
  uint64_t keep = (uint64_t)S->budget;  // keep freed memory in the pool up to the budget
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  S->slots.resize(o->max_inflight);
  bool ok = true;
  for (Slot& sl : S->slots) {
    ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && sl.side.create() && sl.batch.create(S->max_batch);
    ok = ok && cudaEventCreate(&sl.start) == cudaSuccess && cudaEventCreate(&sl.done) == cudaSuccess;
    ok = ok && cudaMalloc(reinterpret_cast<void**>(&sl.param_dev), batch_param_bytes()) == cudaSuccess;
    ok = ok && cudaMallocHost(reinterpret_cast<void**>(&sl.param_host), batch_param_bytes()) == cudaSuccess;
    for (int i = 0; i < kMaxBatch && ok; ++i)
      ok = cudaMallocHost(reinterpret_cast<void**>(&sl.m[i].hdr), sizeof(gs3_ws_header)) == cudaSuccess;
  }
  if (!ok) {
    S->worker = std::thread();
    gs3_server_destroy(S);
    set_last_error("gs3_server_create: stream, event or pinned-memory creation failed");
    return GS3_ERR_CUDA;
  }
  cudaEventCreate(&S->epoch);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return GS3_OK;
}

gs3_status gs3_server_add_scene(gs3_server* S, gs3_scene* scene, int32_t* scene_id) {
  if (!S || !scene || !scene_id) return GS3_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  S->scenes.push_back(scene);
  *scene_id = (int32_t)S->scenes.size() - 1;
  return GS3_OK;
}

gs3_status gs3_server_submit(gs3_server* S, int32_t scene_id, const gs3_camera* cam, const gs3_light* light,
                             const gs3_render_opts* opts, float* out_rgb, uint64_t* ticket) {
  if (!S || !cam || !light || !opts || !out_rgb || !ticket) {
    set_last_error("gs3_server_submit: null argument");
    return GS3_ERR_INVALID_ARG;
  }
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384) {
    set_last_error("gs3_server_submit: image size out of range");
    return GS3_ERR_INVALID_ARG;
  }
  if (!device_range_ok(out_rgb, (size_t)cam->width * cam->height * 3 * sizeof(float))) {
    set_last_error("gs3_server_submit: out_rgb is not device memory of width*height*3 floats");
    return GS3_ERR_INVALID_ARG;
  }
  Request r;
  r.cam = *cam;
  r.light = *light;
  r.opts = *opts;
  r.out = out_rgb;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (scene_id < 0 || scene_id >= (int)S->scenes.size()) {
      set_last_error("gs3_server_submit: unknown scene id");
      return GS3_ERR_INVALID_ARG;
    }
    r.scene = scene_id;
    r.ticket = S->next_ticket++;
    S->results[r.ticket] = Result{};
    S->queue.push_back(r);
    *ticket = r.ticket;
  }
  S->cv_work.notify_one();
  return GS3_OK;
}

gs3_status gs3_server_poll(gs3_server* S, uint64_t ticket, int32_t* state, double* latency_ms) {
  if (!S || !state) return GS3_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) {
    set_last_error("gs3_server_poll: unknown ticket");
    return GS3_ERR_INVALID_ARG;
  }
  *state = it->second.state;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  const gs3_status st = it->second.status;
  if (it->second.state == GS3_REQ_DONE || it->second.state == GS3_REQ_FAILED) S->results.erase(it);
  return st;
}

gs3_status gs3_server_wait(gs3_server* S, uint64_t ticket, double timeout_s, double* latency_ms) {
  if (!S) return GS3_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
      set_last_error("gs3_server_wait: unknown ticket");
      return GS3_ERR_INVALID_ARG;
    }
    if (it->second.state == GS3_REQ_DONE || it->second.state == GS3_REQ_FAILED) {
      if (latency_ms) *latency_ms = it->second.latency_ms;
      const gs3_status st = it->second.status;
      S->results.erase(it);
      return st;
    }
    if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && Clock::now() >= deadline) {
      set_last_error("gs3_server_wait: timed out");
      return GS3_ERR_TIMEOUT;
    }
  }
}

gs3_status gs3_server_stats(gs3_server* S, gs3_server_counters* out) {
  if (!S || !out) return GS3_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  out->completed = S->completed;
  out->failed = S->failed;
  out->retries = S->retries;
  out->queued = S->queue.size();
  int inflight = 0;
  for (Slot& sl : S->slots) inflight += sl.busy ? sl.n : 0;
  out->in_flight = (uint64_t)inflight;
  out->batches = S->batches;
  out->max_batch = (uint64_t)S->max_batch_seen;
  out->light_reuse = S->light_reuse;
  out->max_in_flight = (uint64_t)S->max_inflight_seen;
  out->bytes_in_use = S->in_use;
  out->peak_bytes_in_use = S->peak_in_use;
  out->device_span_ms = S->span_hi > S->span_lo ? S->span_hi - S->span_lo : 0.0;
  return GS3_OK;
}

gs3_status gs3_server_reset_counters(gs3_server* S) {
  if (!S) return GS3_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  S->completed = S->failed = S->retries = 0;
  S->max_inflight_seen = 0;
  S->max_batch_seen = 0;
  S->batches = 0;
  S->light_reuse = 0;
  S->peak_in_use = S->in_use;
  S->epoch_set = false;
  S->span_lo = 1e300;
  S->span_hi = -1e300;
  return GS3_OK;
}

gs3_status gs3_server_destroy(gs3_server* S) {
  if (!S) return GS3_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Slot& sl : S->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  if (!S->slots.empty() && S->slots[0].stream)  // the kept shadow values, once every copy is done
    for (auto& kv : S->light_cache) cudaFreeAsync(kv.second.T, S->slots[0].stream);
  S->light_cache.clear();
  for (Slot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (int i = 0; i < sl.n; ++i)
      if (sl.m[i].ws) cudaFreeAsync(sl.m[i].ws, sl.stream);
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    sl.side.destroy();
    sl.batch.destroy();
    if (sl.param_dev) cudaFree(sl.param_dev);
    if (sl.param_host) cudaFreeHost(sl.param_host);
    for (int i = 0; i < kMaxBatch; ++i)
      if (sl.m[i].hdr) cudaFreeHost(sl.m[i].hdr);
  }
  if (S->epoch) cudaEventDestroy(S->epoch);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
  return GS3_OK;
}

}  // extern "C"
