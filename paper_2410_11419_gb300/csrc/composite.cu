// K6, K7: shadow splatting (Sec. 4.2, Fig. 3) and K9: camera compositing
// (Sec. 3, Eq. 2) with the deferred per-pixel combination (Sec. 4).
//
// Both composites run one 256-thread block per 16x16 tile, one thread per
// pixel, and stream the tile's depth-ordered list through shared memory in
// batches of 256 records.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr float kSkipPower = -5.6f;  // below ln(1/255): alpha < 1/255 for any opacity <= 1

// Evaluate one splat at a pixel centre: beta = exp(power), alpha = min(amax, gamma beta).
// The centre is (a.x + b.w, a.y + vlo): high part first, so the difference to
// the pixel keeps its precision.
__device__ __forceinline__ bool splat_alpha(const float4 a, const float4 b, float vlo, float fx, float fy,
                                            float amin, float amax, float& beta, float& alpha) {
  const float dx = (fx - a.x) - b.w, dy = (fy - a.y) - vlo;
  const float power = -0.5f * (b.x * dx * dx + b.z * dy * dy) - b.y * dx * dy;
  if (power > 0.f || power < kSkipPower) return false;
  beta = __expf(power);
  alpha = fminf(amax, a.z * beta);
  return alpha >= amin;
}

// ---------------------------------------------------------------------------
// K6: shadow composite.
// For every shadow ray m (light pixel) and every list entry j that passes the
// alpha test, T_m(j) = prod (1 - alpha_k,m) over passing k with
// d_k < d_j - bias.  The list is ordered by distance, so the occluder set of
// j is a prefix of the list; an occluder cursor k trails the receiver cursor
// j and advances, block-uniformly, while d_k < d_j - bias.  Each thread keeps
// its ray's product over the consumed occluders.  Per receiver the block sums
// beta T_m and beta over its 256 rays (warp shuffles, then 8 warps in fixed
// order) and writes one (num, den) partial for the (tile, Gaussian) pair.
// ---------------------------------------------------------------------------
struct ShadowParams {
  const uint32_t* list;
  const uint32_t* tile_start;
  const SplatRec* rrec;
  const uint32_t* off;
  float2* partial;
  int W, H, gx;
  float bias, amin, amax;
};

__global__ void __launch_bounds__(256) k_shadow(ShadowParams p) {
  __shared__ float4 Ra[256], Rb[256];
  __shared__ float Rc[256];
  __shared__ uint32_t Rslot[256];
  __shared__ float4 Oa[256], Ob[256];
  __shared__ float Oc[256];
  __shared__ float2 red[8][256];
  const int tile = blockIdx.x;
  const int tx = tile % p.gx, ty = tile / p.gx;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int px = tx * kTile + (t & 15), py = ty * kTile + (t >> 4);
  const bool inside = px < p.W && py < p.H;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const uint32_t b = p.tile_start[tile], e = p.tile_start[tile + 1];
  float A = 1.f;
  uint32_t k = b, ob = b, oc = 0;
  for (uint32_t rb = b; rb < e; rb += 256) {
    const int rc = (int)min(256u, e - rb);
    __syncthreads();
    if (t < rc) {
      const uint32_t rank = p.list[rb + t];
      const SplatRec q = p.rrec[rank];
      Ra[t] = q.a;
      Rb[t] = q.b;
      Rc[t] = q.c.x;
      Rslot[t] = p.off[rank] + (uint32_t)((ty - q.r.y) * (q.r.z - q.r.x + 1) + (tx - q.r.x));
    }
    __syncthreads();
    for (int jj = 0; jj < rc; ++jj) {
      const float thr = __fsub_rn(Ra[jj].w, p.bias);
      while (k < e) {
        if (k >= ob + oc) {
          __syncthreads();
          ob = k;
          oc = min(256u, e - k);
          if (t < (int)oc) {
            const SplatRec q = p.rrec[p.list[ob + t]];
            Oa[t] = q.a;
            Ob[t] = q.b;
            Oc[t] = q.c.x;
          }
          __syncthreads();
        }
        const float4 oa = Oa[k - ob];
        if (!(oa.w < thr)) break;
        float beta, alpha;
        if (splat_alpha(oa, Ob[k - ob], Oc[k - ob], fx, fy, p.amin, p.amax, beta, alpha)) A *= 1.f - alpha;
        ++k;
      }
      float beta = 0.f, alpha;
      const bool pass = inside && splat_alpha(Ra[jj], Rb[jj], Rc[jj], fx, fy, p.amin, p.amax, beta, alpha);
      float cn = pass ? beta * A : 0.f, cd = pass ? beta : 0.f;
      if (__any_sync(0xffffffffu, pass)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cn += __shfl_xor_sync(0xffffffffu, cn, o);
          cd += __shfl_xor_sync(0xffffffffu, cd, o);
        }
      }
      if (lane == 0) red[warp][jj] = make_float2(cn, cd);
    }
    __syncthreads();
    if (t < rc) {
      float2 s = red[0][t];
#pragma unroll
      for (int w = 1; w < 8; ++w) { s.x += red[w][t].x; s.y += red[w][t].y; }
      p.partial[Rslot[t]] = s;
    }
  }
}

// K7: per Gaussian, sum its (tile) partials in tile order; T = num / den, or 1
// when the Gaussian meets no shadow ray.  One warp per Gaussian rank.
__global__ void __launch_bounds__(256) k_shadow_reduce(int n, const uint32_t* __restrict__ off,
                                                       const uint32_t* __restrict__ cnt,
                                                       const float2* __restrict__ partial,
                                                       const uint32_t* __restrict__ order,
                                                       const uint32_t* header, float* __restrict__ T) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const uint32_t P = header[H_PAIRS_LIGHT];
  const uint32_t o = off[r], c = cnt[r];
  float num = 0.f, den = 0.f;
  if (o + c <= P) {
    for (uint32_t i = lane; i < c; i += 32) {
      const float2 v = partial[o + i];
      num += v.x;
      den += v.y;
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, s);
    den += __shfl_xor_sync(0xffffffffu, den, s);
  }
  if (lane == 0) T[order[r]] = den > 0.f ? num / den : 1.f;
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
  const SplatRec* rrec;
  const float4* ccol;
  float* out;
  float* final_t;
  uint32_t* n_contrib;
  int W, H, gx;
  float amin, amax, tstop;
};

__global__ void __launch_bounds__(256) k_camera(CamParams p) {
  __shared__ float4 Ga[256], Gb[256], C0[256], C1[256];
  __shared__ float Gc[256];
  const int tile = blockIdx.x;
  const int tx = tile % p.gx, ty = tile / p.gx;
  const int t = threadIdx.x;
  const int px = tx * kTile + (t & 15), py = ty * kTile + (t >> 4);
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
      Gc[t] = q.c.x;
      C0[t] = p.ccol[2 * rank];
      C1[t] = p.ccol[2 * rank + 1];
    }
    __syncthreads();
    if (!done) {
      for (int jj = 0; jj < rc; ++jj) {
        consumed = rb - b + jj + 1;
        float beta, alpha;
        if (!splat_alpha(Ga[jj], Gb[jj], Gc[jj], fx, fy, p.amin, p.amax, beta, alpha)) continue;
        const float Tn = T * (1.f - alpha);
        if (Tn < p.tstop) {
          done = true;
          consumed -= 1;
          break;
        }
        const float w = alpha * T;
        const float4 c0 = C0[jj], c1 = C1[jj];
        S0 += w * c0.x; S1 += w * c0.y; S2 += w * c0.z;
        Sh += w * c0.w;
        R0 += w * c1.x; R1 += w * c1.y; R2 += w * c1.z;
        T = Tn;
      }
    }
  }
  if (inside) {
    const size_t pix = (size_t)py * p.W + px;
    p.out[3 * pix + 0] = S0 * Sh + R0;
    p.out[3 * pix + 1] = S1 * Sh + R1;
    p.out[3 * pix + 2] = S2 * Sh + R2;
    p.final_t[pix] = T;
    p.n_contrib[pix] = consumed;
  }
}

}  // namespace

void launch_shadow_composite(const FrameArgs& f, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int fin = (f.L->ntiles <= 256 ? 1 : 2) & 1;
  ShadowParams p;
  p.list = at<uint32_t>(ws, b.tv[fin]);
  p.tile_start = at<uint32_t>(ws, b.tile_start);
  p.rrec = at<SplatRec>(ws, b.rrec);
  p.off = at<uint32_t>(ws, b.off);
  p.partial = at<float2>(ws, f.L->partial);
  p.W = f.L->width; p.H = f.L->height; p.gx = f.L->gx;
  p.bias = f.opts.shadow_bias; p.amin = f.opts.alpha_min; p.amax = f.opts.alpha_max;
  k_shadow<<<f.L->ntiles, 256, 0, s>>>(p);
  count_launch();
}

void launch_shadow_reduce(const FrameArgs& f, cudaStream_t s) {
  const SplatBufs& b = f.L->sp[1];
  unsigned char* ws = f.ws;
  const int n = f.sc.n;
  k_shadow_reduce<<<(n * 32 + 255) / 256, 256, 0, s>>>(
      n, at<uint32_t>(ws, b.off), at<uint32_t>(ws, b.cnt), at<float2>(ws, f.L->partial),
      at<uint32_t>(ws, b.sv[1]), at<uint32_t>(ws, f.L->header), at<float>(ws, f.L->T));
  count_launch();
}

void launch_fill_shadow_one(const FrameArgs& f, cudaStream_t s) {
  const int n = f.sc.n;
  k_fill<<<(n + 255) / 256, 256, 0, s>>>(at<float>(f.ws, f.L->T), n, 1.f);
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
  p.W = f.L->width; p.H = f.L->height; p.gx = f.L->gx;
  p.amin = f.opts.alpha_min; p.amax = f.opts.alpha_max; p.tstop = f.opts.t_stop;
  k_camera<<<f.L->ntiles, 256, 0, s>>>(p);
  count_launch();
}

}  // namespace gs3
