// K8 (tensor-core forms): Phi (Sec. 4.2) and Psi (Sec. 4.3) on the
// 5th-generation tensor cores, accumulation in FP32 in tensor memory.
// Operands are BF16 (kind::f16, K = 16 per instruction) or FP8 E4M3 with
// per-tensor scales (kind::f8f6f4, K = 32 per instruction).  Both read the
// same K-major, no-swizzle core-matrix layout (8 rows x 16 bytes).
//
// FP8 scales: hidden layer l computes acc = sum_k q(x_k / sx_l) q(w_jk / sw_l)
// and dequantises h = acc sx_l sw_l + b.  sw_l = max|W_l| / 448 (the E4M3
// maximum); sx_l = 2 max|x| / 448 over a calibration pass at scene creation
// (FP32 evaluation of the network on a strided sample of the Gaussians for
// eight fixed directions), so inputs up to twice the calibrated range stay
// finite; larger ones saturate.
//
// One persistent CTA per SM with up to four warpgroups (128 threads each);
// each warpgroup owns one 128-row tile of Gaussians at a time, thread t of
// the group row t, so that up to four tiles are in flight and one group's
// MMAs run while the others encode their inputs or run their epilogues:
//   - once per CTA: the hidden layers' weights (pre-arranged at scene
//     creation in the K-major, no-swizzle core-matrix layout the MMA reads)
//     arrive by bulk TMA copies on an mbarrier, shared by the groups; biases
//     and the FP32 output layer by plain loads; each group gets its own
//     accumulator columns in TMEM;
//   - per tile, within a group: each thread writes its row's encoded input
//     [T, PE(w), PE(mu), l] (K padded to 64) as BF16 into the group's
//     activation tile; for every hidden layer one thread issues the
//     tcgen05.mma chain (M = 128, N = width, K = 16 per instruction) and
//     commits it to the group's mbarrier; after the wait every thread reads
//     its accumulator row back with tcgen05.ld, adds the bias, applies the
//     activation and stores BF16 into the same activation tile as the next
//     layer's A operand (the MMAs that read it have completed); the last
//     hidden layer feeds the output layer and the sigmoid in FP32 registers.
//     A group synchronises on its own named barrier.
// Phi can run over the Gaussians of several lights at once (rows l N + g).
// Every wait is bounded: a timeout sets GS3_ERR_TIMEOUT in the workspace
// header and the CTA frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "gs3_internal.cuh"
#include "tc_ptx.cuh"

namespace gs3 {
namespace {

using namespace tc;

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;   // one warpgroup: a thread per row of a tile
constexpr int kTcMaxGroups = 4;   // tiles in flight per CTA

// tensor-memory columns of a CTA: a width-W accumulator per group, rounded up
// to a power of two >= 32 (the allocation unit)
__host__ __device__ inline uint32_t tc_tmem_cols(int W, int groups) {
  uint32_t c = 32;
  while (c < (uint32_t)(W * groups)) c <<= 1;
  return c;
}
constexpr int kK0 = 64;  // padded input width (61 / 60 features)
struct TcParams {
  int n, which, nh, width, out_dim, act;
  const unsigned char* wblob;  // hidden-layer weight tiles, canonical layout
  const float* scales;         // FP8: (sx_l, sw_l) per hidden layer; null for BF16
  uint32_t wblob_bytes;
  const float* bias;  // nh x width
  const float* wout;  // out_dim x width
  const float* bout;  // out_dim
  const float4* mean_op;
  const float4* latent;
  int nl;                          // Phi: lights of the batch (row l n + g); Psi: 1
  const float* T[kMaxBatch];       // Phi input T per light, by index
  float* out[kMaxBatch];           // Phi: T' per light; Psi: float4 residual at [0]
  const float4* shade[kMaxBatch];  // shading per light, by index (envcol only)
  float4 light[kMaxBatch];         // homogeneous light per light (light_h)
  float cam_pos[3];
  float4* ccol;    // camera colours by rank (nl = 1)
  float4* envcol;  // non-null (Phi): (shade_l, T'_l) at [r nl + l] instead of ccol
  const uint32_t* rank_of;
  uint32_t* status;
};

// [v, sin(2^q pi v), cos(2^q pi v)], q = 0..3.  Band 0 is evaluated; each
// further band doubles the angle (sin 2a = 2 sin a cos a,
// cos 2a = (cos a - sin a)(cos a + sin a)), which stays within about 1e-6 of
// the direct evaluation after three doublings: far below the rounding of the
// BF16 / E4M3 operands these inputs become.
__device__ __forceinline__ void pe_row(float* x, int base, float v0, float v1, float v2) {
  x[base + 0] = v0; x[base + 1] = v1; x[base + 2] = v2;
  float sn[3], cs[3];
  sincospif(v0, &sn[0], &cs[0]);
  sincospif(v1, &sn[1], &cs[1]);
  sincospif(v2, &sn[2], &cs[2]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = base + 3 + 6 * q;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[o + c] = sn[c];
      x[o + 3 + c] = cs[c];
      const float s2 = 2.f * sn[c] * cs[c], c2 = (cs[c] - sn[c]) * (cs[c] + sn[c]);
      sn[c] = s2;
      cs[c] = c2;
    }
  }
}

// 16 bytes of row `row` starting at element k0: 8 BF16 or 16 E4M3 values (times inv)
template <int EB>
__device__ __forceinline__ void store16(unsigned char* tile, int row, int k0, int kdim, const float* v, float inv) {
  uint4 u;
  if constexpr (EB == 2) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __float22bfloat162_rn(make_float2(v[2 * i], v[2 * i + 1]));
    u = *reinterpret_cast<uint4*>(h);
  } else {
    __nv_fp8x2_storage_t h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      h[i] = __nv_cvt_float2_to_fp8x2(make_float2(v[2 * i] * inv, v[2 * i + 1] * inv), __NV_SATFINITE, __NV_E4M3);
    u = *reinterpret_cast<uint4*>(h);
  }
  *reinterpret_cast<uint4*>(tile + canon_off(row, k0 * EB, kdim * EB)) = u;
}

// Named barrier of one warpgroup (ids 1.. ; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kTcThreads) : "memory");
}

// Encoded input row of Gaussian g (under light li for Phi), K padded to 64:
// Phi [T, PE(w_i), PE(mu), l], Psi [PE(w_o), PE(mu), l]; stored as row `row`
// of the K-major input tile.
template <int EB, int WHICH>
__device__ __forceinline__ void encode_row(const TcParams& p, int li, int g, unsigned char* tile, int row) {
  constexpr int kChunk = 16 / EB;
  float x[kK0];
  const float4 m = p.mean_op[g];
  float sx, sy, sz, sw;
  if (WHICH == 0) {
    const float4 lh = p.light[li];
    sx = lh.x; sy = lh.y; sz = lh.z; sw = lh.w;
  } else {
    sx = p.cam_pos[0]; sy = p.cam_pos[1]; sz = p.cam_pos[2]; sw = 1.f;
  }
  float dx = sx - sw * m.x, dy = sy - sw * m.y, dz = sz - sw * m.z;
  const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
  constexpr int b0 = WHICH == 0 ? 1 : 0;
  if (WHICH == 0) x[0] = p.T[li][g];
  pe_row(x, b0, dx * il, dy * il, dz * il);
  pe_row(x, b0 + 27, m.x, m.y, m.z);
  const float4 l0 = p.latent[g], l1 = p.latent[p.n + g];
  x[b0 + 54] = l0.x; x[b0 + 55] = l0.y; x[b0 + 56] = l0.z; x[b0 + 57] = l0.w;
  x[b0 + 58] = l1.x; x[b0 + 59] = l1.y;
#pragma unroll
  for (int k = b0 + 60; k < kK0; ++k) x[k] = 0.f;
  const float inv0 = EB == 1 ? 1.f / p.scales[0] : 1.f;
#pragma unroll
  for (int k0 = 0; k0 < kK0; k0 += kChunk) store16<EB>(tile, row, k0, kK0, x + k0, inv0);
}

// BF16: a layer's bias becomes the accumulator's initial value: this
// thread's row of the group's accumulator columns is set to b before the
// layer's MMAs, which then all accumulate (the sum b + sum_k a_k w_k is
// formed in FP32 by the tensor core; no per-element add in the epilogue).
__device__ __forceinline__ void tmem_bias(uint32_t lane_addr, const float* b, int W) {
  for (int c0 = 0; c0 < W; c0 += 32) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = b[c0 + i];
    tmem_st32(lane_addr + (uint32_t)c0, v);
  }
}

// One CTA per SM, blockDim = 128 x groups: each warpgroup owns one 128-row
// tile at a time, with its own activation tile in shared memory and its own
// accumulator columns in tensor memory, so that one group's MMAs run while
// the others encode or run their epilogues.  The weights are shared.
template <int EB, int WHICH>
__global__ void __launch_bounds__(kTcThreads * kTcMaxGroups, 1) k_mlp_tc(TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_w, bar_mma[kTcMaxGroups];
  __shared__ uint32_t tmem_slot;
  __shared__ int group_fail[kTcMaxGroups];
  const int t = threadIdx.x, warp = t >> 5;
  const int groups = blockDim.x / kTcThreads, grp = t / kTcThreads, tg = t - grp * kTcThreads;
  const int W = p.width, nh = p.nh;
  constexpr int kOut = WHICH == 0 ? 1 : 3;  // outputs of Phi (T') and Psi (residual rgb)
  const uint32_t ncols = tc_tmem_cols(W, groups);
  const int act_bytes = kTcRows * (W > kK0 ? W : kK0) * EB;
  // shared layout: [weights blob][activation tile per group][bias][wout][bout]
  unsigned char* wsm = sm;
  unsigned char* act = sm + ((p.wblob_bytes + 1023) & ~1023u) + grp * act_bytes;
  float* bsm = reinterpret_cast<float*>(sm + ((p.wblob_bytes + 1023) & ~1023u) + groups * act_bytes);
  float* wosm = bsm + nh * W;
  float* bosm = wosm + p.out_dim * W;

  if (warp == 0) {
    tmem_alloc(smem_u32(&tmem_slot), ncols);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(smem_u32(&bar_w), 1);
    for (int g = 0; g < groups; ++g) mbar_init(smem_u32(&bar_mma[g]), 1);
    fence_mbar_init();
  }
  if (t < kTcMaxGroups) group_fail[t] = 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot + (uint32_t)(grp * W);  // this group's accumulator columns
  if (t == 0) {
    mbar_expect_tx(smem_u32(&bar_w), p.wblob_bytes);
    for (uint32_t off = 0; off < p.wblob_bytes; off += 32768u) {
      const uint32_t nb = min(32768u, p.wblob_bytes - off);
      bulk_g2s(smem_u32(wsm + off), p.wblob + off, nb, smem_u32(&bar_w));
    }
  }
  for (int i = t; i < nh * W; i += blockDim.x) bsm[i] = p.bias[i];
  for (int i = t; i < p.out_dim * W; i += blockDim.x) wosm[i] = p.wout[i];
  if (t < p.out_dim) bosm[t] = p.bout[t];
  const bool w_ok = mbar_wait_bounded(smem_u32(&bar_w), 0);
  const int wfail = __syncthreads_or(!w_ok);
  const uint32_t idesc = idesc_mma(EB, kTcRows, W);
  const uint32_t my_lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
  const uint32_t bar = smem_u32(&bar_mma[grp]);
  uint32_t phase = 0;
  const int rows = p.n * p.nl;
  const int ntiles = (rows + kTcRows - 1) / kTcRows;
  bool fail = wfail != 0;
  for (int tile = blockIdx.x * groups + grp; tile < ntiles && !fail; tile += gridDim.x * groups) {
    const int row = tile * kTcRows + tg;
    const int rc = min(row, rows - 1);
    const int li = rc / p.n, g = rc - li * p.n;
    encode_row<EB, WHICH>(p, li, g, act, tg);
    if (EB == 2) {
      tmem_bias(my_lane_addr, bsm, W);  // layer 0's bias; the previous tile's reads are done
      tmem_wait_st();
    }
    fence_proxy_async();
    tc_fence_before();
    group_sync(1 + grp);
    uint32_t woff = 0;
    float acc_out[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) acc_out[o] = 0.f;
    for (int l = 0; l < nh; ++l) {
      const int kdim = l == 0 ? kK0 : W;
      if (tg == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(act), b0 = smem_u32(wsm + woff);
        const uint32_t sbo = (uint32_t)(kdim * EB * 8);
        for (int s = 0; s < kdim * EB / 32; ++s) {  // 32 bytes of K per instruction
          const uint64_t da = smem_desc(a0 + s * 256, 128, sbo), db = smem_desc(b0 + s * 256, 128, sbo);
          if (EB == 2) tc_mma(tmem, da, db, idesc, 1u);  // onto the bias
          else tc_mma_f8(tmem, da, db, idesc, s > 0 ? 1u : 0u);
        }
        tc_commit(bar);
      }
      woff += (uint32_t)(W * kdim * EB);
      const bool mma_ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      if (!mma_ok) group_fail[grp] = 1;
      tc_fence_after();
      const float* bl = bsm + l * W;
      const float deq = EB == 1 ? p.scales[2 * l] * p.scales[2 * l + 1] : 1.f;
      const float inv_next = EB == 1 && l + 1 < nh ? 1.f / p.scales[2 * l + 2] : 1.f;
      for (int c0 = 0; c0 < W; c0 += 32) {
        float v[32];
        tmem_ld32(my_lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float h = EB == 1 ? fmaf(v[i], deq, bl[c0 + i]) : v[i];  // BF16: the bias is in the sum
          // leaky ReLU as max(h, 0.01 h) (slope below 1), ReLU as max(h, 0)
          v[i] = fmaxf(h, leaky ? 0.01f * h : 0.f);
        }
        if (l + 1 < nh) {
#pragma unroll
          for (int i = 0; i < 32; i += 16 / EB) store16<EB>(act, tg, c0 + i, W, v + i, inv_next);
          if (EB == 2) {  // the next layer's bias into the columns just read
            float bn[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) bn[i] = bl[W + c0 + i];
            tmem_st32(my_lane_addr + (uint32_t)c0, bn);
          }
        } else {
#pragma unroll
          for (int o = 0; o < kOut; ++o) {
            const float* wr = wosm + o * W + c0;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) s = fmaf(v[i], wr[i], s);
            acc_out[o] += s;
          }
        }
      }
      if (EB == 2 && l + 1 < nh) tmem_wait_st();
      tc_fence_before();
      fence_proxy_async();
      group_sync(1 + grp);
      fail = group_fail[grp] != 0;
      if (fail) break;
    }
    if (fail) break;
    if (row < rows) {
      const uint32_t r = p.rank_of[g];
      if (WHICH == 0) {
        const float y = 1.f / (1.f + __expf(-(acc_out[0] + bosm[0])));
        p.out[li][g] = y;
        if (p.envcol) {
          const float4 c = p.shade[li][g];
          p.envcol[(size_t)r * p.nl + li] = make_float4(c.x, c.y, c.z, y);
        } else {
          p.ccol[2 * r].w = y;
        }
      } else {
        float4 y;
        y.x = 1.f / (1.f + __expf(-(acc_out[0] + bosm[0])));
        y.y = 1.f / (1.f + __expf(-(acc_out[1] + bosm[1])));
        y.z = 1.f / (1.f + __expf(-(acc_out[2] + bosm[2])));
        y.w = 0.f;
        reinterpret_cast<float4*>(p.out[0])[g] = y;
        p.ccol[2 * r + 1] = y;
      }
    }
  }
  if (fail) {
    if (tg == 0) atomicCAS(p.status, 0u, (uint32_t)GS3_ERR_TIMEOUT);
    if (!w_ok) mbar_wait_bounded(smem_u32(&bar_w), 0);  // let our own bulk copies land before leaving
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_slot, ncols);
}

// FP32 (out, in) row-major weights -> canonical tile [out rows][kdim] (K
// zero-padded), BF16, or E4M3 of w / sw with sw read from *scale (FP8)
__global__ void k_pack(const float* __restrict__ w, int out, int in, int kdim, int eb, const float* scale,
                       unsigned char* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= out * kdim) return;
  const int r = i / kdim, k = i - r * kdim;
  const float v = k < in ? w[(size_t)r * in + k] : 0.f;
  if (eb == 2) {
    *reinterpret_cast<__nv_bfloat16*>(dst + canon_off(r, 2 * k, 2 * kdim)) = __float2bfloat16_rn(v);
  } else {
    dst[canon_off(r, k, kdim)] = __nv_cvt_float_to_fp8(v / *scale, __NV_SATFINITE, __NV_E4M3);
  }
}

constexpr float kE4M3Max = 448.f;

// sw = max|W| / 448 of one layer (one block; layers hold at most 128 x 128 values)
__global__ void k_weight_scale(const float* __restrict__ w, int count, float* scale) {
  __shared__ float red[256];
  float m = 0.f;
  for (int i = threadIdx.x; i < count; i += blockDim.x) m = fmaxf(m, fabsf(w[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *scale = red[0] > 0.f ? red[0] / kE4M3Max : 1.f;
}

constexpr int kCalibDirs = 8;
constexpr int kCalibSample = 16384;
constexpr int kCalibThreads = 64;  // 64 rows x (width + 1) floats of shared memory: <= 33 KB

// Calibration forward pass in FP32: row = (sample i, direction d); records
// max |input| of every hidden layer (as float bits; all values >= 0) in amax[l].
__global__ void __launch_bounds__(kCalibThreads) k_calib(MlpDev m, int which, int n, const float4* __restrict__ mean_op,
                                               const float4* __restrict__ latent, int samples,
                                               uint32_t* __restrict__ amax) {
  extern __shared__ float hs[];  // [kCalibThreads][W + 1]
  const int W = m.width, t = threadIdx.x;
  const int row = blockIdx.x * kCalibThreads + t;
  const bool live = row < samples * kCalibDirs;
  const int i = live ? row / kCalibDirs : 0, d = row % kCalibDirs;
  const int g = (int)(((long long)i * n) / samples);
  // direction d of a Fibonacci sphere of kCalibDirs points
  const float zc = 1.f - (2.f * d + 1.f) / kCalibDirs, rc = sqrtf(fmaxf(0.f, 1.f - zc * zc));
  const float ph = 2.39996323f * d;
  float x[kK0];
  const float4 mu = mean_op[g];
  const int b0 = which == 0 ? 1 : 0;
  if (which == 0) x[0] = (d & 1) ? 1.f : 0.f;
  pe_row(x, b0, rc * cosf(ph), rc * sinf(ph), zc);
  pe_row(x, b0 + 27, mu.x, mu.y, mu.z);
  const float4 l0 = latent[g], l1 = latent[n + g];
  x[b0 + 54] = l0.x; x[b0 + 55] = l0.y; x[b0 + 56] = l0.z; x[b0 + 57] = l0.w;
  x[b0 + 58] = l1.x; x[b0 + 59] = l1.y;
  float* h = hs + t * (W + 1);
  __shared__ float red[kCalibThreads];
  const float* w = m.w;
  const float* b = m.b;
  const bool leaky = m.act == GS3_ACT_LEAKY_RELU;
  for (int l = 0; l < m.n_hidden; ++l) {
    const int din = l == 0 ? m.in_dim : W;
    float mx = 0.f;
    for (int k = 0; k < din; ++k) mx = fmaxf(mx, fabsf(l == 0 ? x[k] : h[k]));
    red[t] = live ? mx : 0.f;
    __syncthreads();
    for (int o = kCalibThreads / 2; o > 0; o >>= 1) {
      if (t < o) red[t] = fmaxf(red[t], red[t + o]);
      __syncthreads();
    }
    if (t == 0) atomicMax(&amax[l], __float_as_uint(red[0]));
    __syncthreads();  // red is reused by the next layer
    float out[128];
    for (int j = 0; j < W; ++j) {
      float s = b[j];
      for (int k = 0; k < din; ++k) s = fmaf(l == 0 ? x[k] : h[k], w[(size_t)j * din + k], s);
      out[j] = s > 0.f ? s : (leaky ? 0.01f * s : 0.f);
    }
    for (int j = 0; j < W; ++j) h[j] = out[j];
    w += (size_t)W * din;
    b += W;
  }
}

__global__ void k_calib_finish(const uint32_t* amax, int nh, float* scales) {
  const int l = threadIdx.x;
  if (l < nh) {
    const float a = __uint_as_float(amax[l]);
    scales[2 * l] = a > 0.f ? 2.f * a / kE4M3Max : 1.f;
  }
}

}  // namespace

static int elem_bytes(int dtype) { return dtype == GS3_MLP_FP8_E4M3 ? 1 : 2; }

static size_t weight_bytes(const MlpDev& m, int eb) {
  size_t b = 0;
  for (int l = 0; l < m.n_hidden; ++l) b += (size_t)m.width * (l == 0 ? kK0 : m.width) * eb;
  return b;
}
static size_t scale_offset(const MlpDev& m, int eb) { return (weight_bytes(m, eb) + 255) & ~size_t(255); }

size_t mlp_tc_scale_offset(const MlpDev& m, int dtype) { return scale_offset(m, elem_bytes(dtype)); }

// blob = [weight tiles][FP8: scales (sx, sw) x n_hidden][FP8: amax scratch]
size_t mlp_tc_blob_bytes(const MlpDev& m, int dtype) {
  const int eb = elem_bytes(dtype);
  return eb == 2 ? weight_bytes(m, eb) : scale_offset(m, eb) + 2 * 4 * 4 + 4 * 4;
}

// Arrange the hidden layers' weights for the tensor cores (and, for FP8,
// derive the per-tensor scales); stream-ordered.
void pack_mlp_tc(const MlpDev& m, int dtype, const SceneDev& sc, int which, unsigned char* dst, cudaStream_t s) {
  const int eb = elem_bytes(dtype);
  float* scales = reinterpret_cast<float*>(dst + scale_offset(m, eb));
  uint32_t* amax = reinterpret_cast<uint32_t*>(scales + 8);
  if (eb == 1) {
    cudaMemsetAsync(amax, 0, 4 * sizeof(uint32_t), s);
    const int samples = sc.n < kCalibSample ? sc.n : kCalibSample;
    const int rows = samples * kCalibDirs;
    const size_t shm = (size_t)kCalibThreads * (m.width + 1) * sizeof(float);
    k_calib<<<(rows + kCalibThreads - 1) / kCalibThreads, kCalibThreads, shm, s>>>(m, which, sc.n, sc.mean_op,
                                                                                  sc.latent, samples, amax);
    k_calib_finish<<<1, 32, 0, s>>>(amax, m.n_hidden, scales);
    count_launch(2);
  }
  size_t off = 0;
  const float* w = m.w;
  for (int l = 0; l < m.n_hidden; ++l) {
    const int in = l == 0 ? m.in_dim : m.width, kdim = l == 0 ? kK0 : m.width;
    const int nel = m.width * kdim;
    if (eb == 1) {
      k_weight_scale<<<1, 256, 0, s>>>(w, m.width * in, scales + 2 * l + 1);
      count_launch();
    }
    k_pack<<<(nel + 255) / 256, 256, 0, s>>>(w, m.width, in, kdim, eb, scales + 2 * l + 1, dst + off);
    count_launch();
    off += (size_t)nel * eb;
    w += (size_t)m.width * in;
  }
}

// dynamic shared memory of a CTA with `groups` tiles in flight
static size_t tc_smem_bytes(const MlpDev& m, int eb, int groups) {
  const size_t blob = (weight_bytes(m, eb) + 1023) & ~size_t(1023);
  const size_t act = (size_t)kTcRows * (m.width > kK0 ? m.width : kK0) * eb;
  return blob + groups * act + 4 * ((size_t)m.n_hidden * m.width + (size_t)m.out_dim * m.width + m.out_dim);
}

constexpr size_t kTcSmemCap = 220 * 1024;

// Tiles in flight per CTA: as many as fit, up to kTcMaxGroups.
static int tc_groups(const MlpDev& m, int eb) {
  int g = kTcMaxGroups;
  while (g > 1 && tc_smem_bytes(m, eb, g) > kTcSmemCap) --g;
  return g;
}

bool mlp_tc_supported(const MlpDev& m, int dtype) {
  const int eb = elem_bytes(dtype);
  (void)eb;
  // the epilogue moves accumulator columns 32 at a time
  const bool width_ok = m.width == 32 || m.width == 64 || m.width == 128;
  return m.in_dim <= kK0 && m.out_dim <= 4 && m.n_hidden >= 1 && m.n_hidden <= 4 && width_ok &&
         tc_smem_bytes(m, eb, 1) <= kTcSmemCap;
}

namespace {

// parameters of one network over one frame's Gaussians (lights filled by the caller)
TcParams tc_params(const FrameArgs& f, int which, const unsigned char* blob) {
  const int eb = elem_bytes(f.sc.mlp_dtype);
  const MlpDev& m = which == 0 ? f.sc.phi : f.sc.psi;
  TcParams p;
  p.n = f.sc.n;
  p.which = which;
  p.nh = m.n_hidden;
  p.width = m.width;
  p.out_dim = m.out_dim;
  p.act = m.act;
  p.wblob = blob;
  p.wblob_bytes = (uint32_t)weight_bytes(m, eb);
  p.scales = eb == 1 ? reinterpret_cast<const float*>(blob + scale_offset(m, eb)) : nullptr;
  size_t hidden_w = 0;
  for (int l = 0; l < m.n_hidden; ++l) hidden_w += (size_t)m.width * (l == 0 ? m.in_dim : m.width);
  p.bias = m.b;
  p.wout = m.w + hidden_w;
  p.bout = m.b + (size_t)m.n_hidden * m.width;
  p.mean_op = f.sc.mean_op;
  p.latent = f.sc.latent;
  p.nl = 1;
  p.T[0] = at<float>(f.ws, f.L->T);
  p.out[0] = at<float>(f.ws, which == 0 ? f.L->Tp : f.L->res);
  p.shade[0] = at<float4>(f.ws, f.L->shade);
  p.light[0] = light_h(f.light);
  for (int i = 0; i < 3; ++i) p.cam_pos[i] = f.cam.pos[i];
  p.ccol = at<float4>(f.ws, f.L->ccol);
  p.envcol = nullptr;
  p.rank_of = at<uint32_t>(f.ws, f.L->sp[0].rank_of);
  p.status = at<uint32_t>(f.ws, f.L->header) + H_STATUS;
  return p;
}

void launch_tc(const TcParams& p, const MlpDev& m, int eb, cudaStream_t s) {
  const int groups = tc_groups(m, eb);
  size_t smem = tc_smem_bytes(m, eb, groups);
  // CTAs of this kernel (of any launch) that share an SM must fit in its 512
  // tensor-memory columns, or an allocation would wait for another CTA to
  // finish: pad the shared memory so that no more than that many fit
  const int max_ctas = (int)(512 / tc_tmem_cols(m.width, groups));
  const size_t per_sm = 228 * 1024, reserve = 2048;  // reserved and static shared memory per CTA
  const size_t floor_bytes = per_sm / (size_t)(max_ctas + 1) + 1;
  if (smem + reserve < floor_bytes) smem = floor_bytes - reserve;
  auto kern = eb == 2 ? (p.which == 0 ? k_mlp_tc<2, 0> : k_mlp_tc<2, 1>)
                      : (p.which == 0 ? k_mlp_tc<1, 0> : k_mlp_tc<1, 1>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nsm = device_sm_count();
  const int ntiles = (p.n * p.nl + kTcRows - 1) / kTcRows;
  const int ctas = (ntiles + groups - 1) / groups;
  const int grid = ctas < nsm ? ctas : nsm;
  kern<<<grid, kTcThreads * groups, smem, s>>>(p);
  count_launch();
}

}  // namespace

void launch_mlp_tc(const FrameArgs& f, const unsigned char* const blobs[2], cudaStream_t s, int which_mask) {
  const int eb = elem_bytes(f.sc.mlp_dtype);
  for (int which = 0; which < 2; ++which) {
    if (!(which_mask & (1 << which))) continue;
    const bool identity = (f.opts.ablate & (which == 0 ? GS3_ABLATE_PHI : GS3_ABLATE_PSI)) != 0;
    if (identity) continue;  // handled by the FP32 kernel's identity path
    launch_tc(tc_params(f, which, blobs[which]), which == 0 ? f.sc.phi : f.sc.psi, eb, s);
  }
}

void launch_phi_lights_tc(const FrameArgs* const* f, int nl, float4* envcol, const unsigned char* blob,
                          cudaStream_t s) {
  TcParams p = tc_params(*f[0], 0, blob);
  p.nl = nl;
  for (int l = 0; l < nl; ++l) {
    p.T[l] = at<float>(f[l]->ws, f[l]->L->T);
    p.out[l] = at<float>(f[l]->ws, f[l]->L->Tp);
    p.shade[l] = at<float4>(f[l]->ws, f[l]->L->shade);
    p.light[l] = light_h(f[l]->light);
  }
  p.ccol = nullptr;
  p.envcol = envcol;
  launch_tc(p, f[0]->sc.phi, elem_bytes(f[0]->sc.mlp_dtype), s);
}

}  // namespace gs3
