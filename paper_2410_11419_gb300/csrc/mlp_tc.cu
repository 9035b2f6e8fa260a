// K8 (BF16 form): Phi (Sec. 4.2) and Psi (Sec. 4.3) on the 5th-generation
// tensor cores.  Operands in BF16, accumulation in FP32 in tensor memory.
//
// One persistent CTA per SM, 128 threads, thread t owns row t of a 128-row
// tile of Gaussians:
//   - once per CTA: the hidden layers' BF16 weights (pre-arranged at scene
//     creation in the K-major, no-swizzle core-matrix layout the MMA reads)
//     arrive by bulk TMA copies on an mbarrier; biases and the FP32 output
//     layer by plain loads; the accumulator columns are allocated in TMEM;
//   - per tile: each thread writes its row's encoded input [T, PE(w), PE(mu), l]
//     (K padded to 64) as BF16 into shared memory; for every hidden layer one
//     thread issues the tcgen05.mma chain (M = 128, N = width, K = 16 per
//     instruction) and commits it to an mbarrier; after the wait every thread
//     reads its accumulator row back with tcgen05.ld, adds the bias, applies
//     the activation and stores BF16 as the next layer's A operand; the last
//     hidden layer feeds the output layer and the sigmoid in FP32 registers.
// Every wait is bounded: a timeout sets GS3_ERR_TIMEOUT in the workspace
// header and the CTA frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kK0 = 64;  // padded input width (61 / 60 features)
constexpr uint32_t kWaitLimit = 1u << 22;

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major, no swizzle.  Core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// byte offset of element (r, k) in a K-major no-swizzle tile of kdim columns
__host__ __device__ inline uint32_t canon_off(int r, int k, int kdim) {
  return (uint32_t)((r >> 3) * (kdim * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcParams {
  int n, which, nh, width, out_dim, act;
  const unsigned char* wblob;  // BF16 hidden-layer tiles, canonical layout
  uint32_t wblob_bytes;
  const float* bias;  // nh x width
  const float* wout;  // out_dim x width
  const float* bout;  // out_dim
  const float4* mean_op;
  const float4* latent;
  const float* T;
  float light_pos[3], cam_pos[3];
  float* out_idx;
  float4* ccol;
  const uint32_t* rank_of;
  uint32_t* status;
};

__device__ __forceinline__ void pe_row(float* x, int base, float v0, float v1, float v2) {
  x[base + 0] = v0; x[base + 1] = v1; x[base + 2] = v2;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float f = (float)(1 << q);
    const int o = base + 3 + 6 * q;
    sincospif(f * v0, &x[o + 0], &x[o + 3]);
    sincospif(f * v1, &x[o + 1], &x[o + 4]);
    sincospif(f * v2, &x[o + 2], &x[o + 5]);
  }
}

__device__ __forceinline__ void store_bf16x8(unsigned char* tile, int row, int k0, int kdim, const float* v) {
  __nv_bfloat162 h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __float22bfloat162_rn(make_float2(v[2 * i], v[2 * i + 1]));
  *reinterpret_cast<uint4*>(tile + canon_off(row, k0, kdim)) = *reinterpret_cast<uint4*>(h);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc(TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_slot;
  const int t = threadIdx.x, warp = t >> 5;
  const int W = p.width, nh = p.nh;
  const uint32_t ncols = W < 32 ? 32u : (uint32_t)W;
  // shared layout: [weights blob][X 128 x 64][H 128 x W][bias][wout][bout]
  unsigned char* wsm = sm;
  unsigned char* xsm = sm + ((p.wblob_bytes + 1023) & ~1023u);
  unsigned char* hsm = xsm + kTcRows * kK0 * 2;
  float* bsm = reinterpret_cast<float*>(hsm + kTcRows * W * 2);
  float* wosm = bsm + nh * W;
  float* bosm = wosm + p.out_dim * W;

  if (warp == 0) {
    tmem_alloc(smem_u32(&tmem_slot), ncols);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(smem_u32(&bar_w), 1);
    mbar_init(smem_u32(&bar_mma), 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (t == 0) {
    mbar_expect_tx(smem_u32(&bar_w), p.wblob_bytes);
    for (uint32_t off = 0; off < p.wblob_bytes; off += 32768u) {
      const uint32_t nb = min(32768u, p.wblob_bytes - off);
      bulk_g2s(smem_u32(wsm + off), p.wblob + off, nb, smem_u32(&bar_w));
    }
  }
  for (int i = t; i < nh * W; i += kTcThreads) bsm[i] = p.bias[i];
  for (int i = t; i < p.out_dim * W; i += kTcThreads) wosm[i] = p.wout[i];
  if (t < p.out_dim) bosm[t] = p.bout[t];
  const bool w_ok = mbar_wait_bounded(smem_u32(&bar_w), 0);
  int fail = __syncthreads_or(!w_ok);
  const uint32_t idesc = idesc_bf16(kTcRows, W);
  const uint32_t my_lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
  uint32_t phase = 0;
  const int ntiles = (p.n + kTcRows - 1) / kTcRows;
  for (int tile = blockIdx.x; tile < ntiles && !fail; tile += gridDim.x) {
    const int row = tile * kTcRows + t;
    const int g = min(row, p.n - 1);
    // ---- encoded input row, BF16, K padded to 64 ----
    {
      float x[kK0];
      const float4 m = p.mean_op[g];
      const float* src = p.which == 0 ? p.light_pos : p.cam_pos;
      float dx = src[0] - m.x, dy = src[1] - m.y, dz = src[2] - m.z;
      const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
      const int b0 = p.which == 0 ? 1 : 0;
      if (p.which == 0) x[0] = p.T[g];
      pe_row(x, b0, dx * il, dy * il, dz * il);
      pe_row(x, b0 + 27, m.x, m.y, m.z);
      const float4 l0 = p.latent[g], l1 = p.latent[p.n + g];
      x[b0 + 54] = l0.x; x[b0 + 55] = l0.y; x[b0 + 56] = l0.z; x[b0 + 57] = l0.w;
      x[b0 + 58] = l1.x; x[b0 + 59] = l1.y;
#pragma unroll
      for (int k = b0 + 60; k < kK0; ++k) x[k] = 0.f;
#pragma unroll
      for (int k0 = 0; k0 < kK0; k0 += 8) store_bf16x8(xsm, t, k0, kK0, x + k0);
    }
    fence_proxy_async();
    __syncthreads();
    uint32_t woff = 0;
    float acc_out[4] = {0.f, 0.f, 0.f, 0.f};
    for (int l = 0; l < nh; ++l) {
      const int kdim = l == 0 ? kK0 : W;
      if (t == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(l == 0 ? xsm : hsm), b0 = smem_u32(wsm + woff);
        for (int s = 0; s < kdim / 16; ++s)
          tc_mma(tmem, smem_desc(a0 + s * 256, 128, kdim * 16), smem_desc(b0 + s * 256, 128, kdim * 16), idesc,
                 s > 0 ? 1u : 0u);
        tc_commit(smem_u32(&bar_mma));
      }
      woff += (uint32_t)(W * kdim * 2);
      const bool mma_ok = mbar_wait_bounded(smem_u32(&bar_mma), phase);
      phase ^= 1u;
      tc_fence_after();
      const float* bl = bsm + l * W;
      for (int c0 = 0; c0 < W; c0 += 32) {
        float v[32];
        tmem_ld32(my_lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          float h = v[i] + bl[c0 + i];
          v[i] = h > 0.f ? h : (leaky ? 0.01f * h : 0.f);
        }
        if (l + 1 < nh) {
#pragma unroll
          for (int i = 0; i < 32; i += 8) store_bf16x8(hsm, t, c0 + i, W, v + i);
        } else {
          for (int o = 0; o < p.out_dim; ++o) {
            const float* wr = wosm + o * W + c0;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) s = fmaf(v[i], wr[i], s);
            acc_out[o] += s;
          }
        }
      }
      tc_fence_before();
      fence_proxy_async();
      fail = __syncthreads_or(!mma_ok);
      if (fail) break;
    }
    if (fail) break;
    if (row < p.n) {
      const uint32_t r = p.rank_of[row];
      if (p.which == 0) {
        const float y = 1.f / (1.f + __expf(-(acc_out[0] + bosm[0])));
        p.out_idx[row] = y;
        p.ccol[2 * r].w = y;
      } else {
        float4 y;
        y.x = 1.f / (1.f + __expf(-(acc_out[0] + bosm[0])));
        y.y = 1.f / (1.f + __expf(-(acc_out[1] + bosm[1])));
        y.z = 1.f / (1.f + __expf(-(acc_out[2] + bosm[2])));
        y.w = 0.f;
        reinterpret_cast<float4*>(p.out_idx)[row] = y;
        p.ccol[2 * r + 1] = y;
      }
    }
  }
  if (fail) {
    if (t == 0) atomicCAS(p.status, 0u, (uint32_t)GS3_ERR_TIMEOUT);
    if (!w_ok) mbar_wait_bounded(smem_u32(&bar_w), 0);  // let our own bulk copies land before leaving
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// FP32 (out, in) row-major weights -> BF16 canonical tile [out rows][kdim] (K zero-padded)
__global__ void k_pack_bf16(const float* __restrict__ w, int out, int in, int kdim, unsigned char* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= out * kdim) return;
  const int r = i / kdim, k = i - r * kdim;
  const float v = k < in ? w[(size_t)r * in + k] : 0.f;
  *reinterpret_cast<__nv_bfloat16*>(dst + canon_off(r, k, kdim)) = __float2bfloat16_rn(v);
}

}  // namespace

size_t mlp_tc_blob_bytes(const MlpDev& m) {
  size_t b = 0;
  for (int l = 0; l < m.n_hidden; ++l) b += (size_t)m.width * (l == 0 ? kK0 : m.width) * 2;
  return b;
}

// Arrange the hidden layers' weights for the tensor cores; returns the bytes written.
size_t pack_mlp_tc(const MlpDev& m, unsigned char* dst, cudaStream_t s) {
  size_t off = 0;
  const float* w = m.w;
  for (int l = 0; l < m.n_hidden; ++l) {
    const int in = l == 0 ? m.in_dim : m.width, kdim = l == 0 ? kK0 : m.width;
    const int nel = m.width * kdim;
    k_pack_bf16<<<(nel + 255) / 256, 256, 0, s>>>(w, m.width, in, kdim, dst + off);
    count_launch();
    off += (size_t)nel * 2;
    w += (size_t)m.width * in;
  }
  return off;
}

static size_t tc_smem_bytes(const MlpDev& m) {
  const size_t blob = (mlp_tc_blob_bytes(m) + 1023) & ~size_t(1023);
  return blob + kTcRows * kK0 * 2 + (size_t)kTcRows * m.width * 2 +
         4 * ((size_t)m.n_hidden * m.width + (size_t)m.out_dim * m.width + m.out_dim);
}

bool mlp_tc_supported(const MlpDev& m) {
  return m.in_dim <= kK0 && m.out_dim <= 4 && m.n_hidden >= 1 &&
         (m.width == 16 || m.width == 32 || m.width == 64 || m.width == 128) && tc_smem_bytes(m) <= 220 * 1024;
}

void launch_mlp_tc(const FrameArgs& f, const unsigned char* const blobs[2], cudaStream_t s) {
  for (int which = 0; which < 2; ++which) {
    const MlpDev& m = which == 0 ? f.sc.phi : f.sc.psi;
    const bool identity = (f.opts.ablate & (which == 0 ? GS3_ABLATE_PHI : GS3_ABLATE_PSI)) != 0;
    if (identity) continue;  // handled by the FP32 kernel's identity path
    TcParams p;
    p.n = f.sc.n;
    p.which = which;
    p.nh = m.n_hidden;
    p.width = m.width;
    p.out_dim = m.out_dim;
    p.act = m.act;
    p.wblob = blobs[which];
    p.wblob_bytes = (uint32_t)mlp_tc_blob_bytes(m);
    size_t hidden_w = 0;
    for (int l = 0; l < m.n_hidden; ++l) hidden_w += (size_t)m.width * (l == 0 ? m.in_dim : m.width);
    p.bias = m.b;
    p.wout = m.w + hidden_w;
    p.bout = m.b + (size_t)m.n_hidden * m.width;
    p.mean_op = f.sc.mean_op;
    p.latent = f.sc.latent;
    p.T = at<float>(f.ws, f.L->T);
    for (int i = 0; i < 3; ++i) { p.light_pos[i] = f.light.pos[i]; p.cam_pos[i] = f.cam.pos[i]; }
    p.out_idx = at<float>(f.ws, which == 0 ? f.L->Tp : f.L->res);
    p.ccol = at<float4>(f.ws, f.L->ccol);
    p.rank_of = at<uint32_t>(f.ws, f.L->sp[0].rank_of);
    p.status = at<uint32_t>(f.ws, f.L->header) + H_STATUS;
    const size_t smem = tc_smem_bytes(m);
    cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (f.sc.n + kTcRows - 1) / kTcRows;
    const int grid = ntiles < nsm ? ntiles : nsm;
    k_mlp_tc<<<grid, kTcThreads, smem, s>>>(p);
    count_launch();
  }
}

}  // namespace gs3
