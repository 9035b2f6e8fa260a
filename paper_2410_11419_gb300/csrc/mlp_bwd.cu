// K8b: backward of the Phi (Sec. 4.2) and Psi (Sec. 4.3) MLPs in FP32.
//
// The network is x -> h_1 = act(W_1 x + b_1) -> ... -> h_L -> y = sigmoid(W_o h_L + b_o)
// with x = encode(Gaussian) (the positional encoding of the direction and
// the position, and the latent).  Given dL/dy per Gaussian:
//   dz_o = dL/dy * y (1 - y)
//   dz_L = (dz_o W_o) * act'(h_L)
//   dz_l = (dz_{l+1} W_{l+1}) * act'(h_l),      dx = dz_1 W_1
//   dW_l = sum_g dz_l h_{l-1}^T,  db_l = sum_g dz_l   (h_0 = x),  same for W_o
// and dx goes back through the encoding to the Gaussian's position,
// direction and latent.
//
// Every product over the Gaussians is a dense FP32 GEMM with N rows and
// 128 or fewer columns, run by one register-tiled SIMT kernel: a block
// computes a 128 x 128 tile of C = A B, each thread 8 x 8 of it, with the
// contraction staged through double-buffered shared memory in chunks of 16.
// Its two uses:
//   row GEMM (k_rowgemm):  rows = Gaussians; forward recompute h_l = act(h_{l-1} W_l^T + b_l)
//                          and the data gradients dz_{l-1} = (dz_l W_l) * act'(h_{l-1})
//   weight GEMM (k_wgemm): rows = output units, contraction over Gaussians split
//                          across blocks; per-block partials are summed in block order,
//                          so the gradients do not depend on scheduling.
// The activations and data gradients of one network live in the backward
// workspace (about (64 + 4 W) N floats), shared by Phi and Psi in turn.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kTileR = 128, kTileC = 128, kKc = 16, kPad = 4;
constexpr int kGemmThreads = 256;
constexpr int kXdim = 64;  // encoded input, zero-padded (61 / 60 features)
constexpr int kColorStride = 8;
constexpr int kMlpInStride = 24;
constexpr int kWgemmBlocks = 304;  // two per SM

enum { EPI_BIAS_ACT = 0, EPI_DACT = 1, EPI_NONE = 2 };

// One operand chunk: Op[kk][i] for kk in [k0, k0 + kKc), i in [i0, i0 + 128).
// kk_rows = true:  Op[kk][i] = M[kk * ld + i]   (the contraction index is M's row)
// kk_rows = false: Op[kk][i] = M[i * ld + kk]   (the contraction index is M's column)
// Out-of-range elements read as 0.
struct Operand {
  const float* m;
  int ld, ni, nk;  // leading dimension, extent of i, extent of kk
  bool kk_rows;
};

// The chunk is 16 x 128 = 2048 elements, 8 per thread: element e = q 256 + t.
// Consecutive threads read consecutive addresses of M in both layouts.
__device__ __forceinline__ void fetch_chunk(const Operand& o, int i0, int k0, float (&v)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = q * kGemmThreads + t;
    int kk, i;
    if (o.kk_rows) { kk = e >> 7; i = e & 127; }
    else { kk = e & 15; i = e >> 4; }
    const int gk = k0 + kk, gi = i0 + i;
    v[q] = (gk < o.nk && gi < o.ni) ? (o.kk_rows ? o.m[(size_t)gk * o.ld + gi] : o.m[(size_t)gi * o.ld + gk]) : 0.f;
  }
}
__device__ __forceinline__ void store_chunk(const Operand& o, const float (&v)[8], float (*dst)[kTileR + kPad]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = q * kGemmThreads + t;
    if (o.kk_rows) dst[e >> 7][e & 127] = v[q];
    else dst[e & 15][e >> 4] = v[q];
  }
}

struct GemmSmem {
  float a[2][kKc][kTileR + kPad];
  float b[2][kKc][kTileC + kPad];
};

// acc[r][c] += sum over kk in [kbeg, kend) of A[kk][i0 + 8 ty + r] B[kk][j0 + 8 tx + c];
// with ASUM, thread t < 128 also adds up A[kk][i0 + t] into asum.  The next
// chunk is fetched into registers while the current one is multiplied.
template <bool ASUM>
__device__ __forceinline__ void gemm_tile(GemmSmem& S, const Operand& A, const Operand& B, int i0, int j0,
                                          int kbeg, int kend, float (&acc)[8][8], float& asum) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  float ra[8], rb[8];
  fetch_chunk(A, i0, kbeg, ra);
  fetch_chunk(B, j0, kbeg, rb);
  store_chunk(A, ra, S.a[0]);
  store_chunk(B, rb, S.b[0]);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += kKc) {
    const bool more = k0 + kKc < kend;
    if (more) {
      fetch_chunk(A, i0, k0 + kKc, ra);
      fetch_chunk(B, j0, k0 + kKc, rb);
    }
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&S.a[buf][kk][8 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&S.a[buf][kk][8 * ty + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&S.b[buf][kk][8 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&S.b[buf][kk][8 * tx + 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    if (ASUM && t < kTileR) {
#pragma unroll
      for (int kk = 0; kk < kKc; ++kk) asum += S.a[buf][kk][t];
    }
    if (more) {  // the other buffer was last read before the previous barrier
      store_chunk(A, ra, S.a[buf ^ 1]);
      store_chunk(B, rb, S.b[buf ^ 1]);
    }
    __syncthreads();
    buf ^= 1;
  }
}

// C[g][j] (g = Gaussians) = epi(sum_kk A[g][kk] B[kk][j])
//   EPI_BIAS_ACT: act(. + bias[j])            (forward recompute)
//   EPI_DACT:     . * act'(H[g][j])           (data gradient, H = the layer's output)
//   EPI_NONE:     .                           (dx)
struct RowGemm {
  Operand A, B;
  int n, ncols, kdim;
  float* C;
  int ldc;
  const float* bias;
  const float* H;
  int ldh;
  int act;
};

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 2) k_rowgemm(RowGemm p) {
  __shared__ __align__(16) GemmSmem S;
  const int i0 = blockIdx.x * kTileR;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  float unused = 0.f;
  gemm_tile<false>(S, p.A, p.B, i0, 0, 0, p.kdim, acc, unused);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int g = i0 + 8 * ty + r;
    if (g >= p.n) break;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = 8 * tx + c;
      if (j >= p.ncols) break;
      float v = acc[r][c];
      if (EPI == EPI_BIAS_ACT) {
        v += p.bias[j];
        v = v > 0.f ? v : (leaky ? 0.01f * v : 0.f);
      } else if (EPI == EPI_DACT) {
        const float h = p.H[(size_t)g * p.ldh + j];
        v = h > 0.f ? v : (leaky ? 0.01f * v : 0.f);
      }
      p.C[(size_t)g * p.ldc + j] = v;
    }
  }
}

// Block b: partial[b][j][k] = sum over its Gaussians g of dZ[g][j] H[g][k]
// (j < nout, k < nin), and partial bias sums; written in the parameter order
// (weights row-major, then biases).
struct WGemm {
  Operand A, B;  // A: dZ (kk_rows), B: H (kk_rows)
  int n, nout, nin, rows_per_block;
  float* part;   // [gridDim.x][nout * nin + nout]
};

__global__ void __launch_bounds__(kGemmThreads, 2) k_wgemm(WGemm p) {
  __shared__ __align__(16) GemmSmem S;
  const int kbeg = blockIdx.x * p.rows_per_block;
  const int kend = min(p.n, kbeg + p.rows_per_block);
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  float bsum = 0.f;  // thread j < nout: sum of dZ[g][j] over the block's Gaussians
  if (kbeg < kend) gemm_tile<true>(S, p.A, p.B, 0, 0, kbeg, kend, acc, bsum);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const size_t np = (size_t)p.nout * p.nin + p.nout;
  float* out = p.part + (size_t)blockIdx.x * np;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int j = 8 * ty + r;
    if (j >= p.nout) break;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = 8 * tx + c;
      if (k < p.nin) out[(size_t)j * p.nin + k] = acc[r][c];
    }
  }
  if (t < p.nout) out[(size_t)p.nout * p.nin + t] = bsum;
}

// ---- per-Gaussian steps ----------------------------------------------------
struct RowArgs {
  int n, which, nh, width, out_dim, act;
  const float4* mean_op;
  const float4* latent;
  const float* T;
  float light_pos[3], cam_pos[3];
  float light_w;       // 1: point light at light_pos; 0: directional, light_pos = unit direction
  const float* w_out;  // out_dim x width
  const float* b_out;
  const float* color;  // [N][8]: dT' at 3, dres at 4..6
  float* X;            // [N][kXdim]
  const float* Hlast;  // [N][width]
  float* dzo;          // [N][4]
  float* dZlast;       // [N][width]
  const float* dX;     // [N][kXdim]
  float* dT;
  float* mlp_in;       // [N][24]
};

__device__ __forceinline__ void pe_fwd(float* x, int base, float v0, float v1, float v2) {
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

// d/dv of PE(v) given d/dPE
__device__ __forceinline__ void pe_bwd(const float* dpe, float v0, float v1, float v2, float* dv) {
  const float v[3] = {v0, v1, v2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float g = dpe[c];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float f = (float)(1 << q);
      float s, co;
      sincospif(f * v[c], &s, &co);
      const float k = f * 3.14159265358979323846f;
      g += k * (co * dpe[3 + 6 * q + c] - s * dpe[3 + 6 * q + 3 + c]);
    }
    dv[c] = g;
  }
}

// omega = normalize(src - w mu): w = 1 towards a point, w = 0 a fixed direction
__device__ __forceinline__ void unit_dir(const float* src, float w, const float4 m, float& x, float& y, float& z) {
  x = src[0] - w * m.x; y = src[1] - w * m.y; z = src[2] - w * m.z;
  const float il = rsqrtf(x * x + y * y + z * z);
  x *= il; y *= il; z *= il;
}

// x = [T, PE(w_i), PE(mu), l] (Phi) or [PE(w_o), PE(mu), l] (Psi), zero-padded to 64
__global__ void k_encode(RowArgs p) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.n) return;
  float x[kXdim];
#pragma unroll
  for (int k = 0; k < kXdim; ++k) x[k] = 0.f;
  const float4 m = p.mean_op[g];
  float dx, dy, dz;
  unit_dir(p.which == 0 ? p.light_pos : p.cam_pos, p.which == 0 ? p.light_w : 1.f, m, dx, dy, dz);
  const int b0 = p.which == 0 ? 1 : 0;
  if (p.which == 0) x[0] = p.T[g];
  pe_fwd(x, b0, dx, dy, dz);
  pe_fwd(x, b0 + 27, m.x, m.y, m.z);
  const float4 l0 = p.latent[g], l1 = p.latent[p.n + g];
  x[b0 + 54] = l0.x; x[b0 + 55] = l0.y; x[b0 + 56] = l0.z; x[b0 + 57] = l0.w;
  x[b0 + 58] = l1.x; x[b0 + 59] = l1.y;
  float4* dst = reinterpret_cast<float4*>(p.X + (size_t)g * kXdim);
#pragma unroll
  for (int k = 0; k < kXdim / 4; ++k) dst[k] = make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}

// Output layer, one warp per Gaussian (kOutRowsPerWarp Gaussians per warp in
// turn, the weights staged once per block): y = sigmoid(W_o h_L + b_o),
// dz_o = dL/dy y (1 - y), dz_L = (dz_o W_o) * act'(h_L).  Lane l owns the
// columns l, l + 32, l + 64, l + 96 that exist (widths 16..128).
constexpr int kOutRowsPerWarp = 8;
__global__ void __launch_bounds__(256) k_out_layer(RowArgs p) {
  __shared__ float wo[4 * 128];  // the output layer's weights (out_dim <= 3, width <= 128)
  __shared__ float bo[4];
  const int W = p.width, nq = (W + 31) / 32, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < p.out_dim * W; i += blockDim.x) wo[i] = p.w_out[i];
  if (threadIdx.x < p.out_dim) bo[threadIdx.x] = p.b_out[threadIdx.x];
  __syncthreads();
  const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
  const int warp0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kOutRowsPerWarp;
  for (int g = warp0; g < min(p.n, warp0 + kOutRowsPerWarp); ++g) {
    const float* h = p.Hlast + (size_t)g * W;
    float hv[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < nq; ++q)
      if (lane + 32 * q < W) hv[q] = h[lane + 32 * q];
    float dzo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int o = 0; o < p.out_dim; ++o) {
      float s = 0.f;
      for (int q = 0; q < nq; ++q)
        if (lane + 32 * q < W) s = fmaf(hv[q], wo[o * W + lane + 32 * q], s);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      const float y = 1.f / (1.f + expf(-(s + bo[o])));
      const float dy = p.which == 0 ? p.color[(size_t)kColorStride * g + 3] : p.color[(size_t)kColorStride * g + 4 + o];
      dzo[o] = dy * y * (1.f - y);
    }
    if (lane < 4) p.dzo[(size_t)4 * g + lane] = lane < p.out_dim ? dzo[lane] : 0.f;
    for (int q = 0; q < nq; ++q) {
      const int j = lane + 32 * q;
      if (j >= W) break;
      float s = 0.f;
      for (int o = 0; o < p.out_dim; ++o) s = fmaf(dzo[o], wo[o * W + j], s);
      p.dZlast[(size_t)g * W + j] = hv[q] > 0.f ? s : (leaky ? 0.01f * s : 0.f);
    }
  }
}

// dx back through the encoding: d/dmu (from PE(mu) and the direction), d/dw, d/dl, d/dT
__global__ void k_input_grad(RowArgs p) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.n) return;
  float dx[kXdim];
  const float4* src = reinterpret_cast<const float4*>(p.dX + (size_t)g * kXdim);
#pragma unroll
  for (int k = 0; k < kXdim / 4; ++k) {
    const float4 v = src[k];
    dx[4 * k] = v.x; dx[4 * k + 1] = v.y; dx[4 * k + 2] = v.z; dx[4 * k + 3] = v.w;
  }
  const float4 m = p.mean_op[g];
  float vx, vy, vz;
  unit_dir(p.which == 0 ? p.light_pos : p.cam_pos, p.which == 0 ? p.light_w : 1.f, m, vx, vy, vz);
  const int b0 = p.which == 0 ? 1 : 0;
  float dw[3], dm[3];
  pe_bwd(dx + b0, vx, vy, vz, dw);
  pe_bwd(dx + b0 + 27, m.x, m.y, m.z, dm);
  float* out = p.mlp_in + (size_t)kMlpInStride * g + (p.which == 0 ? 0 : 12);
  out[0] = dm[0]; out[1] = dm[1]; out[2] = dm[2];
  out[3] = dw[0]; out[4] = dw[1]; out[5] = dw[2];
#pragma unroll
  for (int k = 0; k < 6; ++k) out[6 + k] = dx[b0 + 54 + k];
  if (p.which == 0) p.dT[g] = dx[0];
}

__global__ void k_sum_parts(const float* part, size_t np, int nblocks, float* red) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * np + i];
  red[i] = s;
}

int wgemm_blocks(int n) {
  const int by_rows = (n + kKc - 1) / kKc;
  return by_rows < kWgemmBlocks ? by_rows : kWgemmBlocks;
}

struct Scratch {
  float *X, *H, *dz[2], *dzo, *part;
};

Scratch carve(void* base, int n, const MlpDev& m) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  unsigned char* c = static_cast<unsigned char*>(base);
  Scratch s;
  s.X = reinterpret_cast<float*>(c); c += al(4ull * n * kXdim);
  s.H = reinterpret_cast<float*>(c); c += al(4ull * n * m.width * m.n_hidden);
  s.dz[0] = reinterpret_cast<float*>(c); c += al(4ull * n * (m.width > kXdim ? m.width : kXdim));
  s.dz[1] = reinterpret_cast<float*>(c); c += al(4ull * n * (m.width > kXdim ? m.width : kXdim));
  s.dzo = reinterpret_cast<float*>(c); c += al(4ull * n * 4);
  s.part = reinterpret_cast<float*>(c);
  return s;
}

}  // namespace

size_t mlp_bwd_scratch_bytes(int n, const MlpDev& m) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t wide = (size_t)(m.width > kXdim ? m.width : kXdim);
  const size_t layer_max = (size_t)m.width * (m.width > m.in_dim ? m.width : m.in_dim) + m.width;
  return al(4ull * n * kXdim) + al(4ull * n * m.width * m.n_hidden) + 2 * al(4ull * n * wide) +
         al(16ull * n) + al(4ull * wgemm_blocks(n) * layer_max);
}

void run_mlp_backward(const MlpArgs& a, void* scratch, float* wred, cudaStream_t s) {
  const MlpDev& m = a.net;
  const int n = a.n, W = m.width, nh = m.n_hidden;
  Scratch S = carve(scratch, n, m);
  RowArgs r;
  r.n = n; r.which = a.which; r.nh = nh; r.width = W; r.out_dim = m.out_dim; r.act = m.act;
  r.mean_op = a.mean_op; r.latent = a.latent; r.T = a.T;
  for (int i = 0; i < 3; ++i) { r.light_pos[i] = a.light_pos[i]; r.cam_pos[i] = a.cam_pos[i]; }
  r.light_w = a.light_w;
  // parameter offsets: hidden layers (weights then biases), then the output layer
  const float* wl[8];
  const float* bl[8];
  size_t poff[9];
  {
    const float* w = m.w;
    const float* b = m.b;
    size_t off = 0;
    int din = m.in_dim;
    for (int l = 0; l <= nh; ++l) {
      const int dout = l == nh ? m.out_dim : W;
      wl[l] = w; bl[l] = b; poff[l] = off;
      w += (size_t)dout * din; b += dout;
      off += (size_t)dout * din + dout;
      din = dout;
    }
  }
  r.w_out = wl[nh]; r.b_out = bl[nh];
  r.color = a.color; r.X = S.X; r.dT = a.dT; r.mlp_in = a.mlp_in;
  const int rows_grid = (n + kTileR - 1) / kTileR;
  // forward recompute
  k_encode<<<(n + 127) / 128, 128, 0, s>>>(r);
  count_launch();
  for (int l = 0; l < nh; ++l) {
    const int din = l == 0 ? m.in_dim : W;
    RowGemm g;
    g.A = {l == 0 ? S.X : S.H + (size_t)(l - 1) * n * W, l == 0 ? kXdim : W, n, din, false};
    g.B = {wl[l], din, W, din, false};  // B[kk][j] = W_l[j][kk]
    g.n = n; g.ncols = W; g.kdim = din;
    g.C = S.H + (size_t)l * n * W; g.ldc = W;
    g.bias = bl[l]; g.H = nullptr; g.ldh = 0; g.act = m.act;
    k_rowgemm<EPI_BIAS_ACT><<<rows_grid, kGemmThreads, 0, s>>>(g);
    count_launch();
  }
  // output layer, then its weight gradient
  r.Hlast = S.H + (size_t)(nh - 1) * n * W;
  r.dzo = S.dzo;
  r.dZlast = S.dz[0];
  const int out_warps = (n + kOutRowsPerWarp - 1) / kOutRowsPerWarp;
  k_out_layer<<<(out_warps * 32 + 255) / 256, 256, 0, s>>>(r);
  count_launch();
  const int nb = wgemm_blocks(n);
  const int rpb = ((n + nb - 1) / nb + kKc - 1) / kKc * kKc;
  auto wgrad = [&](const float* dZ, int ldz, int nout, const float* Hin, int ldhin, int nin, int layer) {
    WGemm w;
    w.A = {dZ, ldz, nout, n, true};
    w.B = {Hin, ldhin, nin, n, true};
    w.n = n; w.nout = nout; w.nin = nin; w.rows_per_block = rpb;
    w.part = S.part;
    k_wgemm<<<nb, kGemmThreads, 0, s>>>(w);
    const size_t np = (size_t)nout * nin + nout;
    k_sum_parts<<<(int)((np + 255) / 256), 256, 0, s>>>(S.part, np, nb, wred + poff[layer]);
    count_launch(2);
  };
  wgrad(S.dzo, 4, m.out_dim, r.Hlast, W, W, nh);
  // hidden layers, last to first
  int cur = 0;
  for (int l = nh - 1; l >= 0; --l) {
    const int din = l == 0 ? m.in_dim : W;
    const float* Hin = l == 0 ? S.X : S.H + (size_t)(l - 1) * n * W;
    const int ldin = l == 0 ? kXdim : W;
    wgrad(S.dz[cur], W, W, Hin, ldin, din, l);
    // data gradient into the layer below (dx for l = 0)
    RowGemm g;
    g.A = {S.dz[cur], W, n, W, false};
    g.B = {wl[l], din, din, W, true};  // B[kk][j] = W_l[kk][j]
    g.n = n; g.ncols = din; g.kdim = W;
    g.C = S.dz[cur ^ 1]; g.ldc = l == 0 ? kXdim : W;
    g.bias = nullptr; g.act = m.act;
    if (l > 0) {
      g.H = Hin; g.ldh = W;
      k_rowgemm<EPI_DACT><<<rows_grid, kGemmThreads, 0, s>>>(g);
    } else {
      g.H = nullptr; g.ldh = 0;  // columns din..63 of dx stay unwritten and unread
      k_rowgemm<EPI_NONE><<<rows_grid, kGemmThreads, 0, s>>>(g);
    }
    count_launch();
    cur ^= 1;
  }
  r.dX = S.dz[cur];
  k_input_grad<<<(n + 127) / 128, 128, 0, s>>>(r);
  count_launch();
}

}  // namespace gs3
