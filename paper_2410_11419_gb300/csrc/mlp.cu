// K8 (FP32 form): the shadow-refinement MLP Phi (Sec. 4.2) and the residual
// MLP Psi (Sec. 4.3) over all spatial Gaussians.
//
// One 256-thread block owns 64 Gaussians.  The prologue builds the inputs in
// shared memory, feature-major:
//   Phi: [T, PE(w_i), PE(mu), l]  (61)      Psi: [PE(w_o), PE(mu), l]  (60)
//   PE(v) = [v, sin(2^k pi v), cos(2^k pi v)], k = 0..3, per component
// with world-space unit directions w_i = (p_L - mu)/|.|, w_o = (p_C - mu)/|.|.
// Each hidden layer is a 64 x width register-tiled FP32 product against the
// layer's weights staged in shared memory, transposed, in rows padded to
// width + 4 floats: the staging stores of a warp (consecutive inputs k, one
// output j) then spread over 8 banks instead of one, and the rows stay
// 16-byte aligned for the vector loads of the product.  The output layer applies the
// sigmoid.  Outputs go both by Gaussian index and, for the camera composite,
// by camera depth rank.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kRows = 64;
constexpr int kHPad = kRows + 4;  // feature-major activations, padded rows

// Phi runs over the Gaussians of nl lights at once (row l n + g: Gaussian g
// under light l); Psi, which does not see the light, over one set (nl = 1).
struct MlpParams {
  MlpDev net;
  int n;
  int which;  // 0 Phi, 1 Psi
  int nl;     // lights of the batch (Phi), 1 for Psi
  const float4* mean_op;
  const float4* latent;
  const float* T[kMaxBatch];       // Phi input T per light, by index
  float* tp[kMaxBatch];            // Phi output T' per light, by index
  const float4* shade[kMaxBatch];  // shading per light, by index (envcol only)
  float4 light[kMaxBatch];         // homogeneous light per light (light_h)
  float cam_pos[3];
  float* res_idx;    // Psi: float4 residual [N] (as floats)
  float4* ccol;      // camera colours by rank: Phi T' into .w of [2r] (nl = 1), Psi residual into [2r + 1]
  float4* envcol;    // non-null (Phi): (shade_l, T'_l) at [r nl + l] instead of ccol
  const uint32_t* rank_of;
  int identity;      // ablation: Phi -> T' = T, Psi -> 0
};

// Phi's output for Gaussian g under light l, camera rank r
__device__ __forceinline__ void put_phi(const MlpParams& p, int l, int g, uint32_t r, float y) {
  p.tp[l][g] = y;
  if (p.envcol) {
    const float4 c = p.shade[l][g];
    p.envcol[(size_t)r * p.nl + l] = make_float4(c.x, c.y, c.z, y);
  } else {
    p.ccol[2 * r].w = y;
  }
}

__device__ __forceinline__ void write_pe(float (*H)[kHPad], int base, int row, int q, float v0, float v1,
                                         float v2) {
  if (q == 0) {
    H[base + 0][row] = v0;
    H[base + 1][row] = v1;
    H[base + 2][row] = v2;
  }
  const float f = (float)(1 << q);
  float s, c;
  const int o = base + 3 + 6 * q;
  sincospif(f * v0, &s, &c); H[o + 0][row] = s; H[o + 3][row] = c;
  sincospif(f * v1, &s, &c); H[o + 1][row] = s; H[o + 4][row] = c;
  sincospif(f * v2, &s, &c); H[o + 2][row] = s; H[o + 5][row] = c;
}

template <int WIDTH>
__global__ void __launch_bounds__(256) k_mlp(MlpParams p) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float (*H)[kHPad] = reinterpret_cast<float (*)[kHPad]>(smem);  // [128][kHPad]
  float* Ws = smem + 128 * kHPad;                                  // [din][dout]
  const int t = threadIdx.x;
  const int g0 = blockIdx.x * kRows;
  const int rows = p.n * p.nl;

  if (p.identity) {
    if (t < kRows && g0 + t < rows) {
      const int l = (g0 + t) / p.n, g = g0 + t - l * p.n;
      const uint32_t r = p.rank_of[g];
      if (p.which == 0) {
        put_phi(p, l, g, r, p.T[l][g]);
      } else {
        reinterpret_cast<float4*>(p.res_idx)[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        p.ccol[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    return;
  }

  // ---- prologue: inputs, 4 threads per row (thread q handles band q) ----
  {
    const int row = t >> 2, q = t & 3;
    const int rc = min(g0 + row, rows - 1);
    const int l = rc / p.n, g = rc - l * p.n;
    const float4 m = p.mean_op[g];
    const float4 lh = p.light[l];
    const float src[3] = {p.which == 0 ? lh.x : p.cam_pos[0], p.which == 0 ? lh.y : p.cam_pos[1],
                          p.which == 0 ? lh.z : p.cam_pos[2]};
    const float sw = p.which == 0 ? lh.w : 1.f;
    float dx = src[0] - sw * m.x, dy = src[1] - sw * m.y, dz = src[2] - sw * m.z;
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il; dy *= il; dz *= il;
    const int b0 = p.which == 0 ? 1 : 0;
    write_pe(H, b0, row, q, dx, dy, dz);
    write_pe(H, b0 + 27, row, q, m.x, m.y, m.z);
    if (q == 0) {
      const float4 l0 = p.latent[g], l1 = p.latent[p.n + g];
      const int lb = b0 + 54;
      H[lb + 0][row] = l0.x; H[lb + 1][row] = l0.y; H[lb + 2][row] = l0.z; H[lb + 3][row] = l0.w;
      H[lb + 4][row] = l1.x; H[lb + 5][row] = l1.y;
      if (p.which == 0) H[0][row] = p.T[l][g];
    }
  }

  constexpr int CPT = WIDTH / 16;  // columns per thread
  const int tcol = t & 15, trow = t >> 4;
  // output column c of thread column tcol: with 8 per thread two runs of 4
  // (tcol 4 + c and 64 + tcol 4 + c - 4), so that 16 threads' 16-byte
  // weight loads cover 256 contiguous bytes (no bank conflict)
  auto out_col = [](int tc, int c) { return CPT == 8 ? (c >> 2) * 64 + tc * 4 + (c & 3) : tc * CPT + c; };
  int din = p.net.in_dim;
  const float* w = p.net.w;
  const float* bias = p.net.b;
  for (int l = 0; l < p.net.n_hidden; ++l) {
    __syncthreads();  // H complete, previous Ws no longer read
    {
      // W row-major (out, in): thread t takes input k = t % kp of rows
      // j = t / kp, + 256 / kp, ... (kp = din rounded up to 64 or 128), so a
      // warp's loads are consecutive and several are in flight
      const int kp = din <= 64 ? 64 : 128, k = t % kp;
      const int rows = 256 / kp;
      if (k < din) {
#pragma unroll 4
        for (int j = t / kp; j < WIDTH; j += rows) Ws[k * (WIDTH + 4) + j] = w[(size_t)j * din + k];
      }
    }
    __syncthreads();
    float acc[4][CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const float bv = bias[out_col(tcol, c)];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r][c] = bv;
    }
    for (int k = 0; k < din; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&H[k][trow * 4]);
      float bv[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) bv[c] = Ws[k * (WIDTH + 4) + out_col(tcol, c)];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        acc[0][c] = fmaf(a.x, bv[c], acc[0][c]);
        acc[1][c] = fmaf(a.y, bv[c], acc[1][c]);
        acc[2][c] = fmaf(a.z, bv[c], acc[2][c]);
        acc[3][c] = fmaf(a.w, bv[c], acc[3][c]);
      }
    }
    __syncthreads();  // all reads of H done
    const bool leaky = p.net.act == GS3_ACT_LEAKY_RELU;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      float v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = acc[r][c] > 0.f ? acc[r][c] : (leaky ? 0.01f * acc[r][c] : 0.f);
      *reinterpret_cast<float4*>(&H[out_col(tcol, c)][trow * 4]) = make_float4(v[0], v[1], v[2], v[3]);
    }
    w += (size_t)din * WIDTH;
    bias += WIDTH;
    din = WIDTH;
  }
  // ---- output layer + sigmoid (its weights staged where the last layer's were) ----
  const int dout = p.net.out_dim;
  for (int i = t; i < dout * din; i += 256) Ws[i] = w[i];
  __syncthreads();
  if (t < kRows * dout) {
    const int row = t % kRows, o = t / kRows;
    float acc = bias[o];
    const float* wr = Ws + o * din;
    for (int k = 0; k < din; ++k) acc = fmaf(H[k][row], wr[k], acc);
    const float y = 1.f / (1.f + __expf(-acc));
    if (g0 + row < rows) {
      const int l = (g0 + row) / p.n, g = g0 + row - l * p.n;
      const uint32_t r = p.rank_of[g];
      if (p.which == 0) {
        put_phi(p, l, g, r, y);
      } else {
        p.res_idx[4 * g + o] = y;
        reinterpret_cast<float*>(&p.ccol[2 * r + 1])[o] = y;
      }
    }
  }
}

template <int WIDTH>
void launch_width(const MlpParams& p, cudaStream_t s) {
  const size_t sm = (size_t)(128 * kHPad + 128 * (WIDTH + 4)) * sizeof(float);
  static DeviceOnce once;
  once.run([sm] {
    return cudaFuncSetAttribute(k_mlp<WIDTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess;
  });
  k_mlp<WIDTH><<<(p.n * p.nl + kRows - 1) / kRows, 256, sm, s>>>(p);
  count_launch();
}

void launch_one(const MlpParams& p, cudaStream_t s) {
  switch (p.net.width) {
    case 16: launch_width<16>(p, s); break;
    case 32: launch_width<32>(p, s); break;
    case 64: launch_width<64>(p, s); break;
    default: launch_width<128>(p, s); break;
  }
}

}  // namespace

void launch_mlp(const FrameArgs& f, cudaStream_t s, bool identity_only, int which_mask) {
  MlpParams p;
  p.n = f.sc.n;
  p.nl = 1;
  p.mean_op = f.sc.mean_op;
  p.latent = f.sc.latent;
  p.T[0] = at<float>(f.ws, f.L->T);
  p.tp[0] = at<float>(f.ws, f.L->Tp);
  p.shade[0] = at<float4>(f.ws, f.L->shade);
  p.light[0] = light_h(f.light);
  for (int i = 0; i < 3; ++i) p.cam_pos[i] = f.cam.pos[i];
  p.res_idx = at<float>(f.ws, f.L->res);
  p.ccol = at<float4>(f.ws, f.L->ccol);
  p.envcol = nullptr;
  p.rank_of = at<uint32_t>(f.ws, f.L->sp[0].rank_of);

  p.net = f.sc.phi;
  p.which = 0;
  p.identity = (f.opts.ablate & GS3_ABLATE_PHI) != 0;
  if ((which_mask & 1) && (p.identity || !identity_only)) launch_one(p, s);

  p.net = f.sc.psi;
  p.which = 1;
  p.identity = (f.opts.ablate & GS3_ABLATE_PSI) != 0;
  if ((which_mask & 2) && (p.identity || !identity_only)) launch_one(p, s);
}

void launch_phi_lights(const FrameArgs* const* f, int nl, float4* envcol, cudaStream_t s) {
  MlpParams p;
  const FrameArgs& f0 = *f[0];
  p.net = f0.sc.phi;
  p.n = f0.sc.n;
  p.which = 0;
  p.nl = nl;
  p.mean_op = f0.sc.mean_op;
  p.latent = f0.sc.latent;
  for (int l = 0; l < nl; ++l) {
    p.T[l] = at<float>(f[l]->ws, f[l]->L->T);
    p.tp[l] = at<float>(f[l]->ws, f[l]->L->Tp);
    p.shade[l] = at<float4>(f[l]->ws, f[l]->L->shade);
    p.light[l] = light_h(f[l]->light);
  }
  for (int i = 0; i < 3; ++i) p.cam_pos[i] = f0.cam.pos[i];
  p.res_idx = nullptr;
  p.ccol = nullptr;
  p.envcol = envcol;
  p.rank_of = at<uint32_t>(f0.ws, f0.L->sp[0].rank_of);
  p.identity = (f0.opts.ablate & GS3_ABLATE_PHI) != 0;
  launch_one(p, s);
}

}  // namespace gs3
