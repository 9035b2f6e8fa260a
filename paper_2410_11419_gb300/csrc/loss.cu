// The training loss of Sec. 4.4 and its image gradient:
//   L = (1 - lambda) mean |I - I*| + lambda (1 - SSIM(I, I*))
// SSIM per pixel and channel with an 11x11 Gaussian window (sigma 1.5),
// C1 = 0.01^2, C2 = 0.03^2, zero padding, averaged over pixels and channels.
//
// Every window sum is a separable blur of planar maps.  With mu = G*I,
// Sxx = G*(I I), Sxy = G*(I I*) (and the same for the target) the SSIM map is
// m = (2 mu mu* + C1)(2 (Sxy - mu mu*) + C2) / ((mu^2 + mu*^2 + C1)(Sxx - mu^2 + Syy - mu*^2 + C2)),
// and dSSIM/dI = (G * dm/dmu) + I* (G * dm/dSxy) + 2 I (G * dm/dSxx), the
// blur being its own adjoint (symmetric kernel, zero padding).  Sums over
// pixels are reduced in a fixed order (per-block partials, one final block).
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

constexpr int kWin = 11, kHalf = 5;

__constant__ float c_gauss[kWin];

// one separable blur pass over nmap planar maps of H x W (dir 0: rows, 1: columns)
__global__ void k_blur(const float* __restrict__ in, float* __restrict__ out, int nmap, int W, int H, int dir) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t plane = (size_t)W * H;
  if (i >= plane * nmap) return;
  const size_t base = (i / plane) * plane;
  const int p = (int)(i - base), x = p % W, y = p / W;
  float s = 0.f;
#pragma unroll
  for (int k = -kHalf; k <= kHalf; ++k) {
    const int xx = dir == 0 ? x + k : x, yy = dir == 0 ? y : y + k;
    if (xx >= 0 && xx < W && yy >= 0 && yy < H) s = fmaf(c_gauss[k + kHalf], in[base + (size_t)yy * W + xx], s);
  }
  out[i] = s;
}

// planar maps per channel c: x, y, x^2, y^2, x y  (5 per channel, 15 maps)
__global__ void k_ssim_inputs(const float* __restrict__ img, const float* __restrict__ tgt, float* maps, int W, int H) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t plane = (size_t)W * H;
  if (p >= (int)plane) return;
  for (int c = 0; c < 3; ++c) {
    const float x = img[3 * (size_t)p + c], y = tgt[3 * (size_t)p + c];
    float* m = maps + (size_t)c * 5 * plane;
    m[p] = x;
    m[plane + p] = y;
    m[2 * plane + p] = x * x;
    m[3 * plane + p] = y * y;
    m[4 * plane + p] = x * y;
  }
}

// SSIM map, its partial derivatives (3 maps per channel) and per-block sums
__global__ void k_ssim_map(const float* __restrict__ img, const float* __restrict__ tgt,
                           const float* __restrict__ blurred, float* __restrict__ dmaps, double* __restrict__ part,
                           int W, int H) {
  __shared__ double s_m[256], s_l1[256];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t plane = (size_t)W * H;
  double sm = 0.0, sl = 0.0;
  if (p < (int)plane) {
    const float C1 = 1e-4f, C2 = 9e-4f;
    for (int c = 0; c < 3; ++c) {
      const float* b = blurred + (size_t)c * 5 * plane;
      const float mx = b[p], my = b[plane + p], sxx = b[2 * plane + p], syy = b[3 * plane + p],
                  sxy = b[4 * plane + p];
      const float A1 = 2.f * mx * my + C1, A2 = 2.f * (sxy - mx * my) + C2;
      const float B1 = mx * mx + my * my + C1, B2 = (sxx - mx * mx) + (syy - my * my) + C2;
      const float iB = 1.f / (B1 * B2);
      const float m = A1 * A2 * iB;
      float* d = dmaps + (size_t)c * 3 * plane;
      d[p] = (2.f * my * A2 - 2.f * my * A1) * iB - m * (2.f * mx / B1 - 2.f * mx / B2);  // dm/dmu
      d[plane + p] = 2.f * A1 * iB;                                                    // dm/dSxy
      d[2 * plane + p] = -m / B2;                                                      // dm/dSxx
      sm += m;
      sl += fabs((double)img[3 * (size_t)p + c] - (double)tgt[3 * (size_t)p + c]);
    }
  }
  s_m[threadIdx.x] = sm;
  s_l1[threadIdx.x] = sl;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_m[threadIdx.x] += s_m[threadIdx.x + o];
      s_l1[threadIdx.x] += s_l1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s_m[0];
    part[2 * blockIdx.x + 1] = s_l1[0];
  }
}

__global__ void k_loss_final(const double* part, int nblocks, double count, float lambda, float* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sm = 0.0, sl = 0.0;
  for (int b = 0; b < nblocks; ++b) { sm += part[2 * b]; sl += part[2 * b + 1]; }
  *loss = (float)((1.0 - lambda) * sl / count + lambda * (1.0 - sm / count));
}

__global__ void k_loss_grad(const float* __restrict__ img, const float* __restrict__ tgt,
                            const float* __restrict__ bd, float* __restrict__ dimg, int W, int H, float lambda) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t plane = (size_t)W * H;
  if (p >= (int)plane) return;
  const float inv = 1.f / (3.f * (float)plane);
  for (int c = 0; c < 3; ++c) {
    const float x = img[3 * (size_t)p + c], y = tgt[3 * (size_t)p + c];
    const float* d = bd + (size_t)c * 3 * plane;
    const float dssim = (d[p] + y * d[plane + p] + 2.f * x * d[2 * plane + p]) * inv;
    const float sgn = x > y ? 1.f : (x < y ? -1.f : 0.f);
    dimg[3 * (size_t)p + c] = (1.f - lambda) * sgn * inv - lambda * dssim;
  }
}

}  // namespace

size_t loss_scratch_bytes(int W, int H) {
  const size_t plane = (size_t)W * H;
  const size_t nb = (plane + 255) / 256;
  return 4 * (15 + 15 + 9 + 9) * plane + 16 * nb + 256;
}

gs3_status run_loss(const float* img, const float* tgt, int W, int H, float lambda, float* loss, float* dimg,
                    void* scratch, cudaStream_t s) {
  // the window lives in constant memory, one copy per device
  static DeviceOnce once;
  const bool ready = once.run([] {
    float g[kWin], sum = 0.f;
    for (int k = 0; k < kWin; ++k) {
      const float d = (float)(k - kHalf);
      g[k] = expf(-d * d / (2.f * 1.5f * 1.5f));
      sum += g[k];
    }
    for (int k = 0; k < kWin; ++k) g[k] /= sum;
    return cudaMemcpyToSymbol(c_gauss, g, sizeof(g)) == cudaSuccess;
  });
  if (!ready) return GS3_ERR_CUDA;
  const size_t plane = (size_t)W * H;
  float* maps = static_cast<float*>(scratch);
  float* tmp = maps + 15 * plane;
  float* dm = tmp + 15 * plane;
  float* dtmp = dm + 9 * plane;
  const int nb = (int)((plane + 255) / 256);
  double* part = reinterpret_cast<double*>(dtmp + 9 * plane);
  k_ssim_inputs<<<nb, 256, 0, s>>>(img, tgt, maps, W, H);
  const int nb15 = (int)((15 * plane + 255) / 256), nb9 = (int)((9 * plane + 255) / 256);
  k_blur<<<nb15, 256, 0, s>>>(maps, tmp, 15, W, H, 0);
  k_blur<<<nb15, 256, 0, s>>>(tmp, maps, 15, W, H, 1);
  k_ssim_map<<<nb, 256, 0, s>>>(img, tgt, maps, dm, part, W, H);
  k_loss_final<<<1, 32, 0, s>>>(part, nb, 3.0 * (double)plane, lambda, loss);
  k_blur<<<nb9, 256, 0, s>>>(dm, dtmp, 9, W, H, 0);
  k_blur<<<nb9, 256, 0, s>>>(dtmp, dm, 9, W, H, 1);
  k_loss_grad<<<nb, 256, 0, s>>>(img, tgt, dm, dimg, W, H, lambda);
  count_launch(8);
  return cudaGetLastError() == cudaSuccess ? GS3_OK : GS3_ERR_CUDA;
}

}  // namespace gs3
