// Adam (Kingma and Ba, 2015), the optimiser of the training in Sec. 4.4,
// applied in place to one parameter array in one pass:
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   p <- max(lo, p - lr (m / c1) / (sqrt(v / c2) + eps)),  c1 = 1 - b1^t, c2 = 1 - b2^t.
// `lo` keeps positive parameters (scales, lobe deviations) positive; -inf
// leaves a parameter unbounded.  Each element is independent, so the update
// is bandwidth-bound: 4 reads and 3 writes of 4 bytes per parameter.
#include "gs3_internal.cuh"

namespace gs3 {
namespace {

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, size_t n, float lr, float b1, float b2,
                                              float eps, float c1, float c2, float lo) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = fmaxf(lo, p[i] - step);
  }
}

}  // namespace

void launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                 int step, float lo, cudaStream_t s) {
  const double c1 = 1.0 - pow((double)b1, (double)step), c2 = 1.0 - pow((double)b2, (double)step);
  const size_t want = (n + 255) / 256;
  const size_t cap_blocks = (size_t)device_sm_count() * 16;
  const int blocks = (int)(want < cap_blocks ? want : cap_blocks);
  k_adam<<<blocks, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, (float)c1, (float)c2, lo);
  count_launch();
}

}  // namespace gs3
