// K8b: backward of the Phi (Sec. 4.2) and Psi (Sec. 4.3) MLPs of an FP32 scene.
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
// Every product over the Gaussians is a dense GEMM with N rows and 128 or
// fewer columns:
//   row GEMM (k_rowgemm_tc):  rows = Gaussians; forward recompute h_l = act(h_{l-1} W_l^T + b_l)
//                             and the data gradients dz_{l-1} = (dz_l W_l) * act'(h_{l-1})
//   weight GEMM (k_wgemm_tc): rows = output units, contraction over Gaussians split
//                             across blocks (the bias sums from a ones column); per-block
//                             partials are summed in block order, so the gradients do not
//                             depend on scheduling.
// Both run on the tensor cores in three-pass TF32 (about 2^-21 relative per
// product, FP32 accumulation).  The output layer (1 or 3 units) and its
// weight gradient run on CUDA cores in k_out_layer.  Hidden widths of 16 take
// their weight gradients from a register-tiled FP32 SIMT kernel (k_wgemm): a
// block owns a 128 x 128 tile of C = A B, each thread 8 x 8 of it, with the
// contraction staged through double-buffered shared memory in chunks of 16.
// The activations and data gradients of one network live in the backward
// workspace (about (64 + 4 W) N floats), shared by Phi and Psi in turn.
#include "gs3_internal.cuh"
#include "tc_ptx.cuh"

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
  const unsigned char* bpack;  // tensor-core form: B pre-split into chunk tiles (tc_pack_b), or null
  int n, ncols, kdim;
  float* C;
  int ldc;
  const float* bias;
  const float* H;
  int ldh;
  int act;
};

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

// ---- the same GEMMs on the tensor cores, three-pass TF32 --------------------
// Every FP32 operand x is split into big = x with its low 13 mantissa bits
// cleared (a TF32 value) and small = x - big (exact in FP32); a product is
// formed as big*big' + big*small' + small*big' by tcgen05.mma kind::tf32
// with FP32 accumulation in tensor memory, which drops only small*small'
// and the bits of small below TF32: about 2^-21 |x y| per product, against
// 2^-24 for an FP32 FMA.
//
// A CTA of 128 threads owns a 128 x npad output tile in TMEM (npad a
// multiple of 32).  The contraction runs in chunks of kTcK elements: each
// thread stages one row of the A chunk and one (or two) rows of the B chunk,
// split, into K-major no-swizzle shared-memory tiles; thread 0 issues the
// chunk's 4 K-steps x 3 passes and commits them to an mbarrier (a bounded,
// sleeping wait); the next chunk is staged once they have completed.  Several
// CTAs per SM overlap one CTA's staging with another's MMAs.
constexpr int kTcK = 32;            // contraction elements per chunk
constexpr int kTcRowBytes = kTcK * 4;  // bytes of a chunk row
constexpr int kTcTile = 128;

__host__ __device__ inline uint32_t tc_alloc_cols(int npad) {
  uint32_t c = 32;
  while (c < (uint32_t)npad) c <<= 1;
  return c;
}
// dynamic shared memory of a CTA: A big/small (128 rows), B big/small (npad rows)
__host__ __device__ inline size_t tc_gemm_smem(int npad) {
  return 2ull * kTcTile * kTcRowBytes + 2ull * npad * kTcRowBytes;
}

__device__ __forceinline__ float tf32_big(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Split four values into big / small and store them as 16 bytes of row r,
// bytes 16 c4 .. 16 c4 + 15, of the big and small chunk tiles.
__device__ __forceinline__ void tc_put4(const float (&v)[4], int r, int c4, unsigned char* big, unsigned char* small) {
  const float4 b4 = make_float4(tf32_big(v[0]), tf32_big(v[1]), tf32_big(v[2]), tf32_big(v[3]));
  const float4 s4 = make_float4(v[0] - b4.x, v[1] - b4.y, v[2] - b4.z, v[3] - b4.w);
  const uint32_t off = tc::canon_off(r, 16 * c4, kTcRowBytes);
  *reinterpret_cast<float4*>(big + off) = b4;
  *reinterpret_cast<float4*>(small + off) = s4;
}

// A thread's share of one operand chunk (elements kk = k0 .. k0 + 31 of
// operand rows i0 + r, r < nrows <= 128; 0 outside the operand or past kend),
// loaded into registers ahead of the chunk that uses it.  Both access
// patterns keep a warp's global loads on few lines and its 16-byte shared
// stores on distinct banks:
//   kk_rows (operand row-major in i): lane = row r = t, consecutive lanes
//     read consecutive i (one line per load), 32 loads per thread;
//   otherwise (row-major in kk): a warp covers 8 rows x 4 float4 per step,
//     lane l row l & 7 and float4 l >> 3 (16-byte loads where aligned); the
//     stores of 8 lanes fill one 128-byte core-matrix row group.
struct TcRegs {
  float4 v[8];
};

__device__ __forceinline__ void tc_load(const Operand& o, int i0, int nrows, int k0, int kend, TcRegs& R) {
  const int t = threadIdx.x;
  const int klim = min(kend, o.nk);
  if (o.kk_rows) {
    const int i = i0 + t;
    const bool row_ok = t < nrows && i < o.ni;
#pragma unroll
    for (int c4 = 0; c4 < kTcK / 4; ++c4) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kk = k0 + 4 * c4 + e;
        v[e] = (row_ok && kk < klim) ? o.m[(size_t)kk * o.ld + i] : 0.f;
      }
      R.v[c4] = make_float4(v[0], v[1], v[2], v[3]);
    }
  } else {
    const int lane = t & 31, warp = t >> 5;
    const int steps = (nrows / 8) * 2;  // (8-row group, half of the chunk's 8 float4) pairs
    const bool vec = (o.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(o.m) & 15) == 0;
#pragma unroll
    for (int qq = 0; qq < 8; ++qq) {
      const int q = warp + 4 * qq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < steps) {
        const int r = (q >> 1) * 8 + (lane & 7), c4 = (q & 1) * 4 + (lane >> 3);
        const int i = i0 + r, kk = k0 + 4 * c4;
        if (i < o.ni) {
          const float* src = o.m + (size_t)i * o.ld + kk;
          if (vec && kk + 4 <= klim) {
            x = *reinterpret_cast<const float4*>(src);
          } else {
            x.x = kk < klim ? src[0] : 0.f;
            x.y = kk + 1 < klim ? src[1] : 0.f;
            x.z = kk + 2 < klim ? src[2] : 0.f;
            x.w = kk + 3 < klim ? src[3] : 0.f;
          }
        }
      }
      R.v[qq] = x;
    }
  }
}

// Split a thread's loaded share into the big and small chunk tiles.  Rows
// [128, nrows) (a weight GEMM's N past 128) hold no operand data: the ones
// row (1 for kk < kend) or zeros.
__device__ __forceinline__ void tc_store(const Operand& o, int nrows, int k0, int kend, int ones_row,
                                         const TcRegs& R, unsigned char* big, unsigned char* small) {
  const int t = threadIdx.x;
  if (o.kk_rows) {
    if (t < nrows) {
#pragma unroll
      for (int c4 = 0; c4 < kTcK / 4; ++c4) {
        float v[4] = {R.v[c4].x, R.v[c4].y, R.v[c4].z, R.v[c4].w};
        if (t == ones_row)
#pragma unroll
          for (int e = 0; e < 4; ++e) v[e] = k0 + 4 * c4 + e < kend ? 1.f : 0.f;
        tc_put4(v, t, c4, big, small);
      }
    }
    for (int r = t + kTcTile; r < nrows; r += kTcTile) {
#pragma unroll
      for (int c4 = 0; c4 < kTcK / 4; ++c4) {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (r == ones_row && k0 + 4 * c4 + e < kend) ? 1.f : 0.f;
        tc_put4(v, r, c4, big, small);
      }
    }
  } else {
    const int lane = t & 31, warp = t >> 5;
    const int steps = (nrows / 8) * 2;
#pragma unroll
    for (int qq = 0; qq < 8; ++qq) {
      const int q = warp + 4 * qq;
      if (q < steps) {
        const int r = (q >> 1) * 8 + (lane & 7), c4 = (q & 1) * 4 + (lane >> 3);
        const float v[4] = {R.v[qq].x, R.v[qq].y, R.v[qq].z, R.v[qq].w};
        tc_put4(v, r, c4, big, small);
      }
    }
  }
}

// A row GEMM's B operand (npad rows n x kdim elements k; element (n, k) =
// W[n ld + k], or W[k ld + n] when transposed; 0 for n >= nvalid or
// k >= kvalid) pre-split once into the chunk tiles the kernel reads: chunk c
// at c * 2 npad 128 bytes, its big tile then its small tile, each in the
// canonical K-major layout.  A CTA then copies a chunk with one bulk copy.
__global__ void k_pack_b(const float* __restrict__ W, int ld, bool transposed, int nvalid, int kvalid, int npad,
                         int nchunks, unsigned char* __restrict__ dst) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npad * nchunks * kTcK) return;
  const int n = idx % npad, k = idx / npad;
  const float x = (n < nvalid && k < kvalid) ? (transposed ? W[(size_t)k * ld + n] : W[(size_t)n * ld + k]) : 0.f;
  const float b = tf32_big(x);
  unsigned char* chunk = dst + (size_t)(k / kTcK) * 2 * npad * kTcRowBytes;
  const uint32_t off = tc::canon_off(n, 4 * (k % kTcK), kTcRowBytes);
  *reinterpret_cast<float*>(chunk + off) = b;
  *reinterpret_cast<float*>(chunk + (size_t)npad * kTcRowBytes + off) = x - b;
}

// 32 accumulator columns of this thread's row into the shared transpose
// buffer (rows of 36 floats: 16-byte stores of 8 consecutive rows hit
// distinct banks), for a write-out where a warp covers 4 rows x 8 float4.
constexpr int kTcOutStride = 36;
__device__ __forceinline__ void tc_rows_to_smem(const float (&v)[32], float* buf) {
  float* row = buf + threadIdx.x * kTcOutStride;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *reinterpret_cast<float4*>(row + 4 * c) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}

// One chunk's MMAs: 4 K-steps of 8 TF32 elements, three passes each
__device__ __forceinline__ void tc_chunk_mma(uint32_t tmem, uint32_t ab, uint32_t as, uint32_t bb, uint32_t bs,
                                             uint32_t idesc, bool first) {
  constexpr uint32_t kSbo = 8 * kTcRowBytes;
#pragma unroll
  for (int st = 0; st < kTcK / 8; ++st) {
    const uint32_t o = (uint32_t)st * 256;  // 32 bytes of K: two core matrices
    const uint64_t dab = tc::smem_desc(ab + o, 128, kSbo), das = tc::smem_desc(as + o, 128, kSbo);
    const uint64_t dbb = tc::smem_desc(bb + o, 128, kSbo), dbs = tc::smem_desc(bs + o, 128, kSbo);
    tc::tc_mma_tf32(tmem, das, dbb, idesc, (first && st == 0) ? 0u : 1u);
    tc::tc_mma_tf32(tmem, dab, dbs, idesc, 1u);
    tc::tc_mma_tf32(tmem, dab, dbb, idesc, 1u);
  }
}

// Shared prologue / epilogue pieces of the two tensor-core GEMM kernels
struct TcCta {
  unsigned char *ab, *as, *bb, *bs;
  uint32_t tmem, ncols;
};
__device__ __forceinline__ TcCta tc_cta_begin(unsigned char* sm, int npad, uint64_t* bar, uint32_t* slot) {
  TcCta c;
  c.ab = sm;
  c.as = sm + kTcTile * kTcRowBytes;
  c.bb = sm + 2 * kTcTile * kTcRowBytes;
  c.bs = c.bb + npad * kTcRowBytes;
  c.ncols = tc_alloc_cols(npad);
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tc::smem_u32(slot), c.ncols);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(bar), 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  c.tmem = *slot;
  return c;
}
__device__ __forceinline__ void tc_cta_end(const TcCta& c, bool ok, uint32_t* status) {
  if (!ok && threadIdx.x == 0 && status) atomicCAS(status, 0u, (uint32_t)GS3_ERR_TIMEOUT);
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(c.tmem, c.ncols);
}
// Issue a staged chunk (thread 0), run `meanwhile` (every thread), wait for
// the chunk (every thread); false on a timeout
template <typename F>
__device__ __forceinline__ bool tc_run_chunk(const TcCta& c, uint32_t bar, uint32_t& phase, uint32_t idesc,
                                             bool first, F&& meanwhile) {
  tc::fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::tc_fence_after();
    tc_chunk_mma(c.tmem, tc::smem_u32(c.ab), tc::smem_u32(c.as), tc::smem_u32(c.bb), tc::smem_u32(c.bs), idesc,
                 first);
    tc::tc_commit(bar);
  }
  meanwhile();
  const bool ok = tc::mbar_wait_bounded(bar, phase);
  phase ^= 1u;
  tc::tc_fence_after();
  return __syncthreads_and(ok) != 0;  // also: every thread is done with the tiles
}

// C[g][j] = epi(sum_kk A[g][kk] B[kk][j]) for the 128 rows of this CTA and
// j < ncols (npad = ncols rounded up to 32); the epilogues of k_rowgemm.
template <int EPI>
__global__ void __launch_bounds__(kTcTile) k_rowgemm_tc(RowGemm p, int npad, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar, bar_b;
  __shared__ uint32_t slot;
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * kTcTile;
  const TcCta c = tc_cta_begin(sm, npad, &bar, &slot);
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(&bar_b), 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  const uint32_t idesc = tc::idesc_tf32(kTcTile, npad);
  const uint32_t chunk_bytes = 2u * npad * kTcRowBytes;
  uint32_t phase = 0, phase_b = 0;
  bool ok = true, b_late = false;
  TcRegs ra, rb;
  tc_load(p.A, i0, kTcTile, 0, p.kdim, ra);
  if (!p.bpack) tc_load(p.B, 0, npad, 0, p.kdim, rb);
  for (int k0 = 0; k0 < p.kdim && ok; k0 += kTcK) {
    if (p.bpack && t == 0) {  // the chunk's B tiles (big, small) by one bulk copy
      tc::mbar_expect_tx(tc::smem_u32(&bar_b), chunk_bytes);
      tc::bulk_g2s(tc::smem_u32(c.bb), p.bpack + (size_t)(k0 / kTcK) * chunk_bytes, chunk_bytes,
                   tc::smem_u32(&bar_b));
    }
    tc_store(p.A, kTcTile, k0, p.kdim, -1, ra, c.ab, c.as);
    if (!p.bpack) tc_store(p.B, npad, k0, p.kdim, -1, rb, c.bb, c.bs);
    if (p.bpack) {  // every thread: the B tiles have landed (a bounded wait)
      const bool b_ok = tc::mbar_wait_bounded(tc::smem_u32(&bar_b), phase_b);
      if (!b_ok) {
        ok = false;
        b_late = true;
      }
      phase_b ^= 1u;
    }
    ok = tc_run_chunk(c, tc::smem_u32(&bar), phase, idesc, k0 == 0, [&] {
      if (k0 + kTcK < p.kdim) {  // the next chunk's loads overlap this chunk's MMAs
        tc_load(p.A, i0, kTcTile, k0 + kTcK, p.kdim, ra);
        if (!p.bpack) tc_load(p.B, 0, npad, k0 + kTcK, p.kdim, rb);
      }
    }) && ok;
  }
  if (ok) {
    // 32 columns at a time: TMEM row -> shared transpose buffer -> a warp
    // applies the epilogue to 4 rows x 8 float4 and writes whole row segments
    float* buf = reinterpret_cast<float*>(sm);  // the operand tiles are free now
    const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
    const uint32_t lane_addr = c.tmem + ((uint32_t)((t >> 5) * 32) << 16);
    const int lane = t & 31, warp = t >> 5;
    for (int c0 = 0; c0 < npad; c0 += 32) {
      float v[32];
      tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
      tc_rows_to_smem(v, buf);
      __syncthreads();
      for (int q = warp; q < kTcTile / 4; q += kTcTile / 32) {
        const int r = q * 4 + (lane >> 3), c4 = lane & 7;
        const int g = i0 + r, j0 = c0 + 4 * c4;
        if (g < p.n && j0 < p.ncols) {
          const float4 a4 = *reinterpret_cast<const float4*>(buf + r * kTcOutStride + 4 * c4);
          float x[4] = {a4.x, a4.y, a4.z, a4.w};
          if (j0 + 4 <= p.ncols && (p.ldc & 3) == 0 && (EPI != EPI_DACT || (p.ldh & 3) == 0)) {
            // whole float4: 8 lanes write one row's 128 contiguous bytes
            float hv[4] = {1.f, 1.f, 1.f, 1.f};
            if (EPI == EPI_DACT) {
              const float4 h4 = *reinterpret_cast<const float4*>(p.H + (size_t)g * p.ldh + j0);
              hv[0] = h4.x; hv[1] = h4.y; hv[2] = h4.z; hv[3] = h4.w;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (EPI == EPI_BIAS_ACT) {
                x[e] += p.bias[j0 + e];
                x[e] = x[e] > 0.f ? x[e] : (leaky ? 0.01f * x[e] : 0.f);
              } else if (EPI == EPI_DACT) {
                x[e] = hv[e] > 0.f ? x[e] : (leaky ? 0.01f * x[e] : 0.f);
              }
            }
            *reinterpret_cast<float4*>(p.C + (size_t)g * p.ldc + j0) = make_float4(x[0], x[1], x[2], x[3]);
            continue;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = j0 + e;
            if (j >= p.ncols) break;
            if (EPI == EPI_BIAS_ACT) {
              x[e] += p.bias[j];
              x[e] = x[e] > 0.f ? x[e] : (leaky ? 0.01f * x[e] : 0.f);
            } else if (EPI == EPI_DACT) {
              const float h = p.H[(size_t)g * p.ldh + j];
              x[e] = h > 0.f ? x[e] : (leaky ? 0.01f * x[e] : 0.f);
            }
            p.C[(size_t)g * p.ldc + j] = x[e];
          }
        }
      }
      __syncthreads();
    }
  }
  if (b_late) tc::mbar_wait_bounded(tc::smem_u32(&bar_b), phase_b ^ 1u);  // our own copy lands before we leave
  tc_cta_end(c, ok, status);
}

// Block b: partial[b][j][k] = sum over its Gaussians g of dZ[g][j] H[g][k]
// (j < nout <= 128, k < nin) and, from a ones column at k = nin, the bias
// partial sum_g dZ[g][j]; the layout of k_wgemm's partials.
__global__ void __launch_bounds__(kTcTile) k_wgemm_tc(WGemm p, int npad, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int t = threadIdx.x;
  const int kbeg = blockIdx.x * p.rows_per_block;
  const int kend = min(p.n, kbeg + p.rows_per_block);
  const TcCta c = tc_cta_begin(sm, npad, &bar, &slot);
  const uint32_t idesc = tc::idesc_tf32(kTcTile, npad);
  uint32_t phase = 0;
  bool ok = true;
  TcRegs ra, rb;
  if (kbeg < kend) {
    tc_load(p.A, 0, kTcTile, kbeg, kend, ra);
    tc_load(p.B, 0, npad, kbeg, kend, rb);
  }
  for (int k0 = kbeg; k0 < kend && ok; k0 += kTcK) {
    tc_store(p.A, kTcTile, k0, kend, -1, ra, c.ab, c.as);
    tc_store(p.B, npad, k0, kend, p.nin, rb, c.bb, c.bs);
    ok = tc_run_chunk(c, tc::smem_u32(&bar), phase, idesc, k0 == kbeg, [&] {
      if (k0 + kTcK < kend) {  // the next chunk's loads overlap this chunk's MMAs
        tc_load(p.A, 0, kTcTile, k0 + kTcK, kend, ra);
        tc_load(p.B, 0, npad, k0 + kTcK, kend, rb);
      }
    });
  }
  const size_t np = (size_t)p.nout * p.nin + p.nout;
  float* out = p.part + (size_t)blockIdx.x * np;
  if (ok && kbeg >= kend) {  // no rows: zero partials
    for (size_t i = t; i < np; i += kTcTile) out[i] = 0.f;
  } else if (ok) {
    float* buf = reinterpret_cast<float*>(sm);
    const uint32_t lane_addr = c.tmem + ((uint32_t)((t >> 5) * 32) << 16);
    const int lane = t & 31, warp = t >> 5;
    for (int c0 = 0; c0 < npad; c0 += 32) {
      float v[32];
      tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
      tc_rows_to_smem(v, buf);
      __syncthreads();
      for (int q = warp; q < kTcTile / 4; q += kTcTile / 32) {
        const int j = q * 4 + (lane >> 3), k0c = c0 + 4 * (lane & 7);
        if (j < p.nout) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = k0c + e;
            const float x = buf[j * kTcOutStride + 4 * (lane & 7) + e];
            if (k < p.nin) out[(size_t)j * p.nin + k] = x;
            else if (k == p.nin) out[(size_t)p.nout * p.nin + j] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  tc_cta_end(c, ok, status);
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

// Output layer and its weight gradient, one warp per Gaussian at a time:
// y = sigmoid(W_o h_L + b_o), dz_o = dL/dy y (1 - y), dz_L = (dz_o W_o) *
// act'(h_L); lane l owns the columns l, l + 32, l + 64, l + 96 that exist
// (widths 16..128).  Block b takes the Gaussians [b rpb, (b + 1) rpb), warp w
// of it every 8th from the w-th (the next one's h_L loaded ahead); each lane
// accumulates dz_o h_L for its columns, and the block adds its warps' sums in
// warp order into partial[b] (the weight gradient's order: W_o row-major,
// then b_o), so the result does not depend on scheduling.
constexpr int kOutWarps = 8;
__global__ void __launch_bounds__(kOutWarps * 32) k_out_layer(RowArgs p, int rows_per_block, float* part) {
  __shared__ float wo[4 * 128];  // the output layer's weights (out_dim <= 3, width <= 128)
  __shared__ float bo[4];
  __shared__ float red[kOutWarps][3 * 128 + 3];
  const int W = p.width, nq = (W + 31) / 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nout = p.out_dim;
  for (int i = threadIdx.x; i < nout * W; i += blockDim.x) wo[i] = p.w_out[i];
  if (threadIdx.x < nout) bo[threadIdx.x] = p.b_out[threadIdx.x];
  __syncthreads();
  const bool leaky = p.act == GS3_ACT_LEAKY_RELU;
  const int kbeg = blockIdx.x * rows_per_block, kend = min(p.n, kbeg + rows_per_block);
  float wacc[3][4], bacc[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    bacc[o] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) wacc[o][q] = 0.f;
  }
  auto load_h = [&](int g, float (&hv)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) hv[q] = (g < kend && q < nq && lane + 32 * q < W) ? p.Hlast[(size_t)g * W + lane + 32 * q] : 0.f;
  };
  float hn[4];
  load_h(kbeg + warp, hn);
  for (int g = kbeg + warp; g < kend; g += kOutWarps) {
    float hv[4] = {hn[0], hn[1], hn[2], hn[3]};
    load_h(g + kOutWarps, hn);
    float dzo[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      if (o >= nout) break;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nq && lane + 32 * q < W) s = fmaf(hv[q], wo[o * W + lane + 32 * q], s);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      const float y = 1.f / (1.f + expf(-(s + bo[o])));
      const float dy = p.which == 0 ? p.color[(size_t)kColorStride * g + 3] : p.color[(size_t)kColorStride * g + 4 + o];
      dzo[o] = dy * y * (1.f - y);
      bacc[o] += dzo[o];
#pragma unroll
      for (int q = 0; q < 4; ++q) wacc[o][q] = fmaf(dzo[o], hv[q], wacc[o][q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = lane + 32 * q;
      if (q >= nq || j >= W) break;
      float s = 0.f;
#pragma unroll
      for (int o = 0; o < 3; ++o)
        if (o < nout) s = fmaf(dzo[o], wo[o * W + j], s);
      p.dZlast[(size_t)g * W + j] = hv[q] > 0.f ? s : (leaky ? 0.01f * s : 0.f);
    }
  }
  // the block's partial weight gradient, its warps added in order
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    if (o >= nout) break;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq && lane + 32 * q < W) red[warp][o * W + lane + 32 * q] = wacc[o][q];
    if (lane == 0) red[warp][nout * W + o] = bacc[o];
  }
  __syncthreads();
  const int np = nout * W + nout;
  float* out = part + (size_t)blockIdx.x * np;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    float v = 0.f;
    for (int w = 0; w < kOutWarps; ++w) v += red[w][i];
    out[i] = v;
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

// red[i] = sum over b of part[b][i], for 32 consecutive i per block: warp w
// adds the partials b = w, w + 8, ... (lane = i, coalesced), then the eight
// warp sums are added in warp order: a fixed order, so the result does not
// depend on scheduling.
constexpr int kSumWarps = 8;
__global__ void __launch_bounds__(kSumWarps * 32) k_sum_parts(const float* part, size_t np, int nblocks, float* red) {
  __shared__ float acc[kSumWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t i = (size_t)blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < np)
    for (int b = warp; b < nblocks; b += kSumWarps) s += part[(size_t)b * np + i];
  acc[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < np) {
    float t = 0.f;
    for (int w = 0; w < kSumWarps; ++w) t += acc[w][lane];
    red[i] = t;
  }
}

int wgemm_blocks(int n) {
  const int by_rows = (n + kKc - 1) / kKc;
  return by_rows < kWgemmBlocks ? by_rows : kWgemmBlocks;
}

struct Scratch {
  float *X, *H, *dz[2], *part;
  unsigned char* bpack;  // pre-split B operands: per hidden layer the forward one, then the data gradient's
};
constexpr size_t kPackBytes = 4ull * 2 * kTcTile * kTcRowBytes;  // a B operand of <= 128 x 128: 4 chunks

Scratch carve(void* base, int n, const MlpDev& m) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  unsigned char* c = static_cast<unsigned char*>(base);
  Scratch s;
  s.X = reinterpret_cast<float*>(c); c += al(4ull * n * kXdim);
  s.H = reinterpret_cast<float*>(c); c += al(4ull * n * m.width * m.n_hidden);
  s.dz[0] = reinterpret_cast<float*>(c); c += al(4ull * n * (m.width > kXdim ? m.width : kXdim));
  s.dz[1] = reinterpret_cast<float*>(c); c += al(4ull * n * (m.width > kXdim ? m.width : kXdim));
  s.bpack = c; c += 2 * kPackBytes * m.n_hidden;
  s.part = reinterpret_cast<float*>(c);
  return s;
}

}  // namespace

size_t mlp_bwd_scratch_bytes(int n, const MlpDev& m) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t wide = (size_t)(m.width > kXdim ? m.width : kXdim);
  const size_t layer_max = (size_t)m.width * (m.width > m.in_dim ? m.width : m.in_dim) + m.width;
  return al(4ull * n * kXdim) + al(4ull * n * m.width * m.n_hidden) + 2 * al(4ull * n * wide) +
         2 * kPackBytes * m.n_hidden + al(4ull * wgemm_blocks(n) * layer_max);
}

namespace {

int round32(int x) { return (x + 31) & ~31; }

// Dynamic shared memory of a tensor-core GEMM launch: the operand tiles,
// padded so that the CTAs that fit on an SM never need more than its 512
// tensor-memory columns at once.
size_t tc_launch_smem(int npad) {
  size_t smem = tc_gemm_smem(npad);
  const int max_ctas = (int)(512 / tc_alloc_cols(npad));
  const size_t per_sm = 228 * 1024, reserve = 2048;
  const size_t floor_bytes = per_sm / (size_t)(max_ctas + 1) + 1;
  if (smem + reserve < floor_bytes) smem = floor_bytes - reserve;
  return smem;
}

template <int EPI>
void launch_rowgemm_tc(const RowGemm& g, int grid, uint32_t* status, cudaStream_t s) {
  const int npad = round32(g.ncols);
  const size_t smem = tc_launch_smem(npad);
  static DeviceOnce once;
  once.run([] {
    return cudaFuncSetAttribute(k_rowgemm_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
           cudaSuccess;
  });
  k_rowgemm_tc<EPI><<<grid, kTcTile, smem, s>>>(g, npad, status);
  count_launch();
}

void launch_wgemm_tc(const WGemm& w, int grid, uint32_t* status, cudaStream_t s) {
  const int npad = round32(w.nin + 1);
  const size_t smem = tc_launch_smem(npad);
  static DeviceOnce once;
  once.run([] {
    return cudaFuncSetAttribute(k_wgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
           cudaSuccess;
  });
  k_wgemm_tc<<<grid, kTcTile, smem, s>>>(w, npad, status);
  count_launch();
}

}  // namespace

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
  // the row GEMMs' B operands, pre-split: forward W_l (n = out unit, k = in),
  // data gradient W_l^T (n = in unit, k = out)
  auto pack = [&](const float* w, int ld, bool tr, int nvalid, int kvalid, unsigned char* dst) {
    const int npad = round32(nvalid), nchunks = (kvalid + kTcK - 1) / kTcK;
    const int total = npad * nchunks * kTcK;
    k_pack_b<<<(total + 255) / 256, 256, 0, s>>>(w, ld, tr, nvalid, kvalid, npad, nchunks, dst);
    count_launch();
  };
  for (int l = 0; l < nh; ++l) {
    const int din = l == 0 ? m.in_dim : W;
    pack(wl[l], din, false, W, din, S.bpack + (size_t)(2 * l) * kPackBytes);
    pack(wl[l], din, true, din, W, S.bpack + (size_t)(2 * l + 1) * kPackBytes);
  }
  // forward recompute
  k_encode<<<(n + 127) / 128, 128, 0, s>>>(r);
  count_launch();
  for (int l = 0; l < nh; ++l) {
    const int din = l == 0 ? m.in_dim : W;
    RowGemm g;
    g.A = {l == 0 ? S.X : S.H + (size_t)(l - 1) * n * W, l == 0 ? kXdim : W, n, din, false};
    g.B = {wl[l], din, W, din, false};  // B[kk][j] = W_l[j][kk]
    g.bpack = S.bpack + (size_t)(2 * l) * kPackBytes;
    g.n = n; g.ncols = W; g.kdim = din;
    g.C = S.H + (size_t)l * n * W; g.ldc = W;
    g.bias = bl[l]; g.H = nullptr; g.ldh = 0; g.act = m.act;
    launch_rowgemm_tc<EPI_BIAS_ACT>(g, rows_grid, a.status, s);
  }
  // output layer, then its weight gradient
  r.Hlast = S.H + (size_t)(nh - 1) * n * W;
  r.dZlast = S.dz[0];
  const int nb = wgemm_blocks(n);
  const int rpb = ((n + nb - 1) / nb + kKc - 1) / kKc * kKc;
  // output layer with its weight gradient's block partials, then their sum
  k_out_layer<<<nb, kOutWarps * 32, 0, s>>>(r, rpb, S.part);
  {
    const size_t np = (size_t)m.out_dim * W + m.out_dim;
    k_sum_parts<<<(int)((np + 31) / 32), kSumWarps * 32, 0, s>>>(S.part, np, nb, wred + poff[nh]);
  }
  count_launch(2);
  auto wgrad = [&](const float* dZ, int ldz, int nout, const float* Hin, int ldhin, int nin, int layer) {
    WGemm w;
    w.A = {dZ, ldz, nout, n, true};
    w.B = {Hin, ldhin, nin, n, true};
    w.n = n; w.nout = nout; w.nin = nin; w.rows_per_block = rpb;
    w.part = S.part;
    if (nout >= 32) {
      launch_wgemm_tc(w, nb, a.status, s);
    } else {  // hidden widths of 16: FP32 SIMT
      k_wgemm<<<nb, kGemmThreads, 0, s>>>(w);
      count_launch();
    }
    const size_t np = (size_t)nout * nin + nout;
    k_sum_parts<<<(int)((np + 31) / 32), kSumWarps * 32, 0, s>>>(S.part, np, nb, wred + poff[layer]);
    count_launch();
  };
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
    g.bpack = S.bpack + (size_t)(2 * l + 1) * kPackBytes;
    g.n = n; g.ncols = din; g.kdim = W;
    g.C = S.dz[cur ^ 1]; g.ldc = l == 0 ? kXdim : W;
    g.bias = nullptr; g.act = m.act;
    if (l > 0) {
      g.H = Hin; g.ldh = W;
      launch_rowgemm_tc<EPI_DACT>(g, rows_grid, a.status, s);
    } else {
      g.H = nullptr; g.ldh = 0;  // columns din..63 of dx stay unwritten and unread
      launch_rowgemm_tc<EPI_NONE>(g, rows_grid, a.status, s);
    }
    cur ^= 1;
  }
  r.dX = S.dz[cur];
  k_input_grad<<<(n + 127) / 128, 128, 0, s>>>(r);
  count_launch();
}

}  // namespace gs3
