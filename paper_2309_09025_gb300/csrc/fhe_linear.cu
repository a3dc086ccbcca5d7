// fhe_linear.cu -- homomorphic WeightSum (paper 4.1, Eq. "noise grows"):
// integer-weighted linear combinations of LWE ciphertexts, modulo 2^32, for
// fully connected and convolutional layers, plus the trivial additions of the
// LIF update (H = V + I, the p/2 centring offset).
#include <cuda_runtime.h>

#include "fhe_internal.cuh"

namespace {

constexpr int kTM = 32;   // outputs (rows of W) per CTA
constexpr int kTC = 128;  // ciphertext words per CTA
constexpr int kTK = 32;   // inputs per smem stage

// out[b][i][c] = sum_j W[i][j] * in[b][j][c] (+ bias[i] * Delta at c == n).
// 256 threads; thread (ty, tx) owns rows ty*4..+4 and words tx + 32*q.
__global__ void __launch_bounds__(256) k_lwe_linear(uint32_t n, uint32_t delta, const int32_t *W,
                                                    uint32_t M, uint32_t K, const int32_t *bias,
                                                    const uint32_t *in, uint32_t *out) {
  __shared__ int32_t Ws[kTM][kTK + 1];
  __shared__ uint32_t Xs[kTK][kTC];
  const uint32_t w = n + 1u;
  const uint32_t b = blockIdx.z;
  const uint32_t i0 = blockIdx.y * kTM, c0 = blockIdx.x * kTC;
  const uint32_t tx = threadIdx.x & 31u, ty = threadIdx.x >> 5;  // ty in [0, 8)
  const uint32_t *X = in + (uint64_t)b * K * w;
  uint32_t acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0u;
  for (uint32_t k0 = 0; k0 < K; k0 += kTK) {
    for (uint32_t e = threadIdx.x; e < kTM * kTK; e += 256u) {
      uint32_t r = e / kTK, cc = e % kTK;
      Ws[r][cc] = (i0 + r < M && k0 + cc < K) ? W[(uint64_t)(i0 + r) * K + k0 + cc] : 0;
    }
    for (uint32_t e = threadIdx.x; e < kTK * kTC; e += 256u) {
      uint32_t r = e / kTC, cc = e % kTC;
      Xs[r][cc] = (k0 + r < K && c0 + cc < w) ? X[(uint64_t)(k0 + r) * w + c0 + cc] : 0u;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTK; ++kk) {
      uint32_t xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = Xs[kk][tx + 32 * q];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t wv = (uint32_t)Ws[ty * 4 + a][kk];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] += wv * xv[q];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    uint32_t i = i0 + ty * 4 + a;
    if (i >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t c = c0 + tx + 32 * q;
      if (c >= w) continue;
      uint32_t v = acc[a][q];
      if (bias && c == n) v += (uint32_t)bias[i] * delta;
      out[((uint64_t)b * M + i) * w + c] = v;
    }
  }
}

// One thread per output word; taps looped (conv layers are tiny next to the
// bootstraps).  in [b][cin][h][w][n+1], W [cout][cin][kh][kw].
__global__ void k_lwe_conv2d(uint32_t n, uint32_t delta, const int32_t *W, uint32_t cin,
                             uint32_t h, uint32_t wd, uint32_t cout, uint32_t kh, uint32_t kw,
                             uint32_t stride, uint32_t pad, uint32_t ho, uint32_t wo,
                             const int32_t *bias, const uint32_t *in, uint64_t total,
                             uint32_t *out) {
  const uint32_t w = n + 1u;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = (uint32_t)(e % w);
    uint64_t pix = e / w;  // ((b * cout + co) * ho + y) * wo + x
    uint32_t x = (uint32_t)(pix % wo);
    uint32_t y = (uint32_t)((pix / wo) % ho);
    uint32_t co = (uint32_t)((pix / ((uint64_t)wo * ho)) % cout);
    uint64_t b = pix / ((uint64_t)wo * ho * cout);
    uint32_t acc = 0u;
    for (uint32_t ci = 0; ci < cin; ++ci)
      for (uint32_t dy = 0; dy < kh; ++dy) {
        int64_t iy = (int64_t)y * stride + dy - pad;
        if (iy < 0 || iy >= (int64_t)h) continue;
        for (uint32_t dx = 0; dx < kw; ++dx) {
          int64_t ix = (int64_t)x * stride + dx - pad;
          if (ix < 0 || ix >= (int64_t)wd) continue;
          uint32_t wt = (uint32_t)W[(((uint64_t)co * cin + ci) * kh + dy) * kw + dx];
          acc += wt * in[((((b * cin + ci) * h) + (uint64_t)iy) * wd + (uint64_t)ix) * w + c];
        }
      }
    if (bias && c == n) acc += (uint32_t)bias[co] * delta;
    out[e] = acc;
  }
}

// out = a + b (+ cst added to every body word), over count ciphertexts.
__global__ void k_lwe_add(uint32_t n, const uint32_t *a, const uint32_t *b, uint32_t cst,
                          uint64_t words, uint32_t *out) {
  const uint32_t w = n + 1u;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < words;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = a[e] + (b ? b[e] : 0u);
    if (e % w == n) v += cst;
    out[e] = v;
  }
}

// out = a + (cst + offs[i % n_in] * delta) on b, per ciphertext i: a public
// per-input plaintext added to every image's ciphertexts (the Poisson
// encoder's thresholds, 2.3).
__global__ void k_lwe_add_offsets(uint32_t n, const uint32_t *a, const int32_t *offs, uint32_t n_in,
                                  uint32_t delta, uint32_t cst, uint64_t words, uint32_t *out) {
  const uint32_t w = n + 1u;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < words;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = a[e];
    if (e % w == n) v += cst + (uint32_t)offs[(e / w) % n_in] * delta;
    out[e] = v;
  }
}

}  // namespace

extern "C" int fhe_lwe_linear(uint32_t n, uint32_t log2_p, const int32_t *W, size_t M, size_t K,
                              const int32_t *bias, const uint32_t *ct_in, size_t batch,
                              uint32_t *ct_out, void *stream) {
  if (!W || !ct_in || !ct_out || n < 1u || n > 2048u || log2_p < 1u || log2_p > 10u)
    return FHE_EINVAL;
  if (M == 0 || batch == 0) return FHE_OK;
  if (M > (1u << 24) || K > (1u << 24) || batch > 65535u) return FHE_EINVAL;
  dim3 grid((n + 1u + kTC - 1u) / kTC, (unsigned)((M + kTM - 1u) / kTM), (unsigned)batch);
  k_lwe_linear<<<grid, 256, 0, (cudaStream_t)stream>>>(n, 1u << (31u - log2_p), W, (uint32_t)M,
                                                       (uint32_t)K, bias, ct_in, ct_out);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

extern "C" int fhe_lwe_conv2d(uint32_t n, uint32_t log2_p, const int32_t *W, uint32_t cin,
                              uint32_t h, uint32_t w, uint32_t cout, uint32_t kh, uint32_t kw,
                              uint32_t stride, uint32_t pad, const int32_t *bias,
                              const uint32_t *ct_in, size_t batch, uint32_t *ct_out,
                              void *stream) {
  if (!W || !ct_in || !ct_out || n < 1u || n > 2048u || log2_p < 1u || log2_p > 10u ||
      stride == 0 || kh == 0 || kw == 0 || h + 2 * pad < kh || w + 2 * pad < kw)
    return FHE_EINVAL;
  const uint32_t ho = (h + 2u * pad - kh) / stride + 1u, wo = (w + 2u * pad - kw) / stride + 1u;
  const uint64_t total = (uint64_t)batch * cout * ho * wo * (n + 1u);
  if (!total) return FHE_OK;
  unsigned blocks = (unsigned)((total + 255u) / 256u);
  if (blocks > 152u * 64u) blocks = 152u * 64u;
  k_lwe_conv2d<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, 1u << (31u - log2_p), W, cin, h, w,
                                                         cout, kh, kw, stride, pad, ho, wo, bias,
                                                         ct_in, total, ct_out);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

namespace fhe {
int lwe_add(uint32_t n, const uint32_t *a, const uint32_t *b, uint32_t cst, uint64_t count,
            uint32_t *out, cudaStream_t st) {
  const uint64_t words = count * (n + 1u);
  if (!words) return FHE_OK;
  unsigned blocks = (unsigned)((words + 255u) / 256u);
  if (blocks > 152u * 32u) blocks = 152u * 32u;
  k_lwe_add<<<blocks, 256, 0, st>>>(n, a, b, cst, words, out);
  note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}
int lwe_add_offsets(uint32_t n, const uint32_t *a, const int32_t *offs, uint32_t n_in,
                    uint32_t delta, uint32_t cst, uint64_t count, uint32_t *out, cudaStream_t st) {
  const uint64_t words = count * (n + 1u);
  if (!words) return FHE_OK;
  unsigned blocks = (unsigned)((words + 255u) / 256u);
  if (blocks > 152u * 32u) blocks = 152u * 32u;
  k_lwe_add_offsets<<<blocks, 256, 0, st>>>(n, a, offs, n_in, delta, cst, words, out);
  note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}
}  // namespace fhe
