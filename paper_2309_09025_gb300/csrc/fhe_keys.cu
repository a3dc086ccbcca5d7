// fhe_keys.cu -- key generation, LWE encryption/decryption and bootstrap
// look-up tables on the GPU (paper 2.1: LWE, RLWE, RGSW keys; Thm 2.1 test
// polynomials).
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "fhe_internal.cuh"

namespace fhe {
static std::atomic<int64_t> g_launches{0};
void note_launches(int64_t n) { g_launches.fetch_add(n); }
uint64_t launches() { return (uint64_t)g_launches.load(); }
}  // namespace fhe

extern "C" uint64_t fhe_kernel_launches(void) { return fhe::launches(); }

using fhe::Params;

namespace {

__global__ void k_secret_keys(Params P, uint64_t seed, uint32_t *s, uint32_t *S) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.n) s[i] = (uint32_t)(fhe::rand64(seed, fhe::kDomLweKey, i) & 1ull);
  if (i < P.k * P.N) S[i] = (uint32_t)(fhe::rand64(seed, fhe::kDomGlweKey, i) & 1ull);
}

// One CTA per GGSW row (i, row): masks from draws, body = sum_j A_j * S_j +
// noise (negacyclic, S binary), then s_i * 2^(32 - lam log2_bg) added to
// component j = row / l at coefficient 0.
__global__ void k_bsk_rows(Params P, uint64_t seed, const uint32_t *s, const uint32_t *S,
                           uint32_t *bsk) {
  extern __shared__ uint32_t sm[];
  const uint32_t N = P.N, k = P.k, rows = P.rows();
  const uint64_t ridx = blockIdx.x;  // i * rows + row
  const uint32_t i = (uint32_t)(ridx / rows), row = (uint32_t)(ridx % rows);
  uint32_t *g = bsk + ridx * (uint64_t)(k + 1u) * N;
  uint32_t *a_s = sm;        // [N]
  uint32_t *key_s = sm + N;  // [N]
  // body accumulators live in registers of the threads owning coefficients
  for (uint32_t c = threadIdx.x; c < N; c += blockDim.x)
    g[(uint64_t)k * N + c] = fhe::noise32(seed, fhe::kDomBskNoise, ridx * N + c, P.glwe_noise_log2);
  for (uint32_t j = 0; j < k; ++j) {
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < N; c += blockDim.x) {
      uint32_t a = (uint32_t)fhe::rand64(seed, fhe::kDomBskMask, (ridx * k + j) * N + c);
      a_s[c] = a;
      key_s[c] = S[(uint64_t)j * N + c];
      g[(uint64_t)j * N + c] = a;
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < N; c += blockDim.x) {
      uint32_t acc = 0;
      for (uint32_t t = 0; t < N; ++t) {
        if (!key_s[t]) continue;  // S binary: add A[c - t] with the X^N = -1 sign
        acc += (c >= t) ? a_s[c - t] : (0u - a_s[c + N - t]);
      }
      g[(uint64_t)k * N + c] += acc;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t j = row / P.l, lam = row % P.l + 1u;
    g[(uint64_t)j * N] += s[i] << (32u - P.log2_bg * lam);
  }
}

// One warp per key-switching row (i, lam): LWE_s(z_i * 2^(32 - lam log2_bks)).
__global__ void k_ksk_rows(Params P, uint64_t seed, const uint32_t *s, const uint32_t *S,
                           uint32_t *ksk) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t ridx = (uint64_t)blockIdx.x * (blockDim.x / 32u) + threadIdx.x / 32u;
  const uint64_t nrows = (uint64_t)P.k * P.N * P.l_ks;
  if (ridx >= nrows) return;
  const uint32_t n = P.n;
  uint32_t *row = ksk + ridx * (n + 1u);
  uint32_t dot = 0;
  for (uint32_t c = lane; c < n; c += 32u) {
    uint32_t a = (uint32_t)fhe::rand64(seed, fhe::kDomKskMask, ridx * n + c);
    row[c] = a;
    dot += a * s[c];
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) {
    const uint32_t i = (uint32_t)(ridx / P.l_ks), lam = (uint32_t)(ridx % P.l_ks) + 1u;
    uint32_t b = fhe::noise32(seed, fhe::kDomKskNoise, ridx, P.lwe_noise_log2) + dot +
                 (S[i] << (32u - P.log2_bks * lam));
    row[n] = b;
  }
}

// One warp per ciphertext.
__global__ void k_encrypt(Params P, const uint32_t *s, const int32_t *msg, size_t count,
                          uint64_t seed, uint32_t *ct) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t idx = (uint64_t)blockIdx.x * (blockDim.x / 32u) + threadIdx.x / 32u;
  if (idx >= count) return;
  const uint32_t n = P.n;
  uint32_t *c = ct + idx * (n + 1u);
  uint32_t dot = 0;
  for (uint32_t t = lane; t < n; t += 32u) {
    uint32_t a = (uint32_t)fhe::rand64(seed, fhe::kDomEncMask, idx * n + t);
    c[t] = a;
    dot += a * s[t];
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0)
    c[n] = fhe::noise32(seed, fhe::kDomEncNoise, idx, P.lwe_noise_log2) + dot +
           (uint32_t)msg[idx] * P.delta();
}

__global__ void k_decrypt(Params P, const uint32_t *s, const uint32_t *ct, size_t count,
                          int32_t *msg) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t idx = (uint64_t)blockIdx.x * (blockDim.x / 32u) + threadIdx.x / 32u;
  if (idx >= count) return;
  const uint32_t n = P.n;
  const uint32_t *c = ct + idx * (n + 1u);
  uint32_t dot = 0;
  for (uint32_t t = lane; t < n; t += 32u) dot += c[t] * s[t];
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) {
    const uint32_t ld = 31u - P.log2_p;
    uint32_t ph = c[n] - dot;
    int32_t m = (int32_t)((uint32_t)(ph + (1u << (ld - 1u))) >> ld);
    const int32_t p = (int32_t)P.p();
    msg[idx] = (m >= p) ? m - 2 * p : m;
  }
}

int validate(const fhe_params *prm) {
  if (!prm) return FHE_EINVAL;
  Params P = fhe::from_abi(*prm);
  if (!fhe::params_supported(P)) return FHE_EINVAL;
  if (P.l_ks > 8u) return FHE_EINVAL;
  return FHE_OK;
}

}  // namespace

extern "C" const char *fhe_strerror(int code) {
  switch (code) {
    case FHE_OK: return "ok";
    case FHE_EINVAL: return "invalid argument or unsupported parameter set";
    case FHE_ENOMEM: return "out of memory";
    case FHE_ECUDA: return "CUDA error";
    case FHE_ETIMEOUT: return "a bounded device wait timed out";
    case FHE_EUNSUPPORTED: return "not supported on this path";
    default: return "unknown error";
  }
}

static void keys_release(fhe_keys *K) {
  if (!K) return;
  cudaFree(K->d_lwe_key);
  cudaFree(K->d_glwe_key);
  cudaFree(K->d_bsk);
  cudaFree(K->d_ksk);
  cudaFree(K->d_big);
  cudaFree(K->d_status);
  cudaFree(K->d_bsk_tc);
  cudaFree(K->d_acc_tc);
  cudaFree(K->d_digits_tc);
  cudaFree(K->d_tsync);
  cudaFree(K->d_fft_twist);
  cudaFree(K->d_fft_tw);
  cudaFree(K->d_fft_kspec);
  cudaFree(K->d_fft_maxerr);
  free(K);
}

extern "C" int fhe_keygen_from_seed(const fhe_params *prm, uint64_t seed, size_t max_batch,
                                    void *stream, fhe_keys **out) {
  if (!out) return FHE_EINVAL;
  *out = NULL;
  int rc = validate(prm);
  if (rc) return rc;
  fhe_keys *K = (fhe_keys *)calloc(1, sizeof(fhe_keys));
  if (!K) return FHE_ENOMEM;
  K->P = fhe::from_abi(*prm);
  const Params &P = K->P;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaGetDevice(&K->device) != cudaSuccess) { free(K); return FHE_ECUDA; }
  K->ws_cap = max_batch ? max_batch : 16384;
  // until fhe_pbs_autotune measures it: tensor cores for every batch (a
  // tensor-core launch of up to 7 tiles runs on 16-CTA clusters, faster than
  // the CUDA-core path at any size on GB300)
  K->tc_min_batch = fhe::tc_available(P) ? 1u : SIZE_MAX;
  K->tc_cl8_max = -1;
  K->tc_cl8_tiles = -1;
  K->tc_force_cl = 0;
  K->tc_cl16_max = -1;
  K->tc_cl16_tiles = -1;
  K->tc_force_mc = -1;
  K->tc_l2_hints = -1;
  K->tc_split_ok = -1;
  K->tc_split_tiles = -1;
  const uint64_t bsk_words = (uint64_t)P.n * P.ggsw_words();
  const uint64_t ksk_words = (uint64_t)P.k * P.N * P.l_ks * (P.n + 1u);
  bool ok = cudaMalloc(&K->d_lwe_key, sizeof(uint32_t) * P.n) == cudaSuccess &&
            cudaMalloc(&K->d_glwe_key, sizeof(uint32_t) * P.k * P.N) == cudaSuccess &&
            cudaMalloc(&K->d_bsk, sizeof(uint32_t) * bsk_words) == cudaSuccess &&
            cudaMalloc(&K->d_ksk, sizeof(uint32_t) * ksk_words) == cudaSuccess &&
            cudaMalloc(&K->d_big, sizeof(uint32_t) * 2ull * K->ws_cap * P.big_words()) == cudaSuccess &&
            cudaMalloc(&K->d_status, sizeof(int)) == cudaSuccess;
  if (!ok) { keys_release(K); return FHE_ENOMEM; }
  cudaMemsetAsync(K->d_status, 0, sizeof(int), st);
  const uint32_t nk = (P.n > P.k * P.N) ? P.n : P.k * P.N;
  k_secret_keys<<<(nk + 255u) / 256u, 256, 0, st>>>(P, seed, K->d_lwe_key, K->d_glwe_key);
  k_bsk_rows<<<(unsigned)(P.n * P.rows()), 256, 2u * P.N * sizeof(uint32_t), st>>>(
      P, seed, K->d_lwe_key, K->d_glwe_key, K->d_bsk);
  const uint64_t ksk_rows = (uint64_t)P.k * P.N * P.l_ks;
  k_ksk_rows<<<(unsigned)((ksk_rows + 7u) / 8u), 256, 0, st>>>(P, seed, K->d_lwe_key,
                                                                 K->d_glwe_key, K->d_ksk);
  fhe::note_launches(3);
  if (cudaGetLastError() != cudaSuccess) { keys_release(K); return FHE_ECUDA; }
  *out = K;
  return FHE_OK;
}

extern "C" void fhe_keys_free(fhe_keys *K) {
  if (!K) return;
  cudaDeviceSynchronize();
  keys_release(K);
}

extern "C" int fhe_keys_params(const fhe_keys *K, fhe_params *out) {
  if (!K || !out) return FHE_EINVAL;
  const Params &P = K->P;
  out->n = P.n; out->k = P.k; out->N = P.N; out->log2_bg = P.log2_bg; out->l = P.l;
  out->log2_bks = P.log2_bks; out->l_ks = P.l_ks; out->log2_p = P.log2_p;
  out->lwe_noise_log2 = P.lwe_noise_log2; out->glwe_noise_log2 = P.glwe_noise_log2;
  return FHE_OK;
}

extern "C" size_t fhe_keys_size(const fhe_keys *K, int which) {
  if (!K) return 0;
  const Params &P = K->P;
  switch (which) {
    case FHE_KEY_LWE: return sizeof(uint32_t) * P.n;
    case FHE_KEY_GLWE: return sizeof(uint32_t) * P.k * P.N;
    case FHE_KEY_BSK: return sizeof(uint32_t) * (size_t)P.n * P.ggsw_words();
    case FHE_KEY_KSK: return sizeof(uint32_t) * (size_t)P.k * P.N * P.l_ks * (P.n + 1u);
    default: return 0;
  }
}

extern "C" int fhe_keys_export(const fhe_keys *K, int which, void *host_dst, size_t bytes) {
  size_t need = fhe_keys_size(K, which);
  if (!need || !host_dst || bytes != need) return FHE_EINVAL;
  const void *src = which == FHE_KEY_LWE ? (const void *)K->d_lwe_key
                    : which == FHE_KEY_GLWE ? (const void *)K->d_glwe_key
                    : which == FHE_KEY_BSK ? (const void *)K->d_bsk : (const void *)K->d_ksk;
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  FHE_CUDA_TRY(cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost));
  return FHE_OK;
}

extern "C" int fhe_encrypt(const fhe_keys *K, const int32_t *msg, size_t count, uint64_t seed,
                           uint32_t *ct, void *stream) {
  if (!K || (!msg && count) || (!ct && count)) return FHE_EINVAL;
  if (!count) return FHE_OK;
  unsigned blocks = (unsigned)((count + 7u) / 8u);
  k_encrypt<<<blocks, 256, 0, (cudaStream_t)stream>>>(K->P, K->d_lwe_key, msg, count, seed, ct);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

extern "C" int fhe_decrypt(const fhe_keys *K, const uint32_t *ct, size_t count, int32_t *msg,
                           void *stream) {
  if (!K || (!msg && count) || (!ct && count)) return FHE_EINVAL;
  if (!count) return FHE_OK;
  unsigned blocks = (unsigned)((count + 7u) / 8u);
  k_decrypt<<<blocks, 256, 0, (cudaStream_t)stream>>>(K->P, K->d_lwe_key, ct, count, msg);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

extern "C" int fhe_status(fhe_keys *K, void *stream) {
  if (!K) return FHE_EINVAL;
  int h = 0;
  FHE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  FHE_CUDA_TRY(cudaMemcpy(&h, K->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  FHE_CUDA_TRY(cudaMemset(K->d_status, 0, sizeof(int)));
  return h ? FHE_ETIMEOUT : FHE_OK;
}

// Test polynomial coefficients (centred boxes) for the message space
// p = 2^log2_p: coeff[c] = f[round(c p / N)] for boxes below p, -f[0] on the
// wrapped half box (Thm 2.1's negacyclic condition with one padding bit).
static void lut_coefficients(uint32_t N, uint32_t log2_p, const int32_t *f,
                             std::vector<int32_t> &co) {
  const uint32_t p = 1u << log2_p;
  co.resize(N);
  for (uint32_t c = 0; c < N; ++c) {
    uint32_t u = (c * p + N / 2u) / N;
    co[c] = (u < p) ? f[u] : (int32_t)(0u - (uint32_t)f[0]);
  }
}

// A bootstrap may read its input in one message space and write each table
// in another (the dynamic message space of DiNN, adopted by the paper in
// 5.2): boxes of p_in = 2^log2_p_in, outputs encoded with
// Delta_j = 2^(31 - log2_p_out[j]).  Multi-value groups rotate
// TV0 = (Delta_min / 2) sum X^i (Delta_min: the group's smallest Delta) and
// apply r_j = (Delta_j / Delta_min) (1 - X) coeffs(f_j), so that
// r_j * TV0 = Delta_j coeffs(f_j) mod X^N + 1.
extern "C" int fhe_lut_create_spaces(const fhe_keys *K, const int32_t *f, uint32_t L,
                                     uint32_t groups, const uint32_t *log2_p_in,
                                     const uint32_t *log2_p_out, fhe_lut **out) {
  if (!K || !f || !out || !log2_p_in || !log2_p_out || (L != 1u && L != 2u) || groups < 1u ||
      groups > fhe::kLutGroups || (L == 1u && groups != 1u))
    return FHE_EINVAL;
  const Params &P = K->P;
  for (uint32_t g = 0; g < groups; ++g) {
    if (log2_p_in[g] < 1u || log2_p_in[g] > 10u || (2u << log2_p_in[g]) > P.N) return FHE_EINVAL;
    for (uint32_t j = 0; j < L; ++j)
      if (log2_p_out[g * L + j] < 1u || log2_p_out[g * L + j] > 10u) return FHE_EINVAL;
  }
  *out = NULL;
  fhe_lut *T = (fhe_lut *)calloc(1, sizeof(fhe_lut));
  if (!T) return FHE_ENOMEM;
  T->L = L;
  T->N = P.N;
  T->groups = groups;
  std::vector<int32_t> co;
  if (L == 1u) {
    lut_coefficients(P.N, log2_p_in[0], f, co);
    const uint32_t delta_out = 1u << (31u - log2_p_out[0]);
    std::vector<uint32_t> tv(P.N);
    for (uint32_t c = 0; c < P.N; ++c) tv[c] = (uint32_t)co[c] * delta_out;
    if (cudaMalloc(&T->d_tv, sizeof(uint32_t) * P.N) != cudaSuccess) { free(T); return FHE_ENOMEM; }
    if (cudaMemcpy(T->d_tv, tv.data(), sizeof(uint32_t) * P.N, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(T->d_tv); free(T); return FHE_ECUDA;
    }
  } else {
    // r_{g,j}, kept sparse (the table's jumps); tables of group g start at
    // f + sum_{h<g} 2 p_h
    std::vector<int32_t> pos, val;
    const int32_t *fg = f;
    for (uint32_t g = 0; g < groups; ++g) {
      const uint32_t p = 1u << log2_p_in[g];
      const uint32_t lp_max = std::max(log2_p_out[2u * g], log2_p_out[2u * g + 1u]);
      T->tv0[g] = 1u << (30u - lp_max);
      for (uint32_t j = 0; j < 2u; ++j) {
        const uint32_t scale = 1u << (lp_max - log2_p_out[2u * g + j]);
        lut_coefficients(P.N, log2_p_in[g], fg + (size_t)j * p, co);
        T->off[g][j] = (uint32_t)pos.size();
        for (uint32_t c = 0; c < P.N; ++c) {
          const uint32_t r = scale * ((c == 0) ? (uint32_t)co[0] + (uint32_t)co[P.N - 1u]
                                               : (uint32_t)co[c] - (uint32_t)co[c - 1u]);
          if (r) { pos.push_back((int32_t)c); val.push_back((int32_t)r); }
        }
        T->nnz[g][j] = (uint32_t)pos.size() - T->off[g][j];
      }
      fg += 2u * (size_t)p;
    }
    size_t bytes = sizeof(int32_t) * (pos.size() ? pos.size() : 1u);
    if (cudaMalloc(&T->d_rpos, bytes) != cudaSuccess || cudaMalloc(&T->d_rval, bytes) != cudaSuccess) {
      cudaFree(T->d_rpos); free(T); return FHE_ENOMEM;
    }
    if (!pos.empty() &&
        (cudaMemcpy(T->d_rpos, pos.data(), sizeof(int32_t) * pos.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(T->d_rval, val.data(), sizeof(int32_t) * val.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
      cudaFree(T->d_rpos); cudaFree(T->d_rval); free(T); return FHE_ECUDA;
    }
  }
  *out = T;
  return FHE_OK;
}

extern "C" int fhe_lut_create(const fhe_keys *K, const int32_t *f, uint32_t L, fhe_lut **out) {
  if (!K) return FHE_EINVAL;
  const uint32_t lp[2] = {K->P.log2_p, K->P.log2_p};
  return fhe_lut_create_spaces(K, f, L, 1u, lp, lp, out);
}

namespace fhe {
LutArgs lut_args(const fhe_lut *T, const uint64_t *seg_end, uint64_t s0) {
  LutArgs a;
  memset(&a, 0, sizeof(a));
  a.L = T->L;
  a.tv = T->d_tv;
  a.rpos = T->d_rpos;
  a.rval = T->d_rval;
  for (uint32_t q = 0; q + 1u < kLutGroups; ++q) {
    uint64_t e = UINT64_MAX;  // past every ciphertext: groups above q + 1 unused
    if (seg_end && q + 1u < T->groups) e = (seg_end[q] > s0) ? seg_end[q] - s0 : 0u;
    a.seg_end[q] = e;
  }
  for (uint32_t g = 0; g < kLutGroups; ++g) {
    a.tv0[g] = T->tv0[g];
    for (uint32_t j = 0; j < 2u; ++j) {
      a.off[g][j] = T->off[g][j];
      a.nnz[g][j] = T->nnz[g][j];
    }
  }
  return a;
}
}  // namespace fhe

extern "C" void fhe_lut_free(fhe_lut *T) {
  if (!T) return;
  cudaDeviceSynchronize();
  cudaFree(T->d_tv);
  cudaFree(T->d_rpos);
  cudaFree(T->d_rval);
  free(T);
}
