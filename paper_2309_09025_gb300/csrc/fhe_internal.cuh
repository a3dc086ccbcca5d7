// fhe_internal.cuh -- shared internals of the sm_103a FHE-DiCSNN library.
//
// Everything here belongs to the product path.  It shares nothing with the
// CPU oracle: the SplitMix64 draw and the noise sampler below are written
// from their published definitions (Steele, Lea & Flood 2014; Irwin-Hall sum)
// so that keys generated here match any other implementation of the same
// definitions bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fhe_dicsnn.h"

namespace fhe {

// ---------------------------------------------------------------- params
struct Params {
  uint32_t n, k, N, log2_bg, l, log2_bks, l_ks, log2_p;
  int32_t lwe_noise_log2, glwe_noise_log2;
  __host__ __device__ uint32_t delta() const { return 1u << (31u - log2_p); }
  __host__ __device__ uint32_t p() const { return 1u << log2_p; }
  __host__ __device__ uint32_t rows() const { return (k + 1u) * l; }
  // words of one GGSW (one bootstrapping-key entry ek_i)
  __host__ __device__ uint64_t ggsw_words() const { return (uint64_t)rows() * (k + 1u) * N; }
  __host__ __device__ uint32_t lwe_words() const { return n + 1u; }
  __host__ __device__ uint32_t big_words() const { return k * N + 1u; }
};

inline Params from_abi(const fhe_params &a) {
  Params p;
  p.n = a.n; p.k = a.k; p.N = a.N; p.log2_bg = a.log2_bg; p.l = a.l;
  p.log2_bks = a.log2_bks; p.l_ks = a.l_ks; p.log2_p = a.log2_p;
  p.lwe_noise_log2 = a.lwe_noise_log2; p.glwe_noise_log2 = a.glwe_noise_log2;
  return p;
}

inline bool params_supported(const Params &p) {
  if (p.k != 1u) return false;
  if (!(p.N == 256u || p.N == 512u || p.N == 1024u || p.N == 2048u)) return false;
  if (p.n < 1u || p.n > 2048u) return false;
  if (p.l < 1u || p.l > 4u || p.log2_bg < 1u || p.log2_bg > 15u || p.log2_bg * p.l > 32u) return false;
  if (p.l_ks < 1u || p.log2_bks < 1u || p.log2_bks > 7u || p.log2_bks * p.l_ks > 32u) return false;
  if (p.log2_p < 1u || p.log2_p > 10u || (2u << p.log2_p) > p.N) return false;
  return true;
}

// Profiling event around a launch: inside a stream capture it must become an
// external event node of the graph; outside a capture a plain record.
inline cudaError_t record_prof_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t q = cudaStreamIsCapturing(st, &cs);
  if (q != cudaSuccess) return q;
  return cudaEventRecordWithFlags(e, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                              : cudaEventRecordDefault);
}

// ---------------------------------------------------------------- randomness
// Domains of the counter-based draws (one independent stream per purpose).
enum Domain : uint32_t {
  kDomLweKey = 0, kDomGlweKey = 1, kDomBskMask = 2, kDomBskNoise = 3,
  kDomKskMask = 4, kDomKskNoise = 5, kDomEncMask = 6, kDomEncNoise = 7
};

__host__ __device__ inline uint64_t splitmix_finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Output number `i` (0-based) of SplitMix64 whose state starts at `state`.
__host__ __device__ inline uint64_t splitmix_nth(uint64_t state, uint64_t i) {
  return splitmix_finalize(state + (i + 1ull) * 0x9E3779B97F4A7C15ull);
}
// Draw for (seed, domain, index): the seed selects a generator, the domain
// selects a sub-generator (its domain-th output), the index its output.
__host__ __device__ inline uint64_t rand64(uint64_t seed, uint32_t domain, uint64_t index) {
  return splitmix_nth(splitmix_nth(seed, domain), index);
}
// Noise: round(sum of 12 uniform signed 32-bit integers / 2^x), x = log2 of
// 1/sigma in torus units; x >= 64 gives 0.
__host__ __device__ inline uint32_t noise32(uint64_t seed, uint32_t domain, uint64_t index,
                                            int32_t x) {
  if (x >= 64) return 0u;
  int64_t acc = 0;
#pragma unroll
  for (uint32_t h = 0; h < 6u; ++h) {
    uint64_t r = rand64(seed, domain, index * 6ull + h);
    acc += (int64_t)(int32_t)(uint32_t)r;
    acc += (int64_t)(int32_t)(uint32_t)(r >> 32);
  }
  if (x <= 0) return (uint32_t)acc;
  int64_t t = acc + ((int64_t)1 << (x - 1));
  // floor division by 2^x of a signed value (arithmetic shift semantics)
  int64_t q = (t >= 0) ? (t >> x) : -((-t - 1) >> x) - 1;
  return (uint32_t)(uint64_t)q;
}

// ---------------------------------------------------------------- TFHE scalar ops
// Round q -> 2N (half up), result in [0, 2N).
__host__ __device__ inline uint32_t mod_switch_2n(uint32_t a, uint32_t log2_2n) {
  return (uint32_t)(a + (1u << (31u - log2_2n))) >> (32u - log2_2n);
}

__host__ inline uint32_t ilog2(uint32_t v) {
  uint32_t r = 0;
  while ((1u << r) < v) ++r;
  return r;
}

}  // namespace fhe

// ---------------------------------------------------------------- handles
struct fhe_keys {
  fhe::Params P;
  int device;
  uint32_t *d_lwe_key;   // [n]
  uint32_t *d_glwe_key;  // [kN]
  uint32_t *d_bsk;       // [n][rows][k+1][N]
  uint32_t *d_ksk;       // [kN][l_ks][n+1]
  // workspace of fhe_pbs_batch
  size_t ws_cap;         // ciphertexts per chunk
  uint32_t *d_big;       // [2][ws_cap][kN+1] extracted LWE_z ciphertexts
  int *d_status;         // device status word (FHE_OK / FHE_ETIMEOUT)
  // FHE_VARIANT_AUTO: batches of at least tc_min_batch ciphertexts run on
  // tensor cores, smaller ones on CUDA cores (SIZE_MAX: tensor-core path
  // not built for these parameters); set by fhe_pbs_autotune
  size_t tc_min_batch;
  // clusters of 8 CTAs of the tensor-core kernel the device holds at once
  // (-1: not queried yet)
  int tc_cl8_max;
  // batches of up to this many 256-ciphertext tiles run on clusters of 8
  // (set by fhe_pbs_autotune from timings; -1: up to tc_cl8_max)
  int tc_cl8_tiles;
  // clusters of 16 CTAs the device holds at once (-1: not queried yet; 0:
  // none) and the most tiles run on them (-1: up to tc_cl16_max)
  int tc_cl16_max;
  int tc_cl16_tiles;
  // force clusters of 4, 8 or 16 (0: the rules above); set by the autotuner
  // while it measures and by fhe_pbs_set_tc_shape
  int tc_force_cl;
  // digit tiles by cluster-multicast copies (1), per CTA (0) or the build's
  // default (-1: multicast where compiled in)
  int tc_force_mc;
  // L2 evict-last policy on the digit operand (1), none (0), default (-1)
  int tc_l2_hints;
  // tiles spread over two 16-CTA clusters: cooperative clustered launches
  // work on this device (1), were refused (0), not tried yet (-1); and the
  // most tiles run that way (-1: up to half the 16-CTA clusters)
  int tc_split_ok;
  int tc_split_tiles;
  uint32_t *d_tsync;     // per-tile barrier counters of the split shape
  // tensor-core key layout (built on first use of FHE_VARIANT_TC)
  void *d_bsk_tc;
  size_t bsk_tc_bytes;
  uint32_t *d_acc_tc;    // accumulators of the tensor-core path
  void *d_digits_tc;     // digit operand of the tensor-core path
  // instrumentation: when set, the next blind-rotation launch is bracketed by
  // this event pair and its ciphertext count stored in prof_count
  cudaEvent_t prof_ev0, prof_ev1;
  size_t prof_count;
  // FP64 FFT variant (built on first use): twist table, FFT twiddles, key
  // spectra, largest rounding distance seen (bits of a double)
  void *d_fft_twist, *d_fft_tw, *d_fft_kspec;
  unsigned long long *d_fft_maxerr;
};

namespace fhe {
// Table groups of one multi-value table set (one per layer of a network
// whose layers have their own message spaces).
constexpr uint32_t kLutGroups = FHE_LUT_MAX_GROUPS;
}  // namespace fhe

struct fhe_lut {
  uint32_t L;
  uint32_t N;
  uint32_t groups;       // table groups (more than one only when L == 2)
  uint32_t *d_tv;        // L == 1: test polynomial [N]
  int32_t *d_rpos;       // L == 2: sparse (Delta_j / Delta_min) (1 - X) coeffs(f_j):
  int32_t *d_rval;       //         positions and values, concatenated per group and j
  uint32_t tv0[fhe::kLutGroups];     // L == 2: TV0 coefficient of each group (Delta_min / 2)
  uint32_t nnz[fhe::kLutGroups][2];
  uint32_t off[fhe::kLutGroups][2];
};

namespace fhe {
// The tables of one bootstrap launch as its kernel reads them (a by-value
// kernel parameter).  L = 1: the test polynomial tv.  L = 2 (multi-value):
// group g rotates TV0 = tv0[g] * sum_i X^i and applies r_{g,j}, the entries
// [off[g][j], off[g][j] + nnz[g][j]) of rpos / rval; ciphertext i of the
// launch belongs to group g = #{q : i >= seg_end[q]}.
struct LutArgs {
  uint32_t L;
  const uint32_t *tv;
  const int32_t *rpos;
  const int32_t *rval;
  uint64_t seg_end[kLutGroups - 1];
  uint32_t tv0[kLutGroups];
  uint32_t off[kLutGroups][2];
  uint32_t nnz[kLutGroups][2];
};

struct LutGroup {
  uint32_t tv0, off0, nnz0, off1, nnz1;
};

// Group of ciphertext i; only compile-time indices into the parameter.
__device__ __forceinline__ LutGroup lut_group(const LutArgs &a, uint64_t i) {
  uint32_t g = 0;
#pragma unroll
  for (uint32_t q = 0; q + 1u < kLutGroups; ++q) g += (i >= a.seg_end[q]) ? 1u : 0u;
  LutGroup s = {a.tv0[0], a.off[0][0], a.nnz[0][0], a.off[0][1], a.nnz[0][1]};
#pragma unroll
  for (uint32_t q = 1; q < kLutGroups; ++q)
    if (g == q) s = LutGroup{a.tv0[q], a.off[q][0], a.nnz[q][0], a.off[q][1], a.nnz[q][1]};
  return s;
}

// Kernel view of `lut` for the ciphertexts [s0, ...) of a call whose group
// boundaries are seg_end (groups - 1 call-relative ends; NULL: one group).
LutArgs lut_args(const fhe_lut *lut, const uint64_t *seg_end, uint64_t s0);
}  // namespace fhe

// On failure, also clear the runtime's last-error slot so that a
// recoverable error does not resurface in later, unrelated checks.
#define FHE_CUDA_TRY(expr)                        \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      (void)cudaGetLastError();                   \
      return FHE_ECUDA;                           \
    }                                             \
  } while (0)

namespace fhe {
// Process-wide kernel-launch counter (fhe_keys.cu).
void note_launches(int64_t n);
uint64_t launches();
// Implemented in fhe_pbs_exact.cu / fhe_pbs_tc.cu.
// Table j of the outputs starts at ct_out + j * table_stride (words).
// seg_end: the group boundaries of a grouped table set (see lut_args).
int pbs_exact(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
              uint32_t *ct_out, size_t table_stride, cudaStream_t st,
              const uint64_t *seg_end = nullptr);
int pbs_tc(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
           uint32_t *ct_out, size_t table_stride, cudaStream_t st,
           const uint64_t *seg_end = nullptr);
int pbs_fft(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
            uint32_t *ct_out, size_t table_stride, cudaStream_t st,
            const uint64_t *seg_end = nullptr);
int fft_prepare(fhe_keys *K);
// Dispatch on the variant (FHE_EINVAL for an unknown one).
int pbs_run(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
            uint32_t *ct_out, size_t table_stride, int variant, cudaStream_t st,
            const uint64_t *seg_end = nullptr);
// Exact bootstrapping with the extracted ciphertexts in a caller buffer
// (fhe_noalloc.cu); single batch, no allocation.
int pbs_exact_into(const fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
                   uint32_t *ct_out, uint32_t *big, cudaStream_t st);
// Builds the variant's key layout and workspace ahead of the first call
// (FHE_OK for variants without one; FHE_EUNSUPPORTED for unsupported sets).
int pbs_prepare(fhe_keys *K, int variant);
bool tc_available(const Params &P);
int key_switch_batch(const fhe_keys *K, const uint32_t *d_big, size_t count, uint32_t *ct_out,
                     cudaStream_t st);
}  // namespace fhe
