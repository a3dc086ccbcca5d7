// fhe_pbs_fft.cu -- blind rotation with the conventional FP64 negacyclic FFT
// product (the paper's "FFT technology", 5.3), kept beside the exact paths as
// the comparison baseline.  It is NOT bit-exact: each external-product output
// is rounded to the nearest integer from a double; the largest distance to an
// integer seen (the torus rounding error, in units of 2^-32) is recorded.
//
// Negacyclic transform of a real polynomial a mod X^N + 1 (M = N/2,
// w = exp(i pi / N), a root of X^N + 1):
//   v_k = (a_k + i a_{k+M}) w^k,  A_j = sum_k v_k exp(+2 pi i jk / M)
// gives A_j = a(w^{4j+1}); the other roots are conjugates, so products of
// real polynomials are pointwise products of A.  Inverse: v = (1/M) sum_j
// C_j exp(-2 pi i jk / M), u_k = v_k w^{-k}, c_k = Re u_k, c_{k+M} = Im u_k.
//
// One CTA per ciphertext, 256 threads; accumulators (uint32), digit spectra
// and the transform of every step in shared memory; the bootstrapping key is
// transformed once (signed 32-bit words) and read from L2 each step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "fhe_internal.cuh"

using fhe::LutArgs;
using fhe::Params;

namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// In-place FFT of `cnt` arrays of M points in shared memory whose inputs
// were stored at bit-reversed positions (decimation in time).  With
// bit-reversed input, the four consecutive blocks B0..B3 of q points in a
// group of 4q hold the q-point transforms D_r of the subsequences x[4m + r]
// in the order D_0, D_2, D_1, D_3; one radix-4 pass merges them:
//   a_r = W^{rp} D_r[p]  (W = exp(+-2 pi i / 4q), p < q),
//   Z[p + kq] = sum_r a_r (+-i)^{rk},  k = 0..3,
// three twiddle products per four points where two radix-2 passes take four
// (none in the first pass, q = 1).  An odd log2 M starts with one radix-2
// pass of unit twiddles.  tw[m] = exp(+2 pi i m / M) for m < 3M/4;
// `inverse` uses the conjugate twiddles (negative exponent).
template <int M, int Q>
__device__ __forceinline__ void fft_radix4_passes(double2 *a, int cnt, const double2 *__restrict__ tw,
                                                  bool inverse) {
  if constexpr (Q < M) {
    constexpr int stride = M / (4 * Q);  // W^{rp} = tw[r p stride]
    for (int t = threadIdx.x; t < cnt * (M / 4); t += kFftThreads) {
      const int arr = t / (M / 4), bt = t % (M / 4);
      const int g = bt / Q, p = bt % Q;
      double2 *x = a + (size_t)arr * M + 4 * Q * g + p;
      double2 a0 = x[0], a1 = x[2 * Q], a2 = x[Q], a3 = x[3 * Q];
      if constexpr (Q > 1) {
        const double2 w1 = __ldg(tw + p * stride), w2 = __ldg(tw + 2 * p * stride),
                      w3 = __ldg(tw + 3 * p * stride);
        a1 = inverse ? cmulc(a1, w1) : cmul(a1, w1);
        a2 = inverse ? cmulc(a2, w2) : cmul(a2, w2);
        a3 = inverse ? cmulc(a3, w3) : cmul(a3, w3);
      }
      const double2 s02 = make_double2(a0.x + a2.x, a0.y + a2.y);
      const double2 d02 = make_double2(a0.x - a2.x, a0.y - a2.y);
      const double2 s13 = make_double2(a1.x + a3.x, a1.y + a3.y);
      // j13 = +i (a1 - a3) forward, -i (a1 - a3) inverse
      const double2 d13 = make_double2(a1.x - a3.x, a1.y - a3.y);
      const double2 j13 = inverse ? make_double2(d13.y, -d13.x) : make_double2(-d13.y, d13.x);
      x[0] = make_double2(s02.x + s13.x, s02.y + s13.y);
      x[Q] = make_double2(d02.x + j13.x, d02.y + j13.y);
      x[2 * Q] = make_double2(s02.x - s13.x, s02.y - s13.y);
      x[3 * Q] = make_double2(d02.x - j13.x, d02.y - j13.y);
    }
    __syncthreads();
    fft_radix4_passes<M, 4 * Q>(a, cnt, tw, inverse);
  }
}

template <int M>
__device__ void fft_stages(double2 *a, int cnt, const double2 *__restrict__ tw, bool inverse) {
  constexpr int LOGM = (M == 512) ? 9 : 10;
  if constexpr ((LOGM & 1) != 0) {
    for (int t = threadIdx.x; t < cnt * (M / 2); t += kFftThreads) {
      double2 *x = a + 2 * t;  // arrays are contiguous: pair t of all of them
      const double2 u = x[0], v = x[1];
      x[0] = make_double2(u.x + v.x, u.y + v.y);
      x[1] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    fft_radix4_passes<M, 2>(a, cnt, tw, inverse);
  } else {
    fft_radix4_passes<M, 1>(a, cnt, tw, inverse);
  }
}

template <int M>
__device__ __forceinline__ int bitrev(int k) {
  constexpr int LOGM = (M == 512) ? 9 : 10;
  return (int)(__brev((unsigned)k) >> (32 - LOGM));
}

// Key spectra: for every GGSW polynomial (i, row, comp) the transform of its
// words read as signed 32-bit integers.  One CTA per polynomial.
template <int M>
__global__ void __launch_bounds__(kFftThreads)
    k_key_spectra(const uint32_t *__restrict__ bsk, const double2 *__restrict__ twist,
                  const double2 *__restrict__ tw, double2 *__restrict__ out) {
  extern __shared__ double2 sh[];
  const uint32_t *K = bsk + (size_t)blockIdx.x * (2 * M);
  for (int k = threadIdx.x; k < M; k += kFftThreads) {
    const double2 v = make_double2((double)(int32_t)K[k], (double)(int32_t)K[k + M]);
    sh[bitrev<M>(k)] = cmul(v, __ldg(twist + k));
  }
  __syncthreads();
  fft_stages<M>(sh, 1, tw, false);
  for (int k = threadIdx.x; k < M; k += kFftThreads) out[(size_t)blockIdx.x * M + k] = sh[k];
}

// Shared memory holds 4 CTAs per SM at N = 1024 (P630: 56 KB each) and 2 at
// N = 2048 (80 KB); the bound of 4 CTAs keeps registers from lowering the
// first (0: no bound for the second, which needs no more than 128).
template <int N>
__global__ void __launch_bounds__(kFftThreads, N == 1024 ? 4 : 0)
    k_blind_rotate_fft(Params P, const double2 *__restrict__ kspec, const double2 *__restrict__ twist,
                       const double2 *__restrict__ tw, const uint32_t *__restrict__ ct_in,
                       size_t count, const __grid_constant__ LutArgs lut,
                       uint32_t *__restrict__ big_out,
                       unsigned long long *max_err_bits) {
  constexpr int M = N / 2;
  constexpr uint32_t LOG2_2N = (N == 1024) ? 11 : 12;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t n = P.n, l = P.l, R = 2u * l;
  double2 *spec = reinterpret_cast<double2 *>(smem);                    // [R][M]
  uint32_t *acc = reinterpret_cast<uint32_t *>(smem + (size_t)R * M * 16);  // [2][N]
  const size_t cti = blockIdx.x;
  const uint32_t *ct = ct_in + cti * (n + 1u);
  const uint32_t total_bits = l * P.log2_bg;
  const uint32_t Bmask = (1u << P.log2_bg) - 1u, Bhalf = 1u << (P.log2_bg - 1u);
  const double inv_m = 1.0 / (double)M;
  double max_err = 0.0;

  // the table group of this CTA's ciphertext (multi-value: TV0 and r_j)
  const fhe::LutGroup grp = fhe::lut_group(lut, cti);
  const uint32_t bb = fhe::mod_switch_2n(ct[n], LOG2_2N);
  for (uint32_t c = threadIdx.x; c < (uint32_t)N; c += kFftThreads) {
    const uint32_t s = (c + bb) & (2u * N - 1u);
    uint32_t v;
    if (lut.L == 1u) v = (s < (uint32_t)N) ? lut.tv[s] : (0u - lut.tv[s - N]);
    else v = (s < (uint32_t)N) ? grp.tv0 : (0u - grp.tv0);
    acc[c] = 0u;
    acc[N + c] = v;
  }
  __syncthreads();

  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t a = fhe::mod_switch_2n(__ldg(ct + i), LOG2_2N);
    // digits of X^a ACC - ACC, folded and twisted, at bit-reversed positions
    for (int k = threadIdx.x; k < M; k += kFftThreads) {
      const double2 w = __ldg(twist + k);
      const int br = bitrev<M>(k);
      for (uint32_t j = 0; j < 2u; ++j) {
        const uint32_t *Pj = acc + j * N;
        uint32_t xr[2];
        for (int h = 0; h < 2; ++h) {
          const uint32_t c = (uint32_t)(k + h * M);
          const uint32_t s = (c + 2u * N - a) & (2u * N - 1u);
          const uint32_t rot = (s < (uint32_t)N) ? Pj[s] : (0u - Pj[s - N]);
          const uint32_t x = rot - Pj[c];
          xr[h] = (total_bits >= 32u) ? x
                                       : ((uint32_t)(x + (1u << (31u - total_bits))) >> (32u - total_bits));
        }
        for (int lam = (int)l - 1; lam >= 0; --lam) {
          int32_t dg[2];
          for (int h = 0; h < 2; ++h) {
            const uint32_t d = xr[h] & Bmask;
            xr[h] >>= P.log2_bg;
            dg[h] = (int32_t)d;
            if (d >= Bhalf) { dg[h] -= (int32_t)(Bmask + 1u); xr[h] += 1u; }
          }
          spec[(size_t)(j * l + (uint32_t)lam) * M + br] =
              cmul(make_double2((double)dg[0], (double)dg[1]), w);
        }
      }
    }
    __syncthreads();
    fft_stages<M>(spec, (int)R, tw, false);
    // pointwise multiply-accumulate with the key spectra of step i; the two
    // outputs are written back at bit-reversed positions of rows 0 and 1
    double2 o0[M / kFftThreads], o1[M / kFftThreads];
#pragma unroll
    for (int q = 0; q < M / kFftThreads; ++q) {
      const int k = threadIdx.x + q * kFftThreads;
      double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
      for (uint32_t r = 0; r < R; ++r) {
        const double2 d = spec[(size_t)r * M + k];
        const double2 *kr = kspec + (((size_t)i * R + r) * 2u) * M;
        const double2 k0 = __ldg(kr + k), k1 = __ldg(kr + M + k);
        s0.x += d.x * k0.x - d.y * k0.y; s0.y += d.x * k0.y + d.y * k0.x;
        s1.x += d.x * k1.x - d.y * k1.y; s1.y += d.x * k1.y + d.y * k1.x;
      }
      o0[q] = s0;
      o1[q] = s1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < M / kFftThreads; ++q) {
      const int k = threadIdx.x + q * kFftThreads;
      const int br = bitrev<M>(k);
      spec[br] = o0[q];
      spec[M + br] = o1[q];
    }
    __syncthreads();
    fft_stages<M>(spec, 2, tw, true);
    // untwist, unfold, round to the nearest integer, add mod 2^32
    for (int k = threadIdx.x; k < M; k += kFftThreads) {
      const double2 w = __ldg(twist + k);
      for (uint32_t j = 0; j < 2u; ++j) {
        const double2 u = cmulc(spec[(size_t)j * M + k], w);
        const double re = u.x * inv_m, im = u.y * inv_m;
        const double rr = rint(re), ri = rint(im);
        max_err = fmax(max_err, fmax(fabs(re - rr), fabs(im - ri)));
        acc[j * N + k] += (uint32_t)(uint64_t)(long long)rr;
        acc[j * N + k + M] += (uint32_t)(uint64_t)(long long)ri;
      }
    }
    __syncthreads();
  }

  // sample extraction (multi-value split when L == 2)
  const uint32_t W = N + 1u;
  for (uint32_t jl = 0; jl < lut.L; ++jl) {
    const uint32_t nnz = jl ? grp.nnz1 : grp.nnz0, off = jl ? grp.off1 : grp.off0;
    for (uint32_t c = threadIdx.x; c < W; c += kFftThreads) {
      const uint32_t *A = acc, *B = acc + N;
      uint32_t v;
      if (lut.L == 1u) {
        v = (c == (uint32_t)N) ? B[0] : (c == 0 ? A[0] : (0u - A[N - c]));
      } else {
        const uint32_t m = (c == (uint32_t)N || c == 0) ? 0u : N - c;
        const uint32_t *Pp = (c == (uint32_t)N) ? B : A;
        uint32_t s = 0;
        for (uint32_t t = 0; t < nnz; ++t) {
          const uint32_t ep = (uint32_t)lut.rpos[off + t];
          const uint32_t val = (uint32_t)lut.rval[off + t];
          s += val * ((m >= ep) ? Pp[m - ep] : (0u - Pp[m + N - ep]));
        }
        v = (c == (uint32_t)N || c == 0) ? s : (0u - s);
      }
      big_out[((size_t)jl * count + cti) * W + c] = v;
    }
  }
  // largest rounding distance seen by this thread (non-negative doubles
  // order like their bit patterns)
  atomicMax(max_err_bits, (unsigned long long)__double_as_longlong(max_err));
}

}  // namespace

namespace fhe {

static bool fft_supported(const Params &P) {
  return P.k == 1u && (P.N == 1024u || P.N == 2048u) && 2u * P.l <= 8u;
}

int fft_prepare(fhe_keys *K) {
  const Params &P = K->P;
  if (K->d_fft_kspec) return FHE_OK;
  const uint32_t M = P.N / 2u;
  std::vector<double2> twist(M), tw(3u * M / 4u);
  const double pi = 3.14159265358979323846264338327950288;
  for (uint32_t k = 0; k < M; ++k)
    twist[k] = make_double2(cos(pi * (double)k / (double)P.N), sin(pi * (double)k / (double)P.N));
  for (uint32_t m = 0; m < 3u * M / 4u; ++m)
    tw[m] = make_double2(cos(2.0 * pi * (double)m / (double)M), sin(2.0 * pi * (double)m / (double)M));
  const size_t polys = (size_t)P.n * P.rows() * 2u;
  if (cudaMalloc(&K->d_fft_twist, sizeof(double2) * M) != cudaSuccess ||
      cudaMalloc(&K->d_fft_tw, sizeof(double2) * (3u * M / 4u)) != cudaSuccess ||
      cudaMalloc(&K->d_fft_kspec, sizeof(double2) * M * polys) != cudaSuccess ||
      cudaMalloc(&K->d_fft_maxerr, sizeof(unsigned long long)) != cudaSuccess)
    return FHE_ENOMEM;
  FHE_CUDA_TRY(cudaMemcpy(K->d_fft_twist, twist.data(), sizeof(double2) * M, cudaMemcpyHostToDevice));
  FHE_CUDA_TRY(cudaMemcpy(K->d_fft_tw, tw.data(), sizeof(double2) * (3u * M / 4u), cudaMemcpyHostToDevice));
  FHE_CUDA_TRY(cudaMemset(K->d_fft_maxerr, 0, sizeof(unsigned long long)));
  if (M == 512u)
    k_key_spectra<512><<<(unsigned)polys, kFftThreads, 512 * 16>>>(
        K->d_bsk, (const double2 *)K->d_fft_twist, (const double2 *)K->d_fft_tw, (double2 *)K->d_fft_kspec);
  else
    k_key_spectra<1024><<<(unsigned)polys, kFftThreads, 1024 * 16>>>(
        K->d_bsk, (const double2 *)K->d_fft_twist, (const double2 *)K->d_fft_tw, (double2 *)K->d_fft_kspec);
  note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  return FHE_OK;
}

int pbs_fft(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
            uint32_t *ct_out, size_t table_stride, cudaStream_t st, const uint64_t *seg_end) {
  const Params &P = K->P;
  if (!fft_supported(P)) return FHE_EUNSUPPORTED;
  int rc = fft_prepare(K);
  if (rc) return rc;
  const uint32_t M = P.N / 2u, R = P.rows();
  const size_t smem = (size_t)R * M * 16u + 2u * P.N * 4u;
  for (size_t s0 = 0; s0 < count; s0 += K->ws_cap) {
    const size_t cnt = (count - s0 < K->ws_cap) ? count - s0 : K->ws_cap;
    const LutArgs la = lut_args(lut, seg_end, s0);
    const bool prof = (s0 == 0) && K->prof_ev0;
    if (prof) { FHE_CUDA_TRY(record_prof_event(K->prof_ev0, st)); K->prof_count = cnt; }
    if (P.N == 1024u) {
      FHE_CUDA_TRY(cudaFuncSetAttribute(k_blind_rotate_fft<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_blind_rotate_fft<1024><<<(unsigned)cnt, kFftThreads, smem, st>>>(
          P, (const double2 *)K->d_fft_kspec, (const double2 *)K->d_fft_twist, (const double2 *)K->d_fft_tw,
          ct_in + s0 * (P.n + 1u), cnt, la, K->d_big, K->d_fft_maxerr);
    } else {
      FHE_CUDA_TRY(cudaFuncSetAttribute(k_blind_rotate_fft<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_blind_rotate_fft<2048><<<(unsigned)cnt, kFftThreads, smem, st>>>(
          P, (const double2 *)K->d_fft_kspec, (const double2 *)K->d_fft_twist, (const double2 *)K->d_fft_tw,
          ct_in + s0 * (P.n + 1u), cnt, la, K->d_big, K->d_fft_maxerr);
    }
    note_launches(1);
    FHE_CUDA_TRY(cudaGetLastError());
    if (prof) FHE_CUDA_TRY(record_prof_event(K->prof_ev1, st));
    for (uint32_t j = 0; j < lut->L; ++j) {
      rc = key_switch_batch(K, K->d_big + (size_t)j * cnt * P.big_words(), cnt,
                            ct_out + (size_t)j * table_stride + s0 * (P.n + 1u), st);
      if (rc) return rc;
    }
  }
  return FHE_OK;
}

}  // namespace fhe

extern "C" int fhe_fft_max_error(fhe_keys *K, double *max_err, int reset) {
  if (!K || !max_err) return FHE_EINVAL;
  *max_err = 0.0;
  if (!K->d_fft_maxerr) return FHE_OK;
  unsigned long long bits = 0;
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  FHE_CUDA_TRY(cudaMemcpy(&bits, K->d_fft_maxerr, sizeof(bits), cudaMemcpyDeviceToHost));
  union { unsigned long long u; double d; } cv;
  cv.u = bits;
  *max_err = cv.d;
  if (reset) FHE_CUDA_TRY(cudaMemset(K->d_fft_maxerr, 0, sizeof(unsigned long long)));
  return FHE_OK;
}
