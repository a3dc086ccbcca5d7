// fhe_pbs_exact.cu -- exact programmable bootstrapping on CUDA cores
// (paper 2.1: Initialization, Blind Rotation, Sample Extraction, Key
// Switching; Thm 2.1).
//
// Blind rotation.  One CTA owns CPC ciphertexts for all n CMux steps; their
// accumulators stay in shared memory.  Per step i:
//   1. digits: every coefficient of X^{a~_i} ACC - ACC is rounded to the top
//      l*log2_bg bits and split into l signed digits (int16), stored twice
//      ([-D | D], the negacyclic extension) so the product needs no sign test;
//   2. the GGSW row ek_i (rows x (k+1) polynomials) arrives in shared memory
//      through one cp.async.bulk copy completed on an mbarrier, issued while
//      the previous step finished;
//   3. external product: each thread owns 8 consecutive output coefficients of
//      both output polynomials for two ciphertexts (32 uint32 accumulators) and
//      walks the key index d; the key word is a shared-memory broadcast, the
//      digit window slides through registers (one 16-byte load per 8 d);
//   4. ACC += product.
// The multiply-accumulates are exact uint32 IMADs (wrap mod 2^32).
#include <cuda_runtime.h>
#include <stdint.h>

#include "fhe_internal.cuh"

using fhe::LutArgs;
using fhe::Params;

namespace {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait (about one second); false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 1000000000ull) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Failure-detection self-test: one thread waits on an mbarrier that nothing
// completes, with the same bounded-wait pattern as the bootstrap kernels but a
// caller-chosen limit; when it gives up it records FHE_ETIMEOUT in the status
// word, which the host reads with fhe_status.  Nothing faults or hangs.
__global__ void k_selftest_timeout(uint64_t limit_ns, int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(&bar, 0u)) {
    if (global_ns() - t0 > limit_ns) {
      atomicExch(status, FHE_ETIMEOUT);
      return;
    }
  }
}

// Unpack 8 int16 (one 16-byte load) into int32.
__device__ __forceinline__ void unpack8(const int16_t *src, int32_t *dst) {
  uint4 v = *reinterpret_cast<const uint4 *>(src);
  uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    dst[2 * q] = ((int32_t)(w[q] << 16)) >> 16;
    dst[2 * q + 1] = ((int32_t)w[q]) >> 16;
  }
}

// Shared-memory plan of the blind-rotation kernel (byte offsets).
struct BrSmem {
  uint32_t acc, key, dig, abar, bar, total;
};
__host__ __device__ inline BrSmem br_smem(uint32_t N, uint32_t CPC, uint32_t R, uint32_t n) {
  BrSmem s;
  uint32_t o = 0;
  s.acc = o; o += CPC * 2u * N * 4u;
  s.key = o; o += R * 2u * N * 4u;
  s.dig = o; o += CPC * R * 2u * N * 2u;
  s.abar = o; o += ((CPC * (n + 1u) * 2u) + 15u) & ~15u;
  s.bar = o; o += 16u;
  s.total = o;
  return s;
}

template <int N, int CPC>
__global__ void __launch_bounds__((N / 8) * (CPC / 2))
    k_blind_rotate_exact(Params P, const uint32_t *__restrict__ bsk,
                         const uint32_t *__restrict__ ct_in, size_t count,
                         const __grid_constant__ LutArgs lut, uint32_t *__restrict__ big_out,
                         int *status) {
  constexpr int THREADS = (N / 8) * (CPC / 2);
  constexpr uint32_t LOG2_2N = (N == 256) ? 9 : (N == 512) ? 10 : (N == 1024) ? 11 : 12;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t n = P.n, l = P.l, R = 2u * l;
  const BrSmem S = br_smem(N, CPC, R, n);
  uint32_t *acc_s = reinterpret_cast<uint32_t *>(smem + S.acc);  // [CPC][2][N]
  uint32_t *key_s = reinterpret_cast<uint32_t *>(smem + S.key);  // [R][2][N]
  int16_t *dig_s = reinterpret_cast<int16_t *>(smem + S.dig);    // [CPC][R][2N]
  uint16_t *abar_s = reinterpret_cast<uint16_t *>(smem + S.abar); // [CPC][n+1]
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S.bar);
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const size_t base = (size_t)blockIdx.x * CPC;
  const uint32_t key_bytes = R * 2u * N * 4u;

  if (tid == 0) {
    s_abort = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // modulus-switched masks and bodies (dummy ciphertexts past `count`: 0)
  for (uint32_t e = tid; e < CPC * (n + 1u); e += THREADS) {
    uint32_t b = e / (n + 1u), i = e % (n + 1u);
    uint32_t v = (base + b < count) ? ct_in[(base + b) * (n + 1u) + i] : 0u;
    abar_s[e] = (uint16_t)fhe::mod_switch_2n(v, LOG2_2N);
  }
  __syncthreads();
  // ACC = (0, X^{-b~} TV); the multi-value case rotates the constant TV0
  // coefficient of the ciphertext's table group
  for (uint32_t e = tid; e < CPC * N; e += THREADS) {
    uint32_t b = e / N, c = e % N;
    uint32_t bb = abar_s[b * (n + 1u) + n];
    uint32_t s = (c + bb) & (2u * N - 1u);
    uint32_t v;
    if (lut.L == 1u) {
      v = (s < N) ? lut.tv[s] : (0u - lut.tv[s - N]);
    } else {
      const uint32_t tv0 = fhe::lut_group(lut, base + b).tv0;
      v = (s < N) ? tv0 : (0u - tv0);
    }
    acc_s[(b * 2u + 0u) * N + c] = 0u;
    acc_s[(b * 2u + 1u) * N + c] = v;
  }
  if (tid == 0) {
    mbar_expect_tx(bar, key_bytes);
    bulk_g2s(key_s, bsk, key_bytes, bar);
  }
  __syncthreads();

  const int g = tid / (N / 8);
  const int c0 = (tid % (N / 8)) * 8;
  const uint32_t total_bits = l * P.log2_bg;
  const uint32_t Bmask = (1u << P.log2_bg) - 1u, Bhalf = 1u << (P.log2_bg - 1u);

  for (uint32_t i = 0; i < n; ++i) {
    // 1. digits of X^{a~} ACC - ACC
    for (uint32_t e = tid; e < CPC * 2u * N; e += THREADS) {
      const uint32_t b = e / (2u * N), j = (e / N) & 1u, c = e % N;
      const uint32_t a = abar_s[b * (n + 1u) + i];
      const uint32_t *Pj = acc_s + (b * 2u + j) * N;
      const uint32_t s = (c + 2u * N - a) & (2u * N - 1u);
      const uint32_t rot = (s < N) ? Pj[s] : (0u - Pj[s - N]);
      const uint32_t x = rot - Pj[c];
      uint32_t xr = (total_bits >= 32u) ? x
                                         : ((uint32_t)(x + (1u << (31u - total_bits))) >> (32u - total_bits));
      int16_t *D = dig_s + (size_t)(b * R + j * l) * 2u * N;
      for (int lam = (int)l - 1; lam >= 0; --lam) {
        uint32_t d = xr & Bmask;
        xr >>= P.log2_bg;
        int32_t sd = (int32_t)d;
        if (d >= Bhalf) { sd -= (int32_t)(Bmask + 1u); xr += 1u; }
        int16_t *Dl = D + (size_t)lam * 2u * N;
        Dl[N + c] = (int16_t)sd;
        Dl[c] = (int16_t)(-sd);
      }
    }
    // 2. the GGSW row of this step
    if (!mbar_wait_bounded(bar, i & 1u)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;

    // 3. external product
    uint32_t accA[2][8], accB[2][8];  // [output poly j][coefficient]
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 8; ++q) { accA[j][q] = 0u; accB[j][q] = 0u; }
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t *K0 = key_s + (r * 2u + 0u) * N;
      const uint32_t *K1 = key_s + (r * 2u + 1u) * N;
      const int16_t *eA = dig_s + (size_t)((2 * g + 0) * R + r) * 2u * N + N;  // x = 0
      const int16_t *eB = dig_s + (size_t)((2 * g + 1) * R + r) * 2u * N + N;
      int32_t wA[16], wB[16];
      unpack8(eA + c0, wA + 8);
      unpack8(eB + c0, wB + 8);
#pragma unroll 1
      for (int d0 = 0; d0 < N; d0 += 8) {
        unpack8(eA + c0 - d0 - 8, wA);
        unpack8(eB + c0 - d0 - 8, wB);
        const uint4 k0a = *reinterpret_cast<const uint4 *>(K0 + d0);
        const uint4 k0b = *reinterpret_cast<const uint4 *>(K0 + d0 + 4);
        const uint4 k1a = *reinterpret_cast<const uint4 *>(K1 + d0);
        const uint4 k1b = *reinterpret_cast<const uint4 *>(K1 + d0 + 4);
        const uint32_t kk0[8] = {k0a.x, k0a.y, k0a.z, k0a.w, k0b.x, k0b.y, k0b.z, k0b.w};
        const uint32_t kk1[8] = {k1a.x, k1a.y, k1a.z, k1a.w, k1b.x, k1b.y, k1b.z, k1b.w};
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t da = (uint32_t)wA[8 + q - dd], db = (uint32_t)wB[8 + q - dd];
            accA[0][q] += kk0[dd] * da;
            accA[1][q] += kk1[dd] * da;
            accB[0][q] += kk0[dd] * db;
            accB[1][q] += kk1[dd] * db;
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) { wA[8 + q] = wA[q]; wB[8 + q] = wB[q]; }
      }
    }
    __syncthreads();  // every read of key_s and dig_s of this step is done
    if (tid == 0 && i + 1u < n) {
      fence_proxy_async();
      mbar_expect_tx(bar, key_bytes);
      bulk_g2s(key_s, bsk + (uint64_t)(i + 1u) * (key_bytes / 4u), key_bytes, bar);
    }
    // 4. ACC += ExtProd
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t *pa = acc_s + ((2 * g + 0) * 2 + j) * N + c0;
      uint32_t *pb = acc_s + ((2 * g + 1) * 2 + j) * N + c0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { pa[q] += accA[j][q]; pb[q] += accB[j][q]; }
    }
    __syncthreads();
  }
  if (s_abort) {
    if (tid == 0) {
      atomicExch(status, FHE_ETIMEOUT);
      // give the copy in flight a bounded chance to land before exiting
      (void)mbar_wait_bounded(bar, 0u);
      (void)mbar_wait_bounded(bar, 1u);
    }
    return;
  }

  // Sample extraction (with the multi-value split r_j * ACC when L == 2):
  // a'_0 = A[0], a'_c = -A[N - c], b' = B[0].
  const uint32_t W = N + 1u;
  for (uint32_t j = 0; j < lut.L; ++j) {
    for (uint32_t e = tid; e < CPC * W; e += THREADS) {
      const uint32_t b = e / W, c = e % W;
      if (base + b >= count) continue;
      const fhe::LutGroup grp = fhe::lut_group(lut, base + b);
      const uint32_t nnz = j ? grp.nnz1 : grp.nnz0, off = j ? grp.off1 : grp.off0;
      const uint32_t *A = acc_s + (b * 2u) * N;
      const uint32_t *B = acc_s + (b * 2u + 1u) * N;
      uint32_t v;
      if (lut.L == 1u) {
        v = (c == N) ? B[0] : (c == 0 ? A[0] : (0u - A[N - c]));
      } else {
        // (r * P)[m] = sum_(e,val) val * (X^e P)[m]
        const uint32_t m = (c == N) ? 0u : ((c == 0) ? 0u : N - c);
        const uint32_t *Pp = (c == N) ? B : A;
        uint32_t s = 0;
        for (uint32_t t = 0; t < nnz; ++t) {
          const uint32_t ep = (uint32_t)lut.rpos[off + t];
          const uint32_t val = (uint32_t)lut.rval[off + t];
          s += val * ((m >= ep) ? Pp[m - ep] : (0u - Pp[m + N - ep]));
        }
        v = (c == N || c == 0) ? s : (0u - s);
      }
      big_out[((size_t)j * count + base + b) * W + c] = v;
    }
  }
}

// Key switching (paper 2.1): out = (0, b') - sum_i sum_lam d_{i,lam} ksk[i][lam]
// with signed digits of base 2^log2_bks.  CTA = TILE ciphertexts x all n+1
// output words; thread owns words tid + 256 q.  Digits of a chunk of CH
// inputs are staged in shared memory as int32 [CH][l_ks][TILE].
template <int TILE, int COLS>
__global__ void __launch_bounds__(256)
    k_key_switch(Params P, const uint32_t *__restrict__ ksk, const uint32_t *__restrict__ big,
                 size_t count, uint32_t *__restrict__ out) {
  constexpr int CH = 32;
  __shared__ __align__(16) int32_t dig[CH * 8 * TILE];
  const uint32_t n = P.n, kN = P.k * P.N, lks = P.l_ks, W = kN + 1u;
  const size_t t0 = (size_t)blockIdx.x * TILE;
  const int tid = threadIdx.x;
  uint32_t acc[TILE][COLS];
#pragma unroll
  for (int t = 0; t < TILE; ++t)
#pragma unroll
    for (int q = 0; q < COLS; ++q) acc[t][q] = 0u;
  const uint32_t tb = P.log2_bks * lks;
  const uint32_t Bm = (1u << P.log2_bks) - 1u, Bh = 1u << (P.log2_bks - 1u);
  for (uint32_t i0 = 0; i0 < kN; i0 += CH) {
    __syncthreads();
    for (uint32_t e = tid; e < (uint32_t)(CH * TILE); e += 256u) {
      const uint32_t ii = e / TILE, t = e % TILE;
      uint32_t x = (t0 + t < count && i0 + ii < kN) ? big[(t0 + t) * W + i0 + ii] : 0u;
      uint32_t xr = (tb >= 32u) ? x : ((uint32_t)(x + (1u << (31u - tb))) >> (32u - tb));
      for (int lam = (int)lks - 1; lam >= 0; --lam) {
        uint32_t d = xr & Bm;
        xr >>= P.log2_bks;
        int32_t sd = (int32_t)d;
        if (d >= Bh) { sd -= (int32_t)(Bm + 1u); xr += 1u; }
        dig[(ii * 8u + (uint32_t)lam) * TILE + t] = sd;
      }
    }
    __syncthreads();
    const uint32_t iend = (kN - i0 < (uint32_t)CH) ? kN - i0 : (uint32_t)CH;
    for (uint32_t ii = 0; ii < iend; ++ii) {
      for (uint32_t lam = 0; lam < lks; ++lam) {
        const uint32_t *row = ksk + ((uint64_t)(i0 + ii) * lks + lam) * (n + 1u);
        uint32_t kv[COLS];
#pragma unroll
        for (int q = 0; q < COLS; ++q) {
          const uint32_t c = tid + 256u * q;
          kv[q] = (c <= n) ? __ldg(row + c) : 0u;
        }
        const int32_t *dl = dig + (ii * 8u + lam) * TILE;
#pragma unroll
        for (int t4 = 0; t4 < TILE; t4 += 4) {
          const int4 d4 = *reinterpret_cast<const int4 *>(dl + t4);
          const int32_t dd[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < COLS; ++q) acc[t4 + u][q] -= (uint32_t)dd[u] * kv[q];
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TILE; ++t) {
    if (t0 + t >= count) break;
#pragma unroll
    for (int q = 0; q < COLS; ++q) {
      const uint32_t c = tid + 256u * q;
      if (c > n) continue;
      uint32_t v = acc[t][q];
      if (c == n) v += big[(t0 + t) * W + kN];
      out[(t0 + t) * (n + 1u) + c] = v;
    }
  }
}

template <int N, int CPC>
int launch_br(const fhe_keys *K, const uint32_t *ct_in, size_t count, const LutArgs &la,
              uint32_t *big, cudaStream_t st) {
  const Params &P = K->P;
  const BrSmem S = br_smem(N, CPC, 2u * P.l, P.n);
  int maxopt = 0;
  FHE_CUDA_TRY(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, K->device));
  if ((int)S.total > maxopt) return FHE_EUNSUPPORTED;
  auto kern = k_blind_rotate_exact<N, CPC>;
  FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total));
  const unsigned blocks = (unsigned)((count + CPC - 1) / CPC);
  kern<<<blocks, (N / 8) * (CPC / 2), S.total, st>>>(P, K->d_bsk, ct_in, count, la, big,
                                                     K->d_status);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

}  // namespace

namespace fhe {

int key_switch_batch(const fhe_keys *K, const uint32_t *d_big, size_t count, uint32_t *ct_out,
                     cudaStream_t st) {
  const Params &P = K->P;
  if (!count) return FHE_OK;
  if (P.n + 1u <= 768u) {
    // 32 ciphertexts per CTA amortise the key's reads; a batch that would
    // leave SMs idle with them (fewer CTAs than SMs) takes 8 per CTA
    // instead: four times the CTAs, a quarter of the time per CTA
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, K->device) != cudaSuccess) {
      (void)cudaGetLastError();
      sms = 152;
    }
    if ((count + 31) / 32 < (size_t)sms)
      k_key_switch<8, 3><<<(unsigned)((count + 7) / 8), 256, 0, st>>>(P, K->d_ksk, d_big, count, ct_out);
    else
      k_key_switch<32, 3><<<(unsigned)((count + 31) / 32), 256, 0, st>>>(P, K->d_ksk, d_big, count, ct_out);
  } else {
    k_key_switch<8, 9><<<(unsigned)((count + 7) / 8), 256, 0, st>>>(P, K->d_ksk, d_big, count, ct_out);
  }
  note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return FHE_OK;
}

int pbs_exact(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
              uint32_t *ct_out, size_t table_stride, cudaStream_t st, const uint64_t *seg_end) {
  const Params &P = K->P;
  for (size_t s0 = 0; s0 < count; s0 += K->ws_cap) {
    const size_t cnt = (count - s0 < K->ws_cap) ? count - s0 : K->ws_cap;
    const LutArgs la = lut_args(lut, seg_end, s0);
    const uint32_t *in = ct_in + s0 * (P.n + 1u);
    int rc;
    const bool prof = (s0 == 0) && K->prof_ev0;
    if (prof) { FHE_CUDA_TRY(record_prof_event(K->prof_ev0, st)); K->prof_count = cnt; }
    switch (P.N) {
      case 256: rc = launch_br<256, 8>(K, in, cnt, la, K->d_big, st); break;
      case 512: rc = launch_br<512, 8>(K, in, cnt, la, K->d_big, st); break;
      case 1024: rc = launch_br<1024, 4>(K, in, cnt, la, K->d_big, st); break;
      case 2048: rc = launch_br<2048, 2>(K, in, cnt, la, K->d_big, st); break;
      default: return FHE_EUNSUPPORTED;
    }
    if (rc) return rc;
    if (prof) FHE_CUDA_TRY(record_prof_event(K->prof_ev1, st));
    for (uint32_t j = 0; j < lut->L; ++j) {
      rc = key_switch_batch(K, K->d_big + (size_t)j * cnt * P.big_words(), cnt,
                            ct_out + (size_t)j * table_stride + s0 * (P.n + 1u), st);
      if (rc) return rc;
    }
  }
  return FHE_OK;
}

// Exact bootstrapping of one batch whose extracted LWE_z ciphertexts go to the
// caller-provided device buffer `big` ([L][count][kN+1] words); no
// workspace of the key handle is touched and nothing is allocated.
int pbs_exact_into(const fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
                   uint32_t *ct_out, uint32_t *big, cudaStream_t st) {
  const Params &P = K->P;
  const LutArgs la = lut_args(lut, nullptr, 0);
  int rc;
  switch (P.N) {
    case 256: rc = launch_br<256, 8>(K, ct_in, count, la, big, st); break;
    case 512: rc = launch_br<512, 8>(K, ct_in, count, la, big, st); break;
    case 1024: rc = launch_br<1024, 4>(K, ct_in, count, la, big, st); break;
    case 2048: rc = launch_br<2048, 2>(K, ct_in, count, la, big, st); break;
    default: return FHE_EUNSUPPORTED;
  }
  if (rc) return rc;
  for (uint32_t j = 0; j < lut->L; ++j) {
    rc = key_switch_batch(K, big + (size_t)j * count * P.big_words(), count,
                          ct_out + (size_t)j * count * (P.n + 1u), st);
    if (rc) return rc;
  }
  return FHE_OK;
}

int pbs_run(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
            uint32_t *ct_out, size_t table_stride, int variant, cudaStream_t st,
            const uint64_t *seg_end) {
  if (!count) return FHE_OK;
  if (variant == FHE_VARIANT_AUTO)  // both exact paths give the same bits
    variant = (count >= K->tc_min_batch) ? FHE_VARIANT_TC : FHE_VARIANT_EXACT;
  if (variant == FHE_VARIANT_EXACT)
    return pbs_exact(K, ct_in, count, lut, ct_out, table_stride, st, seg_end);
  if (variant == FHE_VARIANT_TC) return pbs_tc(K, ct_in, count, lut, ct_out, table_stride, st, seg_end);
  if (variant == FHE_VARIANT_FFT)
    return pbs_fft(K, ct_in, count, lut, ct_out, table_stride, st, seg_end);
  return FHE_EINVAL;
}

}  // namespace fhe

extern "C" int fhe_selftest_timeout(fhe_keys *K, uint32_t limit_us, void *stream) {
  if (!K || limit_us == 0 || limit_us > 1000000u) return FHE_EINVAL;
  k_selftest_timeout<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_us * 1000ull,
                                                         K->d_status);
  fhe::note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  return fhe_status(K, stream);
}

extern "C" int fhe_pbs_batch(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
                             uint32_t *ct_out, int variant, void *stream) {
  if (!K || !lut || (count && (!ct_in || !ct_out)) || lut->N != K->P.N || lut->groups != 1u)
    return FHE_EINVAL;
  if (!count) return FHE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return fhe::pbs_run(K, ct_in, count, lut, ct_out, count * (K->P.n + 1u), variant, st);
}

extern "C" int fhe_pbs_batch_groups(fhe_keys *K, const uint32_t *ct_in, size_t count,
                                    const fhe_lut *lut, const size_t *seg_end, uint32_t *ct_out,
                                    int variant, void *stream) {
  if (!K || !lut || (count && (!ct_in || !ct_out)) || lut->N != K->P.N ||
      (lut->groups > 1u && !seg_end))
    return FHE_EINVAL;
  uint64_t ends[fhe::kLutGroups - 1];
  for (uint32_t q = 0; q + 1u < lut->groups; ++q) {
    if (seg_end[q] > count || (q && seg_end[q] < seg_end[q - 1])) return FHE_EINVAL;
    ends[q] = seg_end[q];
  }
  if (!count) return FHE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return fhe::pbs_run(K, ct_in, count, lut, ct_out, count * (K->P.n + 1u), variant, st,
                      lut->groups > 1u ? ends : nullptr);
}
