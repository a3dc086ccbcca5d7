// fhe_pbs_tc.cu -- blind rotation with the external product on tcgen05 tensor
// cores, bit-exact to the uint32 definition (paper 2.1, Blind Rotation;
// Thm 2.1).
//
// The external product of one CMux step is, per output polynomial j,
//   out_j[c] = sum_r sum_t D_r[t] * ext_{r,j}(c - t),   ext(x) = K[x] (x >= 0),
//                                                        -K[x+N] (x < 0),
// a negacyclic (block-Toeplitz) contraction of small signed gadget digits D
// against 32-bit key words K.  Reversing the digit index (t' = N-1-t) turns
// the key matrix into a Hankel matrix H[c][t'] = h[c + t'].
//
// Exactness.  Key words are split into four balanced 8-bit limbs
// (K = sum_L 2^(8L) K_L mod 2^32, K_L in [-128, 128)); digits lie in
// [-Bg/2, Bg/2).  Both are exact fp16 integers, so a tcgen05 kind::f16 MMA
// with fp32 accumulation is exact as long as every partial sum stays within
// 2^24: the accumulator is drained (cvt to int32, shifted by 8L, added modulo
// 2^32) after at most 2^24 / (Bg/2 * 128) terms.
//
// Operands (SWIZZLE_NONE, K-major, 8x8 fp16 core matrices of 128 bytes), for
// a CTA pair running tcgen05.mma.cta_group::2 with M = 256, N = 256, K = 16:
//  - A = digits of 256 ciphertexts; each CTA holds its 128 rows in tiles of
//    128 x 128 (LBO 128, SBO 2048).  Digits are written once per step to
//    global memory; each CTA copies the tiles of its 128 rows into shared
//    memory, either by cluster-multicast bulk copies (single-GPU library:
//    every CTA sends the rows it generated to all CTAs holding the same rows)
//    or by whole-tile copies per CTA (replica library, or by option).
//  - B = Hankel key, N = 256 output coefficients split 128 + 128 between the
//    two CTAs of the pair.  Core matrix delta holds h[8 delta + rho + kappa];
//    with LBO = SBO = 128 bytes the matrix descriptor walks one strip of core
//    matrices for both the N and K directions, so one 10 KB window per
//    (key row r, limb, 512 K) feeds 32 K16 steps of a 256-coefficient block.
//    Global memory keeps only the 2N distinct entries h[s] per key
//    polynomial and limb (4x the key); a producer warp stages the 640 a
//    window needs and writes the window's core matrices in shared memory.
//  - D = TMEM fp32, 128 lanes (the CTA's ciphertexts) x 256 columns per
//    limb; a unit accumulates two limbs, using all 512 columns (allocated
//    jointly by the pair), so each A tile feeds two MMAs per K16 step.
// Per SM, an M256 N256 K16 step of the pair reads 4 KB of A and 4 KB of B
// from shared memory (64 B/clk at the tensor rate) instead of 4 + 8 KB for a
// single-CTA M128 N256 step.
//
// A cluster of CL = 4, 8 or 16 CTAs (CL/2 pairs) takes one 256-ciphertext
// tile; half the pairs compute output polynomial 0, half polynomial 1, each
// pair a share of the N/256 coefficient blocks (4 CTAs: all blocks, 16 CTAs:
// one block at N = 1024, the lowest latency).  Per step: digits (all warps;
// each CTA makes the digits of 256/CL ciphertexts) -> cluster barrier ->
// units (block, chunk, limb pair) run by a digit-tile producer warp, a
// key-window warp, the leader's MMA warp (the peer's warp 1 relays "A tile
// landed" to the leader) and eight epilogue warps per CTA (TMEM ->
// registers, limb recombination, ACC update in global memory) -> cluster
// barrier.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "fhe_internal.cuh"

using fhe::LutArgs;
using fhe::Params;

namespace {

constexpr int kBt = 256;          // ciphertexts per cluster (MMA M of a CTA pair)
constexpr int kBh = 128;          // ciphertexts per CTA (its half of M)
constexpr int kBN = 256;          // output coefficients per block (MMA N)
constexpr int kKB = 128;          // K elements per A tile
constexpr int kATile = kBh * kKB * 2;   // 32 KB: one CTA's 128 rows x 128 K
// Byte distance between 8-row groups of an A tile (kKB / 8 core matrices).
constexpr uint32_t kASBO = kKB / 8u * 128u;
constexpr uint32_t kAStages = 5;  // A-operand pipeline depth (5 x 32 KB; large tiles keep the
                                  // bulk copies efficient)
// Accumulator staging of the digit phase: six buffers of 32 KB over the (then
// idle) A and B stages.
constexpr uint32_t kGBuf = 6;
// One B window: the 128 columns of a CTA over K = 1024 of a Hankel strip,
// (128 + 1024) / 8 core matrices of 128 bytes.
constexpr uint32_t kBK = 512;
constexpr uint32_t kBWin = (128u + kBK) / 8u * 128u;
constexpr int kThreads = 352;     // warp 0 A producer, warp 1 MMA, warps 2-9 epilogue,
                                  // warp 10 B producer
constexpr uint32_t kBWarp = 10;
constexpr int kTmemCols = 512;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
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
// Acquire at cluster scope: the phase was completed by another CTA's release
// arrive after that CTA's threads wrote shared memory with generic stores.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (two seconds).  Sets *abort and returns false when it gives up;
// returns false immediately once aborted.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (*abort) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (global_ns() - t0 > 2000000000ull) { *abort = 1; return false; }
  }
  return true;
}
__device__ __forceinline__ bool wait_bounded_cluster(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (*abort) return false;
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort) return false;
    if (global_ns() - t0 > 2000000000ull) { *abort = 1; return false; }
  }
  return true;
}
// Bounded wait that does not give up on the abort flag (used to drain the
// tensor pipe before TMEM is released).
__device__ __forceinline__ void wait_time_bounded(uint64_t *bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 2000000000ull) return;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 eviction priority of the digit operand (tc option FHE_TC_OPT_L2_HINTS):
// a cache policy that makes the lines it touches the last to be evicted.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// 8-byte global store, with the policy when `hint`.
__device__ __forceinline__ void st_u2(void *p, uint2 v, bool hint, uint64_t pol) {
  if (hint)
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "l"(pol)
                 : "memory");
  else
    *reinterpret_cast<uint2 *>(p) = v;
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[256 x N] (+)= A[256 x 16] B[16 x N] over the CTA pair: rows 0..127 of A
// and D live in the leader CTA, rows 128..255 in its peer; each CTA holds
// N/2 columns of B; the descriptors give the same offsets in both CTAs.
__device__ __forceinline__ void tc2_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Address of this CTA's shared variable `p` in the CTA of cluster rank `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Completion of every tcgen05.mma this thread issued arrives on the barrier at
// the same offset in each CTA of `mask`: one commit per CTA (the single-GPU
// build uses one multicast commit instead, fhe_tc_multicast.cuh).
__device__ __forceinline__ void tc2_commit_each(uint64_t *bar, uint16_t mask) {
  for (uint32_t r = 0; r < 16u; ++r)
    if (mask & (1u << r))
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              cluster_addr(bar, r))
          : "memory");
}
// One digit tile (kATile bytes, 128 rows x 128 K) into an A stage.  Per-CTA
// form: this CTA copies the whole tile into its own shared memory.  The
// cluster-multicast form (MC = true, defined in fhe_tc_multicast.cuh and
// compiled only into single-GPU builds) copies the share this CTA generated
// into the same stage of every CTA that holds the same rows.
template <bool MC>
struct ATileLoad {
  static __device__ __forceinline__ void run(unsigned char *stage, const __half *tile, uint32_t pr,
                                             uint32_t np, uint64_t *bar, uint16_t mask, bool hint,
                                             uint64_t pol) {
    (void)pr; (void)np; (void)mask;
    if (hint) bulk_g2s_hint(stage, tile, (uint32_t)kATile, bar, pol);
    else bulk_g2s(stage, tile, (uint32_t)kATile, bar);
  }
};
#ifndef FHE_NO_MULTICAST
#include "fhe_tc_multicast.cuh"
constexpr bool kTcMulticast = true;
#else
constexpr bool kTcMulticast = false;
__device__ __forceinline__ void tc2_commit_ctas(uint64_t *bar, uint16_t mask) {
  tc2_commit_each(bar, mask);
}
#endif
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Barrier over the GC clusters that share one tile: the cluster barrier, then
// one thread per cluster publishes its cluster's writes at GPU scope on the
// tile's counter and waits (bounded, two seconds) until every cluster of the
// tile has arrived k times, then the cluster barrier again.  An aborted
// cluster keeps arriving, so its partners never wait for it.  The launch is
// cooperative, so all clusters of a tile are resident together.
template <int GC>
__device__ __forceinline__ void tile_sync(uint32_t *ctr, uint32_t &k, volatile int *abort) {
  cluster_sync_all();
  if constexpr (GC > 1) {
    ++k;
    if (threadIdx.x == 0 && cluster_rank() == 0) {
      __threadfence();
      atomicAdd(ctr, 1u);
      const uint32_t target = (uint32_t)GC * k;
      if (!*abort && ld_acquire_gpu(ctr) < target) {
        const uint64_t t0 = global_ns();
        while (ld_acquire_gpu(ctr) < target)
          if (global_ns() - t0 > 2000000000ull) { *abort = 1; break; }
      }
    }
    cluster_sync_all();
  }
}
// Arrive on this CTA's barrier, releasing this thread's prior writes (and
// those ordered before them) at CTA scope.
__device__ __forceinline__ void mbar_arrive_local(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Arrive on a barrier of another CTA of the cluster, releasing at cluster
// scope (the barrier announces generic shared-memory writes of this CTA).
__device__ __forceinline__ void mbar_arrive_remote_release(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
}
// Arrive on a barrier of another CTA of the cluster (default semantics; the
// operands it announces were written by the async proxy and are read by the
// tensor core, which the barrier phase alone orders).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
// 16 consecutive 32-bit TMEM columns of the warp's 32 lanes, completed by the
// next tc_wait16 on the same registers.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Waits for this thread's outstanding TMEM loads; the registers are operands
// so that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tc_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
// outv[k] += int(r[k]) << shift for the 16 drained fp32 sums (exact integers).
__device__ __forceinline__ void tc_acc16(uint32_t *outv, const uint32_t (&r)[16], uint32_t shift) {
#pragma unroll
  for (int k = 0; k < 16; ++k) outv[k] += (uint32_t)__float2int_rn(__uint_as_float(r[k])) << shift;
}

// Shared-memory matrix descriptor: SWIZZLE_NONE, K-major, version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor: kind::f16, A = B = fp16, D = fp32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Balanced 8-bit limb L of a 32-bit word: w = sum_L 2^(8L) limb_L mod 2^32.
__device__ __forceinline__ int32_t limb8(uint32_t w, uint32_t L) {
  int32_t v = 0;
  for (uint32_t i = 0; i <= L; ++i) {
    v = (int32_t)((w & 0xFFu) ^ 0x80u) - 0x80;
    w = (w - (uint32_t)v) >> 8;
  }
  return v;
}

// ---------------------------------------------------------------- key layout
// hk[((i * R + r) * 2 + j) * 4 + L][s] = limb_L(h[s]) as fp16 for s < 2N,
// h[s] = ext_{r,j}(s - (N - 1)) (h[2N - 1] = 0): the 2N - 1 distinct entries
// of the Hankel key matrix of one key polynomial and limb, 4x the size of
// the key itself.  The kernel builds the 8x8 core matrices of each B window
// from these in shared memory.
__global__ void k_hankel_compact(Params P, const uint32_t *__restrict__ bsk, __half *hk) {
  const uint32_t N = P.N, R = P.rows();
  const uint64_t total = (uint64_t)P.n * R * 2u * 4u * 2u * N;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t sidx = (uint32_t)(e % (2u * N));
    const uint64_t strip = e / (2u * N);  // ((i R + r) 2 + j) 4 + L
    const uint32_t L = (uint32_t)(strip % 4u);
    const uint64_t irj = strip / 4u;      // (i R + r) 2 + j
    const uint32_t *K = bsk + irj * N;
    int32_t v = 0;
    if (sidx <= 2u * N - 2u) {
      const int32_t x = (int32_t)sidx - (int32_t)(N - 1u);
      const uint32_t w = (x >= 0) ? K[x] : (0u - K[x + (int32_t)N]);
      v = limb8(w, L);
    }
    hk[e] = __int2half_rn(v);
  }
}

// Entries of the compact key one B window reads: core matrices 0..78 of a
// window span h[s0 .. s0 + 638] (128 columns + K 512 - 1 + 7 + 7); 640 are
// staged (a 16-byte multiple).
constexpr uint32_t kHWin = 640u;
constexpr uint32_t kHStage = kHWin * 2u;  // bytes
constexpr uint32_t kBCm = 79u;             // core matrices of a window the MMAs read

struct TcSmem {
  uint32_t a, b, h, bars, tmem_slot, total;
};
// A stages, then two B stages of two 128-column windows (one per limb of the
// unit; each window covers K = 512), then the compact key entries staged for
// each B stage.  During the digit phase the A and B regions stage
// accumulators instead (kGBuf buffers of 32 KB).
__host__ __device__ inline TcSmem tc_smem() {
  TcSmem s;
  uint32_t o = 0;
  s.a = o; o += kAStages * kATile;
  s.b = o; o += 2u * 2u * kBWin;
  s.h = o; o += 2u * 2u * kHStage;
  s.bars = o; o += 48u * 8u;   // 3 x kAStages + 6 + 3 + 6 + 2 + 2 mbarriers
  s.tmem_slot = o; o += 16u;
  s.total = o;
  return s;
}

// Global scratch of one cluster tile (256 ciphertexts): ACC [256][2][N] u32,
// then digits [2 halves][RR rows][N/64 tiles][128 x 64] fp16.
__host__ __device__ inline uint64_t tc_tile_acc_words(uint32_t N) { return (uint64_t)kBt * 2u * N; }
__host__ __device__ inline uint64_t tc_tile_dig_halves(uint32_t N, uint32_t RR) {
  return 2ull * RR * (N / kKB) * (kATile / 2);
}

// CL = CTAs per cluster: 4 (two pairs, one per output polynomial), 8 (four
// pairs, each with half the blocks of one polynomial: half the work per CTA
// and step) or 16 (eight pairs, a quarter; a non-portable cluster size, for
// batches that fit in the clusters of 16 the GPU holds at once).  MC: digit
// tiles by cluster-multicast copies (compiled only into single-GPU builds).
template <int N, int CL, int GC, bool MC>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kThreads, 1)
    k_blind_rotate_tc(Params P, const __half *__restrict__ hk,
                      const uint32_t *__restrict__ ct_in, size_t count,
                      const __grid_constant__ LutArgs lut,
                      uint32_t *__restrict__ acc_g, __half *__restrict__ dig_g,
                      uint32_t chunk_r, uint32_t sub_shift, uint32_t *__restrict__ big_out,
                      int *status, uint32_t opts, uint32_t *__restrict__ tsync) {
  constexpr uint32_t LOG2_2N = (N == 1024) ? 11 : 12;
  constexpr uint32_t KBLK = N / kKB;             // A tiles per digit row r
  constexpr uint32_t KH = N / kBK;               // B windows per digit row
  constexpr uint32_t KT = kBK / kKB;             // A tiles per B window
  constexpr uint32_t TILE_H = kATile / 2;        // fp16 elements of one A tile
  constexpr uint32_t NP = CL / 2;                 // CTA pairs per cluster
  constexpr uint32_t TP = GC * NP;                // CTA pairs per tile (GC clusters)
  constexpr uint32_t PPJ = TP / 2;                // pairs per output polynomial
  constexpr uint32_t RPC = kBh / TP;              // digit rows each CTA of a half makes
  constexpr uint32_t UPJ = 2u * (N / kBN);        // (block, limb pair) units per polynomial
  constexpr uint32_t UPP = UPJ / PPJ;             // units per pair
  constexpr uint32_t NLP = (UPP >= 2u) ? 2u : 1u;  // limb pairs per block of a pair
  constexpr uint32_t NBLK = UPP / NLP;            // blocks of 256 coefficients per pair
  // one limb pair per pair: the two pairs of a block add into its accumulators
  constexpr bool RED = (NLP == 1u);
  static_assert(UPP >= 1u && UPJ % PPJ == 0u, "tile shape");
  static_assert(GC == 1 || !MC, "multicast copies stay within one cluster");
  constexpr uint32_t G = 4096u / N;              // ciphertexts per staged group (32 KB)
  constexpr uint32_t NGROUP = RPC / G;
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcSmem S = tc_smem();
  unsigned char *sA = smem + S.a;
  unsigned char *sB = smem + S.b;
  unsigned char *sH = smem + S.h;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S.bars);
  uint64_t *a_full = bars, *a_empty = bars + kAStages, *a_peer = bars + 2 * kAStages;
  uint64_t *b_full = bars + 3 * kAStages, *b_empty = b_full + 2, *b_peer = b_full + 4;
  uint64_t *t_full = b_full + 6, *t_empty = b_full + 7, *done = b_full + 8;
  uint64_t *g_full = b_full + 9;  // staging buffers of the digit phase
  uint64_t *h_full = g_full + kGBuf;  // compact key entries of each B stage
  // t_empty: the epilogue has drained limb 0's accumulator (TMEM columns
  // 0..255) of the unit; t_empty1: limb 1's (256..511)
  uint64_t *t_empty1 = h_full + 2;
  // t_full0: the unit's limb-0 MMAs are complete (its limb-1 MMAs may still run)
  uint64_t *t_full0 = h_full + 3;
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + S.tmem_slot);
  __shared__ int s_abort;
  __shared__ uint32_t s_abar[RPC];  // a~_i of the ciphertexts whose digits this CTA makes
  __shared__ uint32_t s_gdone[kGBuf];  // warps done with each digit-phase staging buffer

  const uint32_t n = P.n, l = P.l, R = 2u * l;
  const uint32_t tid = threadIdx.x, warp = tid / 32u, lane = tid % 32u;
  const uint32_t q = cluster_rank();
  const uint32_t pr = q / 2u;               // pair index within the cluster
  const uint32_t gci = (uint32_t)((blockIdx.x / CL) % GC);  // cluster within the tile
  const uint32_t gp = gci * NP + pr;        // pair index within the tile
  const uint32_t pj = gp / PPJ;             // output polynomial of the pair
  const uint32_t bsub = gp % PPJ;           // which share of the units
  const uint32_t hh = q % 2u;               // ciphertext half (MMA rows 128 hh ..)
  const uint32_t lead = q & ~1u;            // rank of the pair's leader (issues the MMAs)
  const bool leader = (hh == 0u);
  const uint64_t tile = blockIdx.x / (CL * GC);
  const size_t base = (size_t)tile * kBt;
  // With sub_shift > 0 every gadget digit d is split into two signed
  // sub-digits d = hi * 2^sub_shift + lo (rows r and R + r of the digit
  // operand) so that each fp32 partial sum stays within 2^24; chunks never mix
  // low and high rows, and high rows are scaled by 2^sub_shift when drained.
  const uint32_t RR = sub_shift ? 2u * R : R;
  uint32_t *acc = acc_g + tile * tc_tile_acc_words(N);           // [256][2][N]
  __half *dig = dig_g + tile * tc_tile_dig_halves(N, RR);
  __half *dig_h = dig + (uint64_t)hh * RR * KBLK * TILE_H;        // this half's digit rows
  const uint32_t row0 = kBh * hh + RPC * gp;  // first ciphertext whose digits this CTA makes
  // this pair's units: blocks blk0 .. + NBLK, limb pairs lp0 .. + NLP of each
  const uint32_t nblk = NBLK;
  const uint32_t blk0 = bsub * UPP / 2u;
  const uint32_t lp0 = (NLP == 1u) ? (bsub * UPP) % 2u : 0u;
  uint32_t *tile_ctr = (GC > 1) ? tsync + tile : nullptr;
  uint32_t tile_k = 0;  // tile barriers passed
  const uint32_t nchunk = RR / chunk_r;
  const uint64_t strip_halves = 2ull * N;  // compact key entries per strip
  const uint16_t pair_mask = (uint16_t)(3u << lead);
  // every CTA of the same half receives the digit rows this CTA makes
  uint16_t a_mask = 0;
  for (uint32_t k = 0; k < NP; ++k) a_mask |= (uint16_t)(1u << (2u * k + hh));
  const uint16_t all_mask = (uint16_t)((1u << CL) - 1u);
  // A stage release: with multicast copies a stage of every CTA holding the
  // same rows is refilled by all of them, so every pair's MMAs must be done
  // with it; with per-CTA copies only this pair's (the pairs run decoupled)
  const uint16_t ae_mask = MC ? all_mask : pair_mask;
  // opts bit 0: the digit operand is written and copied with an L2
  // evict-last policy (it is read 2 nblk times per step; the accumulators,
  // read once and written once per step, are the lines that leave L2)
  const bool l2keep = (opts & 1u) != 0u;
  const uint64_t pol_keep = l2keep ? l2_policy_keep() : 0ull;

  if (tid == 0) {
    s_abort = 0;
    for (uint32_t b = 0; b < kGBuf; ++b) s_gdone[b] = 0u;
    for (uint32_t s = 0; s < kAStages; ++s) {
      mbar_init(&a_full[s], 1); mbar_init(&a_empty[s], MC ? NP : 1u); mbar_init(&a_peer[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); mbar_init(&b_peer[s], 1);
    }
    for (uint32_t s = 0; s < kGBuf; ++s) mbar_init(&g_full[s], 1);
    for (int s = 0; s < 2; ++s) mbar_init(&h_full[s], 1);
    mbar_init(t_full, 1); mbar_init(t_empty, 16); mbar_init(t_empty1, 16); mbar_init(done, 1);
    mbar_init(t_full0, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // collective over the CTA pair: the same 512 columns in both CTAs
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void *)tmem_slot)),
                 "r"((uint32_t)kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  // initial accumulators of this CTA's RPC ciphertexts: (0, X^{-b~} TV);
  // multi-value: the TV0 coefficient of the ciphertext's table group
  for (uint32_t e = tid; e < RPC * N; e += kThreads) {
    const uint32_t b = row0 + e / N, c = e % N;
    const uint32_t v_ct = (base + b < count) ? ct_in[(base + b) * (n + 1u) + n] : 0u;
    const uint32_t bb = fhe::mod_switch_2n(v_ct, LOG2_2N);
    const uint32_t s = (c + bb) & (2u * N - 1u);
    uint32_t v;
    if (lut.L == 1u) {
      v = (s < N) ? lut.tv[s] : (0u - lut.tv[s - N]);
    } else {
      const uint32_t tv0 = fhe::lut_group(lut, base + b).tv0;
      v = (s < N) ? tv0 : (0u - tv0);
    }
    acc[((uint64_t)b * 2u + 0u) * N + c] = 0u;
    acc[((uint64_t)b * 2u + 1u) * N + c] = v;
  }
  // generic stores of ACC are read by bulk copies (async proxy) in the digit phase
  asm volatile("fence.proxy.async.global;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  tile_sync<GC>(tile_ctr, tile_k, &s_abort);

  const uint32_t total_bits = l * P.log2_bg;
  const uint32_t Bmask = (1u << P.log2_bg) - 1u, Bhalf = 1u << (P.log2_bg - 1u);
  constexpr uint32_t idesc = idesc_f16(2u * kBh, kBN);
  // pipeline positions (each role advances the ones it uses)
  uint32_t a_it = 0, b_it = 0, u_it = 0, g_it = 0;

  for (uint32_t i = 0; i < n; ++i) {
    // ---- digits of X^{a~_i} ACC - ACC for this CTA's RPC ciphertexts.
    // Groups of G ciphertexts (both polynomials, 32 KB) are staged in shared
    // memory by bulk copies, kGBuf groups in flight.  One warp per chunk of 256
    // coefficients of one polynomial; lane L owns c = c_base + 32k + L, so
    // shared-memory reads are conflict free and global stores coalesced.
    if (tid < RPC) {
      const uint32_t b = row0 + tid;
      const uint32_t av = (base + b < count) ? __ldg(ct_in + (base + b) * (n + 1u) + i) : 0u;
      s_abar[tid] = fhe::mod_switch_2n(av, LOG2_2N);
    }
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // accumulator rows other CTAs (other clusters too) updated
      asm volatile("fence.proxy.async.global;" ::: "memory");
      for (uint32_t g = 0; g < kGBuf && g < NGROUP; ++g) {
        const uint32_t bf = (g_it + g) % kGBuf;
        mbar_expect_tx(&g_full[bf], 32768u);
        bulk_g2s(smem + bf * 32768u, acc + (uint64_t)(row0 + g * G) * 2u * N, 32768u, &g_full[bf]);
      }
    }
    __syncthreads();
    for (uint32_t g = 0; g < NGROUP; ++g, ++g_it) {
      const uint32_t buf = g_it % kGBuf;
      const bool got = wait_bounded(&g_full[buf], (g_it / kGBuf) & 1u, &s_abort);
      const uint32_t *sacc = reinterpret_cast<const uint32_t *>(smem + buf * 32768u);
      // Items (ciphertext gi, polynomial j, block of 256 coefficients); lane L
      // owns two runs of 4 consecutive coefficients, c0 = 256 cb + 128 h + 4L
      // (h = 0, 1), computed side by side.  The reversed indices t' = N-1-c
      // of a run form one aligned 8-byte piece of a core-matrix row, so each
      // gadget level is a single 8-byte store per run.
      constexpr uint32_t NB = N / 256u;
      constexpr uint32_t ITEMS = G * 2u * NB;  // = 32
      for (uint32_t item = warp; got && item < ITEMS; item += kThreads / 32u) {
        const uint32_t cb = item % NB, j = (item / NB) & 1u, gi = item / (2u * NB);
        const uint32_t bl = g * G + gi;             // 0..RPC-1
        const uint32_t bm = RPC * gp + bl;          // MMA row within this half
        const uint32_t a = s_abar[bl];
        const uint32_t *Pj = sacc + (gi * 2u + j) * N;
        uint32_t xr[2][4];
        __half *dst0[2];
#pragma unroll
        for (uint32_t h = 0; h < 2u; ++h) {
          const uint32_t c0 = cb * 256u + 128u * h + 4u * lane;
          const uint4 me = *reinterpret_cast<const uint4 *>(Pj + c0);
          // X^{a} P at c0..c0+3 reads P at s = c - a (mod 2N), negated where
          // s >= N.  Aligned runs of 4 never straddle N, so the two aligned
          // runs around s0 give all four values with one sign each (applied
          // as a multiplication by +-1).
          const uint32_t s0 = (c0 + 2u * N - a) & (2u * N - 1u);
          const uint32_t dl = s0 & 3u;               // the same for every lane
          const uint32_t sa = s0 - dl, sb = (sa + 4u) & (2u * N - 1u);
          const uint4 ra = *reinterpret_cast<const uint4 *>(Pj + (sa & (N - 1u)));
          const uint4 rb = *reinterpret_cast<const uint4 *>(Pj + (sb & (N - 1u)));
          const uint32_t ga = (sa >= N) ? 0xFFFFFFFFu : 1u, gb = (sb >= N) ? 0xFFFFFFFFu : 1u;
          const uint32_t w[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
          const uint32_t mev[4] = {me.x, me.y, me.z, me.w};
          uint32_t rot[4];
          // dl is uniform across the warp: one branch, constant indices
#define FHE_ROT(D)                                                               \
  _Pragma("unroll") for (uint32_t k = 0; k < 4u; ++k)                            \
      rot[k] = w[k + (D)] * ((k + (D)) < 4u ? ga : gb);
          switch (dl) {
            case 0u: FHE_ROT(0u) break;
            case 1u: FHE_ROT(1u) break;
            case 2u: FHE_ROT(2u) break;
            default: FHE_ROT(3u) break;
          }
#undef FHE_ROT
#pragma unroll
          for (uint32_t k = 0; k < 4u; ++k) {
            const uint32_t x = rot[k] - mev[k];
            xr[h][k] = (total_bits >= 32u)
                           ? x
                           : ((uint32_t)(x + (1u << (31u - total_bits))) >> (32u - total_bits));
          }
          const uint32_t tpb = N - 4u - c0;  // smallest reversed index of the run
          const uint32_t in_tile = (bm / 8u) * (kKB * 8u) + ((tpb % kKB) / 8u) * 64u + (bm % 8u) * 8u + (tpb % 8u);
          dst0[h] = dig_h + (uint64_t)(tpb / kKB) * TILE_H + in_tile;
        }
        // A digit d with |d| < 512 is the fp16 number (1536 + d) - 1536, and
        // the bits of 1536 + d are 0x6600 + d (1536 <= 1536 + d < 2048 has an
        // ulp of 1), so two digits become fp16 with one exact packed
        // subtraction.
        const __half2 off = __halves2half2(__ushort_as_half(0x6600u), __ushort_as_half(0x6600u));
        auto pack = [&](uint32_t lo16, uint32_t hi16) {  // lo16 at the low half
          const __half2 v = __hsub2(__halves2half2(__ushort_as_half((unsigned short)(lo16 & 0xFFFFu)),
                                                   __ushort_as_half((unsigned short)(hi16 & 0xFFFFu))), off);
          return *reinterpret_cast<const uint32_t *>(&v);
        };
        // least significant level first.  With v = u + B/2, the balanced
        // digit is (v mod B) - B/2 and the carry-propagated rest is v >> beta
        // (a digit d0 >= B/2 becomes d0 - B and carries 1).
        const uint32_t bias = 0x6600u - Bhalf;  // fp16-bit offset minus B/2
        for (int lam = (int)l - 1; lam >= 0; --lam) {
          const uint32_t r = j * l + (uint32_t)lam;
#pragma unroll
          for (uint32_t h = 0; h < 2u; ++h) {
            uint32_t hv[4], hh2[4];
#pragma unroll
            for (uint32_t k = 0; k < 4u; ++k) {
              const uint32_t v = xr[h][k] + Bhalf;
              xr[h][k] = v >> P.log2_bg;
              if (sub_shift == 0u) {
                hv[k] = (v & Bmask) + bias;
                hh2[k] = 0u;
              } else {
                const int32_t sd = (int32_t)(v & Bmask) - (int32_t)Bhalf;
                const uint32_t sm = (1u << sub_shift) - 1u, sh = 1u << (sub_shift - 1u);
                const uint32_t vl = (uint32_t)sd + sh;           // same split for the sub-digits
                const int32_t lo = (int32_t)(vl & sm) - (int32_t)sh;
                const int32_t hi = (sd - lo) >> sub_shift;       // exact: sd - lo is a multiple
                hv[k] = 0x6600u + (uint32_t)lo;
                hh2[k] = 0x6600u + (uint32_t)hi;
              }
            }
            // position tpb + m holds the digit of c0 + 3 - m
            st_u2(dst0[h] + (uint64_t)r * KBLK * TILE_H,
                  make_uint2(pack(hv[3], hv[2]), pack(hv[1], hv[0])), l2keep, pol_keep);
            if (sub_shift != 0u)
              st_u2(dst0[h] + (uint64_t)(R + r) * KBLK * TILE_H,
                    make_uint2(pack(hh2[3], hh2[2]), pack(hh2[1], hh2[0])), l2keep, pol_keep);
          }
        }
      }
      // No CTA-wide barrier per group: each warp counts itself done with the
      // buffer (acquire-release, so the count orders every warp's reads of
      // it), and the last one refills it while the others go on.
      __syncwarp();
      if (lane == 0) {
        uint32_t prev;
        asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;"
                     : "=r"(prev)
                     : "r"(smem_u32(&s_gdone[buf]))
                     : "memory");
        if (prev == kThreads / 32u - 1u) {
          s_gdone[buf] = 0u;
          if (g + kGBuf < NGROUP && !s_abort) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&g_full[buf], 32768u);
            bulk_g2s(smem + buf * 32768u, acc + (uint64_t)(row0 + (g + kGBuf) * G) * 2u * N, 32768u,
                     &g_full[buf]);
          }
        }
      }
    }
    // This CTA multicasts exactly the digit rows it just wrote; the fence and
    // barrier order them (and the staging buffers' last reads) before the
    // bulk copies.  The barrier is cluster-wide because the partner CTA
    // multicasts into this CTA's A stages, which staged accumulators until now.
    asm volatile("fence.proxy.async;" ::: "memory");
    tile_sync<GC>(tile_ctr, tile_k, &s_abort);

    // ---- external product units (block, chunk, limb pair) of output
    // polynomial pj: each A tile feeds both limbs of the pair (accumulators
    // in TMEM columns 0..255 and 256..511).  The two limb pairs of a chunk
    // run back to back, so the second pass over the chunk's digit tiles finds
    // them in L2.
    if (warp == 0) {
      // digit-tile producer
      if (lane == 0) {
        // per-CTA tile copies also read the rows other CTAs generated (their
        // generic stores were fenced for the async proxy before the barrier)
        if (!MC) asm volatile("fence.proxy.async.global;" ::: "memory");
        for (uint32_t blk = blk0; blk < blk0 + nblk; ++blk)
          for (uint32_t ch = 0; ch < nchunk; ++ch)
            for (uint32_t lp = lp0; lp < lp0 + NLP; ++lp) {
              for (uint32_t rr = 0; rr < chunk_r; ++rr)
                for (uint32_t kh = 0; kh < KH; ++kh) {
                  const uint32_t r = ch * chunk_r + rr;
                  for (uint32_t kb = 0; kb < KT; ++kb) {
                    const uint32_t as = a_it % kAStages;
                    if (a_it >= kAStages)
                      wait_bounded(&a_empty[as], ((a_it / kAStages) - 1u) & 1u, &s_abort);
                    if (!s_abort) {
                      const __half *tsrc = dig_h + (uint64_t)(r * KBLK + KT * kh + kb) * TILE_H;
                      mbar_expect_tx(&a_full[as], kATile);
                      ATileLoad<MC>::run(sA + as * kATile, tsrc, pr, NP, &a_full[as], a_mask,
                                         l2keep, pol_keep);
                    }
                    ++a_it;
                  }
                }
            }
      }
      __syncwarp();
    } else if (warp == kBWarp) {
      // key-window producer: per window, the 640 compact entries of both
      // limbs are staged by bulk copies and the warp writes the window's 79
      // core matrices (row rho of core matrix d = entries s0 + 8 d + rho ..
      // + 7; lanes 8g .. 8g + 7 write the 8 rows of one core matrix, 128
      // contiguous bytes).  Generic stores: each lane fences them for the
      // tensor core (async proxy); then the leader's window is announced on
      // its b_full (release, CTA scope) and the peer's on the leader's b_peer
      // (release, cluster scope).
      const uint32_t g = lane >> 3, rho = lane & 7u;
      const uint32_t sh = (rho & 1u) * 16u;  // funnel-shift bits: odd rows start mid-word
      for (uint32_t blk = blk0; blk < blk0 + nblk; ++blk) {
        const uint32_t c0 = blk * kBN + hh * (kBN / 2u);  // this CTA's 128 columns of B
        for (uint32_t ch = 0; ch < nchunk; ++ch)
          for (uint32_t lp = lp0; lp < lp0 + NLP; ++lp)
            for (uint32_t rr = 0; rr < chunk_r; ++rr)
              for (uint32_t kh = 0; kh < KH; ++kh) {
                const uint32_t r = ch * chunk_r + rr;
                const uint32_t bs = b_it & 1u;
                bool go = true;
                if (b_it >= 2u) go = wait_bounded(&b_empty[bs], ((b_it >> 1) - 1u) & 1u, &s_abort);
                go = __all_sync(0xffffffffu, go && !s_abort);
                unsigned char *hst = sH + bs * 2u * kHStage;
                if (go && lane == 0) {
                  // earlier generic reads of this staging buffer precede the copies
                  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                  mbar_expect_tx(&h_full[bs], 2u * kHStage);
                  const uint32_t s0 = c0 + kBK * kh;
                  for (uint32_t z = 0; z < 2u; ++z) {
                    const __half *src =
                        hk + ((((uint64_t)i * R + r % R) * 2u + pj) * 4u + 2u * lp + z) * strip_halves + s0;
                    bulk_g2s(hst + z * kHStage, src, kHStage, &h_full[bs]);
                  }
                }
                __syncwarp();
                if (go) go = __all_sync(0xffffffffu, wait_bounded(&h_full[bs], (b_it >> 1) & 1u, &s_abort));
                if (go) {
                  // both limbs' windows in one pass (two independent chains)
                  const uint32_t *hw0 = reinterpret_cast<const uint32_t *>(hst) + (rho >> 1);
                  const uint32_t *hw1 = reinterpret_cast<const uint32_t *>(hst + kHStage) + (rho >> 1);
                  unsigned char *win0 = sB + bs * 2u * kBWin + rho * 16u;
                  unsigned char *win1 = win0 + kBWin;
#pragma unroll 4
                  for (uint32_t d0 = 0; d0 < kBCm; d0 += 4u) {
                    const uint32_t d = d0 + g;
                    if (d < kBCm) {
                      // entries 8d + rho .. + 7 = halves rho .. rho + 7 of words 4d ..:
                      // a funnel shift by 16 bits for odd rho, by 0 for even
                      const uint32_t *w = hw0 + 4u * d, *v = hw1 + 4u * d;
                      const uint32_t x0 = w[0], x1 = w[1], x2 = w[2], x3 = w[3], x4 = w[4];
                      const uint32_t y0 = v[0], y1 = v[1], y2 = v[2], y3 = v[3], y4 = v[4];
                      *reinterpret_cast<uint4 *>(win0 + d * 128u) =
                          make_uint4(__funnelshift_r(x0, x1, sh), __funnelshift_r(x1, x2, sh),
                                     __funnelshift_r(x2, x3, sh), __funnelshift_r(x3, x4, sh));
                      *reinterpret_cast<uint4 *>(win1 + d * 128u) =
                          make_uint4(__funnelshift_r(y0, y1, sh), __funnelshift_r(y1, y2, sh),
                                     __funnelshift_r(y2, y3, sh), __funnelshift_r(y3, y4, sh));
                    }
                  }
                  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                  __syncwarp();
                  if (lane == 0) {
                    if (leader) mbar_arrive_local(&b_full[bs]);
                    else mbar_arrive_remote_release(cluster_addr(&b_peer[bs], lead));
                  }
                }
                ++b_it;
              }
      }
      __syncwarp();
    } else if (warp == 1) {
      if (lane == 0 && leader) {
        // Limb 0's accumulator is released by the epilogue before limb 1's:
        // a unit starts with limb 0's MMAs as soon as it is free, and the
        // limb-1 MMAs of its first key window's tiles wait (their A stages
        // held) until limb 1's accumulator is drained too, so limb 1's drain
        // overlaps limb 0's MMAs.  Symmetrically, the last key window runs
        // all its limb-0 MMAs first and announces them (t_full0), so limb 0
        // drains while the window's limb-1 MMAs run.  Within a limb every
        // partial sum is an exact fp32 integer, so the order of the additions
        // does not matter.
        for (uint32_t blk = blk0; blk < blk0 + nblk; ++blk)
          for (uint32_t ch = 0; ch < nchunk; ++ch)
            for (uint32_t lp = lp0; lp < lp0 + NLP; ++lp) {
              if (u_it >= 1u) wait_bounded(t_empty, (u_it - 1u) & 1u, &s_abort);
              tc_fence_after();
              bool z1_free = (u_it == 0u);
              uint32_t acc0 = 0, acc1 = 0;
              uint32_t def_as[KT], def_kb[KT], ndef = 0;  // tiles whose limb-1 MMAs wait
              for (uint32_t rr = 0; rr < chunk_r; ++rr)
                for (uint32_t kh = 0; kh < KH; ++kh) {
                  const uint32_t bs = b_it & 1u;
                  wait_bounded(&b_full[bs], (b_it >> 1) & 1u, &s_abort);
                  wait_bounded_cluster(&b_peer[bs], (b_it >> 1) & 1u, &s_abort);
                  tc_fence_after();
                  const uint32_t bbase = smem_u32(sB + bs * 2u * kBWin);
                  // limb z's MMAs of the tile in stage `as` (K position kb of the window)
                  auto mma_tile = [&](uint32_t as, uint32_t kb, uint32_t z, uint32_t &accz) {
                    const uint32_t abase = smem_u32(sA + as * kATile);
#pragma unroll
                    for (uint32_t s = 0; s < kKB / 16u; ++s) {
                      const uint64_t ad = smem_desc(abase + s * 256u, 128u, kASBO);
                      const uint64_t bd = smem_desc(bbase + z * kBWin + ((kKB / 8u) * kb + 2u * s) * 128u,
                                                    128u, 128u);
                      tc2_mma_f16(tmem + z * (uint32_t)kBN, ad, bd, idesc, accz);
                      accz = 1u;
                    }
                  };
                  auto flush = [&]() {
                    for (uint32_t d = 0; d < ndef; ++d) {
                      mma_tile(def_as[d], def_kb[d], 1u, acc1);
                      tc2_commit_ctas(&a_empty[def_as[d]], ae_mask);
                    }
                    ndef = 0;
                  };
                  const bool last = (rr + 1u == chunk_r) && (kh + 1u == KH);
                  uint32_t tail_as[KT], ntail = 0;  // last window: limb-1 MMAs after t_full0
                  for (uint32_t kb = 0; kb < KT; ++kb) {
                    const uint32_t as = a_it % kAStages;
                    wait_bounded(&a_full[as], (a_it / kAStages) & 1u, &s_abort);
                    wait_bounded(&a_peer[as], (a_it / kAStages) & 1u, &s_abort);
                    tc_fence_after();
                    if (!s_abort && last && z1_free) {
                      mma_tile(as, kb, 0u, acc0);
                      tail_as[ntail++] = as;
                    } else if (!s_abort) {
                      mma_tile(as, kb, 0u, acc0);
                      if (!z1_free && mbar_try_wait(t_empty1, (u_it - 1u) & 1u)) {
                        tc_fence_after();
                        z1_free = true;
                      }
                      if (z1_free) {
                        flush();
                        mma_tile(as, kb, 1u, acc1);
                        tc2_commit_ctas(&a_empty[as], ae_mask);
                      } else {
                        def_as[ndef] = as;
                        def_kb[ndef] = kb;
                        ++ndef;
                      }
                    }
                    ++a_it;
                  }
                  // the window's B stage is released only after every MMA
                  // that reads it, deferred ones included
                  if (ndef && !s_abort) {
                    if (wait_bounded(t_empty1, (u_it - 1u) & 1u, &s_abort)) {
                      tc_fence_after();
                      z1_free = true;
                      flush();
                    }
                  }
                  if (last && !s_abort) {
                    // every limb-0 MMA of the unit is issued: announce them,
                    // then the last window's limb-1 MMAs
                    tc2_commit_ctas(t_full0, pair_mask);
                    for (uint32_t d = 0; d < ntail; ++d) {
                      mma_tile(tail_as[d], d, 1u, acc1);
                      tc2_commit_ctas(&a_empty[tail_as[d]], ae_mask);
                    }
                  }
                  if (!s_abort) tc2_commit_ctas(&b_empty[bs], pair_mask);
                  ++b_it;
                }
              if (!s_abort) tc2_commit_ctas(t_full, pair_mask);
              ++u_it;
            }
      } else if (lane == 0) {
        // peer: tell the leader when this CTA's half of each A tile has landed
        // (its B windows are announced by its key-window warp)
        for (uint32_t blk = blk0; blk < blk0 + nblk; ++blk)
          for (uint32_t ch = 0; ch < nchunk; ++ch)
            for (uint32_t lp = lp0; lp < lp0 + NLP; ++lp)
              for (uint32_t rr = 0; rr < chunk_r; ++rr)
                for (uint32_t kh = 0; kh < KH; ++kh) {
                  for (uint32_t kb = 0; kb < KT; ++kb) {
                    const uint32_t as = a_it % kAStages;
                    if (wait_bounded(&a_full[as], (a_it / kAStages) & 1u, &s_abort))
                      mbar_arrive_remote(cluster_addr(&a_peer[as], lead));
                    ++a_it;
                  }
                }
      }
      __syncwarp();
    } else if (warp >= 2u && warp < 10u) {
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +32 (ciphertexts) and
      // columns 128 ((w - 2) / 4) .. +128 of both 256-column accumulators
      const uint32_t quarter = warp % 4u, half = (warp - 2u) / 4u;
      const uint32_t row = kBh * hh + 32u * quarter + lane;  // ciphertext row of the tile
      const uint32_t te = cluster_addr(t_empty, lead), te1 = cluster_addr(t_empty1, lead);
      for (uint32_t blk = blk0; blk < blk0 + nblk; ++blk) {
        uint32_t *dst = acc + ((uint64_t)row * 2u + pj) * N + blk * kBN + half * 128u;
        uint32_t outv[128];
        if (RED) {
          // the other limb pair of this block is another pair's: both add
#pragma unroll
          for (int k = 0; k < 128; ++k) outv[k] = 0u;
        } else {
          // ACC of this block, loaded while the block's MMAs run
#pragma unroll
          for (int k = 0; k < 128; k += 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(dst + k);
            outv[k] = v.x; outv[k + 1] = v.y; outv[k + 2] = v.z; outv[k + 3] = v.w;
          }
        }
        for (uint32_t ch = 0; ch < nchunk; ++ch)
          for (uint32_t lp = lp0; lp < lp0 + NLP; ++lp) {
            const uint32_t sub = (ch * chunk_r >= R) ? sub_shift : 0u;
#pragma unroll 1
            for (uint32_t z = 0; z < 2u; ++z) {
              // limb 0 is complete at t_full0, limb 1 at t_full
              const bool got = wait_bounded(z ? t_full : t_full0, u_it & 1u, &s_abort);
              const bool ok = __all_sync(0xffffffffu, got);  // warp-uniform for tcgen05.ld
              tc_fence_after();
              if (ok) {
                const uint32_t shift = 8u * (2u * lp + z) + sub;
                const uint32_t tbase = tmem + ((32u * quarter) << 16) + z * (uint32_t)kBN + half * 128u;
                // two 16-column buffers: the load of one overlaps the
                // conversion of the other
                uint32_t ra[16], rb[16];
                tc_ld16(tbase, ra);
                tc_wait16(ra);
#pragma unroll
                for (uint32_t c = 0; c < 8u; c += 2u) {
                  tc_ld16(tbase + (c + 1u) * 16u, rb);
                  tc_acc16(outv + c * 16u, ra, shift);
                  tc_wait16(rb);
                  if (c + 2u < 8u) tc_ld16(tbase + (c + 2u) * 16u, ra);
                  tc_acc16(outv + (c + 1u) * 16u, rb, shift);
                  if (c + 2u < 8u) tc_wait16(ra);
                }
              }
              // limb z's accumulator is free for the next unit's MMAs
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive_remote(z ? te1 : te);
            }
            ++u_it;
          }
        if (!__any_sync(0xffffffffu, s_abort != 0)) {
          if (RED) {
            // additions mod 2^32 commute: the result does not depend on
            // which pair adds first
#pragma unroll
            for (int k = 0; k < 128; ++k) atomicAdd(dst + k, outv[k]);
          } else {
#pragma unroll
            for (int k = 0; k < 128; k += 4)
              *reinterpret_cast<uint4 *>(dst + k) = make_uint4(outv[k], outv[k + 1], outv[k + 2], outv[k + 3]);
          }
        }
      }
      // the next step's digit phase reads ACC through bulk copies
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    tile_sync<GC>(tile_ctr, tile_k, &s_abort);
  }

  // Every MMA of the pair has completed before TMEM is released (on the
  // normal path the epilogue already waited for all of them).
  if (warp == 1 && lane == 0 && leader) {
    tc2_commit_ctas(done, (uint16_t)(1u << q));
    wait_time_bounded(done, 0u);
  }

  // ---- sample extraction (with the multi-value split when L == 2)
  const uint32_t W = N + 1u;
  for (uint32_t jl = 0; jl < lut.L; ++jl) {
    for (uint32_t e = tid; e < RPC * W; e += kThreads) {
      const uint32_t b = row0 + e / W, c = e % W;
      if (base + b >= count) continue;
      const fhe::LutGroup grp = fhe::lut_group(lut, base + b);
      const uint32_t nnz = jl ? grp.nnz1 : grp.nnz0, off = jl ? grp.off1 : grp.off0;
      const uint32_t *A = acc + ((uint64_t)b * 2u) * N;
      const uint32_t *B = acc + ((uint64_t)b * 2u + 1u) * N;
      uint32_t v;
      if (lut.L == 1u) {
        v = (c == N) ? B[0] : (c == 0 ? A[0] : (0u - A[N - c]));
      } else {
        const uint32_t m = (c == N || c == 0) ? 0u : N - c;
        const uint32_t *Pp = (c == N) ? B : A;
        uint32_t s = 0;
        for (uint32_t t = 0; t < nnz; ++t) {
          const uint32_t ep = (uint32_t)lut.rpos[off + t];
          const uint32_t val = (uint32_t)lut.rval[off + t];
          s += val * ((m >= ep) ? Pp[m - ep] : (0u - Pp[m + N - ep]));
        }
        v = (c == N || c == 0) ? s : (0u - s);
      }
      big_out[((size_t)jl * count + base + b) * W + c] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)kTmemCols));
  }
  if (tid == 0 && s_abort) atomicExch(status, FHE_ETIMEOUT);
}

}  // namespace

namespace fhe {

// Sub-digit split shift: 0 when the gadget digits (|d| <= Bg/2) keep one key
// row's fp32 partial sums within 2^24, else ceil(log2_bg / 2) (each digit then
// becomes two signed sub-digits of magnitude <= 2^(shift-1)).
static uint32_t tc_sub_shift(const Params &P) {
  const uint64_t per_r = (uint64_t)(1u << (P.log2_bg - 1u)) * 128u * P.N;
  return per_r <= (1ull << 24) ? 0u : (P.log2_bg + 1u) / 2u;
}

// Largest number of digit rows per fp32 accumulation that keeps every partial
// sum within 2^24: max|digit| * 128 * chunk_r * N <= 2^24; the chunk divides
// the key rows so that low and high sub-digit rows never share a chunk.
static uint32_t tc_chunk_r(const Params &P) {
  const uint32_t s = tc_sub_shift(P);
  const uint64_t dmax = s ? (1ull << (s - 1u)) : (1ull << (P.log2_bg - 1u));
  const uint64_t per_r = dmax * 128u * P.N;
  uint32_t cr = 0;
  while ((uint64_t)(cr + 1u) * per_r <= (1ull << 24) && cr + 1u <= P.rows()) ++cr;
  while (cr > 0 && P.rows() % cr) --cr;
  return cr;
}

static bool tc_supported(const Params &P) {
  const uint32_t s = tc_sub_shift(P);
  // digits (or sub-digits) must stay below 512 in magnitude for the fp16
  // conversion of the digit phase
  if ((s ? (1u << (s - 1u)) : (1u << (P.log2_bg - 1u))) >= 512u) return false;
  // the high sub-digit must also fit: |hi| <= 2^(log2_bg - s - 1) + 1 <= 2^(s-1)
  if (s && (1u << (P.log2_bg - s - 1u)) > (1u << (s - 1u))) return false;
  return P.k == 1u && (P.N == 1024u || P.N == 2048u) && tc_chunk_r(P) >= 1u;
}

static uint32_t tc_digit_rows(const Params &P) { return tc_sub_shift(P) ? 2u * P.rows() : P.rows(); }

int tc_prepare(fhe_keys *K) {
  const Params &P = K->P;
  if (K->d_bsk_tc && K->d_acc_tc && K->d_digits_tc && K->d_tsync) return FHE_OK;
  // compact Hankel key: 2N fp16 per (key row, polynomial, limb)
  const uint64_t strips = (uint64_t)P.n * P.rows() * 2u * 4u;
  K->bsk_tc_bytes = strips * 2u * P.N * sizeof(__half);
  const uint64_t tiles = (K->ws_cap + kBt - 1) / kBt;
  if (cudaMalloc(&K->d_bsk_tc, K->bsk_tc_bytes) != cudaSuccess) return FHE_ENOMEM;
  if (cudaMalloc(&K->d_acc_tc, sizeof(uint32_t) * tiles * tc_tile_acc_words(P.N)) != cudaSuccess)
    return FHE_ENOMEM;
  if (cudaMalloc(&K->d_digits_tc, sizeof(__half) * tiles * tc_tile_dig_halves(P.N, tc_digit_rows(P))) !=
      cudaSuccess)
    return FHE_ENOMEM;
  if (cudaMalloc(&K->d_tsync, sizeof(uint32_t) * tiles) != cudaSuccess) return FHE_ENOMEM;
  k_hankel_compact<<<152u * 16u, 256>>>(P, K->d_bsk, (__half *)K->d_bsk_tc);
  note_launches(1);
  FHE_CUDA_TRY(cudaGetLastError());
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  return FHE_OK;
}

bool tc_available(const Params &P) { return tc_supported(P); }

int pbs_prepare(fhe_keys *K, int variant) {
  if (variant == FHE_VARIANT_FFT) return fft_prepare(K);
  if (variant == FHE_VARIANT_AUTO) return tc_supported(K->P) ? tc_prepare(K) : FHE_OK;
  if (variant != FHE_VARIANT_TC) return FHE_OK;
  if (!tc_supported(K->P)) return FHE_EUNSUPPORTED;
  return tc_prepare(K);
}

using TcKernel = decltype(&k_blind_rotate_tc<1024, 4, 1, false>);

// Instance of the blind rotation for ring size N, cluster size cl (4, 8 or
// 16 CTAs per 256-ciphertext tile) and digit-tile copy form, or (split) the
// tile spread over two clusters of 16.  The single-GPU build compiles
// multicast instances for every cluster size and per-CTA ones for clusters
// of 16; the replica build only per-CTA ones.  The split instance copies per
// CTA in both.
template <int N>
static TcKernel tc_kernel(int cl, bool mc, bool split = false) {
  if (split) return k_blind_rotate_tc<N, 16, 2, false>;
#ifndef FHE_NO_MULTICAST
  if (mc) return cl == 16 ? k_blind_rotate_tc<N, 16, 1, true>
                          : (cl == 8 ? k_blind_rotate_tc<N, 8, 1, true> : k_blind_rotate_tc<N, 4, 1, true>);
#else
  (void)mc;
#endif
  return cl == 16 ? k_blind_rotate_tc<N, 16, 1, false>
                  : (cl == 8 ? k_blind_rotate_tc<N, 8, 1, false> : k_blind_rotate_tc<N, 4, 1, false>);
}

// Clusters of `cl` CTAs of `kern` the device holds at once (0 when the
// shape cannot launch, e.g. a 16-CTA cluster where the device does not
// allow that non-portable size).
static int tc_max_clusters(TcKernel kern, int cl, uint32_t smem) {
  if (cl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) { (void)cudaGetLastError(); n = 0; }
  return n;
}

int pbs_tc(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
           uint32_t *ct_out, size_t table_stride, cudaStream_t st, const uint64_t *seg_end) {
  const Params &P = K->P;
  if (!tc_supported(P)) return FHE_EUNSUPPORTED;
  int rc = tc_prepare(K);
  if (rc) return rc;
  const uint32_t chunk_r = tc_chunk_r(P), sub_shift = tc_sub_shift(P);
  const TcSmem S = tc_smem();
  auto pick = [&](int cl, bool mc, bool split = false) {
    return P.N == 1024u ? tc_kernel<1024>(cl, mc, split) : tc_kernel<2048>(cl, mc, split);
  };
  // digit tiles copied as the build does (multicast where compiled in),
  // unless the option asks for per-CTA copies (or multicast)
  const bool mc = (K->tc_force_mc < 0 || !kTcMulticast) ? kTcMulticast : (K->tc_force_mc != 0);
  TcKernel k4 = pick(4, mc), k8 = pick(8, mc), k16 = pick(16, mc);
  TcKernel k32 = pick(16, false, true);
  for (TcKernel k : {k4, k8, k16, k32})
    FHE_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total));
  // 16 CTAs per cluster is a non-portable size (where refused, the occupancy
  // query below reports no such clusters and the shape is never used)
  for (TcKernel k : {k16, k32})
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      (void)cudaGetLastError();
      K->tc_cl16_max = 0;
    }
  // clusters of 8 and 16 the device holds at once (once per key handle)
  if (K->tc_cl8_max < 0) K->tc_cl8_max = tc_max_clusters(k8, 8, S.total);
  if (K->tc_cl16_max < 0) K->tc_cl16_max = tc_max_clusters(k16, 16, S.total);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FHE_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  const bool capturing = (cap != cudaStreamCaptureStatusNone);
  for (size_t s0 = 0; s0 < count; s0 += K->ws_cap) {
    const size_t cnt = (count - s0 < K->ws_cap) ? count - s0 : K->ws_cap;
    const LutArgs la = lut_args(lut, seg_end, s0);
    const int tiles = (int)((cnt + kBt - 1) / kBt);
    // A batch that fits in one wave of 16-CTA clusters runs on them (a
    // quarter of the work per CTA and step of the 4-CTA shape: the lowest
    // latency), one that fits in a wave of 8-CTA clusters on those, larger
    // ones on the 36 clusters of 4.  The autotuner may lower both limits
    // where it measured the smaller shape faster.
    const int lim16 = (K->tc_cl16_tiles >= 0 && K->tc_cl16_tiles < K->tc_cl16_max) ? K->tc_cl16_tiles
                                                                                 : K->tc_cl16_max;
    const int lim8 = (K->tc_cl8_tiles >= 0 && K->tc_cl8_tiles < K->tc_cl8_max) ? K->tc_cl8_tiles
                                                                            : K->tc_cl8_max;
    // Batches of up to half the 16-CTA clusters may spread each tile over
    // two of them (32 CTAs per tile, half the work per CTA and step again),
    // a cooperative launch: tried eagerly first, and used inside a stream
    // capture only once an eager launch has succeeded (a refused launch
    // would invalidate the capture).
    const int split_max = (K->tc_split_ok > 0 || (K->tc_split_ok < 0 && !capturing)) ? K->tc_cl16_max / 2 : 0;
    const int lim32 = (K->tc_split_tiles >= 0 && K->tc_split_tiles < split_max) ? K->tc_split_tiles
                                                                               : split_max;
    int cl = 4;
    if (K->tc_force_cl) {
      if (K->tc_force_cl == 32 && tiles <= split_max) cl = 32;
      else if (K->tc_force_cl >= 16 && tiles <= K->tc_cl16_max) cl = 16;
      else if (K->tc_force_cl >= 8 && tiles <= K->tc_cl8_max) cl = 8;
    } else if (tiles <= lim32) {
      cl = 32;
    } else if (tiles <= lim16) {
      cl = 16;
    } else if (tiles <= lim8) {
      cl = 8;
    }
    const bool prof = (s0 == 0) && K->prof_ev0;
    if (prof) { FHE_CUDA_TRY(record_prof_event(K->prof_ev0, st)); K->prof_count = cnt; }
    const __half *hk = (const __half *)K->d_bsk_tc;
    const uint32_t *in = ct_in + s0 * (P.n + 1u);
    __half *dig = (__half *)K->d_digits_tc;
    const uint32_t opts = K->tc_l2_hints > 0 ? 1u : 0u;
    bool launched = false;
    if (cl == 32) {
      // cooperative: the two clusters of a tile wait on each other
      FHE_CUDA_TRY(cudaMemsetAsync(K->d_tsync, 0, sizeof(uint32_t) * (size_t)tiles, st));
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)tiles * 32u);
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = S.total;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, k32, P, hk, in, cnt, la, K->d_acc_tc, dig, chunk_r, sub_shift, K->d_big,
                             K->d_status, opts, K->d_tsync) == cudaSuccess) {
        launched = true;
        if (!capturing) K->tc_split_ok = 1;
      } else {  // the device refuses a cooperative clustered launch: never again
        (void)cudaGetLastError();
        K->tc_split_ok = 0;
        cl = 16;
      }
    }
    if (!launched) {
      TcKernel kern = (cl == 16) ? k16 : (cl == 8 ? k8 : k4);
      kern<<<(unsigned)tiles * (unsigned)cl, kThreads, S.total, st>>>(
          P, hk, in, cnt, la, K->d_acc_tc, dig, chunk_r, sub_shift, K->d_big, K->d_status, opts, nullptr);
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

// Autotuner of FHE_VARIANT_AUTO: both bit-exact blind rotations are timed on
// this device for doubling batch sizes; the tensor-core path (256 ciphertexts
// per 4-SM cluster, a fixed CMux latency per tile) wins from some batch size
// on, the CUDA-core path (4 ciphertexts per CTA) below it.
extern "C" int fhe_pbs_autotune(fhe_keys *K, uint64_t *tc_min_batch, void *stream) {
  if (!K || !tc_min_batch) return FHE_EINVAL;
  const fhe::Params &P = K->P;
  if (!fhe::tc_available(P)) {
    K->tc_min_batch = SIZE_MAX;
    *tc_min_batch = UINT64_MAX;
    return FHE_OK;
  }
  int rc = fhe::pbs_prepare(K, FHE_VARIANT_TC);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cmax = (K->ws_cap < 4096u) ? K->ws_cap : 4096u;
  const uint32_t W = P.n + 1u;
  std::vector<int32_t> f(P.p());
  for (uint32_t u = 0; u < P.p(); ++u) f[u] = (int32_t)u;
  fhe_lut *lut = nullptr;
  rc = fhe_lut_create(K, f.data(), 1u, &lut);
  if (rc) return rc;
  uint32_t *d_in = nullptr, *d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // the blind rotation's cost does not depend on the ciphertext values
  bool ok = cudaMalloc(&d_in, sizeof(uint32_t) * cmax * W) == cudaSuccess &&
            cudaMalloc(&d_out, sizeof(uint32_t) * cmax * W) == cudaSuccess &&
            cudaMemsetAsync(d_in, 0, sizeof(uint32_t) * cmax * W, st) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  size_t best = SIZE_MAX;
  int wins = 0;
  // Below one tile the tensor-core launch takes the latency of one tile (on
  // a cluster of 16 about a third of a CUDA-core launch of even 4
  // ciphertexts), so sampling starts at 16 ciphertexts; a tensor-core win
  // there holds for every smaller batch.
  const size_t c_first = 16;
  for (size_t c = c_first; ok && rc == FHE_OK && c <= cmax; c *= 2) {
    float t[2] = {0.f, 0.f};
    for (int v = 0; v < 2 && rc == FHE_OK; ++v) {
      const int variant = v ? FHE_VARIANT_TC : FHE_VARIANT_EXACT;
      rc = fhe::pbs_run(K, d_in, c, lut, d_out, c * W, variant, st);  // warm-up
      if (rc) break;
      ok = cudaEventRecord(e0, st) == cudaSuccess;
      rc = fhe::pbs_run(K, d_in, c, lut, d_out, c * W, variant, st);
      ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&t[v], e0, e1) == cudaSuccess;
    }
    if (!ok || rc) break;
    if (t[1] <= t[0]) {
      if (best == SIZE_MAX) best = c;
      if (++wins == 2) break;  // the tensor-core path only gains with size
    } else {
      best = SIZE_MAX;
      wins = 0;
    }
  }
  // cluster shape of the tensor-core tiles: a batch of t tiles that fits in
  // one wave of the larger shape runs on t clusters of 8 (half the work per
  // CTA and step of clusters of 4) or of 16 (a quarter); time each larger
  // shape against the next smaller one at t = 1, 4 and its largest t, and
  // keep it up to the largest sampled t at and below which it was never slower
  auto tune_shape = [&](int small, int large, int max_large) {
    std::vector<int> samples;  // 1, 4 and the largest t, those that fit
    for (int t : {1, 4, max_large})
      if (t <= max_large && (size_t)t * 256u <= cmax && (samples.empty() || t > samples.back()))
        samples.push_back(t);
    int keep = 0;
    for (int v = 0; v < 2 && rc == FHE_OK; ++v) {  // warm both instances
      K->tc_force_cl = v ? large : small;
      rc = fhe::pbs_run(K, d_in, 256u, lut, d_out, 256u * W, FHE_VARIANT_TC, st);
    }
    for (size_t si = 0; si < samples.size() && ok && rc == FHE_OK; ++si) {
      const size_t c = (size_t)samples[si] * 256u;
      float t[2] = {0.f, 0.f};
      for (int v = 0; v < 2 && ok && rc == FHE_OK; ++v) {
        K->tc_force_cl = v ? large : small;
        ok = cudaEventRecord(e0, st) == cudaSuccess;
        rc = fhe::pbs_run(K, d_in, c, lut, d_out, c * W, FHE_VARIANT_TC, st);
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&t[v], e0, e1) == cudaSuccess;
      }
      if (!ok || rc) break;
      if (t[1] > t[0]) break;
      keep = samples[si];
    }
    K->tc_force_cl = 0;
    return keep;
  };
  int cl8_tiles = -1, cl16_tiles = -1;
  if (ok && rc == FHE_OK && K->tc_cl8_max > 0 && cmax >= 256u) cl8_tiles = tune_shape(4, 8, K->tc_cl8_max);
  if (ok && rc == FHE_OK && K->tc_cl16_max > 0 && cmax >= 256u)
    cl16_tiles = tune_shape(K->tc_cl8_max > 0 ? 8 : 4, 16, K->tc_cl16_max);
  int split_tiles = -1;
  if (ok && rc == FHE_OK && K->tc_split_ok != 0 && K->tc_cl16_max >= 2 && cmax >= 256u)
    split_tiles = tune_shape(16, 32, K->tc_cl16_max / 2);
  if (!ok && rc == FHE_OK) { (void)cudaGetLastError(); rc = FHE_ECUDA; }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_in);
  cudaFree(d_out);
  fhe_lut_free(lut);
  if (rc) return rc;
  K->tc_cl8_tiles = cl8_tiles;
  K->tc_cl16_tiles = cl16_tiles;
  K->tc_split_tiles = split_tiles;
  // tensor cores never won up to cmax: use them only above it
  K->tc_min_batch = (best == SIZE_MAX) ? 2 * cmax : (best == c_first ? 1u : best);
  *tc_min_batch = K->tc_min_batch;
  return fhe_status(K, stream);
}

extern "C" int fhe_pbs_tuning(const fhe_keys *K, uint64_t *tc_min_batch, int32_t *tc_cl8_tiles,
                              int32_t *tc_cl16_tiles, int32_t *tc_split_tiles) {
  if (!K || !tc_min_batch || !tc_cl8_tiles) return FHE_EINVAL;
  *tc_min_batch = (K->tc_min_batch == SIZE_MAX) ? UINT64_MAX : (uint64_t)K->tc_min_batch;
  *tc_cl8_tiles = (K->tc_cl8_tiles >= 0 && K->tc_cl8_tiles < K->tc_cl8_max) ? K->tc_cl8_tiles
                                                                           : K->tc_cl8_max;
  if (tc_cl16_tiles)
    *tc_cl16_tiles = (K->tc_cl16_tiles >= 0 && K->tc_cl16_tiles < K->tc_cl16_max) ? K->tc_cl16_tiles
                                                                                 : K->tc_cl16_max;
  if (tc_split_tiles) {
    const int smax = (K->tc_split_ok == 0 || K->tc_cl16_max < 0) ? 0 : K->tc_cl16_max / 2;
    *tc_split_tiles = (K->tc_split_ok < 0 && K->tc_cl16_max < 0) ? -1
                      : ((K->tc_split_tiles >= 0 && K->tc_split_tiles < smax) ? K->tc_split_tiles : smax);
  }
  return FHE_OK;
}

extern "C" int fhe_pbs_set_tc_option(fhe_keys *K, int option, int value) {
  if (!K) return FHE_EINVAL;
  switch (option) {
    case FHE_TC_OPT_CLUSTER:
      if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32) return FHE_EINVAL;
      K->tc_force_cl = value;
      return FHE_OK;
    case FHE_TC_OPT_MULTICAST:
      if (value < -1 || value > 1) return FHE_EINVAL;
      if (value == 1 && !kTcMulticast) return FHE_EUNSUPPORTED;
      K->tc_force_mc = value;
      return FHE_OK;
    case FHE_TC_OPT_L2_HINTS:
      if (value < -1 || value > 1) return FHE_EINVAL;
      K->tc_l2_hints = value;
      return FHE_OK;
    default:
      return FHE_EINVAL;
  }
}

extern "C" int fhe_tc_plan_query(const fhe_params *params, fhe_tc_plan *out) {
  if (!params || !out) return FHE_EINVAL;
  const Params P = fhe::from_abi(*params);
  if (!fhe::params_supported(P)) return FHE_EINVAL;
  memset(out, 0, sizeof(*out));
  out->available = tc_supported(P) ? 1 : 0;
  out->key_rows = P.rows();
  out->digit_rows = tc_digit_rows(P);
  out->sub_shift = tc_sub_shift(P);
  out->max_digit = out->sub_shift ? (1u << (out->sub_shift - 1u)) : (1u << (P.log2_bg - 1u));
  out->chunk_rows = tc_chunk_r(P);
  out->max_partial = (uint64_t)out->max_digit * 128u * out->chunk_rows * P.N;
  return FHE_OK;
}
