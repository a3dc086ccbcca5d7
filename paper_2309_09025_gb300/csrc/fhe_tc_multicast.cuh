// fhe_tc_multicast.cuh -- cluster-multicast forms used by the tensor-core
// blind rotation: the digit-tile copy and the MMA completion commit.
// Included by fhe_pbs_tc.cu only when FHE_NO_MULTICAST is not defined: the
// single-GPU library uses them, the replica library (one process per GPU) is
// built without them (every CTA copies whole digit tiles, and MMA completion
// is committed to each CTA's barrier separately).  The copy's source is this
// GPU's own digit workspace.
#pragma once

// Completion of every tcgen05.mma this thread issued arrives on the barrier at
// the same offset in each CTA of `mask`.
__device__ __forceinline__ void tc2_commit_ctas(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s_multicast(void *dst, const void *src, uint32_t bytes,
                                                   uint64_t *bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Each of the np CTAs holding the same 128 rows sends the rows it generated
// (share pr of the tile) to all of them; the tile is complete in every CTA
// once all np shares have landed (kATile bytes on each CTA's barrier).
__device__ __forceinline__ void bulk_g2s_multicast_hint(void *dst, const void *src, uint32_t bytes,
                                                        uint64_t *bar, uint16_t mask, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      ".L2::cache_hint [%0], [%1], %2, [%3], %4, %5;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask), "l"(pol)
      : "memory");
}

template <>
struct ATileLoad<true> {
  static __device__ __forceinline__ void run(unsigned char *stage, const __half *tile, uint32_t pr,
                                             uint32_t np, uint64_t *bar, uint16_t mask, bool hint,
                                             uint64_t pol) {
    const uint32_t share = (uint32_t)kATile / np;  // bytes
    if (hint)
      bulk_g2s_multicast_hint(stage + pr * share, tile + pr * (share / 2u), share, bar, mask, pol);
    else
      bulk_g2s_multicast(stage + pr * share, tile + pr * (share / 2u), share, bar, mask);
  }
};
