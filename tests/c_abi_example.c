/* A plain C client of libfhe_dicsnn: keys from a seed, encryption of every
 * message of Z_2p, one batch of bootstraps with the LIF Fire / Reset tables
 * (Thm 2.1, one multi-value blind rotation, 4.2), decryption, and a check of
 * every output against the tables.  Uses only the C ABI and the CUDA runtime
 * for device buffers.
 *
 * Exit status: 0 when every output decrypts to its table value, 1 on a
 * mismatch, 2 when the library or the CUDA runtime reports an error (for
 * instance on a machine without a GPU), after printing it. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include "fhe_dicsnn.h"

static int fail(const char *what, int rc) {
  fprintf(stderr, "%s: %s (%d)\n", what, fhe_strerror(rc), rc);
  return 2;
}

int main(void) {
  /* the test-only low-noise set: n = 32, N = 1024, p = 32 */
  const fhe_params P = {32u, 1u, 1024u, 8u, 3u, 4u, 5u, 5u, 25, 30};
  const int32_t p = 1 << P.log2_p, v_th = 4;
  const size_t count = 2u * (size_t)p, W = P.n + 1u;
  fhe_keys *keys = NULL;
  int rc = fhe_keygen_from_seed(&P, 7u, 0u, NULL, &keys);
  if (rc) return fail("fhe_keygen_from_seed", rc);

  /* Fire and Reset on the centred input u = H + p/2, v = u - p/2 */
  int32_t *f = (int32_t *)malloc(sizeof(int32_t) * 2u * (size_t)p);
  for (int32_t u = 0; u < p; ++u) {
    const int32_t v = u - p / 2;
    f[u] = v >= v_th;
    f[p + u] = v >= v_th ? 0 : (v >= 0 ? v >> 1 : 0);
  }
  fhe_lut *lut = NULL;
  rc = fhe_lut_create(keys, f, 2u, &lut);
  if (rc) return fail("fhe_lut_create", rc);

  int32_t *msg = (int32_t *)malloc(sizeof(int32_t) * count);
  for (size_t i = 0; i < count; ++i) msg[i] = (int32_t)i;
  int32_t *d_msg = NULL, *d_dec = NULL;
  uint32_t *d_ct = NULL, *d_out = NULL;
  if (cudaMalloc((void **)&d_msg, sizeof(int32_t) * 2u * count) != cudaSuccess ||
      cudaMalloc((void **)&d_dec, sizeof(int32_t) * 2u * count) != cudaSuccess ||
      cudaMalloc((void **)&d_ct, sizeof(uint32_t) * count * W) != cudaSuccess ||
      cudaMalloc((void **)&d_out, sizeof(uint32_t) * 2u * count * W) != cudaSuccess)
    return fail("cudaMalloc", FHE_ENOMEM);
  if (cudaMemcpy(d_msg, msg, sizeof(int32_t) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail("cudaMemcpy", FHE_ECUDA);
  if ((rc = fhe_encrypt(keys, d_msg, count, 11u, d_ct, NULL))) return fail("fhe_encrypt", rc);
  if ((rc = fhe_pbs_batch(keys, d_ct, count, lut, d_out, FHE_VARIANT_EXACT, NULL)))
    return fail("fhe_pbs_batch", rc);
  if ((rc = fhe_decrypt(keys, d_out, 2u * count, d_dec, NULL))) return fail("fhe_decrypt", rc);
  int32_t *dec = (int32_t *)malloc(sizeof(int32_t) * 2u * count);
  if (cudaMemcpy(dec, d_dec, sizeof(int32_t) * 2u * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail("cudaMemcpy", FHE_ECUDA);

  /* messages in [p, 2p) land on the negacyclic half: -f(m - p) */
  int bad = 0;
  for (int j = 0; j < 2; ++j)
    for (size_t i = 0; i < count; ++i) {
      const int32_t m = (int32_t)i;
      int32_t want = m < p ? f[j * p + m] : -f[j * p + m - p];
      want = ((want + p) % (2 * p) + 2 * p) % (2 * p) - p;
      if (dec[(size_t)j * count + i] != want) ++bad;
    }
  printf("%d of %zu outputs differ from the tables\n", bad, 2u * count);
  fhe_lut_free(lut);
  fhe_keys_free(keys);
  cudaFree(d_msg);
  cudaFree(d_dec);
  cudaFree(d_ct);
  cudaFree(d_out);
  free(f);
  free(msg);
  free(dec);
  return bad ? 1 : 0;
}
