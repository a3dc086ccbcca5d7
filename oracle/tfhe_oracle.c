/*
 * tfhe_oracle.c -- plain, slow, obviously-correct CPU reference of the
 * FHE-DiCSNN hot path (TFHE programmable bootstrapping over the uint32 torus
 * plus the integer-weighted LWE sums that feed it).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may load this library.  The product path
 * (paper_2309_09025_gb300) never links, imports or calls it, and it shares no
 * code, header, table or helper with the CUDA implementation.
 *
 * Every function follows the plain mathematical definition in the paper's
 * notation; polynomial products are the schoolbook negacyclic sum (no FFT, no
 * blocking).  All ciphertext arithmetic is in Z_q with q = 2^32, i.e. uint32_t
 * with wrap-around.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - noise: the paper asks for a discrete Gaussian (paper 2.1, RLWE) without a
 *     sampler; we use an integer Irwin-Hall(12) sum of uniform signed 32-bit
 *     integers scaled by 2^-noise_log2 (std = 2^-noise_log2 torus units);
 *   - keys: binary uniform LWE key s and GLWE key S;
 *   - encoding: one padding bit, Delta = q / (2p);
 *   - gadget and key-switch digits: signed, in [-B/2, B/2), value first
 *     rounded to the top (levels*log2 B) bits, carries propagated from the
 *     least significant level, the final carry dropped;
 *   - modulus switch: round half up;
 *   - test polynomial: centred boxes round(i*p/N) with the negacyclic wrap
 *     (-f(0)) on the last half box (the paper's floor(i*p/2N) boxes are
 *     uncentred and misdecode message 0 with negative noise).
 *
 * Parity status: every function below is pinned by the CPU test-suite
 * (published SplitMix64 vectors, enc/dec round trip, linearity, brute-force
 * negacyclic products, exhaustive decomposition, brute-force PBS over every
 * message, noise variance against the closed form, hand-worked LIF example).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
  uint32_t n;        /* LWE dimension                                   */
  uint32_t k;        /* GLWE dimension                                  */
  uint32_t N;        /* polynomial size (power of two)                  */
  uint32_t log2_bg;  /* gadget base Bg = 2^log2_bg                      */
  uint32_t l;        /* gadget levels                                   */
  uint32_t log2_bks; /* key-switch base                                 */
  uint32_t l_ks;     /* key-switch levels                               */
  uint32_t log2_p;   /* message modulus p = 2^log2_p (plus padding bit) */
  int32_t lwe_noise_log2;  /* sigma_lwe  = 2^-x torus units; x>=64: none */
  int32_t glwe_noise_log2; /* sigma_glwe = 2^-x torus units; x>=64: none */
} orc_params;

enum {
  ORC_DOM_LWE_KEY = 0,
  ORC_DOM_GLWE_KEY = 1,
  ORC_DOM_BSK_MASK = 2,
  ORC_DOM_BSK_NOISE = 3,
  ORC_DOM_KSK_MASK = 4,
  ORC_DOM_KSK_NOISE = 5,
  ORC_DOM_ENC_MASK = 6,
  ORC_DOM_ENC_NOISE = 7
};

/* ------------------------------------------------------------------ */
/* Counter-based randomness: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
 * splitmix_out(s, i) is the i-th (0-based) output of the generator whose
 * state starts at s.  A draw for (seed, domain, index) is output `index` of
 * the generator seeded with output `domain` of the generator seeded with
 * `seed`.                                                              */
static uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t orc_splitmix_out(uint64_t state, uint64_t i) {
  return orc_mix64(state + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

uint64_t orc_draw(uint64_t seed, uint32_t domain, uint64_t index) {
  return orc_splitmix_out(orc_splitmix_out(seed, domain), index);
}

/* floor(x / 2^s) for signed 64-bit x, written without relying on the
 * implementation-defined right shift of negative values.               */
static int64_t orc_floor_shift(int64_t x, int s) {
  if (x >= 0) return x >> s;
  return -(((-x) - 1) >> s) - 1;
}

/* Noise sample (reading of the paper's discrete Gaussian, 2.1 RLWE):
 * e = round_half_up( sum_{j<12} u_j / 2^noise_log2 ), u_j uniform signed
 * 32-bit integers taken from six 64-bit draws (low half, then high half).
 * The sum has variance (2^64-1) ~ (q)^2, so e has std ~ q * 2^-noise_log2. */
uint32_t orc_noise(uint64_t seed, uint32_t domain, uint64_t index, int32_t noise_log2) {
  if (noise_log2 >= 64) return 0u;
  int64_t sum = 0;
  for (uint32_t j = 0; j < 6; ++j) {
    uint64_t u = orc_draw(seed, domain, index * 6u + j);
    sum += (int64_t)(int32_t)(uint32_t)(u & 0xFFFFFFFFu);
    sum += (int64_t)(int32_t)(uint32_t)(u >> 32);
  }
  if (noise_log2 <= 0) return (uint32_t)sum;
  int64_t e = orc_floor_shift(sum + ((int64_t)1 << (noise_log2 - 1)), noise_log2);
  return (uint32_t)(uint64_t)e;
}

/* ------------------------------------------------------------------ */
/* Ring R_{q,N} = Z_q[X]/(X^N+1) (paper 2.1).                          */

/* out = a * b mod (X^N + 1), schoolbook: X^N = -1.                     */
void orc_negacyclic_mul(const uint32_t *a, const uint32_t *b, uint32_t N, uint32_t *out) {
  for (uint32_t c = 0; c < N; ++c) out[c] = 0;
  for (uint32_t t = 0; t < N; ++t) {
    for (uint32_t u = 0; u < N; ++u) {
      uint32_t prod = a[t] * b[u];
      uint32_t s = t + u;
      if (s < N) out[s] += prod;
      else out[s - N] -= prod;
    }
  }
}

/* out += d * key mod (X^N + 1) for a signed small-integer polynomial d.  */
static void orc_negacyclic_mul_acc_signed(const int32_t *d, const uint32_t *key, uint32_t N,
                                          uint32_t *out) {
  for (uint32_t t = 0; t < N; ++t) {
    uint32_t dt = (uint32_t)d[t];
    if (dt == 0) continue;
    for (uint32_t u = 0; u < N; ++u) {
      uint32_t prod = dt * key[u];
      uint32_t s = t + u;
      if (s < N) out[s] += prod;
      else out[s - N] -= prod;
    }
  }
}

/* out = X^e * P mod (X^N + 1), e in [0, 2N).                             */
void orc_poly_rotate(const uint32_t *P, uint32_t N, uint32_t e, uint32_t *out) {
  for (uint32_t t = 0; t < N; ++t) {
    uint32_t s = (t + e) % (2u * N);
    if (s < N) out[s] = P[t];
    else out[s - N] = (uint32_t)0u - P[t];
  }
}

/* ------------------------------------------------------------------ */
/* Signed gadget decomposition (reading of the RGSW external product,
 * paper 2.1 GSW): digits[lam-1] is level lam (lam = 1 most significant),
 * sum_lam digits[lam-1] * 2^(32 - lam*log2_base) = x rounded to the top
 * levels*log2_base bits, mod 2^32; every digit in [-B/2, B/2).          */
void orc_decompose(uint32_t x, uint32_t log2_base, uint32_t levels, int32_t *digits) {
  uint32_t total = log2_base * levels;
  uint32_t xr;
  if (total >= 32u) xr = x;
  else xr = (uint32_t)(x + (1u << (31u - total))) >> (32u - total);
  uint32_t B = 1u << log2_base;
  uint32_t half = B >> 1;
  for (uint32_t lam = levels; lam >= 1u; --lam) {
    uint32_t d = xr & (B - 1u);
    xr >>= log2_base;
    if (d >= half) {
      digits[lam - 1u] = (int32_t)d - (int32_t)B;
      xr += 1u;
    } else {
      digits[lam - 1u] = (int32_t)d;
    }
  }
}

/* Modulus switch q -> 2N with round half up (implicit in the accumulator
 * index ACC[-b + sum a_i s_i], paper 2.1 Initialization/Blind Rotation). */
uint32_t orc_mod_switch(uint32_t a, uint32_t N) {
  uint32_t w = 0;
  while ((1u << w) < 2u * N) ++w; /* w = log2(2N) */
  return (uint32_t)(a + (1u << (31u - w))) >> (32u - w);
}

/* ------------------------------------------------------------------ */
/* LWE (paper 2.1, LWE): (a, b = <a,s> + e + Delta*m) mod q.             */

static uint32_t orc_delta(const orc_params *P) { return 1u << (31u - P->log2_p); }

void orc_keygen(const orc_params *P, uint64_t seed, uint32_t *lwe_key, uint32_t *glwe_key,
                uint32_t *bsk, uint32_t *ksk) {
  const uint32_t n = P->n, k = P->k, N = P->N, l = P->l;
  for (uint32_t i = 0; i < n; ++i) lwe_key[i] = (uint32_t)(orc_draw(seed, ORC_DOM_LWE_KEY, i) & 1u);
  for (uint32_t i = 0; i < k * N; ++i)
    glwe_key[i] = (uint32_t)(orc_draw(seed, ORC_DOM_GLWE_KEY, i) & 1u);

  /* Bootstrapping key ek_i = RGSW(X^{s_i}) (paper 2.1, Blind Rotation).
   * Layout bsk[i][row][comp][c], row = j*l + (lam-1), comp 0..k-1 masks,
   * comp k body.  Row (j, lam) is a GLWE encryption of zero with
   * s_i * q/Bg^lam added to component j at coefficient 0.              */
  const uint32_t rows = (k + 1u) * l;
  uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * N);
  for (uint32_t i = 0; i < n; ++i) {
    for (uint32_t row = 0; row < rows; ++row) {
      uint64_t ridx = (uint64_t)i * rows + row;
      uint32_t *g = bsk + ridx * (k + 1u) * N;
      uint32_t *body = g + (uint64_t)k * N;
      for (uint32_t c = 0; c < N; ++c)
        body[c] = orc_noise(seed, ORC_DOM_BSK_NOISE, ridx * N + c, P->glwe_noise_log2);
      for (uint32_t jj = 0; jj < k; ++jj) {
        uint32_t *a = g + (uint64_t)jj * N;
        for (uint32_t c = 0; c < N; ++c)
          a[c] = (uint32_t)orc_draw(seed, ORC_DOM_BSK_MASK, (ridx * k + jj) * N + c);
        orc_negacyclic_mul(a, glwe_key + (uint64_t)jj * N, N, tmp);
        for (uint32_t c = 0; c < N; ++c) body[c] += tmp[c];
      }
      uint32_t j = row / l, lam = row % l + 1u;
      uint32_t mu = lwe_key[i] << (32u - P->log2_bg * lam);
      g[(uint64_t)j * N] += mu;
    }
  }
  free(tmp);

  /* Key-switching key: ksk[i][lam-1] = LWE_s(z_i * q/Bks^lam), z = S's
   * coefficients (paper 2.1, Key Switching).                           */
  for (uint32_t i = 0; i < k * N; ++i) {
    for (uint32_t lam = 1; lam <= P->l_ks; ++lam) {
      uint64_t ridx = (uint64_t)i * P->l_ks + (lam - 1u);
      uint32_t *c = ksk + ridx * (n + 1u);
      uint32_t b = orc_noise(seed, ORC_DOM_KSK_NOISE, ridx, P->lwe_noise_log2);
      for (uint32_t t = 0; t < n; ++t) {
        c[t] = (uint32_t)orc_draw(seed, ORC_DOM_KSK_MASK, ridx * n + t);
        b += c[t] * lwe_key[t];
      }
      b += glwe_key[i] << (32u - P->log2_bks * lam);
      c[n] = b;
    }
  }
}

void orc_encrypt(const orc_params *P, const uint32_t *lwe_key, const int32_t *msg, uint64_t count,
                 uint64_t seed, uint32_t *ct) {
  const uint32_t n = P->n;
  for (uint64_t idx = 0; idx < count; ++idx) {
    uint32_t *c = ct + idx * (n + 1u);
    uint32_t b = orc_noise(seed, ORC_DOM_ENC_NOISE, idx, P->lwe_noise_log2);
    for (uint32_t t = 0; t < n; ++t) {
      c[t] = (uint32_t)orc_draw(seed, ORC_DOM_ENC_MASK, idx * n + t);
      b += c[t] * lwe_key[t];
    }
    b += (uint32_t)msg[idx] * orc_delta(P);
    c[n] = b;
  }
}

/* phase = b - <a, s> mod q                                             */
void orc_phase(uint32_t n, const uint32_t *lwe_key, const uint32_t *ct, uint64_t count,
               uint32_t *phase) {
  for (uint64_t idx = 0; idx < count; ++idx) {
    const uint32_t *c = ct + idx * (n + 1u);
    uint32_t ph = c[n];
    for (uint32_t t = 0; t < n; ++t) ph -= c[t] * lwe_key[t];
    phase[idx] = ph;
  }
}

/* m = round(phase / Delta) mod 2p, returned as a signed value in [-p, p). */
void orc_decrypt(const orc_params *P, const uint32_t *lwe_key, const uint32_t *ct, uint64_t count,
                 int32_t *msg) {
  const uint32_t log2_delta = 31u - P->log2_p;
  const int32_t p = 1 << P->log2_p;
  for (uint64_t idx = 0; idx < count; ++idx) {
    uint32_t ph;
    orc_phase(P->n, lwe_key, ct + idx * (P->n + 1u), 1, &ph);
    uint32_t m = (uint32_t)(ph + (1u << (log2_delta - 1u))) >> log2_delta; /* [0, 2p) */
    int32_t s = (int32_t)m;
    if (s >= p) s -= 2 * p;
    msg[idx] = s;
  }
}

/* GLWE phase B - sum_j A_j * S_j (used by the tests)                   */
void orc_glwe_phase(const orc_params *P, const uint32_t *glwe_key, const uint32_t *glwe,
                    uint32_t *phase) {
  const uint32_t N = P->N, k = P->k;
  uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * N);
  for (uint32_t c = 0; c < N; ++c) phase[c] = glwe[(uint64_t)k * N + c];
  for (uint32_t j = 0; j < k; ++j) {
    orc_negacyclic_mul(glwe + (uint64_t)j * N, glwe_key + (uint64_t)j * N, N, tmp);
    for (uint32_t c = 0; c < N; ++c) phase[c] -= tmp[c];
  }
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* Test polynomial (paper 2.1, Initialization, read with centred boxes).
 * f gives p values f(u), u in [0,p), as signed integers of Z_{2p}.
 * coeffs[c] = f(round(c*p/N)) for round(c*p/N) < p, else -f(0).        */
void orc_lut_coeffs(const orc_params *P, const int32_t *f, int32_t *coeffs) {
  const uint32_t N = P->N, p = 1u << P->log2_p;
  for (uint32_t c = 0; c < N; ++c) {
    uint32_t u = (c * p + N / 2u) / N;
    coeffs[c] = (u < p) ? f[u] : -f[0];
  }
}

void orc_test_poly(const orc_params *P, const int32_t *f, uint32_t *tv) {
  int32_t *co = (int32_t *)malloc(sizeof(int32_t) * P->N);
  orc_lut_coeffs(P, f, co);
  for (uint32_t c = 0; c < P->N; ++c) tv[c] = (uint32_t)co[c] * orc_delta(P);
  free(co);
}

/* External product GLWE x GGSW (paper 2.1, GSW):
 * out_comp = sum_{j, lam} Dec_{j,lam}(glwe_j) * ggsw[(j,lam)][comp].    */
void orc_external_product(const orc_params *P, const uint32_t *ggsw, const uint32_t *glwe,
                          uint32_t *out) {
  const uint32_t N = P->N, k = P->k, l = P->l;
  int32_t *dig = (int32_t *)malloc(sizeof(int32_t) * (uint64_t)(k + 1u) * l * N);
  int32_t tmpd[32];
  for (uint32_t j = 0; j <= k; ++j)
    for (uint32_t c = 0; c < N; ++c) {
      orc_decompose(glwe[(uint64_t)j * N + c], P->log2_bg, l, tmpd);
      for (uint32_t lam = 0; lam < l; ++lam) dig[((uint64_t)j * l + lam) * N + c] = tmpd[lam];
    }
  for (uint64_t c = 0; c < (uint64_t)(k + 1u) * N; ++c) out[c] = 0;
  for (uint32_t row = 0; row < (k + 1u) * l; ++row)
    for (uint32_t comp = 0; comp <= k; ++comp)
      orc_negacyclic_mul_acc_signed(dig + (uint64_t)row * N,
                                    ggsw + ((uint64_t)row * (k + 1u) + comp) * N, N,
                                    out + (uint64_t)comp * N);
  free(dig);
}

/* Blind rotation (paper 2.1, Initialization + Blind Rotation):
 * ACC = (0, X^{-b~} TV); for i < n: ACC += ExtProd(ek_i, X^{a~_i} ACC - ACC)
 * so that ACC ends at X^{-(b~ - sum a~_i s_i)} TV.                      */
void orc_blind_rotate(const orc_params *P, const uint32_t *bsk, const uint32_t *ct,
                      const uint32_t *tv, uint32_t *acc) {
  const uint32_t n = P->n, k = P->k, N = P->N, l = P->l;
  const uint64_t glwe_sz = (uint64_t)(k + 1u) * N;
  const uint64_t ggsw_sz = (uint64_t)(k + 1u) * l * glwe_sz;
  uint32_t *diff = (uint32_t *)malloc(sizeof(uint32_t) * glwe_sz);
  uint32_t *prod = (uint32_t *)malloc(sizeof(uint32_t) * glwe_sz);
  uint32_t bbar = orc_mod_switch(ct[n], N);
  for (uint64_t c = 0; c < glwe_sz; ++c) acc[c] = 0;
  orc_poly_rotate(tv, N, (2u * N - bbar) % (2u * N), acc + (uint64_t)k * N);
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t abar = orc_mod_switch(ct[i], N);
    for (uint32_t j = 0; j <= k; ++j) {
      orc_poly_rotate(acc + (uint64_t)j * N, N, abar, diff + (uint64_t)j * N);
      for (uint32_t c = 0; c < N; ++c) diff[(uint64_t)j * N + c] -= acc[(uint64_t)j * N + c];
    }
    orc_external_product(P, bsk + (uint64_t)i * ggsw_sz, diff, prod);
    for (uint64_t c = 0; c < glwe_sz; ++c) acc[c] += prod[c];
  }
  free(diff);
  free(prod);
}

/* Sample extraction (paper 2.1): LWE under z = (S_0, ..., S_{k-1}) from
 * coefficient 0: a'_{jN} = A_j[0], a'_{jN+c} = -A_j[N-c], b' = B[0].     */
void orc_sample_extract(const orc_params *P, const uint32_t *acc, uint32_t *big) {
  const uint32_t N = P->N, k = P->k;
  for (uint32_t j = 0; j < k; ++j) {
    const uint32_t *A = acc + (uint64_t)j * N;
    big[(uint64_t)j * N] = A[0];
    for (uint32_t c = 1; c < N; ++c) big[(uint64_t)j * N + c] = (uint32_t)0u - A[N - c];
  }
  big[(uint64_t)k * N] = acc[(uint64_t)k * N];
}

/* Key switching LWE_z -> LWE_s (paper 2.1):
 * out = (0, b') - sum_i sum_lam d_{i,lam} ksk[i][lam].                  */
void orc_key_switch(const orc_params *P, const uint32_t *ksk, const uint32_t *big,
                    uint32_t *out) {
  const uint32_t n = P->n, kN = P->k * P->N;
  int32_t d[32];
  for (uint32_t c = 0; c < n; ++c) out[c] = 0;
  out[n] = big[kN];
  for (uint32_t i = 0; i < kN; ++i) {
    orc_decompose(big[i], P->log2_bks, P->l_ks, d);
    for (uint32_t lam = 0; lam < P->l_ks; ++lam) {
      const uint32_t *row = ksk + ((uint64_t)i * P->l_ks + lam) * (n + 1u);
      uint32_t dl = (uint32_t)d[lam];
      for (uint32_t c = 0; c <= n; ++c) out[c] -= dl * row[c];
    }
  }
}

/* Programmable bootstrapping (paper Thm 2.1 and
 * bootstrapping = KeySwitch o Extract o BlindRotate o Initialize), from the
 * message space p_in = 2^P->log2_p of the input into the spaces of the
 * outputs: table j is written in the encoding Delta_j = 2^(31 - log2_p_out[j])
 * (the dynamic message space of DiNN that the paper adopts, 5.2: a
 * bootstrap reads its input with the boxes of one space and may write its
 * result in another).
 * L = 1: one LUT, test polynomial TV = Delta_0 * coeffs(f).
 * L = 2: multi-value reading of the two PBS per LIF neuron (FHE-Fire and
 *        FHE-Reset, paper 4.2): one blind rotation of
 *        TV0 = (Delta_min / 2) sum X^i, Delta_min = min_j Delta_j, then
 *        ACC_j = r_j * ACC with r_j = (Delta_j / Delta_min) (1 - X) coeffs(f_j),
 *        because (1 - X) sum X^i = 2 mod X^N + 1 gives
 *        r_j * TV0 = Delta_j coeffs(f_j).
 * luts: L x p_in signed values; out: L consecutive LWE_s ciphertexts.    */
void orc_pbs_spaces(const orc_params *P, const uint32_t *bsk, const uint32_t *ksk,
                    const uint32_t *ct, const int32_t *luts, uint32_t L,
                    const uint32_t *log2_p_out, uint32_t *out) {
  const uint32_t N = P->N, k = P->k, n = P->n;
  const uint32_t p = 1u << P->log2_p;
  const uint64_t glwe_sz = (uint64_t)(k + 1u) * N;
  uint32_t *tv = (uint32_t *)malloc(sizeof(uint32_t) * N);
  uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * glwe_sz);
  uint32_t *accj = (uint32_t *)malloc(sizeof(uint32_t) * glwe_sz);
  uint32_t *big = (uint32_t *)malloc(sizeof(uint32_t) * ((uint64_t)k * N + 1u));
  uint32_t *rj = (uint32_t *)malloc(sizeof(uint32_t) * N);
  int32_t *co = (int32_t *)malloc(sizeof(int32_t) * N);
  if (L == 1u) {
    const uint32_t delta_out = 1u << (31u - log2_p_out[0]);
    orc_lut_coeffs(P, luts, co);
    for (uint32_t c = 0; c < N; ++c) tv[c] = (uint32_t)co[c] * delta_out;
    orc_blind_rotate(P, bsk, ct, tv, acc);
    orc_sample_extract(P, acc, big);
    orc_key_switch(P, ksk, big, out);
  } else {
    uint32_t log2_p_max = 0;
    for (uint32_t j = 0; j < L; ++j)
      if (log2_p_out[j] > log2_p_max) log2_p_max = log2_p_out[j];
    const uint32_t half_delta_min = 1u << (30u - log2_p_max);
    for (uint32_t c = 0; c < N; ++c) tv[c] = half_delta_min;
    orc_blind_rotate(P, bsk, ct, tv, acc);
    for (uint32_t j = 0; j < L; ++j) {
      const uint32_t scale = 1u << (log2_p_max - log2_p_out[j]);  /* Delta_j / Delta_min */
      orc_lut_coeffs(P, luts + (uint64_t)j * p, co);
      rj[0] = scale * ((uint32_t)co[0] + (uint32_t)co[N - 1u]);
      for (uint32_t c = 1; c < N; ++c) rj[c] = scale * ((uint32_t)co[c] - (uint32_t)co[c - 1u]);
      for (uint32_t comp = 0; comp <= k; ++comp)
        orc_negacyclic_mul(rj, acc + (uint64_t)comp * N, N, accj + (uint64_t)comp * N);
      orc_sample_extract(P, accj, big);
      orc_key_switch(P, ksk, big, out + (uint64_t)j * (n + 1u));
    }
  }
  free(tv);
  free(acc);
  free(accj);
  free(big);
  free(rj);
  free(co);
}

/* Bootstrapping within the input's own message space (every table written
 * with the input's Delta).                                               */
void orc_pbs(const orc_params *P, const uint32_t *bsk, const uint32_t *ksk, const uint32_t *ct,
             const int32_t *luts, uint32_t L, uint32_t *out) {
  uint32_t same[2] = {P->log2_p, P->log2_p};
  orc_pbs_spaces(P, bsk, ksk, ct, luts, L, same, out);
}

/* Batched PBS over independent ciphertexts with plain worker threads (the
 * paper's "parallel computing" of bootstraps, 5.3).  out layout:
 * [L][count][n+1].                                                       */
typedef struct {
  const orc_params *P;
  const uint32_t *bsk, *ksk, *ct;
  const int32_t *luts;
  uint32_t L;
  const uint32_t *log2_p_out;
  uint32_t *out;
  uint64_t count, begin, end;
} orc_batch_job;

static void *orc_batch_worker(void *arg) {
  orc_batch_job *J = (orc_batch_job *)arg;
  const uint32_t w = J->P->n + 1u;
  uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (uint64_t)J->L * w);
  for (uint64_t idx = J->begin; idx < J->end; ++idx) {
    orc_pbs_spaces(J->P, J->bsk, J->ksk, J->ct + idx * w, J->luts, J->L, J->log2_p_out, tmp);
    for (uint32_t j = 0; j < J->L; ++j)
      memcpy(J->out + ((uint64_t)j * J->count + idx) * w, tmp + (uint64_t)j * w,
             sizeof(uint32_t) * w);
  }
  free(tmp);
  return NULL;
}

/* log2_p_out: L output spaces, or NULL for the input's own space.        */
void orc_pbs_batch(const orc_params *P, const uint32_t *bsk, const uint32_t *ksk,
                   const uint32_t *ct, uint64_t count, const int32_t *luts, uint32_t L,
                   const uint32_t *log2_p_out, uint32_t *out, int nthreads) {
  uint32_t same[2] = {P->log2_p, P->log2_p};
  if (!log2_p_out) log2_p_out = same;
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > count) nthreads = (int)(count ? count : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  orc_batch_job *jobs = (orc_batch_job *)malloc(sizeof(orc_batch_job) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].P = P;
    jobs[t].bsk = bsk;
    jobs[t].ksk = ksk;
    jobs[t].ct = ct;
    jobs[t].luts = luts;
    jobs[t].L = L;
    jobs[t].log2_p_out = log2_p_out;
    jobs[t].out = out;
    jobs[t].count = count;
    jobs[t].begin = count * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].end = count * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, orc_batch_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------ */
/* Homomorphic WeightSum (paper 4.1, Eq. noise grows):
 * sum_j w_j LWE(x_j) = LWE(sum_j w_j x_j); bias (nullable) adds
 * Delta * bias_i to the body (a trivial encryption of the constant).    */
void orc_lwe_linear(uint32_t n, uint32_t log2_p, const int32_t *W, uint64_t M, uint64_t K,
                    const int32_t *bias, const uint32_t *ct_in, uint32_t *ct_out) {
  const uint32_t w = n + 1u;
  const uint32_t delta = 1u << (31u - log2_p);
  for (uint64_t i = 0; i < M; ++i) {
    uint32_t *o = ct_out + i * w;
    for (uint32_t c = 0; c < w; ++c) o[c] = 0;
    for (uint64_t j = 0; j < K; ++j) {
      uint32_t wij = (uint32_t)W[i * K + j];
      const uint32_t *x = ct_in + j * w;
      for (uint32_t c = 0; c < w; ++c) o[c] += wij * x[c];
    }
    if (bias) o[n] += (uint32_t)bias[i] * delta;
  }
}

/* Convolution as WeightSum over each receptive field (paper 4.1, conv
 * layers).  ct_in [cin][h][w][n+1]; W [cout][cin][kh][kw]; zero padding
 * reads trivial encryptions of 0; ct_out [cout][ho][wo][n+1].            */
void orc_lwe_conv2d(uint32_t n, uint32_t log2_p, uint32_t cin, uint32_t h, uint32_t wd,
                    uint32_t cout, uint32_t kh, uint32_t kw, uint32_t stride, uint32_t pad,
                    const int32_t *W, const int32_t *bias, const uint32_t *ct_in,
                    uint32_t *ct_out) {
  const uint32_t w = n + 1u;
  const uint32_t delta = 1u << (31u - log2_p);
  const uint32_t ho = (h + 2u * pad - kh) / stride + 1u;
  const uint32_t wo = (wd + 2u * pad - kw) / stride + 1u;
  for (uint32_t co = 0; co < cout; ++co)
    for (uint32_t y = 0; y < ho; ++y)
      for (uint32_t x = 0; x < wo; ++x) {
        uint32_t *o = ct_out + (((uint64_t)co * ho + y) * wo + x) * w;
        for (uint32_t c = 0; c < w; ++c) o[c] = 0;
        for (uint32_t ci = 0; ci < cin; ++ci)
          for (uint32_t dy = 0; dy < kh; ++dy)
            for (uint32_t dx = 0; dx < kw; ++dx) {
              int64_t iy = (int64_t)y * stride + dy - pad;
              int64_t ix = (int64_t)x * stride + dx - pad;
              if (iy < 0 || ix < 0 || iy >= (int64_t)h || ix >= (int64_t)wd) continue;
              uint32_t wt = (uint32_t)W[(((uint64_t)co * cin + ci) * kh + dy) * kw + dx];
              const uint32_t *src = ct_in + (((uint64_t)ci * h + (uint64_t)iy) * wd + (uint64_t)ix) * w;
              for (uint32_t c = 0; c < w; ++c) o[c] += wt * src[c];
            }
        if (bias) o[n] += (uint32_t)bias[co] * delta;
      }
}

/* Trivial constant addition: b += Delta * value (the +1 of FHE-Fire, the
 * centring offset p/2 before each LIF bootstrap).                        */
void orc_lwe_add_const(uint32_t n, uint32_t log2_p, uint32_t *ct, uint64_t count, int32_t value) {
  const uint32_t delta = 1u << (31u - log2_p);
  for (uint64_t i = 0; i < count; ++i) ct[i * (n + 1u) + n] += (uint32_t)value * delta;
}
