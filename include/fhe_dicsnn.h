/*
 * fhe_dicsnn.h -- C ABI of the GB300 (sm_103a) FHE-DiCSNN hot path.
 *
 * The library evaluates the paper's encrypted spiking network (FHE-DiCSNN):
 * TFHE programmable bootstrapping of LWE ciphertexts over the uint32 torus
 * (paper 2.1, Thm 2.1), the integer-weighted LWE sums that feed it (4.1,
 * Eq. "noise grows"), and the LIF neuron's Fire/Reset as bootstrap test
 * polynomials (4.2, Eqs. FHE-Fire / FHE-Reset; discretized LIF of Thm 3.2).
 *
 * Conventions shared by every entry point
 *  - Torus: q = 2^32; ciphertext words are uint32_t and wrap modulo 2^32.
 *  - LWE ciphertext: n+1 consecutive uint32_t, mask a[0..n-1] then body b.
 *    Arrays of ciphertexts are dense [count][n+1] (no padding).
 *  - Messages: p = 2^log2_p with one padding bit, Delta = 2^(31 - log2_p);
 *    a message m is encoded as m * Delta (mod 2^32), so messages live in
 *    Z_{2p} and decrypt to the signed range [-p, p).
 *  - Pointers documented "device" must be CUDA device memory of the current
 *    device (for instance torch tensors' data_ptr()); "host" pointers are
 *    ordinary host memory.  The caller owns every buffer it passes; the
 *    library owns the opaque handles it returns.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work is enqueued asynchronously on it; the functions return
 *    once the work is enqueued, except where stated.
 *  - Errors: functions return 0 (FHE_OK) or a negative FHE_E* code; they
 *    never throw.  An asynchronous kernel failure is reported by the next
 *    call that synchronizes (fhe_status, fhe_keys_export, fhe_snn_infer).
 *  - Handles are not thread-safe: a fhe_keys (and its workspace) must not be
 *    used by two calls that overlap in time.
 */
#ifndef FHE_DICSNN_H
#define FHE_DICSNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FHE_OK 0
#define FHE_EINVAL (-1)        /* bad argument, size or parameter set          */
#define FHE_ENOMEM (-2)        /* device or host allocation failed             */
#define FHE_ECUDA (-3)         /* a CUDA runtime call or kernel failed         */
#define FHE_ETIMEOUT (-4)      /* a bounded device wait gave up (status word)  */
#define FHE_EUNSUPPORTED (-5)  /* valid but not implemented on this path       */

/* Blind-rotation variants accepted by fhe_pbs_batch / fhe_snn_create. */
#define FHE_VARIANT_EXACT 0 /* exact uint32 external product on CUDA cores (IMAD) */
#define FHE_VARIANT_TC 1    /* exact external product on tcgen05 tensor cores,
                               key split into 8-bit limbs (fp16 operands, fp32
                               accumulation kept below 2^24)                 */
#define FHE_VARIANT_FFT 2   /* conventional FP64 negacyclic FFT product (the
                               paper's "FFT technology", 5.3): NOT bit-exact,
                               outputs rounded from doubles; see
                               fhe_fft_max_error                              */
#define FHE_VARIANT_AUTO 3  /* EXACT or TC per launch by batch size (same bits
                               either way): tensor cores from the key
                               handle's crossover up (fhe_pbs_autotune)       */

/* Which key to export (fhe_keys_export / fhe_keys_size). */
#define FHE_KEY_LWE 0  /* s:   uint32_t[n], entries 0/1                        */
#define FHE_KEY_GLWE 1 /* S:   uint32_t[k*N], entries 0/1                      */
#define FHE_KEY_BSK 2  /* ek:  uint32_t[n][(k+1)*l][k+1][N]: row (j, lam) at
                          index j*l + lam-1 is a GLWE encryption of zero with
                          s_i * 2^(32 - lam*log2_bg) added to component j  */
#define FHE_KEY_KSK 3  /* ksk: uint32_t[k*N][l_ks][n+1]: LWE_s(z_i * 2^(32 -
                          lam*log2_bks)) for lam = 1..l_ks                   */

/* TFHE parameter set.  Noise standard deviations are powers of two given by
 * their negative log2 in torus units (sigma = 2^-x); x >= 64 means no noise.
 * Supported: k = 1; N in {256, 512, 1024, 2048}; log2_bg * l <= 32,
 * log2_bg <= 15, l <= 4; log2_bks * l_ks <= 32, log2_bks <= 7; 1 <= log2_p
 * <= 10 with 2p <= N; 1 <= n <= 2048.                                     */
typedef struct fhe_params {
  uint32_t n;        /* LWE dimension                                        */
  uint32_t k;        /* GLWE dimension (must be 1)                           */
  uint32_t N;        /* polynomial size                                      */
  uint32_t log2_bg;  /* gadget base Bg = 2^log2_bg                           */
  uint32_t l;        /* gadget levels                                        */
  uint32_t log2_bks; /* key-switching base                                   */
  uint32_t l_ks;     /* key-switching levels                                 */
  uint32_t log2_p;   /* message modulus p = 2^log2_p                         */
  int32_t lwe_noise_log2;
  int32_t glwe_noise_log2;
} fhe_params;

typedef struct fhe_keys fhe_keys; /* opaque: device keys + PBS workspace   */
typedef struct fhe_lut fhe_lut;   /* opaque: device test polynomial(s)     */
typedef struct fhe_snn fhe_snn;   /* opaque: encrypted network + state     */

/* Human-readable text of an FHE_E* code (static storage). */
const char *fhe_strerror(int code);

/* Key generation from a seed (paper 2.1: LWE/RLWE keys, bootstrapping key
 * ek = (RGSW(X^s_1), ..., RGSW(X^s_n)), key-switching key).  All draws are
 * SplitMix64 outputs addressed by (seed, domain, index), so the keys are a
 * pure function of (params, seed).  Runs on the current CUDA device, on
 * `stream`, and allocates the device keys plus a PBS workspace for
 * `max_batch` ciphertexts (0 = 16384).  *out receives the handle.
 * Errors: FHE_EINVAL (NULL pointer, unsupported parameter set),
 * FHE_ENOMEM, FHE_ECUDA. */
int fhe_keygen_from_seed(const fhe_params *params, uint64_t seed, size_t max_batch,
                         void *stream, fhe_keys **out);

/* Free a key handle (synchronizes the device first).  NULL is ignored. */
void fhe_keys_free(fhe_keys *keys);

/* Parameter set the keys were generated for. */
int fhe_keys_params(const fhe_keys *keys, fhe_params *out);

/* Size in bytes of key `which` (FHE_KEY_*); 0 on a bad argument. */
size_t fhe_keys_size(const fhe_keys *keys, int which);

/* Copy key `which` in the layout documented at FHE_KEY_* to host memory
 * `host_dst` of `bytes` bytes (must equal fhe_keys_size).  Synchronizes.
 * Errors: FHE_EINVAL, FHE_ECUDA. */
int fhe_keys_export(const fhe_keys *keys, int which, void *host_dst, size_t bytes);

/* LWE encryption (paper 2.1, LWE): ct[i] = (a, <a,s> + e + msg[i]*Delta).
 * msg: device int32[count], any integer (reduced mod 2p).  ct: device
 * uint32[count][n+1].  Masks and noise are draws of (seed, index i), so the
 * same seed re-encrypts identically.  Errors: FHE_EINVAL, FHE_ECUDA. */
int fhe_encrypt(const fhe_keys *keys, const int32_t *msg, size_t count, uint64_t seed,
                uint32_t *ct, void *stream);

/* LWE decryption: msg[i] = round((b - <a,s>) / Delta) as a signed value in
 * [-p, p).  ct: device uint32[count][n+1]; msg: device int32[count]. */
int fhe_decrypt(const fhe_keys *keys, const uint32_t *ct, size_t count, int32_t *msg,
                void *stream);

/* Homomorphic WeightSum for a fully connected layer (paper 4.1, Eq. "noise
 * grows"): for every batch item b and output i,
 *   ct_out[b][i] = sum_j W[i][j] * ct_in[b][j]  (+ bias[i] * Delta on b),
 * componentwise modulo 2^32.  W: device int32[M][K] row-major; bias: device
 * int32[M] or NULL; ct_in: device uint32[batch][K][n+1]; ct_out: device
 * uint32[batch][M][n+1] (must not alias ct_in). */
int fhe_lwe_linear(uint32_t n, uint32_t log2_p, const int32_t *W, size_t M, size_t K,
                   const int32_t *bias, const uint32_t *ct_in, size_t batch, uint32_t *ct_out,
                   void *stream);

/* Convolution as WeightSum over receptive fields (paper 4.1; conv layer of
 * 3.1).  ct_in: device uint32[batch][cin][h][w][n+1]; W: device
 * int32[cout][cin][kh][kw]; bias: device int32[cout] or NULL; zero padding
 * reads trivial encryptions of 0; ct_out: device
 * uint32[batch][cout][ho][wo][n+1] with ho = (h + 2 pad - kh)/stride + 1. */
int fhe_lwe_conv2d(uint32_t n, uint32_t log2_p, const int32_t *W, uint32_t cin, uint32_t h,
                   uint32_t w, uint32_t cout, uint32_t kh, uint32_t kw, uint32_t stride,
                   uint32_t pad, const int32_t *bias, const uint32_t *ct_in, size_t batch,
                   uint32_t *ct_out, void *stream);

/* Bootstrap look-up tables.  f: host int32[L][p], f[j][u] is the value
 * (any integer, reduced mod 2p) the bootstrap returns for message u in
 * [0, p); messages u in [p, 2p) return -f[j][u - p] (negacyclic half of
 * Thm 2.1).  L = 1: the test polynomial is Delta * f on centred boxes
 * round(i p / N).  L = 2: one blind rotation serves both tables (the
 * FHE-Fire / FHE-Reset pair of 4.2) through the multi-value split
 * ACC_j = (1 - X) coeffs(f_j) * ACC of the constant test polynomial
 * (Delta/2) sum X^i.  The handle uploads the tables once (synchronous). */
int fhe_lut_create(const fhe_keys *keys, const int32_t *f, uint32_t L, fhe_lut **out);
void fhe_lut_free(fhe_lut *lut);

/* Tables between message spaces (the dynamic message space of DiNN, which
 * the paper adopts in 5.2, Parameters Selection): group g reads its input
 * in Z_{2 p_g}, p_g = 2^log2_p_in[g] (boxes round(i p_g / N), padding
 * Delta_in = 2^31 / p_g), and writes table j with the encoding
 * Delta = 2^(31 - log2_p_out[g*L + j]), i.e. ct_out decrypts to f_j(m) in
 * Z_{2 p_out}.  A multi-value group rotates TV0 = (Delta_min / 2) sum X^i,
 * Delta_min the group's smallest output Delta, and applies
 * r_j = (Delta_j / Delta_min) (1 - X) coeffs(f_j).  f: host int32, the
 * groups one after another, group g holding L tables of p_g values.
 * groups (1 .. FHE_LUT_MAX_GROUPS) > 1 only with L = 2; fhe_pbs_batch_groups
 * says which ciphertexts use which group.  fhe_lut_create(keys, f, L, out)
 * is one group in the key's space.  Errors: FHE_EINVAL (null pointer, L not
 * 1 or 2, group count out of range, a log2 value outside [1, 10], or
 * 2 p_in > N), FHE_ENOMEM, FHE_ECUDA. */
#define FHE_LUT_MAX_GROUPS 8
int fhe_lut_create_spaces(const fhe_keys *keys, const int32_t *f, uint32_t L, uint32_t groups,
                          const uint32_t *log2_p_in, const uint32_t *log2_p_out, fhe_lut **out);

/* Programmable bootstrapping of a batch (paper Thm 2.1, bootstrapping =
 * KeySwitch o Extract o BlindRotate o Initialize): for every input i and
 * table j, ct_out[j][i] = LWE_s(f_j(m_i)).  ct_in: device uint32[count][n+1];
 * ct_out: device uint32[L][count][n+1] (must not alias ct_in).  variant:
 * FHE_VARIANT_EXACT, FHE_VARIANT_TC or FHE_VARIANT_AUTO (bit-identical), or
 * FHE_VARIANT_FFT (decrypts the same, not bit-identical).  Uses the key
 * handle's workspace; batches above its capacity run in chunks.
 * Errors: FHE_EINVAL, FHE_EUNSUPPORTED (variant not built for these
 * parameters), FHE_ECUDA. */
int fhe_pbs_batch(fhe_keys *keys, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
                  uint32_t *ct_out, int variant, void *stream);

/* fhe_pbs_batch with a grouped table set (fhe_lut_create_spaces): inputs
 * [seg_end[g-1], seg_end[g]) use group g (seg_end[-1] = 0; the last group
 * runs to count).  seg_end: host size_t[groups - 1], non-decreasing, each
 * <= count (empty groups allowed); NULL only for one group.  One launch
 * serves every group (a network bootstraps all its layers at once).
 * fhe_pbs_batch and fhe_pbs_batch_noalloc reject grouped sets.
 * Errors: as fhe_pbs_batch, FHE_EINVAL for bad segment ends. */
int fhe_pbs_batch_groups(fhe_keys *keys, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
                         const size_t *seg_end, uint32_t *ct_out, int variant, void *stream);

/* Autotuner of FHE_VARIANT_AUTO (no counterpart in the paper): times the
 * CUDA-core and tensor-core blind rotations on this device for batches of
 * 16, 32, ... ciphertexts (up to 4096 and the workspace), and stores in the
 * key handle the smallest batch from which the tensor-core path is faster
 * (1 when it is already faster at 16: a launch below one tile costs one
 * tile; written to *tc_min_batch; UINT64_MAX when the tensor-core path is not
 * built for these parameters).  Before tuning, AUTO uses tensor cores for
 * every batch.  It also times the tile shapes of the tensor-core path (a
 * 256-ciphertext tile on a cluster of 4, 8 or 16 SMs): each larger shape
 * against the next smaller one at 1, 4 and the most tiles that fit at once
 * in the larger shape, keeping the larger one only up to where it was
 * measured no slower (before tuning: whenever the batch fits).
 * Synchronous; allocates and frees temporary buffers; takes seconds (longest
 * at N = 2048).  Errors: FHE_EINVAL, FHE_ENOMEM, FHE_ECUDA, FHE_ETIMEOUT. */
int fhe_pbs_autotune(fhe_keys *keys, uint64_t *tc_min_batch, void *stream);

/* Exactness plan of the tensor-core blind rotation for a parameter set (no
 * counterpart in the paper; host only, no device needed).  The external
 * product runs on fp16 tensor cores with fp32 accumulation: key words are
 * four balanced 8-bit limbs (|limb| <= 128), gadget digits are balanced
 * (|d| <= Bg/2) or, when Bg/2 * 128 * N exceeds 2^24, split into two
 * sub-digits of sub_shift bits; the fp32 accumulator is drained after every
 * chunk_rows digit rows, so that no partial sum exceeds max_partial <= 2^24
 * and every fp32 result is the exact integer.  available = 0 when the path
 * does not cover the set (N not 1024 or 2048, digits that do not fit).
 * Errors: FHE_EINVAL (null pointer, parameters the library does not support
 * at all, as fhe_keygen_from_seed). */
typedef struct fhe_tc_plan {
  int32_t available;     /* 1: FHE_VARIANT_TC covers these parameters        */
  uint32_t key_rows;     /* (k+1) l GGSW rows                                */
  uint32_t digit_rows;   /* key_rows, doubled when digits are split          */
  uint32_t sub_shift;    /* 0, or the bits of the low sub-digit              */
  uint32_t max_digit;    /* largest |digit| (or |sub-digit|) multiplied      */
  uint32_t chunk_rows;   /* digit rows accumulated in fp32 per drain         */
  uint64_t max_partial;  /* max_digit * 128 * chunk_rows * N                 */
} fhe_tc_plan;
int fhe_tc_plan_query(const fhe_params *params, fhe_tc_plan *out);

/* What FHE_VARIANT_AUTO and the tensor-core path currently use: the batch
 * size from which AUTO picks tensor cores (UINT64_MAX: never) and the most
 * 256-ciphertext tiles a batch may have to run on clusters of 8, of 16, and
 * spread over two clusters of 16 (the device limit before fhe_pbs_autotune;
 * 0: never, e.g. the device refused a cooperative clustered launch; -1: the
 * device limit, not yet queried).  tc_cl16_tiles and tc_split_tiles may be
 * NULL.  Host only.  Errors: FHE_EINVAL. */
int fhe_pbs_tuning(const fhe_keys *keys, uint64_t *tc_min_batch, int32_t *tc_cl8_tiles,
                   int32_t *tc_cl16_tiles, int32_t *tc_split_tiles);

/* Options of the tensor-core path, for measurements and tuning (no
 * counterpart in the paper); results are bit-identical under every option.
 *   FHE_TC_OPT_CLUSTER: 4, 8 or 16 CTAs per 256-ciphertext tile for every
 *     batch that fits in one wave of that shape (others use clusters of 4),
 *     32 for each tile spread over two clusters of 16 (a cooperative launch;
 *     batches of up to half the 16-CTA clusters, else clusters of 16), or 0
 *     for the tuned rule (32 up to its limit, then 16, 8, 4).
 *   FHE_TC_OPT_MULTICAST: 1 = digit tiles copied to all CTAs that hold the
 *     same rows by cluster-multicast copies (each stage refilled once every
 *     pair of the cluster is done with it), 0 = each CTA copies whole tiles
 *     (the pairs run decoupled), -1 = the build's default (multicast in the
 *     single-GPU library; the replica library has no multicast and returns
 *     FHE_EUNSUPPORTED for 1).  The split shape always copies per CTA.
 *   FHE_TC_OPT_L2_HINTS: 1 = the digit operand is stored and copied with an
 *     L2 evict-last cache policy, 0 = no policy, -1 = the default (none).
 * Host only; applies from the next call.  Errors: FHE_EINVAL (unknown
 * option or value), FHE_EUNSUPPORTED. */
#define FHE_TC_OPT_CLUSTER 0
#define FHE_TC_OPT_MULTICAST 1
#define FHE_TC_OPT_L2_HINTS 2
int fhe_pbs_set_tc_option(fhe_keys *keys, int option, int value);

/* Bootstrapping that allocates nothing (no counterpart in the paper: an
 * integration aid).  Some callers cannot call cudaMalloc at the point where
 * they bootstrap: a host framework that owns the whole device memory budget
 * through its own allocator, or a latency-critical serving loop where an
 * allocation (which can synchronize the device or fail under memory pressure)
 * is not acceptable.  This call computes exactly what fhe_pbs_batch computes
 * with FHE_VARIANT_EXACT (bit-identical outputs, same argument layouts), but
 * keeps its intermediate ciphertexts in one fixed scratch array compiled into
 * the library (FHE_PBS_NOALLOC_MAX_WORDS 32-bit words = 4 MiB, held by every
 * GPU that loads the library until the process exits) instead of the key
 * handle's workspace.  The caller still provides inputs, outputs, keys and
 * table, created beforehand.
 * Limit: L * count * (k*N + 1) <= FHE_PBS_NOALLOC_MAX_WORDS, e.g. count <= 511
 * for two tables at N = 1024; larger batches return FHE_EINVAL (split them).
 * The first call on a device resolves the scratch address on that device
 * (make that first call before any stream capture).  With CUDA's lazy module
 * loading (the default), that first call is also where the library's device
 * code, and with it the 4 MiB array, is loaded onto the device: "allocates
 * nothing" holds from the first call on; a caller that must not see even
 * that can make one call with count = 1 at start-up.  All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other threads)
 * race on it and must be serialized by the caller.
 * Errors: FHE_EINVAL (bad argument, batch above the limit, keys of another
 * device), FHE_ECUDA. */
#define FHE_PBS_NOALLOC_MAX_WORDS (1u << 20)
int fhe_pbs_batch_noalloc(const fhe_keys *keys, const uint32_t *ct_in, size_t count,
                          const fhe_lut *lut, uint32_t *ct_out, void *stream);

/* Largest distance to the nearest integer of any external-product output of
 * the FFT variant since the last reset (units of 2^-32 torus, i.e. of one
 * uint32 step): below 0.5 every output was rounded to the exact value.
 * Synchronizes; reset != 0 clears it.  0.0 before the first FFT call. */
int fhe_fft_max_error(fhe_keys *keys, double *max_err, int reset);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * thread that waits, with the bounded-wait pattern of the bootstrap kernels,
 * on an mbarrier that nothing completes; after `limit_us` microseconds
 * (1 .. 1e6) it gives up and records FHE_ETIMEOUT in the status word.  Then
 * returns fhe_status(keys, stream), i.e. FHE_ETIMEOUT when the path works.
 * No fault, trap or endless wait is involved. */
int fhe_selftest_timeout(fhe_keys *keys, uint32_t limit_us, void *stream);

/* Device status word: FHE_OK, or FHE_ETIMEOUT if a bounded device wait gave
 * up since the last call.  Synchronizes `stream`, then clears the word. */
int fhe_status(fhe_keys *keys, void *stream);

/* ------------------------------------------------------------------------
 * Encrypted DiCSNN inference (paper 3.1-3.3 network, 4.1-4.2 evaluation,
 * 5.3 client/server flow).  A network is a chain of layers, each a WeightSum
 * (conv or fully connected) followed by a LIF spiking activation layer:
 *   I = WeightSum(x);  H = V + I;
 *   (S, V) = bootstrap(H + p/2) with the FHE-Fire / FHE-Reset tables;
 *   x_next = S;  scores += S of the last layer.
 * The first layer's input is either static (pixel ciphertexts reused every
 * step, the conv output computed once) or a per-step spike train.
 *
 * FHE_LAYER_POISSON (first layer only, static input): the Poisson encoder of
 * 2.3 (Eq. Poisson-coding), S[t] = [x > M_t] per pixel, where M_t is the
 * server's public random matrix of step t (drawn by the caller); one
 * comparison bootstrap per pixel and step (5.1, Table Poisson).  It has no
 * WeightSum and no membrane: with FHE_LIF_MULTI_VALUE the comparison is the
 * Fire table on x - M_t + V_th - 1 (>= V_th exactly when x > M_t); with
 * FHE_LIF_TWO_PBS it is the sign bootstrap of x - M_t - 1, plus 1.
 * Pixel levels and M_t must keep these inputs inside the table's range
 * ([-p/2, p/2) resp. [-p, p)), as Thm 4.1 does for the LIF layers.
 *
 * lif_mode selects how one LIF neuron-step is bootstrapped:
 *  FHE_LIF_MULTI_VALUE: one blind rotation of H + p/2 with a multi-value test
 *    polynomial gives FHE-Fire and FHE-Reset (tables on v in [-p/2, p/2));
 *  FHE_LIF_TWO_PBS: the paper's two bootstraps (4.2, Eq. FHE-Fire and
 *    FHE-Reset) with negacyclic program functions, no centring:
 *    S = bootstrap_sign(H - V_th) + 1 = 2 Spike, V = bootstrap_g(H), valid for
 *    H in [V_th - p, p) (Thm 4.1 with the paper's modulus 2p).  Requires
 *    spike_scale == 2 (the spike value the construction produces).
 */
#define FHE_LAYER_FC 0
#define FHE_LAYER_CONV 1
#define FHE_LAYER_POISSON 2
#define FHE_LIF_MULTI_VALUE 0
#define FHE_LIF_TWO_PBS 1

typedef struct fhe_layer_desc {
  int32_t type;            /* FHE_LAYER_FC, FHE_LAYER_CONV or FHE_LAYER_POISSON */
  const int32_t *weights;  /* HOST int32: FC [out][in]; conv [cout][cin][kh][kw];
                              Poisson: thresholds M [T][in_size]              */
  uint32_t in_size;        /* FC, Poisson: number of inputs                  */
  uint32_t out_size;       /* FC: number of outputs; Poisson: = in_size      */
  uint32_t cin, h, w, cout, kh, kw, stride, pad; /* conv geometry          */
  uint32_t log2_p;         /* the layer's message space p_l = 2^log2_p (DiNN's
                              dynamic message space, 5.2); 0: the key's.  The
                              layer's currents, membranes and bootstrap boxes
                              live in Z_{2 p_l}; its spikes are written in the
                              space of the next layer (the key's for the last
                              layer: the scores).  The first layer reads the
                              input in the key's space: a WeightSum first layer
                              needs p_0 <= p (its weights are applied times
                              p / p_0), a Poisson layer p_0 = p.  Other spaces
                              than the key's need FHE_LIF_MULTI_VALUE and at
                              most FHE_LUT_MAX_GROUPS layers.                 */
} fhe_layer_desc;

typedef struct fhe_snn_desc {
  uint32_t n_layers;
  const fhe_layer_desc *layers; /* host array of n_layers descriptors        */
  int32_t v_th;                 /* LIF threshold V_th (Thm 3.2)               */
  int32_t leak_shift;           /* leak(v) = v >> leak_shift; 0 = IF model    */
  int32_t spike_scale;          /* value of an output spike (1 or 2)         */
  uint32_t T;                   /* time steps                                */
  int32_t static_input;         /* 1: input reused every step (pixels)       */
  uint32_t max_images;          /* capacity: images per inference call       */
  int32_t variant;              /* FHE_VARIANT_* of the bootstraps           */
  int32_t use_graph;            /* bit 0: run each time step as a captured
                                   CUDA graph (fhe_snn_step, and the streamed
                                   steps once every layer is active); bit 1
                                   (FHE_SNN_PROFILE): time the blind
                                   rotations (fhe_snn_profile)               */
  int32_t lif_mode;             /* FHE_LIF_MULTI_VALUE or FHE_LIF_TWO_PBS     */
} fhe_snn_desc;

/* Build a network on `keys` (uploads weights, allocates state for
 * max_images images; synchronous).  Errors: FHE_EINVAL (bad geometry, a
 * Poisson layer that is not the first or without static input, an unknown
 * lif_mode, FHE_LIF_TWO_PBS with spike_scale != 2, a layer message space
 * that breaks the rules of fhe_layer_desc.log2_p), FHE_ENOMEM. */
int fhe_snn_create(fhe_keys *keys, const fhe_snn_desc *desc, fhe_snn **out);
void fhe_snn_free(fhe_snn *net);

/* Number of bootstraps (blind rotations) one inference of one image runs:
 * per step one per neuron (two per LIF neuron with FHE_LIF_TWO_PBS). */
uint64_t fhe_snn_pbs_per_image(const fhe_snn *net);

/* Encrypted inference of `n_images` images (<= max_images).
 * ct_input: uint32 [n_images][n_in][n+1] if static_input, else
 *           [T][n_images][n_in][n+1] (time-major);
 * scores:   uint32 [n_images][n_out][n+1] (encrypted spike counts).
 * If inputs_on_host != 0 both pointers are HOST memory: the call copies the
 * inputs to the device, runs the network and copies the scores back, then
 * synchronizes `stream` (end-to-end client/server round trip, 5.3).
 * Otherwise both are device pointers and the call only enqueues work.
 * Errors: FHE_EINVAL, FHE_ECUDA, FHE_ETIMEOUT. */
int fhe_snn_infer(fhe_snn *net, const uint32_t *ct_input, size_t n_images, uint32_t *scores,
                  int inputs_on_host, void *stream);

/* The same inference split into its steps (fhe_snn_infer = begin, step until
 * it returns 0, end).  Layer-skewed schedule: step tau advances every layer l
 * whose time step t = tau - l lies in [0, T) -- layer l at t needs only layer
 * l-1 at t and itself at t-1 (Thm 3.2 recurrence) -- so one bootstrap launch
 * serves all active layers; an inference is T + n_layers - 1 steps.
 * begin: stages the input (layouts as in fhe_snn_infer) and resets the state.
 * step:  enqueues the next step (its CUDA graph when use_graph bit 0 is set);
 *        returns the number of steps still to run (>= 0) or an FHE_E* code.
 * end:   copies the encrypted scores out (synchronizing when on host). */
int fhe_snn_begin(fhe_snn *net, const uint32_t *ct_input, size_t n_images, int inputs_on_host,
                  void *stream);
int fhe_snn_step(fhe_snn *net, void *stream);
int fhe_snn_end(fhe_snn *net, uint32_t *scores, int inputs_on_host, void *stream);
/* Number of steps of one inference (T + n_layers - 1). */
uint32_t fhe_snn_iterations(const fhe_snn *net);

/* Streamed inference of a sequence of batches (no counterpart in the paper:
 * the serving form of the same computation).  Each push enqueues the T
 * layer-skewed steps that start batch k and, in the same bootstrap launches,
 * advance the layers of the batches still in flight, so that every launch
 * holds every layer's neurons; each push runs exactly one batch's worth of
 * bootstraps.  Batch k's encrypted scores [n_images][n_out][n+1] are written
 * to `scores` (host memory if on_host, device otherwise; the input layout and
 * on_host rule are those of fhe_snn_infer) by copies enqueued on `stream`
 * once the batch completes, during a later push or the flush; host results
 * are valid after `stream` synchronizes.  All batches of a stream have the
 * same n_images (<= max_images).  The caller keeps `scores` valid until the
 * batch completes.  fhe_snn_stream_flush runs the remaining steps so every
 * pushed batch completes, synchronizes `stream` when any destination is host
 * memory (returning the device status), and ends the stream.  While a stream
 * runs, fhe_snn_infer / fhe_snn_begin return FHE_EINVAL (and vice versa).
 * With use_graph bit 0 set, a step in which every layer is active (every
 * step but the stream's first n_layers - 1 and those of the flush) launches
 * exactly the work of the step T * slots later on the same buffers, slots =
 * 1 + ceil((n_layers - 1) / T) being the batches in flight at once: each of
 * those T * slots step kinds is captured as a CUDA graph on its first use
 * and replayed after that (a new n_images or a change of the keys' tuning
 * settings captures them again); the copy of a completed batch's scores to
 * its caller stays outside the graph.  Graph memory is kept until
 * fhe_snn_free;
 * fhe_snn_profile covers the launches since the stream's first push (with
 * profiling on, two events are kept per bootstrap launch of the stream:
 * meant for bounded measurement runs, not for unbounded serving).
 * Errors: FHE_EINVAL, FHE_ENOMEM (first push allocates the stream state),
 * FHE_ECUDA, FHE_ETIMEOUT. */
int fhe_snn_stream_push(fhe_snn *net, const uint32_t *ct_input, size_t n_images, uint32_t *scores,
                        int on_host, void *stream);
int fhe_snn_stream_flush(fhe_snn *net, void *stream);

/* The streamed inference one iteration at a time (no counterpart in the
 * paper: lets a test or a scheduler observe every layer-skewed step of the
 * same code path as fhe_snn_stream_push).  fhe_snn_stream_stage stages the
 * next batch (arguments and rules of fhe_snn_stream_push) without running
 * any step; a batch must be staged before its first step runs (FHE_EINVAL
 * otherwise).  fhe_snn_stream_push = stage + the steps up to the end of the
 * staged batch's T steps.  fhe_snn_stream_iterate runs the next step of the
 * stream (including the last layers' steps after the last staged batch, as
 * the flush does) and returns how many steps can still run without staging
 * (0: nothing ran), or a negative error.
 * fhe_snn_stream_state copies, for batch `batch` (0 = the stream's first
 * batch) while it holds its slot (staged, and fewer than `slots` batches
 * staged after it), layer `layer`'s latest spikes (FHE_STATE_SPIKES),
 * membranes V (FHE_STATE_MEMBRANES) or WeightSum currents I
 * (FHE_STATE_CURRENTS; a static first layer keeps its step-0 current) to the
 * device buffer dst [n_images][out_size][n+1] on `stream`.  A Poisson layer
 * has spikes only.  Errors: FHE_EINVAL, FHE_ECUDA, FHE_ETIMEOUT. */
#define FHE_STATE_SPIKES 0
#define FHE_STATE_MEMBRANES 1
#define FHE_STATE_CURRENTS 2
int fhe_snn_stream_stage(fhe_snn *net, const uint32_t *ct_input, size_t n_images, uint32_t *scores,
                         int on_host, void *stream);
int fhe_snn_stream_iterate(fhe_snn *net, void *stream);
int fhe_snn_stream_state(const fhe_snn *net, uint64_t batch, uint32_t layer, int kind,
                         uint32_t *dst, void *stream);

/* Optional: device spike ciphertexts of layer `layer` at the last step of
 * the last inference, copied to device buffer dst [n_images][size][n+1]. */
int fhe_snn_layer_spikes(const fhe_snn *net, uint32_t layer, uint32_t *dst, void *stream);

/* Blind-rotation kernel time of the last inference (instrumentation).  When
 * the network was created with profiling on (FHE_SNN_PROFILE in use_graph's
 * bit 1), every blind-rotation launch is bracketed by a CUDA event pair on its
 * stream, inside the captured graphs too.  Synchronizes, then writes the
 * summed milliseconds, the number of launches and the number of bootstrapped
 * ciphertexts of the last fhe_snn_infer call.  Errors: FHE_EINVAL when
 * profiling is off, FHE_ECUDA. */
#define FHE_SNN_PROFILE 2
int fhe_snn_profile(const fhe_snn *net, double *br_ms, uint64_t *br_launches,
                    uint64_t *br_ciphertexts);

/* Process-wide count of kernels this library has launched (graph replays
 * count every kernel node of the graph). */
uint64_t fhe_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* FHE_DICSNN_H */
