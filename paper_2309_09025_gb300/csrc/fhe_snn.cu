// fhe_snn.cu -- encrypted DiCSNN inference (paper 3.1-3.3 network, 4.1
// WeightSum, 4.2 FHE-Fire / FHE-Reset, 5.3 client/server flow).
//
// Per layer l and time step t:  I = WeightSum(x);  H = V + I + (p/2) Delta;
// (S, V) = bootstrap(H) with the Fire and Reset tables from ONE blind rotation
// (multi-value split);  x_next = S;  scores += S of the last layer.  In the
// two-bootstrap mode (4.2 as printed) S = bootstrap_sign(V + I - V_th) + 1 and
// V = bootstrap_g(V + I) with negacyclic tables and no centring.  A Poisson
// encoder first layer (2.3) bootstraps the comparison x > M_t per pixel.
//
// Layer-skewed schedule.  Layer l at step t only needs layer l-1 at step t
// and itself at step t-1, so iteration tau runs every layer l with
// t = tau - l in [0, T): all active layers' neurons (of all images) go through
// ONE bootstrap launch per iteration, T + layers - 1 iterations in total,
// instead of one mostly-empty launch per layer and step.  Each iteration is
// captured once as a CUDA graph per batch size and replayed; a stream of
// batches replays one graph per kind of steady-state iteration.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <vector>

#include "fhe_internal.cuh"

namespace fhe {
int lwe_add(uint32_t n, const uint32_t *a, const uint32_t *b, uint32_t cst, uint64_t count,
            uint32_t *out, cudaStream_t st);
int lwe_add_offsets(uint32_t n, const uint32_t *a, const int32_t *offs, uint32_t n_in,
                    uint32_t delta, uint32_t cst, uint64_t count, uint32_t *out, cudaStream_t st);
}

namespace {
struct Layer {
  int type;
  uint32_t log2_p;  // the layer's message space
  int32_t *d_w;   // weights; Poisson: thresholds M [T][in_size]
  uint32_t in_size, out_size;
  uint32_t cin, h, w, cout, kh, kw, stride, pad;
  uint32_t *d_I;  // [max_images][out][n+1] (not used by a Poisson layer)
};

// One captured streamed iteration: its executable graph (and the graph it was
// instantiated from, whose event-record nodes are re-pointed before every
// replay), its kernel count, and per bracketed bootstrap launch the two
// event-record nodes and the launch's ciphertext count.
struct IterGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  std::vector<cudaGraphNode_t> ev_nodes;  // [launch][2]
  std::vector<size_t> ev_counts;          // [launch]
};

// Streamed inference: batch b lives in slot b % nslots while its layers are
// in flight (T + layers - 1 iterations); every iteration gathers the active
// (layer, batch) segments into one contiguous bootstrap launch.
struct StreamState {
  size_t ni = 0;            // images per batch of the running stream (0: idle)
  uint32_t nslots = 0;
  uint64_t pushed = 0;      // batches pushed since the stream started
  uint64_t next_iter = 0;   // next iteration of the stream
  std::vector<std::vector<uint32_t *>> spk, mem, I;  // [slot][layer]
  std::vector<uint32_t *> in, scores, dst;           // [slot]
  std::vector<int> dst_host;                         // [slot]
  uint32_t *stage_H = nullptr, *stage_Hf = nullptr, *pout = nullptr;
  std::vector<cudaEvent_t> ev;   // [launch][2]
  std::vector<size_t> ev_count;  // ciphertexts of each bracketed launch
  size_t ev_used = 0;
  // Steady state (every layer active): iteration j launches the same work on
  // the same buffers as iteration j + T * nslots, so with use_graph bit 0 one
  // graph per residue j mod (T * nslots) is captured on first use and
  // replayed; captured for batches of graph_ni images under the keys' tuning
  // settings graph_tuning.
  std::vector<IterGraph> graphs;
  size_t graph_ni = 0;
  std::vector<int64_t> graph_tuning;
};

static void drop_graphs(std::vector<IterGraph> &v) {
  for (auto &g : v) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  v.clear();
}
}  // namespace

struct fhe_snn {
  fhe_keys *K;
  fhe_snn_desc desc;
  std::vector<Layer> layers;
  int mode;               // FHE_LIF_MULTI_VALUE or FHE_LIF_TWO_PBS
  fhe_lut *lut;           // multi-value: Fire and Reset tables (L = 2), one
                          // group per layer when the layers have their own
                          // message spaces
  fhe_lut *lut_fire;      // two bootstraps: sign table (L = 1)
  fhe_lut *lut_reset;     // two bootstraps: reset table (L = 1)
  uint32_t n_in, n_out;
  uint64_t neurons;    // sum of the layers' sizes (per image)
  uint32_t *d_H;       // bootstrap inputs, all layers: [max_images * neurons][n+1]
  uint32_t *d_Hf;      // two bootstraps: Fire inputs H - V_th, same layout
  uint32_t *d_out;     // [2][max_images * neurons][n+1]: spikes, then membrane V
  uint32_t *d_input;   // staging copy of the caller's input
  uint32_t *d_scores;  // [max_images][n_out][n+1]
  // inference in progress
  size_t cur_images;
  uint32_t next_iter;
  // captured graphs per batch size: one executable graph per iteration, its
  // kernel-node count and its bracketed bootstrap counts (two per iteration)
  struct GraphSet {
    std::vector<int64_t> tuning;  // the keys' tuning settings at capture
    std::vector<cudaGraphExec_t> execs;
    std::vector<int64_t> kernels;
    std::vector<size_t> pbs_counts;
  };
  std::map<size_t, GraphSet> graphs;
  // Graphs are captured and replayed on a library-owned non-blocking stream
  // (the legacy default stream cannot be captured), joined to the caller's
  // stream by the two events below.
  cudaStream_t gs;
  cudaEvent_t join_in, join_out;
  size_t last_images;
  // streamed inference state (allocated on the first push)
  StreamState *stream;
  bool prof_stream;    // the last inference activity was a stream
  // instrumentation: one event pair per bootstrap launch of an iteration
  bool profile;
  std::vector<cudaEvent_t> ev;   // [iterations][2 launches][2]
  std::vector<size_t> ev_count;  // [iterations][2]: ciphertexts of each bracketed launch
};

// Centring offset (p_l / 2) * Delta_l of a layer's bootstrap input (q / 4
// whatever the space).
static uint32_t half_space(uint32_t log2_p) {
  return (1u << (log2_p - 1u)) * (1u << (31u - log2_p));
}

// The keys' settings that pick the launched blind-rotation kernels (variant
// threshold, cluster shapes and their limits, forced options): a CUDA graph
// captured under other values is captured again.
static std::vector<int64_t> tuning_of(const fhe_keys *K) {
  return {(int64_t)K->tc_min_batch, K->tc_cl8_tiles, K->tc_cl16_tiles, K->tc_split_ok,
          K->tc_split_tiles, K->tc_force_cl, K->tc_force_mc, K->tc_l2_hints};
}

static uint32_t snn_iterations(const fhe_snn *S) {
  return S->desc.T + (uint32_t)S->layers.size() - 1u;
}

static void stream_release(StreamState *Z) {
  if (!Z) return;
  drop_graphs(Z->graphs);
  for (auto *v : {&Z->spk, &Z->mem, &Z->I})
    for (auto &slot : *v)
      for (auto p : slot) cudaFree(p);
  for (auto p : Z->in) cudaFree(p);
  for (auto p : Z->scores) cudaFree(p);
  cudaFree(Z->stage_H);
  cudaFree(Z->stage_Hf);
  cudaFree(Z->pout);
  for (auto e : Z->ev)
    if (e) cudaEventDestroy(e);
  delete Z;
}

static void snn_release(fhe_snn *S) {
  if (!S) return;
  stream_release(S->stream);
  for (auto &kv : S->graphs)
    for (auto &g : kv.second.execs)
      if (g) cudaGraphExecDestroy(g);
  for (auto &e : S->ev)
    if (e) cudaEventDestroy(e);
  if (S->join_in) cudaEventDestroy(S->join_in);
  if (S->join_out) cudaEventDestroy(S->join_out);
  if (S->gs) cudaStreamDestroy(S->gs);
  for (auto &L : S->layers) {
    cudaFree(L.d_w);
    cudaFree(L.d_I);
  }
  cudaFree(S->d_H);
  cudaFree(S->d_Hf);
  cudaFree(S->d_out);
  cudaFree(S->d_input);
  cudaFree(S->d_scores);
  fhe_lut_free(S->lut);
  fhe_lut_free(S->lut_fire);
  fhe_lut_free(S->lut_reset);
  delete S;
}

extern "C" int fhe_snn_create(fhe_keys *K, const fhe_snn_desc *d, fhe_snn **out) {
  if (!K || !d || !out || !d->layers || d->n_layers == 0 || d->T == 0 || d->max_images == 0)
    return FHE_EINVAL;
  if (d->variant != FHE_VARIANT_EXACT && d->variant != FHE_VARIANT_TC &&
      d->variant != FHE_VARIANT_FFT && d->variant != FHE_VARIANT_AUTO)
    return FHE_EINVAL;
  if (d->lif_mode != FHE_LIF_MULTI_VALUE && d->lif_mode != FHE_LIF_TWO_PBS) return FHE_EINVAL;
  if (d->lif_mode == FHE_LIF_TWO_PBS && d->spike_scale != 2) return FHE_EINVAL;
  *out = NULL;
  const fhe::Params &P = K->P;
  const int32_t p = (int32_t)P.p();
  // message spaces of the layers (DiNN's dynamic message space, 5.2)
  const uint32_t nl = d->n_layers;
  std::vector<uint32_t> lp(nl);
  bool spaces = false;
  for (uint32_t i = 0; i < nl; ++i) {
    const fhe_layer_desc &ld = d->layers[i];
    lp[i] = ld.log2_p ? ld.log2_p : P.log2_p;
    if (lp[i] > 10u || (2u << lp[i]) > P.N) return FHE_EINVAL;
    if (i == 0 && (lp[0] > P.log2_p || (ld.type == FHE_LAYER_POISSON && lp[0] != P.log2_p)))
      return FHE_EINVAL;
    spaces = spaces || lp[i] != P.log2_p;
  }
  if (spaces && (d->lif_mode != FHE_LIF_MULTI_VALUE || nl > fhe::kLutGroups)) return FHE_EINVAL;
  fhe_snn *S = new fhe_snn();
  S->K = K;
  S->desc = *d;
  S->desc.layers = NULL;
  S->mode = d->lif_mode;
  int rc = fhe::pbs_prepare(K, d->variant);
  if (rc) { snn_release(S); return rc; }
  std::vector<int32_t> f(2u * (size_t)p);
  if (S->mode == FHE_LIF_MULTI_VALUE) {
    // LIF tables on the centred input u = H + p_l/2, v = u - p_l/2 (Thm 3.2 /
    // 4.2); one group per layer when the spaces differ: Fire written in the
    // next layer's space (the key's after the last layer), Reset in its own
    const uint32_t groups = spaces ? nl : 1u;
    std::vector<uint32_t> lp_in(groups), lp_out(2u * groups);
    f.clear();
    for (uint32_t g = 0; g < groups; ++g) {
      lp_in[g] = lp[g];
      lp_out[2u * g] = (g + 1u < groups) ? lp[g + 1u] : P.log2_p;
      lp_out[2u * g + 1u] = lp[g];
      const int32_t pg = 1 << lp[g];
      const size_t at = f.size();
      f.resize(at + 2u * (size_t)pg);
      for (int32_t u = 0; u < pg; ++u) {
        const int32_t v = u - pg / 2;
        f[at + u] = (v >= d->v_th) ? d->spike_scale : 0;
        f[at + pg + u] = (v >= d->v_th) ? 0 : (v >= 0 ? (v >> d->leak_shift) : 0);
      }
    }
    rc = fhe_lut_create_spaces(K, f.data(), 2u, groups, lp_in.data(), lp_out.data(), &S->lut);
  } else {
    // Negacyclic program functions on u in [0, p) (4.2); the bootstrap gives
    // -g(u) on the other half [-p, 0).  Sign: g = 1.  Reset: 0 from V_th up,
    // leak(u) below.
    for (int32_t u = 0; u < p; ++u) {
      f[u] = 1;
      f[p + u] = (u >= d->v_th) ? 0 : (u >> d->leak_shift);
    }
    rc = fhe_lut_create(K, f.data(), 1u, &S->lut_fire);
    if (!rc) rc = fhe_lut_create(K, f.data() + p, 1u, &S->lut_reset);
  }
  if (rc) { snn_release(S); return rc; }
  uint32_t prev = 0;
  const uint32_t W = P.n + 1u;
  for (uint32_t i = 0; i < d->n_layers; ++i) {
    const fhe_layer_desc &ld = d->layers[i];
    Layer L;
    memset(&L, 0, sizeof(L));
    L.type = ld.type;
    L.log2_p = lp[i];
    size_t wcount;
    if (ld.type == FHE_LAYER_FC) {
      L.in_size = ld.in_size; L.out_size = ld.out_size;
      wcount = (size_t)ld.in_size * ld.out_size;
    } else if (ld.type == FHE_LAYER_POISSON) {
      if (i != 0 || !d->static_input || ld.out_size != ld.in_size) { snn_release(S); return FHE_EINVAL; }
      L.in_size = L.out_size = ld.in_size;
      wcount = (size_t)d->T * ld.in_size;
    } else if (ld.type == FHE_LAYER_CONV) {
      if (!ld.stride || !ld.kh || !ld.kw || ld.h + 2 * ld.pad < ld.kh || ld.w + 2 * ld.pad < ld.kw) {
        snn_release(S); return FHE_EINVAL;
      }
      L.cin = ld.cin; L.h = ld.h; L.w = ld.w; L.cout = ld.cout; L.kh = ld.kh; L.kw = ld.kw;
      L.stride = ld.stride; L.pad = ld.pad;
      L.in_size = ld.cin * ld.h * ld.w;
      const uint32_t ho = (ld.h + 2 * ld.pad - ld.kh) / ld.stride + 1;
      const uint32_t wo = (ld.w + 2 * ld.pad - ld.kw) / ld.stride + 1;
      L.out_size = ld.cout * ho * wo;
      wcount = (size_t)ld.cout * ld.cin * ld.kh * ld.kw;
    } else {
      snn_release(S); return FHE_EINVAL;
    }
    if (!ld.weights || L.out_size == 0 || (i > 0 && L.in_size != prev)) {
      S->layers.push_back(L); snn_release(S); return FHE_EINVAL;
    }
    prev = L.out_size;
    S->neurons += L.out_size;
    const size_t cts = (size_t)d->max_images * L.out_size;
    bool ok = cudaMalloc(&L.d_w, sizeof(int32_t) * wcount) == cudaSuccess &&
              (L.type == FHE_LAYER_POISSON ||
               cudaMalloc(&L.d_I, sizeof(uint32_t) * cts * W) == cudaSuccess);
    S->layers.push_back(L);
    if (!ok) { snn_release(S); return FHE_ENOMEM; }
    // a WeightSum first layer in a smaller space than the input's: the
    // input's Delta times p / p_0 is the layer's
    std::vector<int32_t> scaled;
    const int32_t *wsrc = ld.weights;
    if (i == 0 && L.type != FHE_LAYER_POISSON && lp[0] != P.log2_p) {
      scaled.assign(ld.weights, ld.weights + wcount);
      for (auto &w : scaled) w = (int32_t)((uint32_t)w << (P.log2_p - lp[0]));
      wsrc = scaled.data();
    }
    if (cudaMemcpy(L.d_w, wsrc, sizeof(int32_t) * wcount, cudaMemcpyHostToDevice) != cudaSuccess) {
      snn_release(S); return FHE_ECUDA;
    }
  }
  S->n_in = S->layers.front().in_size;
  S->n_out = S->layers.back().out_size;
  const size_t all = (size_t)d->max_images * S->neurons;
  const size_t in_words = (size_t)d->max_images * (d->static_input ? 1u : d->T) * S->n_in * W;
  if (cudaMalloc(&S->d_H, sizeof(uint32_t) * all * W) != cudaSuccess ||
      (S->mode == FHE_LIF_TWO_PBS && cudaMalloc(&S->d_Hf, sizeof(uint32_t) * all * W) != cudaSuccess) ||
      cudaMalloc(&S->d_out, sizeof(uint32_t) * 2u * all * W) != cudaSuccess ||
      cudaMalloc(&S->d_input, sizeof(uint32_t) * in_words) != cudaSuccess ||
      cudaMalloc(&S->d_scores, sizeof(uint32_t) * (size_t)d->max_images * S->n_out * W) != cudaSuccess) {
    snn_release(S); return FHE_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&S->gs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->join_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->join_out, cudaEventDisableTiming) != cudaSuccess) {
    snn_release(S); return FHE_ECUDA;
  }
  S->profile = (d->use_graph & FHE_SNN_PROFILE) != 0;
  if (S->profile) {
    S->ev.assign((size_t)snn_iterations(S) * 4u, (cudaEvent_t)0);
    S->ev_count.assign((size_t)snn_iterations(S) * 2u, 0);
    for (auto &e : S->ev)
      if (cudaEventCreate(&e) != cudaSuccess) { snn_release(S); return FHE_ECUDA; }
  }
  *out = S;
  return FHE_OK;
}

extern "C" void fhe_snn_free(fhe_snn *S) {
  if (!S) return;
  cudaDeviceSynchronize();
  snn_release(S);
}

extern "C" uint64_t fhe_snn_pbs_per_image(const fhe_snn *S) {
  if (!S) return 0;
  uint64_t per_step = 0;
  for (const Layer &L : S->layers)
    per_step += (uint64_t)L.out_size *
                ((S->mode == FHE_LIF_TWO_PBS && L.type != FHE_LAYER_POISSON) ? 2u : 1u);
  return per_step * S->desc.T;
}

extern "C" uint32_t fhe_snn_iterations(const fhe_snn *S) { return S ? snn_iterations(S) : 0u; }

extern "C" int fhe_snn_profile(const fhe_snn *S, double *br_ms, uint64_t *br_launches,
                               uint64_t *br_ciphertexts) {
  if (!S || !S->profile || !br_ms || !br_launches || !br_ciphertexts) return FHE_EINVAL;
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  double ms = 0.0;
  uint64_t launches = 0, cts = 0;
  if (S->prof_stream && S->stream) {
    const StreamState &Z = *S->stream;
    for (size_t e = 0; e < Z.ev_used; ++e) {
      if (!Z.ev_count[e]) continue;
      float t = 0.f;
      FHE_CUDA_TRY(cudaEventElapsedTime(&t, Z.ev[2 * e], Z.ev[2 * e + 1]));
      ms += t;
      launches += 1;
      cts += Z.ev_count[e];
    }
    *br_ms = ms;
    *br_launches = launches;
    *br_ciphertexts = cts;
    return FHE_OK;
  }
  for (size_t e = 0; e < S->ev_count.size(); ++e) {
    if (!S->ev_count[e]) continue;
    float t = 0.f;
    FHE_CUDA_TRY(cudaEventElapsedTime(&t, S->ev[2 * e], S->ev[2 * e + 1]));
    ms += t;
    launches += 1;
    cts += S->ev_count[e];
  }
  *br_ms = ms;
  *br_launches = launches;
  *br_ciphertexts = cts;
  return FHE_OK;
}

// Bootstrap the ciphertexts [lo, hi) of `in` with `lut` into `out` (table
// stride `stride`), bracketed by profiling slot `slot` of iteration tau.
// seg_end: the launch-relative layer boundaries of a grouped table set.
static int snn_bootstrap(fhe_snn *S, uint32_t tau, uint32_t slot, const uint32_t *in, size_t lo,
                         size_t hi, const fhe_lut *lut, uint32_t *out, size_t stride,
                         cudaStream_t st, const uint64_t *seg_end = nullptr) {
  const uint32_t W = S->K->P.n + 1u;
  if (hi <= lo) return FHE_OK;
  const size_t e = 2u * tau + slot;
  if (S->profile) {
    S->K->prof_ev0 = S->ev[2u * e];
    S->K->prof_ev1 = S->ev[2u * e + 1u];
  }
  const int rc = fhe::pbs_run(S->K, in + lo * W, hi - lo, lut, out + lo * W, stride,
                              S->desc.variant, st, seg_end);
  if (S->profile) {
    S->ev_count[e] = S->K->prof_count;
    S->K->prof_ev0 = S->K->prof_ev1 = (cudaEvent_t)0;
  }
  return rc;
}

// Enqueue iteration tau for `ni` images: every layer l with t = tau - l in
// [0, T) advances one step; their bootstraps share one launch (two in the
// two-bootstrap mode: Fire over all active layers, Reset over the LIF ones).
static int snn_iteration(fhe_snn *S, uint32_t tau, size_t ni, cudaStream_t st) {
  const fhe::Params &P = S->K->P;
  const uint32_t W = P.n + 1u;
  const uint32_t delta = P.delta();
  const uint32_t half_p = delta * (P.p() / 2u);  // (p/2) * Delta
  const uint32_t T = S->desc.T, nl = (uint32_t)S->layers.size();
  const uint32_t lo = (tau >= T) ? tau - T + 1u : 0u;
  const uint32_t hi = (tau < nl - 1u) ? tau : nl - 1u;
  const size_t all = ni * S->neurons;
  const bool two = (S->mode == FHE_LIF_TWO_PBS);
  uint32_t *spk = S->d_out, *mem = S->d_out + all * W;
  uint32_t *fire_in = two ? S->d_Hf : S->d_H;
  // segment offsets of the layers (ciphertexts) for this batch size
  std::vector<size_t> off(nl + 1u, 0);
  for (uint32_t l = 0; l < nl; ++l) off[l + 1] = off[l] + ni * S->layers[l].out_size;
  int rc;
  // 1. WeightSums of the active layers, from the spikes of the previous
  //    iteration (read before this iteration's bootstrap overwrites them)
  for (uint32_t l = lo; l <= hi; ++l) {
    Layer &L = S->layers[l];
    const uint32_t t = tau - l;
    if (L.type == FHE_LAYER_POISSON) continue;  // no WeightSum: compares pixels
    const bool static_first = (l == 0 && S->desc.static_input);
    if (static_first && t > 0) continue;  // the conv of the pixels is time-invariant
    const uint32_t *x = (l == 0)
                            ? S->d_input + (S->desc.static_input ? 0 : (size_t)t * ni * S->n_in * W)
                            : spk + off[l - 1] * W;
    if (L.type == FHE_LAYER_FC)
      rc = fhe_lwe_linear(P.n, P.log2_p, L.d_w, L.out_size, L.in_size, NULL, x, ni, L.d_I, st);
    else
      rc = fhe_lwe_conv2d(P.n, P.log2_p, L.d_w, L.cin, L.h, L.w, L.cout, L.kh, L.kw, L.stride,
                          L.pad, NULL, x, ni, L.d_I, st);
    if (rc) return rc;
  }
  // 2. bootstrap inputs.  LIF: H = V + I (V = 0 at the layer's first step),
  //    centred by +p/2 (multi-value) or also H - V_th for the sign bootstrap
  //    (two bootstraps).  Poisson: x - M_t + V_th - 1, centred (multi-value),
  //    or x - M_t - 1 (two bootstraps).
  for (uint32_t l = lo; l <= hi; ++l) {
    const Layer &L = S->layers[l];
    const uint32_t t = tau - l;
    const uint64_t cnt = ni * L.out_size;
    if (L.type == FHE_LAYER_POISSON) {
      const uint32_t cst = two ? (0u - delta) : ((uint32_t)(S->desc.v_th - 1) * delta + half_p);
      rc = fhe::lwe_add_offsets(P.n, S->d_input, L.d_w + (size_t)t * L.in_size, L.in_size, 0u - delta,
                                cst, cnt, fire_in + off[l] * W, st);
      if (rc) return rc;
      continue;
    }
    rc = fhe::lwe_add(P.n, L.d_I, t ? mem + off[l] * W : NULL, two ? 0u : half_space(L.log2_p), cnt,
                      S->d_H + off[l] * W, st);
    if (!rc && two)
      rc = fhe::lwe_add(P.n, S->d_H + off[l] * W, NULL, 0u - (uint32_t)S->desc.v_th * delta, cnt,
                        S->d_Hf + off[l] * W, st);
    if (rc) return rc;
  }
  // 3. bootstraps for every active neuron: spikes and V in place
  if (!two) {
    std::vector<uint64_t> seg(nl, 0);  // layer boundaries relative to off[lo]
    for (uint32_t q = 0; q + 1u < nl; ++q) seg[q] = (off[q + 1] > off[lo]) ? off[q + 1] - off[lo] : 0u;
    rc = snn_bootstrap(S, tau, 0u, S->d_H, off[lo], off[hi + 1], S->lut, spk, all * W, st,
                       S->lut->groups > 1u ? seg.data() : nullptr);
    if (rc) return rc;
  } else {
    rc = snn_bootstrap(S, tau, 0u, S->d_Hf, off[lo], off[hi + 1], S->lut_fire, spk, all * W, st);
    if (!rc)  // 2 FHE-Fire = bootstrap_sign + 1
      rc = fhe::lwe_add(P.n, spk + off[lo] * W, NULL, delta, off[hi + 1] - off[lo], spk + off[lo] * W, st);
    const uint32_t lr = (S->layers[lo].type == FHE_LAYER_POISSON) ? lo + 1u : lo;
    if (!rc && lr <= hi)
      rc = snn_bootstrap(S, tau, 1u, S->d_H, off[lr], off[hi + 1], S->lut_reset, mem, all * W, st);
    if (rc) return rc;
  }
  // 4. spike-count scores of the last layer
  if (hi == nl - 1u) {
    const uint32_t t = tau - (nl - 1u);
    rc = fhe::lwe_add(P.n, spk + off[nl - 1u] * W, t ? S->d_scores : NULL, 0u, ni * S->n_out,
                      S->d_scores, st);
    if (rc) return rc;
  }
  return FHE_OK;
}

// Capture the iterations for batch size ni (kept for later calls of the same
// size; at most max_images sets exist).
static int snn_capture(fhe_snn *S, size_t ni, cudaStream_t st) {
  const uint32_t iters = snn_iterations(S);
  fhe_snn::GraphSet set;
  set.tuning = tuning_of(S->K);
  set.execs.assign(iters, (cudaGraphExec_t)0);
  set.kernels.assign(iters, 0);
  set.pbs_counts.assign(2u * iters, 0);
  int rc = FHE_OK;
  for (uint32_t tau = 0; tau < iters && rc == FHE_OK; ++tau) {
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = FHE_ECUDA;
      break;
    }
    // launches enqueued while capturing run only when the graph is replayed
    const int64_t before = (int64_t)fhe::launches();
    rc = snn_iteration(S, tau, ni, st);
    set.kernels[tau] = (int64_t)fhe::launches() - before;
    fhe::note_launches(-set.kernels[tau]);
    if (S->profile)
      for (uint32_t k = 0; k < 2u; ++k) set.pbs_counts[2u * tau + k] = S->ev_count[2u * tau + k];
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) { if (e == cudaSuccess) cudaGraphDestroy(graph); break; }
    if (e != cudaSuccess) { (void)cudaGetLastError(); rc = FHE_ECUDA; break; }
    cudaError_t ie = cudaGraphInstantiate(&set.execs[tau], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { (void)cudaGetLastError(); rc = FHE_ECUDA; }
  }
  if (rc) {
    for (auto &g : set.execs)
      if (g) cudaGraphExecDestroy(g);
    return rc;
  }
  S->graphs[ni] = set;
  return FHE_OK;
}

extern "C" int fhe_snn_begin(fhe_snn *S, const uint32_t *ct_input, size_t ni, int inputs_on_host,
                             void *stream) {
  if (!S || !ct_input || ni == 0 || ni > S->desc.max_images) return FHE_EINVAL;
  if (S->stream && S->stream->ni) return FHE_EINVAL;  // a stream is running
  S->prof_stream = false;
  const uint32_t W = S->K->P.n + 1u;
  const size_t in_words = ni * (S->desc.static_input ? 1u : S->desc.T) * S->n_in * W;
  FHE_CUDA_TRY(cudaMemcpyAsync(S->d_input, ct_input, sizeof(uint32_t) * in_words,
                               inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  S->cur_images = ni;
  S->next_iter = 0;
  return FHE_OK;
}

extern "C" int fhe_snn_step(fhe_snn *S, void *stream) {
  if (!S || !S->cur_images) return FHE_EINVAL;
  const uint32_t iters = snn_iterations(S);
  if (S->next_iter >= iters) return FHE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ni = S->cur_images;
  const uint32_t tau = S->next_iter;
  if (S->desc.use_graph & 1) {
    auto old = S->graphs.find(ni);
    if (old != S->graphs.end() && old->second.tuning != tuning_of(S->K)) {
      // captured under other tuning settings: capture again (a graph still
      // running is freed when it completes)
      for (auto &g : old->second.execs)
        if (g) cudaGraphExecDestroy(g);
      S->graphs.erase(old);
    }
    if (S->graphs.find(ni) == S->graphs.end()) {
      FHE_CUDA_TRY(cudaEventRecord(S->join_in, st));
      FHE_CUDA_TRY(cudaStreamWaitEvent(S->gs, S->join_in, 0));
      int rc = snn_capture(S, ni, S->gs);
      if (rc) return rc;
    }
    const fhe_snn::GraphSet &set = S->graphs[ni];
    FHE_CUDA_TRY(cudaEventRecord(S->join_in, st));
    FHE_CUDA_TRY(cudaStreamWaitEvent(S->gs, S->join_in, 0));
    FHE_CUDA_TRY(cudaGraphLaunch(set.execs[tau], S->gs));
    fhe::note_launches(set.kernels[tau]);
    if (S->profile)
      for (uint32_t k = 0; k < 2u; ++k) S->ev_count[2u * tau + k] = set.pbs_counts[2u * tau + k];
    FHE_CUDA_TRY(cudaEventRecord(S->join_out, S->gs));
    FHE_CUDA_TRY(cudaStreamWaitEvent(st, S->join_out, 0));
  } else {
    int rc = snn_iteration(S, tau, ni, st);
    if (rc) return rc;
  }
  S->next_iter = tau + 1u;
  return (int)(iters - S->next_iter);
}

extern "C" int fhe_snn_end(fhe_snn *S, uint32_t *scores, int inputs_on_host, void *stream) {
  if (!S || !scores || !S->cur_images || S->next_iter != snn_iterations(S)) return FHE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t out_words = S->cur_images * S->n_out * (S->K->P.n + 1u);
  FHE_CUDA_TRY(cudaMemcpyAsync(scores, S->d_scores, sizeof(uint32_t) * out_words,
                               inputs_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  S->last_images = S->cur_images;
  S->cur_images = 0;
  if (inputs_on_host) {
    FHE_CUDA_TRY(cudaStreamSynchronize(st));
    return fhe_status(S->K, stream);
  }
  return FHE_OK;
}

extern "C" int fhe_snn_infer(fhe_snn *S, const uint32_t *ct_input, size_t ni, uint32_t *scores,
                             int inputs_on_host, void *stream) {
  if (!S || !scores) return FHE_EINVAL;
  int rc = fhe_snn_begin(S, ct_input, ni, inputs_on_host, stream);
  if (rc) return rc;
  do {
    rc = fhe_snn_step(S, stream);
  } while (rc > 0);
  if (rc < 0) { S->cur_images = 0; return rc; }
  return fhe_snn_end(S, scores, inputs_on_host, stream);
}

extern "C" int fhe_snn_layer_spikes(const fhe_snn *S, uint32_t layer, uint32_t *dst,
                                    void *stream) {
  if (!S || !dst || layer >= S->layers.size() || !S->last_images) return FHE_EINVAL;
  size_t off = 0;
  for (uint32_t l = 0; l < layer; ++l) off += S->last_images * S->layers[l].out_size;
  const uint32_t W = S->K->P.n + 1u;
  const size_t words = S->last_images * S->layers[layer].out_size * W;
  FHE_CUDA_TRY(cudaMemcpyAsync(dst, S->d_out + off * W, sizeof(uint32_t) * words,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return FHE_OK;
}

// ---------------------------------------------------------------- streaming
static int stream_alloc(fhe_snn *S) {
  if (S->stream) return FHE_OK;
  StreamState *Z = new StreamState();
  const uint32_t T = S->desc.T, nl = (uint32_t)S->layers.size();
  const uint32_t W = S->K->P.n + 1u;
  const size_t mi = S->desc.max_images;
  Z->nslots = 1u + (nl - 1u + T - 1u) / T;  // batches in flight at once
  const size_t in_words = mi * (S->desc.static_input ? 1u : T) * S->n_in * W;
  const size_t all = mi * S->neurons;
  bool ok = true;
  auto get = [&](uint32_t **p, size_t words) {
    if (ok && cudaMalloc(p, sizeof(uint32_t) * words) != cudaSuccess) { *p = nullptr; ok = false; }
  };
  Z->spk.assign(Z->nslots, std::vector<uint32_t *>(nl, nullptr));
  Z->mem = Z->spk;
  Z->I = Z->spk;
  Z->in.assign(Z->nslots, nullptr);
  Z->scores.assign(Z->nslots, nullptr);
  Z->dst.assign(Z->nslots, nullptr);
  Z->dst_host.assign(Z->nslots, 0);
  for (uint32_t sl = 0; sl < Z->nslots; ++sl) {
    for (uint32_t l = 0; l < nl; ++l) {
      const size_t words = mi * S->layers[l].out_size * W;
      get(&Z->spk[sl][l], words);
      if (S->layers[l].type != FHE_LAYER_POISSON) {
        get(&Z->mem[sl][l], words);
        get(&Z->I[sl][l], words);
      }
    }
    get(&Z->in[sl], in_words);
    get(&Z->scores[sl], mi * S->n_out * W);
  }
  get(&Z->stage_H, all * W);
  if (S->mode == FHE_LIF_TWO_PBS) get(&Z->stage_Hf, all * W);
  get(&Z->pout, 2u * all * W);
  if (!ok) { stream_release(Z); return FHE_ENOMEM; }
  S->stream = Z;
  return FHE_OK;
}

// Make sure an event pair exists for the next bracketed launch (slot ev_used).
static int stream_event_pair(StreamState &Z) {
  if (2u * Z.ev_used + 2u <= Z.ev.size()) return FHE_OK;
  cudaEvent_t a, b;
  FHE_CUDA_TRY(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    (void)cudaGetLastError();
    return FHE_ECUDA;
  }
  Z.ev.push_back(a);
  Z.ev.push_back(b);
  Z.ev_count.push_back(0);
  return FHE_OK;
}

static int stream_bootstrap(fhe_snn *S, const uint32_t *in, size_t lo, size_t hi, const fhe_lut *lut,
                            uint32_t *out, size_t stride, cudaStream_t st,
                            const uint64_t *seg_end = nullptr) {
  if (hi <= lo) return FHE_OK;
  StreamState &Z = *S->stream;
  const uint32_t W = S->K->P.n + 1u;
  if (S->profile) {
    const int rc = stream_event_pair(Z);
    if (rc) return rc;
    S->K->prof_ev0 = Z.ev[2u * Z.ev_used];
    S->K->prof_ev1 = Z.ev[2u * Z.ev_used + 1u];
  }
  const int rc = fhe::pbs_run(S->K, in + lo * W, hi - lo, lut, out + lo * W, stride, S->desc.variant, st,
                              seg_end);
  if (S->profile) {
    Z.ev_count[Z.ev_used++] = S->K->prof_count;
    S->K->prof_ev0 = S->K->prof_ev1 = (cudaEvent_t)0;
  }
  return rc;
}

// Iteration j of the stream: layer l runs batch b = (j - l) / T at time
// t = (j - l) mod T for every pushed batch b (same recurrence as the
// layer-skewed schedule of one inference).  Everything but the copy of a
// completed batch's scores to its caller (stream_deliver).
static int stream_body(fhe_snn *S, uint64_t j, cudaStream_t st) {
  StreamState &Z = *S->stream;
  const fhe::Params &P = S->K->P;
  const uint32_t W = P.n + 1u, delta = P.delta();
  const uint32_t half_p = delta * (P.p() / 2u);
  const uint32_t T = S->desc.T, nl = (uint32_t)S->layers.size();
  const bool two = (S->mode == FHE_LIF_TWO_PBS);
  const size_t ni = Z.ni, all = S->desc.max_images * S->neurons;
  std::vector<int> on(nl, 0);
  std::vector<uint32_t> slot(nl, 0), tt(nl, 0);
  std::vector<size_t> off(nl + 1u, 0);
  for (uint32_t l = 0; l < nl; ++l) {
    if (j >= l) {
      const uint64_t b = (j - l) / T;
      if (b < Z.pushed) {
        on[l] = 1;
        slot[l] = (uint32_t)(b % Z.nslots);
        tt[l] = (uint32_t)((j - l) % T);
      }
    }
    off[l + 1] = off[l] + (on[l] ? ni * S->layers[l].out_size : 0);
  }
  if (off[nl] == 0) return FHE_OK;
  int rc;
  // 1. WeightSums of the active layers from the previous iteration's spikes
  for (uint32_t l = 0; l < nl; ++l) {
    if (!on[l]) continue;
    Layer &L = S->layers[l];
    const uint32_t sl = slot[l], t = tt[l];
    if (L.type == FHE_LAYER_POISSON) continue;
    if (l == 0 && S->desc.static_input && t > 0) continue;  // time-invariant conv
    const uint32_t *x = (l == 0) ? Z.in[sl] + (S->desc.static_input ? 0 : (size_t)t * ni * S->n_in * W)
                                 : Z.spk[sl][l - 1];
    if (L.type == FHE_LAYER_FC)
      rc = fhe_lwe_linear(P.n, P.log2_p, L.d_w, L.out_size, L.in_size, NULL, x, ni, Z.I[sl][l], st);
    else
      rc = fhe_lwe_conv2d(P.n, P.log2_p, L.d_w, L.cin, L.h, L.w, L.cout, L.kh, L.kw, L.stride, L.pad,
                          NULL, x, ni, Z.I[sl][l], st);
    if (rc) return rc;
  }
  // 2. bootstrap inputs, gathered contiguously in layer order
  for (uint32_t l = 0; l < nl; ++l) {
    if (!on[l]) continue;
    const Layer &L = S->layers[l];
    const uint32_t sl = slot[l], t = tt[l];
    const uint64_t cnt = ni * L.out_size;
    uint32_t *h = Z.stage_H + off[l] * W, *hf = two ? Z.stage_Hf + off[l] * W : nullptr;
    if (L.type == FHE_LAYER_POISSON) {
      const uint32_t cst = two ? (0u - delta) : ((uint32_t)(S->desc.v_th - 1) * delta + half_p);
      rc = fhe::lwe_add_offsets(P.n, Z.in[sl], L.d_w + (size_t)t * L.in_size, L.in_size, 0u - delta, cst,
                                cnt, two ? hf : h, st);
      if (rc) return rc;
      continue;
    }
    rc = fhe::lwe_add(P.n, Z.I[sl][l], t ? Z.mem[sl][l] : NULL, two ? 0u : half_space(L.log2_p), cnt,
                      h, st);
    if (!rc && two) rc = fhe::lwe_add(P.n, h, NULL, 0u - (uint32_t)S->desc.v_th * delta, cnt, hf, st);
    if (rc) return rc;
  }
  // 3. one launch for every active neuron (two in the two-bootstrap mode)
  uint32_t *pout_v = Z.pout + all * W;
  if (!two) {
    // layer boundaries of the gathered launch (inactive layers: empty)
    const std::vector<uint64_t> seg(off.begin() + 1, off.end());
    rc = stream_bootstrap(S, Z.stage_H, 0, off[nl], S->lut, Z.pout, all * W, st,
                          S->lut->groups > 1u ? seg.data() : nullptr);
  } else {
    rc = stream_bootstrap(S, Z.stage_Hf, 0, off[nl], S->lut_fire, Z.pout, all * W, st);
    if (!rc) rc = fhe::lwe_add(P.n, Z.pout, NULL, delta, off[nl], Z.pout, st);
    const size_t lr = (on[0] && S->layers[0].type == FHE_LAYER_POISSON) ? off[1] : 0;
    if (!rc) rc = stream_bootstrap(S, Z.stage_H, lr, off[nl], S->lut_reset, pout_v, all * W, st);
  }
  if (rc) return rc;
  // 4. spikes and membranes back to their batch slots
  for (uint32_t l = 0; l < nl; ++l) {
    if (!on[l]) continue;
    const size_t bytes = sizeof(uint32_t) * ni * S->layers[l].out_size * W;
    FHE_CUDA_TRY(cudaMemcpyAsync(Z.spk[slot[l]][l], Z.pout + off[l] * W, bytes, cudaMemcpyDeviceToDevice, st));
    if (S->layers[l].type != FHE_LAYER_POISSON)
      FHE_CUDA_TRY(cudaMemcpyAsync(Z.mem[slot[l]][l], pout_v + off[l] * W, bytes, cudaMemcpyDeviceToDevice, st));
  }
  // 5. spike-count scores of the last layer
  const uint32_t lo = nl - 1u;
  if (on[lo]) {
    const uint32_t sl = slot[lo], t = tt[lo];
    rc = fhe::lwe_add(P.n, Z.spk[sl][lo], t ? Z.scores[sl] : NULL, 0u, ni * S->n_out, Z.scores[sl], st);
    if (rc) return rc;
  }
  return FHE_OK;
}

// A batch is complete after the last layer's step T - 1: iteration j copies
// its scores to the caller's buffer (host or device, given at staging).
static int stream_deliver(fhe_snn *S, uint64_t j, cudaStream_t st) {
  StreamState &Z = *S->stream;
  const uint32_t T = S->desc.T, lo = (uint32_t)S->layers.size() - 1u;
  if (j < lo || (j - lo) % T != T - 1u) return FHE_OK;
  const uint64_t b = (j - lo) / T;
  if (b >= Z.pushed) return FHE_OK;
  const uint32_t sl = (uint32_t)(b % Z.nslots);
  FHE_CUDA_TRY(cudaMemcpyAsync(Z.dst[sl], Z.scores[sl],
                               sizeof(uint32_t) * Z.ni * S->n_out * (S->K->P.n + 1u),
                               Z.dst_host[sl] ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  return FHE_OK;
}

// Capture iteration j's body on the library stream into G.  The capture runs
// nothing: the profiling event slots it took are handed back, and the graph's
// event-record nodes that stand for them are located so that every replay
// can point them at fresh events.
static int stream_capture(fhe_snn *S, uint64_t j, IterGraph &G) {
  StreamState &Z = *S->stream;
  const size_t u0 = Z.ev_used;
  // an iteration brackets two bootstrap launches at most: their event pairs
  // are created before the capture starts
  for (int k = 0; S->profile && k < 2; ++k, ++Z.ev_used) {
    const int rc = stream_event_pair(Z);
    if (rc) { Z.ev_used = u0; return rc; }
  }
  Z.ev_used = u0;
  if (cudaStreamBeginCapture(S->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    return FHE_ECUDA;
  }
  const int64_t before = (int64_t)fhe::launches();
  int rc = stream_body(S, j, S->gs);
  G.kernels = (int64_t)fhe::launches() - before;
  fhe::note_launches(-G.kernels);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(S->gs, &graph);
  const size_t u1 = Z.ev_used;
  Z.ev_used = u0;
  if (rc || e != cudaSuccess) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    else (void)cudaGetLastError();
    return rc ? rc : FHE_ECUDA;
  }
  G.ev_nodes.assign(2u * (u1 - u0), (cudaGraphNode_t)0);
  G.ev_counts.assign(Z.ev_count.begin() + u0, Z.ev_count.begin() + u1);
  if (u1 > u0) {
    size_t nn = 0;
    bool ok = cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess;
    std::vector<cudaGraphNode_t> nodes(nn);
    ok = ok && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess;
    for (size_t q = 0; ok && q < nn; ++q) {
      cudaGraphNodeType ty;
      cudaEvent_t ev = nullptr;
      ok = cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess;
      if (!ok || ty != cudaGraphNodeTypeEventRecord) continue;
      ok = cudaGraphEventRecordNodeGetEvent(nodes[q], &ev) == cudaSuccess;
      for (size_t k = 0; ok && k < G.ev_nodes.size(); ++k)
        if (Z.ev[2u * u0 + k] == ev) G.ev_nodes[k] = nodes[q];
    }
    for (auto nd : G.ev_nodes) ok = ok && nd != nullptr;
    if (!ok) {
      (void)cudaGetLastError();
      cudaGraphDestroy(graph);
      return FHE_ECUDA;
    }
  }
  if (cudaGraphInstantiate(&G.exec, graph, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    G.exec = nullptr;
    cudaGraphDestroy(graph);
    return FHE_ECUDA;
  }
  G.graph = graph;
  return FHE_OK;
}

// Run iteration j: its cached graph in the steady state when graphs are on,
// else its launches directly; then the score delivery.
static int stream_iteration(fhe_snn *S, uint64_t j, cudaStream_t st) {
  StreamState &Z = *S->stream;
  const uint32_t T = S->desc.T, nl = (uint32_t)S->layers.size();
  const bool steady = (S->desc.use_graph & 1) && j + 1u >= nl && j < Z.pushed * T;
  if (!steady) {
    const int rc = stream_body(S, j, st);
    return rc ? rc : stream_deliver(S, j, st);
  }
  const size_t period = (size_t)T * Z.nslots;
  std::vector<int64_t> tuning = tuning_of(S->K);
  if (Z.graph_ni != Z.ni || Z.graph_tuning != tuning || Z.graphs.size() != period) {
    drop_graphs(Z.graphs);  // graphs still running are freed when they complete
    Z.graphs.resize(period);
    Z.graph_ni = Z.ni;
    Z.graph_tuning.swap(tuning);
  }
  IterGraph &G = Z.graphs[j % period];
  FHE_CUDA_TRY(cudaEventRecord(S->join_in, st));
  FHE_CUDA_TRY(cudaStreamWaitEvent(S->gs, S->join_in, 0));
  if (!G.exec) {
    const int rc = stream_capture(S, j, G);
    if (rc) { G = IterGraph(); return rc; }
  }
  // this replay's bootstrap launches are timed by the next free event pairs
  for (size_t k = 0; S->profile && k < G.ev_counts.size(); ++k) {
    const int rc = stream_event_pair(Z);
    if (rc) return rc;
    FHE_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.ev_nodes[2u * k], Z.ev[2u * Z.ev_used]));
    FHE_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.ev_nodes[2u * k + 1u],
                                                      Z.ev[2u * Z.ev_used + 1u]));
    Z.ev_count[Z.ev_used++] = G.ev_counts[k];
  }
  FHE_CUDA_TRY(cudaGraphLaunch(G.exec, S->gs));
  fhe::note_launches(G.kernels);
  FHE_CUDA_TRY(cudaEventRecord(S->join_out, S->gs));
  FHE_CUDA_TRY(cudaStreamWaitEvent(st, S->join_out, 0));
  return stream_deliver(S, j, st);
}

extern "C" int fhe_snn_stream_stage(fhe_snn *S, const uint32_t *ct_input, size_t ni, uint32_t *scores,
                                    int on_host, void *stream) {
  if (!S || !ct_input || !scores || ni == 0 || ni > S->desc.max_images || S->cur_images)
    return FHE_EINVAL;
  int rc = stream_alloc(S);
  if (rc) return rc;
  StreamState &Z = *S->stream;
  const uint32_t T = S->desc.T, W = S->K->P.n + 1u;
  if (Z.ni == 0) {  // a new stream
    Z.ni = ni;
    Z.pushed = 0;
    Z.next_iter = 0;
    Z.ev_used = 0;
    S->prof_stream = true;
  } else if (ni != Z.ni || Z.next_iter > Z.pushed * T) {
    // other batch size, or the new batch's first iteration has already run
    return FHE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t b = Z.pushed;
  const uint32_t sl = (uint32_t)(b % Z.nslots);
  const size_t in_words = ni * (S->desc.static_input ? 1u : T) * S->n_in * W;
  FHE_CUDA_TRY(cudaMemcpyAsync(Z.in[sl], ct_input, sizeof(uint32_t) * in_words,
                               on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  Z.dst[sl] = scores;
  Z.dst_host[sl] = on_host;
  Z.pushed = b + 1u;
  return FHE_OK;
}

extern "C" int fhe_snn_stream_push(fhe_snn *S, const uint32_t *ct_input, size_t ni, uint32_t *scores,
                                   int on_host, void *stream) {
  int rc = fhe_snn_stream_stage(S, ct_input, ni, scores, on_host, stream);
  if (rc) return rc;
  StreamState &Z = *S->stream;
  const uint64_t end = Z.pushed * S->desc.T;  // the staged batch's T iterations
  for (uint64_t j = Z.next_iter; j < end; ++j) {
    rc = stream_iteration(S, j, (cudaStream_t)stream);
    if (rc) return rc;
  }
  Z.next_iter = end;
  return FHE_OK;
}

extern "C" int fhe_snn_stream_iterate(fhe_snn *S, void *stream) {
  if (!S || !S->stream || !S->stream->ni) return FHE_EINVAL;
  StreamState &Z = *S->stream;
  const uint64_t end = Z.pushed * S->desc.T + S->layers.size() - 1u;
  if (Z.next_iter >= end) return 0;
  const int rc = stream_iteration(S, Z.next_iter, (cudaStream_t)stream);
  if (rc) return rc;
  ++Z.next_iter;
  return (int)(end - Z.next_iter);
}

extern "C" int fhe_snn_stream_state(const fhe_snn *S, uint64_t batch, uint32_t layer, int kind,
                                    uint32_t *dst, void *stream) {
  if (!S || !dst || !S->stream || !S->stream->ni || layer >= S->layers.size()) return FHE_EINVAL;
  const StreamState &Z = *S->stream;
  if (batch >= Z.pushed || Z.pushed > batch + Z.nslots) return FHE_EINVAL;  // not in its slot
  const uint32_t sl = (uint32_t)(batch % Z.nslots);
  const bool poisson = S->layers[layer].type == FHE_LAYER_POISSON;
  const uint32_t *src = nullptr;
  if (kind == FHE_STATE_SPIKES) src = Z.spk[sl][layer];
  else if (kind == FHE_STATE_MEMBRANES && !poisson) src = Z.mem[sl][layer];
  else if (kind == FHE_STATE_CURRENTS && !poisson) src = Z.I[sl][layer];
  if (!src) return FHE_EINVAL;
  const size_t words = Z.ni * S->layers[layer].out_size * (S->K->P.n + 1u);
  FHE_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return FHE_OK;
}

extern "C" int fhe_snn_stream_flush(fhe_snn *S, void *stream) {
  if (!S) return FHE_EINVAL;
  if (!S->stream || !S->stream->ni) return FHE_OK;
  StreamState &Z = *S->stream;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t end = Z.pushed * S->desc.T + S->layers.size() - 1u;
  for (uint64_t j = Z.next_iter; j < end; ++j) {
    const int rc = stream_iteration(S, j, st);
    if (rc) { Z.ni = 0; return rc; }
  }
  Z.next_iter = end;
  bool host = false;
  for (uint32_t sl = 0; sl < Z.nslots; ++sl) host = host || Z.dst_host[sl];
  Z.ni = 0;
  if (host) {
    FHE_CUDA_TRY(cudaStreamSynchronize(st));
    return fhe_status(S->K, stream);
  }
  return FHE_OK;
}
