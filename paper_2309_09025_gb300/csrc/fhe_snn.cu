// fhe_snn.cu -- encrypted DiCSNN inference (paper 3.1-3.3 network, 4.1
// WeightSum, 4.2 FHE-Fire / FHE-Reset, 5.3 client/server flow).
//
// Per time step and layer:  I = WeightSum(x);  H = V + I + (p/2) Delta;
// (S, V) = bootstrap(H) with the Fire and Reset tables from ONE blind
// rotation (multi-value split);  x_next = S;  scores += S of the last layer.
// Each time step is captured once as a CUDA graph per batch size and replayed.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "fhe_internal.cuh"

namespace fhe {
int lwe_add(uint32_t n, const uint32_t *a, const uint32_t *b, uint32_t cst, uint64_t count,
            uint32_t *out, cudaStream_t st);
}

namespace {
struct Layer {
  int type;
  int32_t *d_w;
  uint32_t in_size, out_size;
  uint32_t cin, h, w, cout, kh, kw, stride, pad;
  uint32_t *d_I;    // [max_images][out][n+1]
  uint32_t *d_H;    // [max_images][out][n+1]
  uint32_t *d_out;  // [2][max_images * out][n+1]: spikes then membrane V
};
}  // namespace

struct fhe_snn {
  fhe_keys *K;
  fhe_snn_desc desc;
  std::vector<Layer> layers;
  fhe_lut *lut;
  uint32_t n_in, n_out;
  uint32_t *d_input;   // staging copy of the caller's input
  uint32_t *d_scores;  // [max_images][n_out][n+1]
  size_t graph_images;
  std::vector<cudaGraphExec_t> graphs;  // one per time step
  std::vector<int64_t> graph_kernels;   // kernel nodes of each graph
  // Graphs are captured and replayed on a library-owned non-blocking stream
  // (the legacy default stream cannot be captured), joined to the caller's
  // stream by the two events below.
  cudaStream_t gs;
  cudaEvent_t join_in, join_out;
  size_t last_images;
  // instrumentation: one event pair per (step, layer) blind rotation
  bool profile;
  std::vector<cudaEvent_t> ev;  // [T][layers][2]
  std::vector<size_t> ev_count; // ciphertexts of each bracketed launch
};

static void snn_release(fhe_snn *S) {
  if (!S) return;
  for (auto &g : S->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (auto &e : S->ev)
    if (e) cudaEventDestroy(e);
  if (S->join_in) cudaEventDestroy(S->join_in);
  if (S->join_out) cudaEventDestroy(S->join_out);
  if (S->gs) cudaStreamDestroy(S->gs);
  for (auto &L : S->layers) {
    cudaFree(L.d_w); cudaFree(L.d_I); cudaFree(L.d_H); cudaFree(L.d_out);
  }
  cudaFree(S->d_input);
  cudaFree(S->d_scores);
  fhe_lut_free(S->lut);
  delete S;
}

extern "C" int fhe_snn_create(fhe_keys *K, const fhe_snn_desc *d, fhe_snn **out) {
  if (!K || !d || !out || !d->layers || d->n_layers == 0 || d->T == 0 || d->max_images == 0)
    return FHE_EINVAL;
  if (d->variant != FHE_VARIANT_EXACT && d->variant != FHE_VARIANT_TC) return FHE_EINVAL;
  *out = NULL;
  const fhe::Params &P = K->P;
  const int32_t p = (int32_t)P.p();
  fhe_snn *S = new fhe_snn();
  S->K = K;
  S->desc = *d;
  S->desc.layers = NULL;
  // LIF tables on the centred input u = H + p/2, v = u - p/2 (Thm 3.2 / 4.2)
  std::vector<int32_t> f(2u * (size_t)p);
  for (int32_t u = 0; u < p; ++u) {
    const int32_t v = u - p / 2;
    f[u] = (v >= d->v_th) ? d->spike_scale : 0;
    f[p + u] = (v >= d->v_th) ? 0 : (v >= 0 ? (v >> d->leak_shift) : 0);
  }
  int rc = fhe::pbs_prepare(K, d->variant);
  if (rc) { snn_release(S); return rc; }
  rc = fhe_lut_create(K, f.data(), 2u, &S->lut);
  if (rc) { snn_release(S); return rc; }
  uint32_t prev = 0;
  const uint32_t W = P.n + 1u;
  for (uint32_t i = 0; i < d->n_layers; ++i) {
    const fhe_layer_desc &ld = d->layers[i];
    Layer L;
    memset(&L, 0, sizeof(L));
    L.type = ld.type;
    size_t wcount;
    if (ld.type == FHE_LAYER_FC) {
      L.in_size = ld.in_size; L.out_size = ld.out_size;
      wcount = (size_t)ld.in_size * ld.out_size;
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
    const size_t cts = (size_t)d->max_images * L.out_size;
    bool ok = cudaMalloc(&L.d_w, sizeof(int32_t) * wcount) == cudaSuccess &&
              cudaMalloc(&L.d_I, sizeof(uint32_t) * cts * W) == cudaSuccess &&
              cudaMalloc(&L.d_H, sizeof(uint32_t) * cts * W) == cudaSuccess &&
              cudaMalloc(&L.d_out, sizeof(uint32_t) * 2u * cts * W) == cudaSuccess;
    S->layers.push_back(L);
    if (!ok) { snn_release(S); return FHE_ENOMEM; }
    if (cudaMemcpy(L.d_w, ld.weights, sizeof(int32_t) * wcount, cudaMemcpyHostToDevice) != cudaSuccess) {
      snn_release(S); return FHE_ECUDA;
    }
  }
  S->n_in = S->layers.front().in_size;
  S->n_out = S->layers.back().out_size;
  const size_t in_words = (size_t)d->max_images * (d->static_input ? 1u : d->T) * S->n_in * W;
  if (cudaMalloc(&S->d_input, sizeof(uint32_t) * in_words) != cudaSuccess ||
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
    S->ev.assign((size_t)d->T * S->layers.size() * 2u, (cudaEvent_t)0);
    S->ev_count.assign((size_t)d->T * S->layers.size(), 0);
    for (auto &e : S->ev)
      if (cudaEventCreate(&e) != cudaSuccess) { snn_release(S); return FHE_ECUDA; }
  }
  *out = S;
  return FHE_OK;
}

extern "C" int fhe_snn_profile(const fhe_snn *S, double *br_ms, uint64_t *br_launches,
                               uint64_t *br_ciphertexts) {
  if (!S || !S->profile || !br_ms || !br_launches || !br_ciphertexts) return FHE_EINVAL;
  FHE_CUDA_TRY(cudaDeviceSynchronize());
  double ms = 0.0;
  uint64_t launches = 0, cts = 0;
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

extern "C" void fhe_snn_free(fhe_snn *S) {
  if (!S) return;
  cudaDeviceSynchronize();
  snn_release(S);
}

extern "C" uint64_t fhe_snn_pbs_per_image(const fhe_snn *S) {
  if (!S) return 0;
  uint64_t per_step = 0;
  for (const auto &L : S->layers) per_step += L.out_size;
  return per_step * S->desc.T;
}

// Enqueue one time step t for `ni` images.
static int snn_step(fhe_snn *S, uint32_t t, size_t ni, cudaStream_t st) {
  const fhe::Params &P = S->K->P;
  const uint32_t W = P.n + 1u;
  const uint32_t half_p = P.delta() * (P.p() / 2u);  // (p/2) * Delta
  const uint32_t *x = S->d_input + (S->desc.static_input ? 0 : (size_t)t * ni * S->n_in * W);
  int rc;
  for (size_t li = 0; li < S->layers.size(); ++li) {
    Layer &L = S->layers[li];
    const size_t cts = ni * L.out_size;
    const bool static_first = (li == 0 && S->desc.static_input);
    if (!(static_first && t > 0)) {
      if (L.type == FHE_LAYER_FC)
        rc = fhe_lwe_linear(P.n, P.log2_p, L.d_w, L.out_size, L.in_size, NULL, x, ni, L.d_I, st);
      else
        rc = fhe_lwe_conv2d(P.n, P.log2_p, L.d_w, L.cin, L.h, L.w, L.cout, L.kh, L.kw, L.stride,
                            L.pad, NULL, x, ni, L.d_I, st);
      if (rc) return rc;
    }
    uint32_t *V = L.d_out + cts * W;  // membrane potentials from the previous step
    // H = V + I, centred by +p/2 (V = 0 at t = 0)
    rc = fhe::lwe_add(P.n, L.d_I, t ? V : NULL, half_p, cts, L.d_H, st);
    if (rc) return rc;
    if (S->profile) {
      const size_t e = (size_t)t * S->layers.size() + li;
      S->K->prof_ev0 = S->ev[2 * e];
      S->K->prof_ev1 = S->ev[2 * e + 1];
    }
    rc = fhe_pbs_batch(S->K, L.d_H, cts, S->lut, L.d_out, S->desc.variant, st);
    if (S->profile) {
      S->ev_count[(size_t)t * S->layers.size() + li] = S->K->prof_count;
      S->K->prof_ev0 = S->K->prof_ev1 = (cudaEvent_t)0;
    }
    if (rc) return rc;
    x = L.d_out;  // spikes
  }
  const Layer &last = S->layers.back();
  const size_t cts = ni * last.out_size;
  return fhe::lwe_add(P.n, last.d_out, t ? S->d_scores : NULL, 0u, cts, S->d_scores, st);
}

static int snn_capture(fhe_snn *S, size_t ni, cudaStream_t st) {
  for (auto &g : S->graphs)
    if (g) cudaGraphExecDestroy(g);
  S->graphs.assign(S->desc.T, (cudaGraphExec_t)0);
  S->graph_kernels.assign(S->desc.T, 0);
  for (uint32_t t = 0; t < S->desc.T; ++t) {
    cudaGraph_t graph;
    FHE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    // launches enqueued while capturing run only when the graph is replayed
    const int64_t before = (int64_t)fhe::launches();
    int rc = snn_step(S, t, ni, st);
    S->graph_kernels[t] = (int64_t)fhe::launches() - before;
    fhe::note_launches(-S->graph_kernels[t]);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
    FHE_CUDA_TRY(e);
    cudaError_t ie = cudaGraphInstantiate(&S->graphs[t], graph, 0);
    cudaGraphDestroy(graph);
    FHE_CUDA_TRY(ie);
  }
  S->graph_images = ni;
  return FHE_OK;
}

extern "C" int fhe_snn_infer(fhe_snn *S, const uint32_t *ct_input, size_t ni, uint32_t *scores,
                             int inputs_on_host, void *stream) {
  if (!S || !ct_input || !scores || ni == 0 || ni > S->desc.max_images) return FHE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const fhe::Params &P = S->K->P;
  const uint32_t W = P.n + 1u;
  const size_t in_words = ni * (S->desc.static_input ? 1u : S->desc.T) * S->n_in * W;
  FHE_CUDA_TRY(cudaMemcpyAsync(S->d_input, ct_input, sizeof(uint32_t) * in_words,
                               inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  if (S->desc.use_graph & 1) {
    FHE_CUDA_TRY(cudaEventRecord(S->join_in, st));
    FHE_CUDA_TRY(cudaStreamWaitEvent(S->gs, S->join_in, 0));
    if (S->graph_images != ni || S->graphs.size() != S->desc.T) {
      int rc = snn_capture(S, ni, S->gs);
      if (rc) return rc;
    }
    for (uint32_t t = 0; t < S->desc.T; ++t) {
      FHE_CUDA_TRY(cudaGraphLaunch(S->graphs[t], S->gs));
      fhe::note_launches(S->graph_kernels[t]);
    }
    FHE_CUDA_TRY(cudaEventRecord(S->join_out, S->gs));
    FHE_CUDA_TRY(cudaStreamWaitEvent(st, S->join_out, 0));
  } else {
    for (uint32_t t = 0; t < S->desc.T; ++t) {
      int rc = snn_step(S, t, ni, st);
      if (rc) return rc;
    }
  }
  const size_t out_words = ni * S->n_out * W;
  FHE_CUDA_TRY(cudaMemcpyAsync(scores, S->d_scores, sizeof(uint32_t) * out_words,
                               inputs_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  S->last_images = ni;
  if (inputs_on_host) {
    FHE_CUDA_TRY(cudaStreamSynchronize(st));
    return fhe_status(S->K, stream);
  }
  return FHE_OK;
}

extern "C" int fhe_snn_layer_spikes(const fhe_snn *S, uint32_t layer, uint32_t *dst,
                                    void *stream) {
  if (!S || !dst || layer >= S->layers.size() || !S->last_images) return FHE_EINVAL;
  const Layer &L = S->layers[layer];
  const size_t words = S->last_images * L.out_size * (S->K->P.n + 1u);
  FHE_CUDA_TRY(cudaMemcpyAsync(dst, L.d_out, sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return FHE_OK;
}
