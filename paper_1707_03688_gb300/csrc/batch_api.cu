// Batched NsDLCT over fields of uneven sizes, each with its own ABCD matrix:
// nslct_plan_batch / nslct_batch_* (see include/nslct.h).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "batch_common.h"
#include "fft_pass.cuh"

using namespace nslct;

struct nslct_batch_s {
  int n = 0;
  int device = 0;
  int num_sms = 0;
  std::vector<nslct_plan_t> plans;
  PassDesc* d_descs = nullptr;      // [5][n]
  BatchItem* d_items = nullptr;     // all passes' work lists back to back
  // per pass, up to two work lists: [0] the lines of the configuration
  // `threads`; [1] (128-thread CTAs) the 3*2^a lines, which run packed in the
  // kB3K configuration on a second stream, beside list [0]
  int item_off[5][2] = {};
  int nitems[5][2] = {};
  int* d_counters = nullptr;        // one per pass and list
  // fields whose shorter side is >= split run through their own plan's fused
  // kernels (nslct_forward) instead of the batched launches; chosen by
  // nslct_batch_tune (default: every field batched)
  int split = 1 << 30;
  int threads = 512;   // CTA size of the batched kernels: the smallest that handles every line (tuned)
  std::vector<int> Nx, Ny;
  // the fields that run alone are spread over these streams (forked from and
  // joined to the caller's stream by events), so their passes overlap
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  cudaStream_t xs = nullptr;        // the second list's stream
  cudaEvent_t xfork = nullptr, xjoin = nullptr;
  bool bound = false;
  std::vector<const void*> in;
  std::vector<void*> out;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
};

namespace {


void free_batch(nslct_batch_s* b) {
  if (!b) return;
  for (int k = 0; k < nslct_batch_s::kSide; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->xs) cudaStreamDestroy(b->xs);
  if (b->xfork) cudaEventDestroy(b->xfork);
  if (b->xjoin) cudaEventDestroy(b->xjoin);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counters) cudaFree(b->d_counters);
  for (auto p : b->plans) nslct_destroy(p);
  delete b;
}

bool runs_alone(const nslct_batch_s* b, int f) { return std::min(b->Nx[f], b->Ny[f]) >= b->split; }

#ifndef NSLCT_BATCH_B3K
#define NSLCT_BATCH_B3K 1
#endif
// The configuration that runs lines of length L in a pass when the batch's CTA
// size is `threads`: with 128 threads, the 3*2^a lines of column passes go to
// the packed kB3K kernel (measured on the 256-field workload: column passes
// 20 % faster for those fields; their one-FFT row passes 10-15 % slower at
// three CTAs per SM, so rows stay in the four-CTA kernel).
int line_config(int threads, int L, bool col) {
  return (NSLCT_BATCH_B3K && threads == 128 && col && (L & (L - 1)) != 0 && batch_panel_lines(L, kB3K) > 0)
             ? kB3K
             : threads;
}

// (Re)build the per-pass work lists of the batched fields: every field's
// panels, longest lines first, in the list of the configuration that runs
// their lines.
int build_items(nslct_batch_s* b) {
  std::vector<BatchItem> all;
  for (int k = 0; k < 5; ++k) {
    const bool col = chain_pass_is_column(k);
    std::vector<int> order;
    for (int f = 0; f < b->n; ++f)
      if (!runs_alone(b, f)) order.push_back(f);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      const int la = col ? b->Nx[a] : b->Ny[a], lc = col ? b->Nx[c] : b->Ny[c];
      return la > lc;
    });
    for (int li = 0; li < 2; ++li) {
      b->item_off[k][li] = (int)all.size();
      for (int f : order) {
        const int L = col ? b->Nx[f] : b->Ny[f];
        const int cfg = line_config(b->threads, L, col);
        if ((cfg == kB3K) != (li == 1)) continue;
        const int lines = col ? b->Ny[f] : b->Nx[f];
        const int P = batch_panel_lines(L, cfg);
        for (int panel = 0; panel * P < lines; ++panel) all.push_back(BatchItem{f, panel});
      }
      b->nitems[k][li] = (int)all.size() - b->item_off[k][li];
    }
  }
  if (b->d_items) { cudaFree(b->d_items); b->d_items = nullptr; }
  if (all.empty()) return NSLCT_OK;
  if (cudaMalloc(&b->d_items, all.size() * sizeof(BatchItem)) != cudaSuccess) { b->d_items = nullptr; return NSLCT_E_NOMEM; }
  return cudaMemcpy(b->d_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) == cudaSuccess
             ? NSLCT_OK
             : NSLCT_E_CUDA;
}

void drop_graph(nslct_batch_s* b) {
  if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
}

// Pass k of the batched fields: one persistent launch over each non-empty work
// list (their counters must be zero); the second list runs on its own stream,
// forked from and joined back to `s`.
int launch_list(nslct_batch_s* b, int k, int li, cudaStream_t s) {
  const int n = b->nitems[k][li];
  if (n == 0) return NSLCT_OK;
  const int cfg = li == 1 ? kB3K : b->threads;
  const int per_sm = cfg == kB3K ? 3 : cfg == 128 ? 4 : cfg == 256 ? 2 : 1;
  const int grid = std::min(n, per_sm * b->num_sms);
  const PassDesc* descs = b->d_descs + (size_t)k * b->n;
  const BatchItem* items = b->d_items + b->item_off[k][li];
  int* counter = b->d_counters + 2 * k + li;
  return chain_pass_is_column(k) ? launch_batch_col(grid, cfg, descs, items, n, counter, s)
                                 : launch_batch_row(grid, cfg, descs, items, n, counter, s);
}

int launch_batched_pass(nslct_batch_s* b, int k, cudaStream_t s) {
  if (b->nitems[k][1] == 0) return launch_list(b, k, 0, s);
  if (cudaEventRecord(b->xfork, s) != cudaSuccess || cudaStreamWaitEvent(b->xs, b->xfork, 0) != cudaSuccess)
    return NSLCT_E_CUDA;
  int rc = launch_list(b, k, 1, b->xs);
  if (rc == NSLCT_OK) rc = launch_list(b, k, 0, s);
  if (cudaEventRecord(b->xjoin, b->xs) != cudaSuccess || cudaStreamWaitEvent(s, b->xjoin, 0) != cudaSuccess)
    return NSLCT_E_CUDA;
  return rc;
}

int enqueue(nslct_batch_s* b, cudaStream_t s) {
  // the large fields, each through its own fused passes, round-robin over the
  // side streams; the batched launches run on `s` meanwhile
  int nalone = 0;
  for (int f = 0; f < b->n; ++f) nalone += runs_alone(b, f) ? 1 : 0;
  const int nside = std::min(nalone, (int)nslct_batch_s::kSide);
  if (nside > 0 && cudaEventRecord(b->fork, s) != cudaSuccess) return NSLCT_E_CUDA;
  for (int k = 0; k < nside; ++k)
    if (cudaStreamWaitEvent(b->side[k], b->fork, 0) != cudaSuccess) return NSLCT_E_CUDA;
  for (int f = 0, i = 0; f < b->n; ++f) {
    if (!runs_alone(b, f)) continue;
    const int rc = nslct_forward(b->plans[f], b->in[f], b->out[f], b->side[i++ % nside]);
    if (rc != NSLCT_OK) return rc;
  }
  if (cudaMemsetAsync(b->d_counters, 0, 10 * sizeof(int), s) != cudaSuccess) return NSLCT_E_CUDA;
  for (int k = 0; k < 5; ++k) {
    const int rc = launch_batched_pass(b, k, s);
    if (rc != NSLCT_OK) return rc;
  }
  for (int k = 0; k < nside; ++k)
    if (cudaEventRecord(b->join[k], b->side[k]) != cudaSuccess || cudaStreamWaitEvent(s, b->join[k], 0) != cudaSuccess)
      return NSLCT_E_CUDA;
  return NSLCT_OK;
}

}  // namespace

extern "C" {

int nslct_plan_batch(nslct_batch_t* out, int nfields, const double* abcd, const int* Nx, const int* Ny,
                     const double* dx, const double* dy, unsigned flags) {
  if (!out) return NSLCT_E_ARG;
  *out = nullptr;
  if (nfields <= 0 || !abcd || !Nx || !Ny || !dx || !dy) return NSLCT_E_ARG;
  if ((flags & NSLCT_PREC_MASK) != NSLCT_PREC_FP32) return NSLCT_E_UNSUPPORTED;
  if (flags & (NSLCT_TYPE2 | NSLCT_TYPE_BY_TRACE)) return NSLCT_E_UNSUPPORTED;
  for (int f = 0; f < nfields; ++f)
    if (batch_panel_lines(Nx[f], 512) == 0 || batch_panel_lines(Ny[f], 512) == 0) return NSLCT_E_SIZE;
  nslct_batch_s* b = new (std::nothrow) nslct_batch_s();
  if (!b) return NSLCT_E_NOMEM;
  b->n = nfields;
  // the smallest CTA size that handles every line (the tuner may change it)
  b->threads = 512;
  for (int th : {256, 128}) {
    bool fits = true;
    for (int f = 0; f < nfields && fits; ++f)
      fits = batch_panel_lines(Nx[f], th) != 0 && batch_panel_lines(Ny[f], th) != 0;
    if (!fits) break;
    b->threads = th;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    free_batch(b);
    return NSLCT_E_CUDA;
  }
  for (int f = 0; f < nfields; ++f) {
    nslct_plan_t p = nullptr;
    const int rc = nslct_plan(&p, abcd + 16 * (size_t)f, Nx[f], Ny[f], dx[f], dy[f], flags);
    if (rc != NSLCT_OK) { free_batch(b); return rc; }
    b->plans.push_back(p);
  }
  b->Nx.assign(Nx, Nx + nfields);
  b->Ny.assign(Ny, Ny + nfields);
  bool ev_ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < nslct_batch_s::kSide && ev_ok; ++k)
    ev_ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  ev_ok = ev_ok && cudaStreamCreateWithFlags(&b->xs, cudaStreamNonBlocking) == cudaSuccess &&
          cudaEventCreateWithFlags(&b->xfork, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventCreateWithFlags(&b->xjoin, cudaEventDisableTiming) == cudaSuccess;
  if (!ev_ok) {
    free_batch(b);
    return NSLCT_E_CUDA;
  }
  if (cudaMalloc(&b->d_descs, 5 * (size_t)nfields * sizeof(PassDesc)) != cudaSuccess ||
      cudaMalloc(&b->d_counters, 10 * sizeof(int)) != cudaSuccess) {
    free_batch(b);
    return NSLCT_E_NOMEM;
  }
  int rc = build_items(b);
  if (rc == NSLCT_OK && (prepare_batch_row() != NSLCT_OK || prepare_batch_col() != NSLCT_OK)) rc = NSLCT_E_CUDA;
  if (rc != NSLCT_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return NSLCT_OK;
}

int nslct_batch_size(nslct_batch_t b) { return b ? b->n : 0; }

int nslct_batch_plan(nslct_batch_t b, int field, nslct_plan_t* plan) {
  if (!b || !plan || field < 0 || field >= b->n) return NSLCT_E_ARG;
  *plan = b->plans[field];
  return NSLCT_OK;
}

int nslct_batch_bind(nslct_batch_t b, const void* const* in, void* const* out) {
  if (!b || !in || !out) return NSLCT_E_ARG;
  std::vector<PassDesc> descs(5 * (size_t)b->n);
  for (int f = 0; f < b->n; ++f) {
    if (!in[f] || !out[f]) return NSLCT_E_ARG;
    if ((reinterpret_cast<uintptr_t>(in[f]) | reinterpret_cast<uintptr_t>(out[f])) & 15u) return NSLCT_E_ARG;
    PassDesc d[5];
    build_chain_descs(b->plans[f], in[f], out[f], false, d);
    // the batched kernels run elems_per_thread(L) per thread: their twiddle tables
    for (int k = 0; k < 5; ++k) {
      d[k].tw = chain_pass_is_column(k) ? b->plans[f]->tw16_x : b->plans[f]->tw16_y;
      // the packed batched kernel runs the pass as a program (x2.ntr = 0: not one)
      const int mode = x2_program(d[k], d[k].x2);
      if (mode == 0) d[k].x2.ntr = 0;
      d[k].x2_first_inv = (mode == 2 || mode == 3) ? 1 : 0;
      descs[(size_t)k * b->n + f] = d[k];
    }
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  const bool ok = cudaMemcpy(b->d_descs, descs.data(), descs.size() * sizeof(PassDesc), cudaMemcpyHostToDevice) ==
                  cudaSuccess;
  if (prev != b->device) cudaSetDevice(prev);
  if (!ok) return NSLCT_E_CUDA;
  b->in.assign(in, in + b->n);
  b->out.assign(out, out + b->n);
  b->bound = true;
  drop_graph(b);
  return NSLCT_OK;
}

int nslct_batch_set_split(nslct_batch_t b, int split) {
  if (!b || split < 1) return NSLCT_E_ARG;
  b->split = split;
  drop_graph(b);
  return build_items(b);
}

int nslct_batch_get_split(nslct_batch_t b) { return b ? b->split : 0; }

int nslct_batch_set_threads(nslct_batch_t b, int threads) {
  if (!b || (threads != 128 && threads != 256 && threads != 512)) return NSLCT_E_ARG;
  for (int f = 0; f < b->n; ++f)
    if (batch_panel_lines(b->Nx[f], threads) == 0 || batch_panel_lines(b->Ny[f], threads) == 0) return NSLCT_E_SIZE;
  b->threads = threads;
  drop_graph(b);
  return build_items(b);
}

int nslct_batch_threads(nslct_batch_t b) { return b ? b->threads : 0; }

int nslct_batch_tune(nslct_batch_t b, nslct_stream_t stream, int iters, int* chosen, float* ms_per_forward) {
  if (!b || !b->bound || iters < 1) return NSLCT_E_ARG;
  for (int f = 0; f < b->n; ++f)
    if (b->in[f] == b->out[f]) return NSLCT_E_ARG;  // the timing runs must not feed outputs back in
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  drop_graph(b);
  // candidate thresholds: the distinct shorter sides, and "none"
  std::vector<int> cands;
  for (int f = 0; f < b->n; ++f) cands.push_back(std::min(b->Nx[f], b->Ny[f]));
  std::sort(cands.begin(), cands.end());
  cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
  cands.push_back(1 << 30);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NSLCT_E_CUDA;
  }
  // the batched kernels' CTA size is the other tuned choice: 128 threads
  // (four CTAs per SM, packed line pairs), 256 (two CTAs per SM) or 512,
  // each where every field's lines fit it
  std::vector<int> tile = {512};
  for (int th : {256, 128}) {
    bool fits = true;
    for (int f = 0; f < b->n && fits; ++f)
      fits = batch_panel_lines(b->Nx[f], th) != 0 && batch_panel_lines(b->Ny[f], th) != 0;
    if (fits) tile.push_back(th);
  }
  int best = 1 << 30, best_th = b->threads, rc = NSLCT_OK;
  float best_ms = 0.0f;
  for (int th : tile) {
    for (int c : cands) {
      b->threads = th;
      b->split = c;
      rc = build_items(b);
      if (rc == NSLCT_OK) rc = enqueue(b, s);  // warm-up
      if (rc == NSLCT_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = NSLCT_E_CUDA;
      for (int i = 0; rc == NSLCT_OK && i < iters; ++i) rc = enqueue(b, s);
      if (rc == NSLCT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        rc = NSLCT_E_CUDA;
      float ms = 0.0f;
      if (rc == NSLCT_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = NSLCT_E_CUDA;
      if (rc != NSLCT_OK) break;
      ms /= (float)iters;
      if (best_ms == 0.0f || ms < best_ms) { best_ms = ms; best = c; best_th = th; }
    }
    if (rc != NSLCT_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->split = best;
  b->threads = best_th;
  const int rc2 = build_items(b);
  if (rc == NSLCT_OK) rc = rc2;
  if (chosen) *chosen = best;
  if (ms_per_forward) *ms_per_forward = best_ms;
  return rc;
}

int nslct_batch_capture(nslct_batch_t b, nslct_stream_t stream) {
  if (!b || !b->bound) return NSLCT_E_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!s) return NSLCT_E_ARG;  // the legacy default stream cannot be captured
  drop_graph(b);
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NSLCT_E_CUDA;
  const int rc = enqueue(b, s);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc != NSLCT_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != NSLCT_OK ? rc : NSLCT_E_CUDA;
  }
  if (cudaGraphInstantiate(&b->graph_exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->graph_exec = nullptr;
    return NSLCT_E_CUDA;
  }
  b->graph = g;
  return NSLCT_OK;
}

int nslct_batch_forward(nslct_batch_t b, nslct_stream_t stream) {
  if (!b || !b->bound) return NSLCT_E_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (b->graph_exec) return cudaGraphLaunch(b->graph_exec, s) == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
  return enqueue(b, s);
}

int nslct_batch_forward_pass(nslct_batch_t b, int pass, nslct_stream_t stream) {
  if (!b || !b->bound || pass < 0 || pass > 4) return NSLCT_E_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int f = 0; f < b->n; ++f) {
    if (!runs_alone(b, f)) continue;
    const int rc = nslct_forward_pass(b->plans[f], pass, b->in[f], b->out[f], stream);
    if (rc != NSLCT_OK) return rc;
  }
  if (cudaMemsetAsync(b->d_counters + 2 * pass, 0, 2 * sizeof(int), s) != cudaSuccess) return NSLCT_E_CUDA;
  return launch_batched_pass(b, pass, s);
}

int nslct_batch_forward_each(nslct_batch_t b, nslct_stream_t stream) {
  if (!b || !b->bound) return NSLCT_E_ARG;
  for (int f = 0; f < b->n; ++f) {
    const int rc = nslct_forward(b->plans[f], b->in[f], b->out[f], stream);
    if (rc != NSLCT_OK) return rc;
  }
  return NSLCT_OK;
}

int nslct_batch_destroy(nslct_batch_t b) {
  free_batch(b);
  return NSLCT_OK;
}

}  // extern "C"
