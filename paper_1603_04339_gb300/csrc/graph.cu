// Filter graphs: the Chebyshev filters of a batch of independent cells (each its
// own grid, projectors, ns and m) captured once into one CUDA graph whose
// branches run concurrently, then replayed with one launch per step.  Each cell
// owns its workspace, so concurrent branches share nothing but read-only tables.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ham.cuh"
#include "rr.cuh"

using namespace sparc;

struct sparc_filter_graph {
  sparc_ctx* ctx = nullptr;
  int device = 0;                     // destroy needs no live context
  sparc_dtype dtype = SPARC_F32;
  int ncell = 0, nbranch = 1;
  long long kernels = 0;              // kernel nodes of the graph
  std::vector<sparc_ham*> H;
  std::vector<int> m, ns;
  std::vector<long long> ld;
  std::vector<const void*> X;
  std::vector<void*> Y;
  std::vector<double> a, b, a0;
  std::vector<void*> ws;              // per-cell workspace (device)
  std::vector<cudaStream_t> streams;  // capture branches
  std::vector<cudaEvent_t> events;    // fork + one join event per branch
  cudaGraphExec_t exec = nullptr;
};

namespace {

void release(sparc_filter_graph* G) {
  if (G->exec) cudaGraphExecDestroy(G->exec);
  for (cudaEvent_t e : G->events) cudaEventDestroy(e);
  for (cudaStream_t s : G->streams) cudaStreamDestroy(s);
  for (void* p : G->ws) cudaFree(p);
  G->exec = nullptr;
  G->events.clear();
  G->streams.clear();
  G->ws.clear();
}

// Capture the cells' filters: streams[0] forks to every branch, cell i runs on
// branch i % nbranch, every branch joins back into streams[0].
sparc_status capture(sparc_filter_graph* G, cudaGraph_t* out) {
  sparc_ctx* ctx = G->ctx;
  const bool timing = ctx->timing;
  ctx->timing = false;   // no event records inside the graph
  cudaStream_t s0 = G->streams[0];
  const long long l0 = ctx->launches;   // captured launches are counted when the graph runs
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { ctx->timing = timing; return cuda_fail(ctx, e, "cudaStreamBeginCapture"); }
  sparc_status st = SPARC_OK;
  cudaEventRecord(G->events[0], s0);
  for (int j = 1; j < G->nbranch; ++j) cudaStreamWaitEvent(G->streams[j], G->events[0], 0);
  for (int i = 0; i < G->ncell && st == SPARC_OK; ++i) {
    BlockWs w;
    filter_ws(G->H[i], G->dtype, G->ns[i], (char*)G->ws[i], &w);
    st = filter_run(G->H[i], G->dtype, G->m[i], G->a[i], G->b[i], G->a0[i], G->X[i], G->Y[i], G->ns[i], G->ld[i],
                    G->streams[i % G->nbranch], w);
  }
  for (int j = 1; j < G->nbranch; ++j) {
    cudaEventRecord(G->events[j], G->streams[j]);
    cudaStreamWaitEvent(s0, G->events[j], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s0, &g);
  ctx->timing = timing;
  G->kernels = ctx->launches - l0;
  ctx->launches = l0;
  if (st != SPARC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
  *out = g;
  return SPARC_OK;
}

sparc_status check_bounds(sparc_ctx* ctx, int n, const double* a, const double* b, const double* a0) {
  if (!a || !b || !a0) return fail(ctx, SPARC_ERR_INVALID_ARG, "null bounds array");
  for (int i = 0; i < n; ++i)
    if (!(a0[i] < a[i] && a[i] < b[i]) || !isfinite(a0[i]) || !isfinite(b[i]))
      return fail(ctx, SPARC_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
  return SPARC_OK;
}

}  // namespace

extern "C" {

sparc_status sparc_filter_graph_create(sparc_ham* const* H, int ncell, sparc_dtype dtype, const int* m,
                                       const double* a, const double* b, const double* a0,
                                       const void* const* X, void* const* Y, const int* ns, const int64_t* ld,
                                       int nbranch, sparc_filter_graph** out) {
  if (!out) return SPARC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!H || ncell < 1 || !H[0] || !m || !X || !Y || !ns || !ld) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H[0]->ctx;
  if (nbranch < 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "nbranch must be >= 1");
  sparc_status s = check_bounds(ctx, ncell, a, b, a0);
  if (s != SPARC_OK) return s;
  for (int i = 0; i < ncell; ++i) {
    if (!H[i] || H[i]->ctx != ctx) return fail(ctx, SPARC_ERR_INVALID_ARG, "cells must share one context");
    if (m[i] < 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "m must be >= 1");
    s = check_block_args(H[i], dtype, X[i], Y[i], ns[i], ld[i]);
    if (s != SPARC_OK) return s;
  }
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  sparc_filter_graph* G = new (std::nothrow) sparc_filter_graph();
  if (!G) return fail(ctx, SPARC_ERR_OOM, "graph allocation failed");
  G->ctx = ctx;
  G->device = ctx->device;
  G->dtype = dtype;
  G->ncell = ncell;
  G->nbranch = std::min(nbranch, ncell);
  G->H.assign(H, H + ncell);
  G->m.assign(m, m + ncell);
  G->ns.assign(ns, ns + ncell);
  G->ld.assign(ld, ld + ncell);
  G->X.assign(X, X + ncell);
  G->Y.assign(Y, Y + ncell);
  G->a.assign(a, a + ncell);
  G->b.assign(b, b + ncell);
  G->a0.assign(a0, a0 + ncell);
  auto bail = [&](sparc_status st, const char* msg) {
    cudaGetLastError();
    release(G);
    delete G;
    return msg ? fail(ctx, st, msg) : st;
  };
  for (int i = 0; i < ncell; ++i) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(256, filter_ws(H[i], dtype, ns[i], nullptr, nullptr))) != cudaSuccess)
      return bail(SPARC_ERR_OOM, "graph workspace allocation failed");
    G->ws.push_back(p);
  }
  for (int j = 0; j < G->nbranch; ++j) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(SPARC_ERR_CUDA, "stream creation failed");
    G->streams.push_back(st);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(SPARC_ERR_CUDA, "event creation failed");
    G->events.push_back(ev);
  }
  cudaGraph_t g = nullptr;
  s = capture(G, &g);
  if (s != SPARC_OK) return bail(s, nullptr);
  cudaError_t e = cudaGraphInstantiate(&G->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    G->exec = nullptr;
    return bail(SPARC_ERR_CUDA, "cudaGraphInstantiate failed");
  }
  *out = G;
  return SPARC_OK;
}

sparc_status sparc_filter_graph_set_bounds(sparc_filter_graph* G, const double* a, const double* b,
                                           const double* a0) {
  if (!G) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = G->ctx;
  sparc_status s = check_bounds(ctx, G->ncell, a, b, a0);
  if (s != SPARC_OK) return s;
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  const std::vector<double> oa = G->a, ob = G->b, oa0 = G->a0;
  G->a.assign(a, a + G->ncell);
  G->b.assign(b, b + G->ncell);
  G->a0.assign(a0, a0 + G->ncell);
  cudaGraph_t g = nullptr;
  s = capture(G, &g);
  if (s != SPARC_OK) {
    G->a = oa; G->b = ob; G->a0 = oa0;
    return s;
  }
  // same topology, new kernel arguments: update the executable graph in place
  cudaGraphExecUpdateResultInfo info;
  cudaError_t e = cudaGraphExecUpdate(G->exec, g, &info);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) {
      cudaGraphExecDestroy(G->exec);
      G->exec = ex;
    }
  }
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "filter graph update");
  return SPARC_OK;
}

sparc_status sparc_filter_graph_launch(sparc_filter_graph* G, void* stream) {
  if (!G || !G->exec) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(G->ctx, cudaSetDevice(G->ctx->device));
  SPARC_CUDA(G->ctx, cudaGraphLaunch(G->exec, (cudaStream_t)stream));
  G->ctx->launches += G->kernels;
  ++G->ctx->graph_launches;
  return SPARC_OK;
}

void sparc_filter_graph_destroy(sparc_filter_graph* G) {
  if (!G) return;
  cudaSetDevice(G->device);
  cudaDeviceSynchronize();
  release(G);
  delete G;
}

}  // extern "C"
