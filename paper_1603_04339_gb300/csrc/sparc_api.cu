// C ABI of libsparc: contexts, H(k) construction, H-apply and the Chebyshev filter.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <new>

#include "ham.cuh"
#include "fast.cuh"
#include "rr.cuh"

namespace sparc {

bool sync_check() {
  static const bool on = [] {
    const char* v = getenv("SPARC_SYNC_CHECK");
    return v != nullptr && v[0] == '1';
  }();
  return on;
}

sparc_status fail(sparc_ctx* ctx, sparc_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

sparc_status cuda_fail(sparc_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? SPARC_ERR_OOM : SPARC_ERR_CUDA, m);
}

cudaEvent_t timing_begin(sparc_ctx* ctx, cudaStream_t st) {
  if (!ctx->timing) return nullptr;
  // launches being captured into a CUDA graph are not timed (an event recorded during
  // capture would become a graph node, not a timestamp)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cs != cudaStreamCaptureStatusNone) return nullptr;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaEventRecord(e, st);
  return e;
}

void timing_end(sparc_ctx* ctx, int which, cudaEvent_t begin, cudaStream_t st) {
  if (!ctx->timing || begin == nullptr) return;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    ctx->ev_pool.push_back(begin);
    return;
  }
  cudaEventRecord(e, st);
  ctx->ev[which].emplace_back(begin, e);
}

static void timing_reset(sparc_ctx* ctx) {
  for (int w = 0; w < sparc_ctx::NTIMED; ++w) {
    for (auto& pr : ctx->ev[w]) {
      ctx->ev_pool.push_back(pr.first);
      ctx->ev_pool.push_back(pr.second);
    }
    ctx->ev[w].clear();
  }
}

bool ensure_ws(sparc_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return true;
  if (ctx->inject_alloc_fail > 0) {   // injected failure: the workspace is left as it is
    --ctx->inject_alloc_fail;
    return false;
  }
  if (ctx->ws) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = std::max(bytes, (size_t)1 << 20);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return false;
  }
  ctx->ws_bytes = want;
  return true;
}

namespace {

__global__ void k_d2f(const double* a, float* b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Central FD weights of the second derivative, Eq. weightsLap.
void fd_weights(int no, double h, double* w) {
  double s = 0.0;
  for (int q = 1; q <= no; ++q) s += 1.0 / ((double)q * q);
  w[0] = -s / (h * h);
  double fo = 1.0;
  for (int q = 2; q <= no; ++q) fo *= q;
  for (int p = 1; p <= no; ++p) {
    double fm = 1.0, fp = 1.0;
    for (int q = 2; q <= no - p; ++q) fm *= q;
    for (int q = 2; q <= no + p; ++q) fp *= q;
    double sign = (p % 2 == 1) ? 1.0 : -1.0;
    w[p] = 2.0 * sign * fo * fo / (h * h * (double)p * p * fm * fp);
  }
}

long long floordiv(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

template <class T>
T make_val(double re, double im);
template <> double make_val<double>(double re, double) { return re; }
template <> float make_val<float>(double re, double) { return (float)re; }
template <> cf64 make_val<cf64>(double re, double im) { return {re, im}; }
template <> cf32 make_val<cf32>(double re, double im) { return {(float)re, (float)im}; }

template <class T>
sparc_status upload_vals(sparc_ham* H, const std::vector<double>& re, const std::vector<double>& im,
                         void** dst) {
  std::vector<T> v(re.size());
  for (size_t e = 0; e < re.size(); ++e) v[e] = make_val<T>(re[e], im.empty() ? 0.0 : im[e]);
  SPARC_CUDA(H->ctx, cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T)));
  SPARC_CUDA(H->ctx, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SPARC_OK;
}

}  // namespace

// Make the chi~ values of H available in the element type `dt` (first use only).
sparc_status ensure_vals(sparc_ham* H, sparc_dtype dt) {
  if (H->nproj == 0 || H->d_p_val[dt] != nullptr) return SPARC_OK;
  sparc_status st = SPARC_OK;
  switch (dt) {
    case SPARC_F64:
      st = upload_vals<double>(H, H->h_p_re, H->h_p_im, &H->d_p_val[dt]);
      if (st == SPARC_OK) st = upload_vals<double>(H, H->h_pt_re, H->h_pt_im, &H->d_pt_val[dt]);
      break;
    case SPARC_F32:
      st = upload_vals<float>(H, H->h_p_re, H->h_p_im, &H->d_p_val[dt]);
      if (st == SPARC_OK) st = upload_vals<float>(H, H->h_pt_re, H->h_pt_im, &H->d_pt_val[dt]);
      break;
    case SPARC_C128:
      st = upload_vals<cf64>(H, H->h_p_re, H->h_p_im, &H->d_p_val[dt]);
      if (st == SPARC_OK) st = upload_vals<cf64>(H, H->h_pt_re, H->h_pt_im, &H->d_pt_val[dt]);
      break;
    case SPARC_C64:
      st = upload_vals<cf32>(H, H->h_p_re, H->h_p_im, &H->d_p_val[dt]);
      if (st == SPARC_OK) st = upload_vals<cf32>(H, H->h_pt_re, H->h_pt_im, &H->d_pt_val[dt]);
      break;
  }
  return st;
}

sparc_status check_block_args(sparc_ham* H, sparc_dtype dt, const void* X, const void* Y, int ns,
                              int64_t ld) {
  sparc_ctx* ctx = H->ctx;
  if ((int)dt < 0 || (int)dt > 3) return fail(ctx, SPARC_ERR_INVALID_ARG, "unknown dtype");
  if (H->gd.cplx && (dt == SPARC_F64 || dt == SPARC_F32))
    return fail(ctx, SPARC_ERR_INVALID_ARG, "real dtype needs k = 0 (Gamma point)");
  if (ns < 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "ns must be >= 1");
  if (ld < H->gd.nd) return fail(ctx, SPARC_ERR_INVALID_ARG, "ld must be >= Nd");
  if (X == nullptr || Y == nullptr) return fail(ctx, SPARC_ERR_INVALID_ARG, "null X or Y");
  const size_t es = dtype_size(dt);
  const char* x0 = (const char*)X;
  const char* y0 = (const char*)Y;
  const size_t span = ((size_t)(ns - 1) * (size_t)ld + (size_t)H->gd.nd) * es;
  if (x0 < y0 + span && y0 < x0 + span) return fail(ctx, SPARC_ERR_INVALID_ARG, "X and Y overlap");
  return ensure_vals(H, dt);
}

sparc_status block_ws(sparc_ham* H, sparc_dtype dt, int ns, size_t extra, BlockWs* w, char** tail) {
  const size_t es = dtype_size(dt);
  const int nblk = ceil_div(ns, NB);
  const size_t bb = align256((size_t)nblk * H->gd.nd * NB * es);
  const size_t gb = align256((size_t)std::max(1, H->nproj) * nblk * NB * es);
  if (!ensure_ws(H->ctx, 2 * bb + gb + extra))
    return fail(H->ctx, SPARC_ERR_OOM, "workspace allocation failed");
  char* p = (char*)H->ctx->ws;
  w->b0 = p;
  w->b1 = p + bb;
  w->gc = p + 2 * bb;
  w->tail = p + 2 * bb + gb;
  if (tail) *tail = p + 2 * bb + gb;
  return SPARC_OK;
}

template <class T>
sparc_status apply_block(sparc_ham* H, const T* X, T* Y, int ns, long long ld, cudaStream_t st,
                         const BlockWs& w) {
  const int nblk = ceil_div(ns, NB);
  T* b0 = (T*)w.b0;
  T* b1 = (T*)w.b1;
  T* gc = (T*)w.gc;
  SPARC_CUDA(H->ctx, launch_to_blocks<T>(X, ld, ns, b0, H->gd.nd, nblk, st));
  ++H->ctx->launches;
  if constexpr (std::is_same<T, float>::value) {
    if (w.gs && fast::usable(H)) {   // the tiled pass in difference form, all blocks in one launch
      SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, b0, nblk, 0, nblk, gc, (T*)w.gs, st));
      SPARC_CUDA(H->ctx, fast::launch_pass<T>(H, b0, nullptr, b1, gc, nblk, 0, nblk, 1.0, 0.0, 0.0, st,
                                              fast::SHAPE_DIFF));
      SPARC_CUDA(H->ctx, launch_from_blocks<T>(b1, H->gd.nd, nblk, Y, ld, ns, st));
      ++H->ctx->launches;
      SPARC_LAUNCH(H->ctx, "H apply");
      return SPARC_OK;
    }
  }
  SPARC_CUDA(H->ctx, launch_nl_gather<T>(H, b0, NB, nblk, gc, st));
  SPARC_CUDA(H->ctx, launch_hpass<T>(H, b0, nullptr, b1, gc, NB, nblk, 1.0, 0.0, 0.0, true, st));
  SPARC_CUDA(H->ctx, launch_from_blocks<T>(b1, H->gd.nd, nblk, Y, ld, ns, st));
  ++H->ctx->launches;
  SPARC_LAUNCH(H->ctx, "H apply");
  return SPARC_OK;
}

// Scaled Chebyshev filter (Eq. ChebFilter), three-term recurrence in the
// normalised form: sigma_1 = e/(a0-c), sigma_{j+1} = 1/(2/sigma_1 - sigma_j),
// Y_1 = (sigma_1/e)(H-c)X, Y_{j+1} = (2 sigma_{j+1}/e)(H-c)Y_j - sigma_j sigma_{j+1} Y_{j-1}.
template <class T>
sparc_status filter_block(sparc_ham* H, int m, double a, double b, double a0, const T* X, T* Y,
                          int ns, long long ld, cudaStream_t st, const BlockWs& w) {
  const int nblk = ceil_div(ns, NB);
  T* prev = (T*)w.b0;
  T* cur = (T*)w.b1;
  T* gc = (T*)w.gc;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double sigma1 = e / (a0 - c);
  double sigma = sigma1;
  SPARC_CUDA(H->ctx, launch_to_blocks<T>(X, ld, ns, prev, H->gd.nd, nblk, st));
  ++H->ctx->launches;
  SPARC_CUDA(H->ctx, launch_nl_gather<T>(H, prev, NB, nblk, gc, st));
  SPARC_CUDA(H->ctx, launch_hpass<T>(H, prev, nullptr, cur, gc, NB, nblk, sigma1 / e, c, 0.0, false, st));
  for (int j = 1; j < m; ++j) {
    const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
    SPARC_CUDA(H->ctx, launch_nl_gather<T>(H, cur, NB, nblk, gc, st));
    SPARC_CUDA(H->ctx, launch_hpass<T>(H, cur, prev, prev, gc, NB, nblk, 2.0 * sigma_new / e, c,
                                       -sigma * sigma_new, false, st));
    std::swap(cur, prev);
    sigma = sigma_new;
  }
  SPARC_CUDA(H->ctx, launch_from_blocks<T>(cur, H->gd.nd, nblk, Y, ld, ns, st));
  ++H->ctx->launches;
  SPARC_LAUNCH(H->ctx, "filter");
  return SPARC_OK;
}

template sparc_status apply_block<double>(sparc_ham*, const double*, double*, int, long long,
                                          cudaStream_t, const BlockWs&);
template sparc_status apply_block<float>(sparc_ham*, const float*, float*, int, long long,
                                         cudaStream_t, const BlockWs&);
template sparc_status apply_block<cf64>(sparc_ham*, const cf64*, cf64*, int, long long,
                                        cudaStream_t, const BlockWs&);
template sparc_status apply_block<cf32>(sparc_ham*, const cf32*, cf32*, int, long long,
                                        cudaStream_t, const BlockWs&);

// The filter on the tiled FP32 / complex64 kernels: per degree one projection and
// one pass launch over a group of blocks (all blocks unless a tuned configuration
// groups them; a group runs all m degrees before the next group starts).
template <class T>
sparc_status filter_block_fast(sparc_ham* H, int m, double a, double b, double a0, const T* X, T* Y,
                               int ns, long long ld, cudaStream_t st, const BlockWs& w) {
  const int nblk = ceil_div(ns, NB);
  T* B0 = (T*)w.b0;
  T* B1 = (T*)w.b1;
  T* gc = (T*)w.gc;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double sigma1 = e / (a0 - c);
  // Blocks per launch.  The pass and the projection are issue-bound far below HBM
  // bandwidth, so keeping a group of blocks L2-resident across degrees does not pay
  // for the partial last wave of every group launch: by default one launch per degree
  // covers all blocks.  A tuned configuration (sparc_autotune_filter) may group blocks
  // and, for FP32, choose the pass tile shape.
  int shape = 0, G = nblk;
  if constexpr (std::is_same<T, float>::value)
    if (fast::tma_usable(H)) shape = fast::SHAPE_TMA;   // the default where it applies
  const auto tu = H->ctx->tuned.find(std::make_tuple((int)DtypeOf<T>::v, H->gd.nd, ns, 1));
  if (tu != H->ctx->tuned.end()) {
    const int tunedG = tu->second & (TUNE_SHAPE - 1);
    if (tunedG > 0) G = std::min(nblk, tunedG);
    if constexpr (!std::is_same<T, cf32>::value) shape = tu->second / TUNE_SHAPE;
  }
  // a tuned configuration is keyed by (dtype, Nd, ns), which other Hamiltonians may share:
  // a tile shape that this H cannot take falls back to the 16 x 16 tiled pass
  if constexpr (std::is_same<T, float>::value)
    if (!fast::shape_usable(H, shape)) shape = 0;
  T* scratch = (T*)w.tail;
  if constexpr (std::is_same<T, float>::value) {
    if (shape == fast::SHAPE_TMA) {
      // the TMA pass on x-padded block buffers (ghost nodes at both ends of every row)
      SPARC_CUDA(H->ctx, fast::launch_to_blocks_px(H, X, ld, ns, B0, nblk, st));
      ++H->ctx->launches;
      T* res = B1;
      for (int g0 = 0; g0 < nblk; g0 += G) {
        const int nb = std::min(G, nblk - g0);
        T* prev = B0;
        T* cur = B1;
        double sigma = sigma1;
        SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, prev, nblk, g0, nb, gc, scratch, st, true));
        SPARC_CUDA(H->ctx, fast::launch_pass_tma(H, prev, nullptr, cur, gc, nblk, g0, nb, sigma1 / e, c, 0.0, st));
        for (int j = 1; j < m; ++j) {
          const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
          SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, cur, nblk, g0, nb, gc, scratch, st, true));
          SPARC_CUDA(H->ctx, fast::launch_pass_tma(H, cur, prev, prev, gc, nblk, g0, nb, 2.0 * sigma_new / e, c,
                                                   -sigma * sigma_new, st));
          std::swap(cur, prev);
          sigma = sigma_new;
        }
        res = cur;
      }
      SPARC_CUDA(H->ctx, fast::launch_from_blocks_px(H, res, nblk, Y, ld, ns, st));
      ++H->ctx->launches;
      return SPARC_OK;
    }
  } else if constexpr (std::is_same<T, cf32>::value) {
    if (fast::tma_usable_c(H)) {
      // the complex TMA pass on x-padded block buffers (ghost nodes carry the Bloch factor)
      SPARC_CUDA(H->ctx, fast::launch_to_blocks_px(H, X, ld, ns, B0, nblk, st));
      ++H->ctx->launches;
      T* res = B1;
      for (int g0 = 0; g0 < nblk; g0 += G) {
        fast::KSlots ks;
        ks.nk = 1;
        ks.nbk = std::min(G, nblk - g0);
        fast::kslot(H, ks.s[0]);
        ks.s[0].ubase = g0;
        ks.s[0].shift = (float)c;
        T* prev = B0;
        T* cur = B1;
        double sigma = sigma1;
        ks.s[0].alpha = (float)(sigma1 / e);
        ks.s[0].beta = 0.f;
        SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, prev, nblk, g0, ks.nbk, gc, scratch, st, true));
        SPARC_CUDA(H->ctx, fast::launch_pass_tma_k(H, prev, nullptr, cur, gc, nblk, ks, st));
        for (int j = 1; j < m; ++j) {
          const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
          ks.s[0].alpha = (float)(2.0 * sigma_new / e);
          ks.s[0].beta = (float)(-sigma * sigma_new);
          SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, cur, nblk, g0, ks.nbk, gc, scratch, st, true));
          SPARC_CUDA(H->ctx, fast::launch_pass_tma_k(H, cur, prev, prev, gc, nblk, ks, st));
          std::swap(cur, prev);
          sigma = sigma_new;
        }
        res = cur;
      }
      SPARC_CUDA(H->ctx, fast::launch_from_blocks_px(H, res, nblk, Y, ld, ns, st));
      ++H->ctx->launches;
      return SPARC_OK;
    }
  }
  SPARC_CUDA(H->ctx, launch_to_blocks<T>(X, ld, ns, B0, H->gd.nd, nblk, st));
  ++H->ctx->launches;
  T* res = B1;
  for (int g0 = 0; g0 < nblk; g0 += G) {
    const int nb = std::min(G, nblk - g0);
    T* prev = B0;
    T* cur = B1;
    double sigma = sigma1;
    SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, prev, nblk, g0, nb, gc, scratch, st));
    SPARC_CUDA(H->ctx, fast::launch_pass<T>(H, prev, nullptr, cur, gc, nblk, g0, nb, sigma1 / e, c, 0.0, st, shape));
    for (int j = 1; j < m; ++j) {
      const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
      SPARC_CUDA(H->ctx, fast::launch_gather<T>(H, cur, nblk, g0, nb, gc, scratch, st));
      SPARC_CUDA(H->ctx, fast::launch_pass<T>(H, cur, prev, prev, gc, nblk, g0, nb, 2.0 * sigma_new / e, c,
                                              -sigma * sigma_new, st, shape));
      std::swap(cur, prev);
      sigma = sigma_new;
    }
    res = cur;
  }
  SPARC_CUDA(H->ctx, launch_from_blocks<T>(res, H->gd.nd, nblk, Y, ld, ns, st));
  ++H->ctx->launches;
  return SPARC_OK;
}

size_t apply_scratch_bytes(sparc_ham* H, sparc_dtype dt, int ns) {
  if (dt == SPARC_F32 && fast::usable(H))
    return align256(fast::gather_scratch_bytes(H, ceil_div(ns, NB), sizeof(float)));
  return 0;
}

size_t filter_ws(sparc_ham* H, sparc_dtype dt, int ns, char* base, BlockWs* w) {
  const size_t es = dtype_size(dt);
  const int nblk = ceil_div(ns, NB);
  // FP32 and complex64 block buffers hold the x-padded layout of the TMA pass where it applies
  const bool tma = (dt == SPARC_F32 && fast::tma_usable(H)) || (dt == SPARC_C64 && fast::tma_usable_c(H));
  const long long ndb = tma ? fast::padded_nd(H) : H->gd.nd;
  const size_t bb = align256((size_t)nblk * ndb * NB * es);
  const size_t gb = align256((size_t)std::max(1, H->nproj) * nblk * NB * es);
  size_t extra = 0;
  if ((dt == SPARC_F32 || dt == SPARC_C64) && fast::usable(H)) extra = fast::gather_scratch_bytes(H, nblk, es);
  if (base) {
    w->b0 = base;
    w->b1 = base + bb;
    w->gc = base + 2 * bb;
    w->tail = base + 2 * bb + gb;
  }
  return 2 * bb + gb + extra;
}

sparc_status filter_run(sparc_ham* H, sparc_dtype dtype, int m, double a, double b, double a0, const void* X,
                        void* Y, int ns, long long ld, cudaStream_t st, const BlockWs& w) {
  switch (dtype) {
    case SPARC_F64:
      return filter_block<double>(H, m, a, b, a0, (const double*)X, (double*)Y, ns, ld, st, w);
    case SPARC_F32:
      if (fast::usable(H)) return filter_block_fast<float>(H, m, a, b, a0, (const float*)X, (float*)Y, ns, ld, st, w);
      return filter_block<float>(H, m, a, b, a0, (const float*)X, (float*)Y, ns, ld, st, w);
    case SPARC_C128:
      return filter_block<cf64>(H, m, a, b, a0, (const cf64*)X, (cf64*)Y, ns, ld, st, w);
    case SPARC_C64:
      if (fast::usable(H)) return filter_block_fast<cf32>(H, m, a, b, a0, (const cf32*)X, (cf32*)Y, ns, ld, st, w);
      return filter_block<cf32>(H, m, a, b, a0, (const cf32*)X, (cf32*)Y, ns, ld, st, w);
  }
  return fail(H->ctx, SPARC_ERR_INVALID_ARG, "unknown dtype");
}

// Launch grouping of a k batch: nkg k-points x nbk of their blocks per launch.
// Minimises the modelled time -- waves of one-CTA-per-SM work items plus 0.05
// wave per launch pair -- over groupings of at most `upl` units (0: any).
struct KGroup { int nkg, nbk; };
static KGroup kbatch_grouping(int nk, int nblk, int items_per_blk, int nsm, int upl) {
  KGroup g{1, 1};
  double best = 1e300;
  for (int nkg = 1; nkg <= std::min(nk, fast::KMAX); ++nkg)
    for (int d = 1; d <= nblk; ++d) {
      const int nbk = ceil_div(nblk, d);
      if (d > 1 && ceil_div(nblk, d - 1) == nbk) continue;
      if (upl > 0 && nkg * nbk > upl && !(nkg == 1 && nbk == 1)) continue;
      double cost = 0.0;
      for (int k0 = 0; k0 < nk; k0 += nkg)
        for (int b0 = 0; b0 < nblk; b0 += nbk) {
          const long long it = (long long)std::min(nkg, nk - k0) * std::min(nbk, nblk - b0) * items_per_blk;
          cost += (double)((it + nsm - 1) / nsm) + 0.05;
        }
      if (cost < best - 1e-9) { best = cost; g = {nkg, nbk}; }
    }
  return g;
}

// The launches of the k-point batch filter below, issued on st.
// tma: every H passes fast::tma_batch_compatible with H0 and the block buffers hold the
// x-padded layout of the TMA pass.
static sparc_status kbatch_launches(sparc_ham* const* Hs, int nk, int m, const double* a, const double* b,
                                    const double* a0, const cf32* X, cf32* Y, int ns, long long ld, const KGroup& G,
                                    size_t bb, size_t gb, bool tma, cudaStream_t st) {
  sparc_ham* H0 = Hs[0];
  sparc_ctx* ctx = H0->ctx;
  const int nblk = ceil_div(ns, NB);
  const long long nd = tma ? fast::padded_nd(H0) : H0->gd.nd;
  const long long U = (long long)nk * nblk;
  char* p = (char*)ctx->ws;
  cf32* B0 = (cf32*)p;
  cf32* B1 = (cf32*)(p + bb);
  cf32* gc = (cf32*)(p + 2 * bb);
  cf32* scratch = (cf32*)(p + 2 * bb + gb);
  const size_t kx = (size_t)ns * (size_t)ld, kb = (size_t)nblk * nd * NB;
  for (int k = 0; k < nk; ++k) {
    if (tma) SPARC_CUDA(ctx, fast::launch_to_blocks_px(Hs[k], X + k * kx, ld, ns, B0 + k * kb, nblk, st));
    else SPARC_CUDA(ctx, launch_to_blocks<cf32>(X + k * kx, ld, ns, B0 + k * kb, nd, nblk, st));
    ++ctx->launches;
  }
  std::vector<double> e(nk), c(nk), s1(nk), sg(nk);
  for (int k = 0; k < nk; ++k) {
    e[k] = 0.5 * (b[k] - a[k]);
    c[k] = 0.5 * (b[k] + a[k]);
    s1[k] = e[k] / (a0[k] - c[k]);
  }
  cf32* res = B1;
  for (int k0 = 0; k0 < nk; k0 += G.nkg)
    for (int b0 = 0; b0 < nblk; b0 += G.nbk) {
      fast::KSlots ks;
      ks.nk = std::min(G.nkg, nk - k0);
      ks.nbk = std::min(G.nbk, nblk - b0);
      for (int kk = 0; kk < ks.nk; ++kk) {
        fast::kslot(Hs[k0 + kk], ks.s[kk]);
        ks.s[kk].ubase = (long long)(k0 + kk) * nblk + b0;
      }
      auto coefs = [&](int j) {   // degree j + 1 of the recurrence, per k
        for (int kk = 0; kk < ks.nk; ++kk) {
          const int k = k0 + kk;
          fast::KSlot& S = ks.s[kk];
          S.shift = (float)c[k];
          if (j == 0) {
            sg[k] = s1[k];
            S.alpha = (float)(s1[k] / e[k]);
            S.beta = 0.f;
          } else {
            const double sn = 1.0 / (2.0 / s1[k] - sg[k]);
            S.alpha = (float)(2.0 * sn / e[k]);
            S.beta = (float)(-sg[k] * sn);
            sg[k] = sn;
          }
        }
      };
      cf32* prev = B0;
      cf32* cur = B1;
      auto pass = [&](const cf32* in, const cf32* pv, cf32* out) {
        return tma ? fast::launch_pass_tma_k(H0, in, pv, out, gc, U, ks, st)
                   : fast::launch_pass_k(H0, in, pv, out, gc, U, ks, st);
      };
      coefs(0);
      SPARC_CUDA(ctx, fast::launch_gather_k(H0, prev, U, ks, nblk, gc, scratch, st, tma));
      SPARC_CUDA(ctx, pass(prev, nullptr, cur));
      for (int j = 1; j < m; ++j) {
        coefs(j);
        SPARC_CUDA(ctx, fast::launch_gather_k(H0, cur, U, ks, nblk, gc, scratch, st, tma));
        SPARC_CUDA(ctx, pass(cur, prev, prev));
        std::swap(cur, prev);
      }
      res = cur;
    }
  for (int k = 0; k < nk; ++k) {
    if (tma) SPARC_CUDA(ctx, fast::launch_from_blocks_px(Hs[k], res + k * kb, nblk, Y + k * kx, ld, ns, st));
    else SPARC_CUDA(ctx, launch_from_blocks<cf32>(res + k * kb, nd, nblk, Y + k * kx, ld, ns, st));
    ++ctx->launches;
  }
  SPARC_LAUNCH(ctx, "filter batch");
  return SPARC_OK;
}

// The complex64 filter of nk Hamiltonians that share the grid and projector
// geometry: the same recurrence as filter_block_fast per k, with every gather
// and pass launch covering the blocks of up to KMAX k-points.  Its launches are
// captured into one CUDA graph and replayed, so that a call is one host launch; a
// call with the same arguments but new bounds updates the graph's parameters.  With
// per-kernel timing on (or the synchronous debug check) the launches are issued
// directly.
static sparc_status filter_kbatch(sparc_ham* const* Hs, int nk, int m, const double* a, const double* b,
                                  const double* a0, const cf32* X, cf32* Y, int ns, long long ld,
                                  cudaStream_t st) {
  sparc_ham* H0 = Hs[0];
  sparc_ctx* ctx = H0->ctx;
  const int nblk = ceil_div(ns, NB);
  const long long nd = H0->gd.nd;
  const long long U = (long long)nk * nblk;
  int upl = 0;
  const auto tu = ctx->tuned.find(std::make_tuple((int)SPARC_C64, nd, ns, nk));
  if (tu != ctx->tuned.end()) upl = tu->second & (TUNE_SHAPE - 1);
  const bool tma = fast::tma_usable_c(H0);
  const int ipu = tma ? fast::tma_items_per_unit(H0) : fast::items_per_block<cf32>(H0);
  const KGroup G = kbatch_grouping(nk, nblk, ipu, ctx->nsm, upl);
  const long long ndb = tma ? fast::padded_nd(H0) : nd;
  const size_t bb = align256((size_t)U * ndb * NB * sizeof(cf32));
  const size_t gb = align256((size_t)std::max(1, H0->nproj) * U * NB * sizeof(cf32));
  const size_t sb = align256(fast::gather_scratch_bytes(H0, G.nkg * G.nbk, sizeof(cf32)));
  if (!ensure_ws(ctx, 2 * bb + gb + sb)) return fail(ctx, SPARC_ERR_OOM, "workspace allocation failed");
  if (ctx->timing || sync_check())
    return kbatch_launches(Hs, nk, m, a, b, a0, X, Y, ns, ld, G, bb, gb, tma, st);
  sparc_ctx::KBatchGraph& K = ctx->kbg;
  const bool same = K.exec && (int)K.H.size() == nk && std::equal(K.H.begin(), K.H.end(), (const void* const*)Hs) &&
                    K.m == m && K.ns == ns && K.ld == ld && K.X == X && K.Y == Y && K.ws == ctx->ws &&
                    K.nkg == G.nkg && K.nbk == G.nbk;
  const bool bounds = same && std::equal(K.a.begin(), K.a.end(), a) && std::equal(K.b.begin(), K.b.end(), b) &&
                      std::equal(K.a0.begin(), K.a0.end(), a0);
  if (!bounds) {
    if (!ctx->cap_stream) SPARC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const long long l0 = ctx->launches;
    SPARC_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    sparc_status s = kbatch_launches(Hs, nk, m, a, b, a0, X, Y, ns, ld, G, bb, gb, tma, ctx->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    const long long kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (s != SPARC_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    SPARC_CUDA(ctx, e);
    bool updated = false;
    if (same) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(K.exec, g, &info) == cudaSuccess;
      if (!updated) cudaGetLastError();
    }
    if (!updated) {
      if (K.exec) cudaGraphExecDestroy(K.exec);
      K.exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&K.exec, g, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        K.exec = nullptr;
        return cuda_fail(ctx, ei, "k-point batch graph instantiation");
      }
    }
    cudaGraphDestroy(g);
    K.H.assign((const void* const*)Hs, (const void* const*)Hs + nk);
    K.m = m;
    K.ns = ns;
    K.ld = ld;
    K.X = X;
    K.Y = Y;
    K.ws = ctx->ws;
    K.nkg = G.nkg;
    K.nbk = G.nbk;
    K.a.assign(a, a + nk);
    K.b.assign(b, b + nk);
    K.a0.assign(a0, a0 + nk);
    K.kernels = kernels;
  }
  SPARC_CUDA(ctx, cudaGraphLaunch(K.exec, st));
  ctx->launches += K.kernels;
  ++ctx->graph_launches;
  return SPARC_OK;
}

}  // namespace sparc

using namespace sparc;

extern "C" {

sparc_status sparc_create(sparc_ctx** out, int device) {
  if (!out) return SPARC_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SPARC_ERR_INVALID_ARG;
  }
  sparc_ctx* ctx = new (std::nothrow) sparc_ctx();
  if (!ctx) return SPARC_ERR_OOM;
  ctx->device = device;
  // status word + 15 words of diagnostics (used only with SPARC_SYNC_CHECK=1)
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->d_status, 16 * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, 16 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SPARC_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
  *out = ctx;
  return SPARC_OK;
}

sparc_status sparc_timing_enable(sparc_ctx* ctx, int on) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  SPARC_CUDA(ctx, cudaDeviceSynchronize());
  timing_reset(ctx);
  ctx->timing = (on != 0);
  return SPARC_OK;
}

sparc_status sparc_last_sweeps(const sparc_ctx* ctx, int* sweeps) {
  if (!ctx || !sweeps) return SPARC_ERR_INVALID_ARG;
  *sweeps = ctx->last_sweeps;
  return SPARC_OK;
}

sparc_status sparc_graph_launch_count(const sparc_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return SPARC_ERR_INVALID_ARG;
  *launches = ctx->graph_launches;
  return SPARC_OK;
}

sparc_status sparc_last_ortho_err(const sparc_ctx* ctx, double* err) {
  if (!ctx || !err) return SPARC_ERR_INVALID_ARG;
  *err = ctx->last_ortho_err;
  return SPARC_OK;
}

sparc_status sparc_debug_inject(sparc_ctx* ctx, int what, int64_t value) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  switch (what) {
    case SPARC_INJECT_ALLOC_FAIL: ctx->inject_alloc_fail = (int)std::max<int64_t>(0, value); return SPARC_OK;
    case SPARC_INJECT_WAIT_LIMIT: ctx->inject_wait_limit = std::max<int64_t>(0, value); return SPARC_OK;
    case SPARC_INJECT_STALL: ctx->inject_stall = value < 0 ? -1 : (int)value; return SPARC_OK;
    case SPARC_INJECT_CG_MAX_ITERS: ctx->inject_cg_max = (int)std::max<int64_t>(0, value); return SPARC_OK;
    case SPARC_INJECT_FP64_ORTHO: ctx->inject_fp64_ortho = (int)std::min<int64_t>(2, std::max<int64_t>(0, value)); return SPARC_OK;
  }
  return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_debug_inject: unknown injection");
}

sparc_status sparc_launch_count(const sparc_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return SPARC_ERR_INVALID_ARG;
  *launches = (int64_t)ctx->launches;
  return SPARC_OK;
}

sparc_status sparc_timing_read(sparc_ctx* ctx, int which, double* ms_total, int64_t* launches) {
  if (!ctx || which < 0 || which >= sparc_ctx::NTIMED || !ms_total || !launches)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "bad timing query");
  double tot = 0.0;
  for (auto& pr : ctx->ev[which]) {
    SPARC_CUDA(ctx, cudaEventSynchronize(pr.second));
    float ms = 0.f;
    SPARC_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
  }
  *ms_total = tot;
  *launches = (int64_t)ctx->ev[which].size();
  return SPARC_OK;
}

void sparc_destroy(sparc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  timing_reset(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  if (ctx->kbg.exec) cudaGraphExecDestroy(ctx->kbg.exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
  for (cudaStream_t& a : ctx->aux_stream)
    if (a) cudaStreamDestroy(a);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx;
}

const char* sparc_last_error(const sparc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

sparc_status sparc_sync(sparc_ctx* ctx, void* stream) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  int word = 0;
  SPARC_CUDA(ctx, cudaMemcpy(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  SPARC_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  if (word & STATUS_TIMEOUT) return fail(ctx, SPARC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (word & STATUS_NOT_POSDEF) return fail(ctx, SPARC_ERR_NOT_POSDEF, "M~ not positive definite");
  if (word & STATUS_BAD_INDEX) return fail(ctx, SPARC_ERR_INVALID_ARG, "a row index was outside its array");
  if (word & STATUS_NO_CONVERGENCE)
    return fail(ctx, SPARC_ERR_NO_CONVERGENCE, "subspace eigensolver did not converge");
  return SPARC_OK;
}

sparc_status sparc_ham_create(sparc_ctx* ctx, const sparc_grid* grid, const double* veff,
                              const sparc_nonlocal* nl, sparc_ham** out) {
  if (!ctx || !grid || !veff || !out) return fail(ctx, SPARC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const sparc_grid& gr = *grid;
  if (gr.fd_radius < 1 || gr.fd_radius > MAX_FD)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "fd_radius must be in 1..8");
  for (int s = 0; s < 3; ++s) {
    if (gr.n[s] < 2 * gr.fd_radius + 1)
      return fail(ctx, SPARC_ERR_INVALID_ARG, "each n_s must be >= 2*fd_radius+1");
    if (!(gr.h[s] > 0.0)) return fail(ctx, SPARC_ERR_INVALID_ARG, "h_s must be > 0");
    if (!isfinite(gr.k[s])) return fail(ctx, SPARC_ERR_INVALID_ARG, "k must be finite");
  }
  const long long nd = (long long)gr.n[0] * gr.n[1] * gr.n[2];
  if (nd > (1LL << 31) - 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "grid too large");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  sparc_ham* H = new (std::nothrow) sparc_ham();
  if (!H) return fail(ctx, SPARC_ERR_OOM, "host allocation failed");
  H->ctx = ctx;
  H->device = ctx->device;
  H->grid = gr;
  GridDev& gd = H->gd;
  gd.n1 = gr.n[0];
  gd.n2 = gr.n[1];
  gd.n3 = gr.n[2];
  gd.no = gr.fd_radius;
  gd.nd = nd;
  gd.cplx = (gr.k[0] != 0.0 || gr.k[1] != 0.0 || gr.k[2] != 0.0) ? 1 : 0;
  for (int s = 0; s < 3; ++s) {
    double w[MAX_FD + 1];
    fd_weights(gr.fd_radius, gr.h[s], w);
    for (int p = 0; p <= MAX_FD; ++p) gd.coef[s][p] = (p <= gr.fd_radius) ? -0.5 * w[p] : 0.0;
    const double kL = gr.k[s] * gr.n[s] * gr.h[s];
    gd.ph_re[s] = cos(kL);
    gd.ph_im[s] = sin(kL);
  }
  auto bail = [&](sparc_status st) {
    sparc_ham_destroy(H);
    return st;
  };
  if (cudaMalloc(&H->d_veff, nd * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&H->d_veff32, nd * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(ctx, SPARC_ERR_OOM, "V_eff allocation failed"));
  }
  sparc_status st = sparc_ham_set_veff(H, veff, 0, nullptr);
  if (st != SPARC_OK) return bail(st);

  // ---- projectors: chi~_p[g] = exp(-i k.(t L)) chi_p[q], g = q mod n, t = floor(q/n)
  const int np = nl ? nl->nproj : 0;
  if (np < 0) return bail(fail(ctx, SPARC_ERR_INVALID_ARG, "nproj < 0"));
  H->nproj = np;
  if (np > 0) {
    if (!nl->box_lo || !nl->box_n || !nl->chi_off || !nl->chi || !nl->gamma)
      return bail(fail(ctx, SPARC_ERR_INVALID_ARG, "null projector array"));
    std::vector<long long> p_off(np + 1, 0);
    for (int p = 0; p < np; ++p) {
      long long sz = 1;
      for (int s = 0; s < 3; ++s) {
        const int nb = nl->box_n[3 * p + s];
        if (nb < 1 || nb > gr.n[s])
          return bail(fail(ctx, SPARC_ERR_INVALID_ARG, "projector box size must be in 1..n_s"));
        sz *= nb;
      }
      if (nl->chi_off[p] < 0 || nl->chi_off[p] + sz > nl->chi_len)
        return bail(fail(ctx, SPARC_ERR_INVALID_ARG, "projector box outside chi"));
      p_off[p + 1] = p_off[p] + sz;
    }
    const long long ne = p_off[np];
    if (ne > (1LL << 31) - 1) return bail(fail(ctx, SPARC_ERR_INVALID_ARG, "too many box nodes"));
    H->n_ent = ne;
    std::vector<int> pg(ne);
    H->h_p_re.resize(ne);
    if (gd.cplx) H->h_p_im.resize(ne);
    const double L[3] = {gr.n[0] * gr.h[0], gr.n[1] * gr.h[1], gr.n[2] * gr.h[2]};
    for (int p = 0; p < np; ++p) {
      const int* lo = nl->box_lo + 3 * p;
      const int* nb = nl->box_n + 3 * p;
      long long e = p_off[p];
      for (int c = 0; c < nb[2]; ++c)
        for (int b = 0; b < nb[1]; ++b)
          for (int a = 0; a < nb[0]; ++a, ++e) {
            const long long q[3] = {(long long)lo[0] + a, (long long)lo[1] + b, (long long)lo[2] + c};
            long long gidx[3];
            double kt = 0.0;
            for (int s = 0; s < 3; ++s) {
              const long long t = floordiv(q[s], gr.n[s]);
              gidx[s] = q[s] - t * gr.n[s];
              kt += gr.k[s] * L[s] * (double)t;
            }
            pg[e] = (int)(gidx[0] + gr.n[0] * (gidx[1] + (long long)gr.n[1] * gidx[2]));
            const double v = nl->chi[nl->chi_off[p] + a + (long long)nb[0] * (b + (long long)nb[1] * c)];
            if (gd.cplx) {
              H->h_p_re[e] = v * cos(kt);
              H->h_p_im[e] = -v * sin(kt);
            } else {
              H->h_p_re[e] = v;
            }
          }
    }
    // node-major copy for the scatter (stable in p)
    std::vector<int> ptr(nd + 1, 0), pp(ne);
    H->h_pt_re.resize(ne);
    if (gd.cplx) H->h_pt_im.resize(ne);
    for (long long e = 0; e < ne; ++e) ptr[pg[e] + 1]++;
    for (long long g = 0; g < nd; ++g) ptr[g + 1] += ptr[g];
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int p = 0; p < np; ++p)
      for (long long e = p_off[p]; e < p_off[p + 1]; ++e) {
        const int slot = fill[pg[e]]++;
        pp[slot] = p;
        H->h_pt_re[slot] = H->h_p_re[e];
        if (gd.cplx) H->h_pt_im[slot] = H->h_p_im[e];
      }
    std::vector<float> g32(np);
    for (int p = 0; p < np; ++p) g32[p] = (float)nl->gamma[p];
    if (cudaMalloc(&H->d_gamma, np * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->d_gamma32, np * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&H->d_p_off, (np + 1) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&H->d_p_g, ne * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&H->d_pt_ptr, (nd + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&H->d_pt_p, ne * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(ctx, SPARC_ERR_OOM, "projector allocation failed"));
    }
    if (cudaMemcpy(H->d_gamma, nl->gamma, np * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_gamma32, g32.data(), np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_p_off, p_off.data(), (np + 1) * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_p_g, pg.data(), ne * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_pt_ptr, ptr.data(), (nd + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_pt_p, pp.data(), ne * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      return bail(cuda_fail(ctx, cudaGetLastError(), "projector upload"));
    }
  }
  {
    const sparc_status fst = fast::build_tables(H, nl);
    if (fst != SPARC_OK) return bail(fst);
  }
  *out = H;
  return SPARC_OK;
}

sparc_status sparc_ham_set_veff(sparc_ham* H, const double* veff, int on_device, void* stream) {
  if (!H || !veff) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nd = H->gd.nd;
  if (on_device) {
    SPARC_CUDA(ctx, cudaMemcpyAsync(H->d_veff, veff, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    SPARC_CUDA(ctx, cudaMemcpy(H->d_veff, veff, nd * sizeof(double), cudaMemcpyHostToDevice));
  }
  k_d2f<<<ceil_div(nd, 256), 256, 0, st>>>(H->d_veff, H->d_veff32, nd);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "veff conversion");
  if (!on_device) SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  return SPARC_OK;
}

void sparc_ham_destroy(sparc_ham* H) {
  if (!H) return;
  cudaSetDevice(H->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {H->d_veff, H->d_veff32, H->d_gamma, H->d_gamma32, H->d_p_off, H->d_p_g,
                  H->d_pt_ptr, H->d_pt_p};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < 4; ++i) {
    if (H->d_p_val[i]) cudaFree(H->d_p_val[i]);
    if (H->d_pt_val[i]) cudaFree(H->d_pt_val[i]);
  }
  if (H->fast) {
    fast::free_tables(*(fast::Tables*)H->fast);
    delete (fast::Tables*)H->fast;
  }
  delete H;
}

sparc_status sparc_apply_H(sparc_ham* H, sparc_dtype dtype, const void* X, void* Y, int ns,
                           int64_t ld, void* stream) {
  if (!H) return SPARC_ERR_INVALID_ARG;
  sparc_status s = check_block_args(H, dtype, X, Y, ns, ld);
  if (s != SPARC_OK) return s;
  SPARC_CUDA(H->ctx, cudaSetDevice(H->ctx->device));
  BlockWs w;
  const size_t gsb = apply_scratch_bytes(H, dtype, ns);
  s = block_ws(H, dtype, ns, gsb, &w, nullptr);
  if (s != SPARC_OK) return s;
  if (gsb) w.gs = w.tail;
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case SPARC_F64: return apply_block<double>(H, (const double*)X, (double*)Y, ns, ld, st, w);
    case SPARC_F32: return apply_block<float>(H, (const float*)X, (float*)Y, ns, ld, st, w);
    case SPARC_C128: return apply_block<cf64>(H, (const cf64*)X, (cf64*)Y, ns, ld, st, w);
    case SPARC_C64: return apply_block<cf32>(H, (const cf32*)X, (cf32*)Y, ns, ld, st, w);
  }
  return SPARC_ERR_INVALID_ARG;
}

sparc_status sparc_cheb_filter(sparc_ham* H, sparc_dtype dtype, int m, double a, double b,
                               double a0, const void* X, void* Y, int ns, int64_t ld,
                               void* stream) {
  if (!H) return SPARC_ERR_INVALID_ARG;
  if (m < 1) return fail(H->ctx, SPARC_ERR_INVALID_ARG, "m must be >= 1");
  if (!(a0 < a && a < b) || !isfinite(a0) || !isfinite(b))
    return fail(H->ctx, SPARC_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
  sparc_status s = check_block_args(H, dtype, X, Y, ns, ld);
  if (s != SPARC_OK) return s;
  SPARC_CUDA(H->ctx, cudaSetDevice(H->ctx->device));
  if (!ensure_ws(H->ctx, filter_ws(H, dtype, ns, nullptr, nullptr)))
    return fail(H->ctx, SPARC_ERR_OOM, "workspace allocation failed");
  BlockWs w;
  filter_ws(H, dtype, ns, (char*)H->ctx->ws, &w);
  return filter_run(H, dtype, m, a, b, a0, X, Y, ns, ld, (cudaStream_t)stream, w);
}

sparc_status sparc_cheb_filter_batch(sparc_ham* const* H, int nk, sparc_dtype dtype, int m, const double* a,
                                     const double* b, const double* a0, const void* X, void* Y, int ns,
                                     int64_t ld, void* stream) {
  if (!H || nk < 1 || !H[0]) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H[0]->ctx;
  if (!a || !b || !a0) return fail(ctx, SPARC_ERR_INVALID_ARG, "null bounds array");
  if ((int)dtype < 0 || (int)dtype > 3) return fail(ctx, SPARC_ERR_INVALID_ARG, "unknown dtype");
  if (m < 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "m must be >= 1");
  if (ns < 1 || ld < H[0]->gd.nd || !X || !Y) return fail(ctx, SPARC_ERR_INVALID_ARG, "bad ns, ld, X or Y");
  const size_t es = dtype_size(dtype);
  const size_t kx = (size_t)ns * (size_t)ld;
  const size_t span = ((size_t)(nk - 1) * kx + (size_t)(ns - 1) * (size_t)ld + (size_t)H[0]->gd.nd) * es;
  const char* x0 = (const char*)X;
  const char* y0 = (const char*)Y;
  if (x0 < y0 + span && y0 < x0 + span) return fail(ctx, SPARC_ERR_INVALID_ARG, "X and Y overlap");
  bool batch = dtype == SPARC_C64;
  for (int k = 0; k < nk; ++k) {
    sparc_ham* Hk = H[k];
    if (!Hk || Hk->ctx != ctx) return fail(ctx, SPARC_ERR_INVALID_ARG, "Hamiltonians must share one context");
    for (int s3 = 0; s3 < 3; ++s3)
      if (Hk->grid.n[s3] != H[0]->grid.n[s3] || Hk->grid.h[s3] != H[0]->grid.h[s3])
        return fail(ctx, SPARC_ERR_INVALID_ARG, "Hamiltonians of a batch must share the grid");
    if (Hk->grid.fd_radius != H[0]->grid.fd_radius || Hk->nproj != H[0]->nproj)
      return fail(ctx, SPARC_ERR_INVALID_ARG, "Hamiltonians of a batch must share the stencil and projectors");
    if (!(a0[k] < a[k] && a[k] < b[k]) || !isfinite(a0[k]) || !isfinite(b[k]))
      return fail(ctx, SPARC_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
    sparc_status s = check_block_args(Hk, dtype, x0 + k * kx * es, y0 + k * kx * es, ns, ld);
    if (s != SPARC_OK) return s;
    batch = batch && fast::usable(Hk) && fast::geometry_hash(Hk) == fast::geometry_hash(H[0]);
    // the TMA pass serves the batch with the tables of H[0]: every H[k] on it, with the
    // same records (projector values at the nodes), so that each k's result is that of
    // its own filter
    if (batch && (fast::tma_usable_c(Hk) || fast::tma_usable_c(H[0])))
      batch = fast::tma_batch_compatible(H[0], Hk);
  }
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (!batch) {
    for (int k = 0; k < nk; ++k) {
      sparc_status s = sparc_cheb_filter(H[k], dtype, m, a[k], b[k], a0[k], x0 + k * kx * es,
                                         (char*)Y + k * kx * es, ns, ld, stream);
      if (s != SPARC_OK) return s;
    }
    return SPARC_OK;
  }
  return filter_kbatch(H, nk, m, a, b, a0, (const cf32*)X, (cf32*)Y, ns, ld, st);
}

sparc_status sparc_filter_kernel(const sparc_ham* H, sparc_dtype dtype, int* out) {
  if (!H || !out || (int)dtype < 0 || (int)dtype > 3) return SPARC_ERR_INVALID_ARG;
  if (H->gd.cplx && (dtype == SPARC_F64 || dtype == SPARC_F32)) return SPARC_ERR_INVALID_ARG;
  *out = SPARC_KERNEL_GENERIC;
  if (dtype == SPARC_F32 && fast::usable(H)) *out = fast::tma_usable(H) ? SPARC_KERNEL_TMA : SPARC_KERNEL_TILED;
  if (dtype == SPARC_C64 && fast::usable(H)) *out = fast::tma_usable_c(H) ? SPARC_KERNEL_TMA : SPARC_KERNEL_TILED;
  return SPARC_OK;
}

sparc_status sparc_set_filter_units(sparc_ctx* ctx, sparc_dtype dtype, int64_t nd, int ns, int nk, int units) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  if ((int)dtype < 0 || (int)dtype > 3 || nd < 1 || ns < 1 || nk < 1 || units < 0)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "bad filter-units key or value");
  const auto key = std::make_tuple((int)dtype, (long long)nd, ns, nk);
  if (units == 0) ctx->tuned.erase(key);
  else ctx->tuned[key] = units;
  return SPARC_OK;
}

sparc_status sparc_autotune_filter(sparc_ham* const* H, int nk, sparc_dtype dtype, int m, const double* a,
                                   const double* b, const double* a0, const void* X, void* Y, int ns,
                                   int64_t ld, void* stream, int* units, double* ms) {
  if (!H || nk < 1 || !H[0]) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H[0]->ctx;
  const bool kb = dtype == SPARC_C64 && nk > 1;
  const bool f32 = dtype == SPARC_F32 && nk == 1;
  const int nblk = ceil_div(std::max(ns, 1), NB);
  const auto key = std::make_tuple((int)dtype, H[0]->gd.nd, ns, nk);
  // candidate units per launch: multiples and fractions of the L2-sized group
  const size_t per_unit = 2 * (size_t)H[0]->gd.nd * NB * (dtype == SPARC_F32 ? 4 : 8);
  const int l2u = (int)std::max<size_t>(1, (size_t)90 * 1024 * 1024 / per_unit);
  std::vector<int> cand;
  if (kb || f32) {
    for (int f : {1, 2, 4}) cand.push_back(std::max(1, l2u / f));
    for (int f : {2, 4, 8}) cand.push_back(l2u * f);
    cand.push_back(nblk);
    if (kb) cand.push_back(nk * nblk);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    if (f32) cand.erase(std::remove_if(cand.begin(), cand.end(), [&](int u) { return u > nblk; }), cand.end());
  }
  // FP32: every blocks-per-launch candidate with each pass tile shape the grid allows
  if (f32) {
    const size_t nc = cand.size();
    for (int sh = 1; sh < fast::NSHAPE_F32; ++sh)
      if (fast::shape_usable(H[0], sh))
        for (size_t i = 0; i < nc; ++i) cand.push_back(cand[i] + sh * TUNE_SHAPE);
  }
  // preference among near-equal times: the TMA pass, then the 16 x 16 and 16 x 8 tiles
  auto shape_rank = [](int code) {
    const int sh = code / TUNE_SHAPE;
    return sh == fast::SHAPE_TMA ? 0 : sh + 1;
  };
  const int mt = std::min(m, 4);
  cudaStream_t st = (cudaStream_t)stream;
  ctx->tuned.erase(key);
  if (cand.empty()) {   // nothing to tune for this type: the filter has one launch shape
    if (units) *units = 0;
    if (ms) *ms = 0.0;
    return sparc_cheb_filter_batch(H, nk, dtype, mt, a, b, a0, X, Y, ns, ld, stream);
  }
  cudaEvent_t e0, e1;
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  SPARC_CUDA(ctx, cudaEventCreate(&e0));
  SPARC_CUDA(ctx, cudaEventCreate(&e1));
  std::vector<double> tms;
  for (int u : cand) {
    ctx->tuned[key] = u;
    double tmin = 1e300;
    for (int rep = 0; rep < 3; ++rep) {   // the first run warms up
      cudaEventRecord(e0, st);
      sparc_status s = sparc_cheb_filter_batch(H, nk, dtype, mt, a, b, a0, X, Y, ns, ld, stream);
      if (s != SPARC_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); ctx->tuned.erase(key); return s; }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0); cudaEventDestroy(e1);
        ctx->tuned.erase(key);
        return cuda_fail(ctx, cudaGetLastError(), "autotune timing");
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) tmin = std::min(tmin, (double)t);
    }
    tms.push_back(tmin);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the fastest, except that a configuration within 3% of it with more blocks per
  // launch (fewer launches; then the preferred tile shape) is preferred: the timed
  // filter is short, and differences that small are within its run-to-run spread
  const double tbest = *std::min_element(tms.begin(), tms.end());
  int best_u = 0;
  double best_ms = 1e300;
  for (size_t i = 0; i < cand.size(); ++i) {
    if (tms[i] > 1.03 * tbest) continue;
    const int u = cand[i], ub = best_u;
    const bool more = best_u == 0 || (u & (TUNE_SHAPE - 1)) > (ub & (TUNE_SHAPE - 1)) ||
                      ((u & (TUNE_SHAPE - 1)) == (ub & (TUNE_SHAPE - 1)) && shape_rank(u) < shape_rank(ub));
    if (more) { best_u = u; best_ms = tms[i]; }
  }
  ctx->tuned[key] = best_u;
  if (units) *units = best_u;
  if (ms) *ms = best_ms;
  return SPARC_OK;
}

}  // extern "C"
