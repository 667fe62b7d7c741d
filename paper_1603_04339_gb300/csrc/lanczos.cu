// Lanczos estimate of the extremal eigenvalues of H(k), used as Chebyshev
// filter bounds (Section 4: "the Lanczos method for calculating the extremal
// eigenvalues of the Hamiltonian").  FP64 (complex128 at k != 0), one vector,
// full reorthogonalisation, all scalars kept on the device.
#include <math.h>

#include <algorithm>

#include "rr.cuh"

namespace sparc {
namespace {

constexpr int RB = 256;     // threads per reduction block
constexpr int RPARTS = 304; // reduction blocks (2 per SM)

template <class T> __device__ __forceinline__ T lz_zero();
template <> __device__ __forceinline__ double lz_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ cf64 lz_zero<cf64>() { return {0.0, 0.0}; }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cf64 shfl_xor(cf64 v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

// part[b][i] = sum over this block's share of g of conj(V_i[g]) w[g], i < nv
template <class T>
__global__ void __launch_bounds__(RB) k_multidot_part(const T* __restrict__ V, int nv,
                                                      long long vs, const T* __restrict__ w,
                                                      long long nd, T* __restrict__ part) {
  __shared__ T sm[RB];
  for (int i = 0; i < nv; ++i) {
    T acc = lz_zero<T>();
    for (long long g = (long long)blockIdx.x * RB + threadIdx.x; g < nd; g += (long long)gridDim.x * RB)
      acc = fmacj(acc, V[(size_t)i * vs + g], w[g]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RB / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sm[threadIdx.x] = add(sm[threadIdx.x], sm[threadIdx.x + s]);
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 64 + i] = sm[0];
    __syncthreads();
  }
}

// out[i] = sum_b part[b][i] in a fixed order (deterministic).
template <class T>
__global__ void k_multidot_final(const T* __restrict__ part, int nparts, int nv, T* __restrict__ out) {
  // one warp per dot product: lane-strided partial sums, then a fixed butterfly
  const int i = blockIdx.x, lane = threadIdx.x;
  if (i >= nv) return;
  T acc = lz_zero<T>();
  for (int b = lane; b < nparts; b += 32) acc = add(acc, part[(size_t)b * 64 + i]);
  for (int o = 16; o > 0; o >>= 1) acc = add(acc, shfl_xor(acc, o));
  if (lane == 0) out[i] = acc;
}

// alpha_j = Re(dot); w -= alpha_j v_j + beta_{j-1} v_{j-1}
template <class T>
__global__ void k_three_term(T* __restrict__ w, const T* __restrict__ vj, const T* __restrict__ vjm1,
                             const T* __restrict__ dot, double* __restrict__ alpha,
                             const double* __restrict__ beta, int j, long long nd) {
  const double a = Tr<T>::re(dot[0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) alpha[j] = a;
  const double bm = (j > 0) ? beta[j - 1] : 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nd;
       g += (long long)gridDim.x * blockDim.x) {
    T x = axpy(w[g], -a, vj[g]);
    if (j > 0) x = axpy(x, -bm, vjm1[g]);
    w[g] = x;
  }
}

// w -= sum_i h_i V_i (classical Gram-Schmidt against all Lanczos vectors)
template <class T>
__global__ void k_reorth(T* __restrict__ w, const T* __restrict__ V, int nv, long long vs,
                         const T* __restrict__ h, long long nd) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nd;
       g += (long long)gridDim.x * blockDim.x) {
    T s = lz_zero<T>();
    for (int i = 0; i < nv; ++i) s = fmac(s, V[(size_t)i * vs + g], h[i]);
    w[g] = w[g] - s;
  }
}

// beta_j = ||w|| (from dot = w^H w); v_{j+1} = w / beta_j
template <class T>
__global__ void k_normalise(const T* __restrict__ w, T* __restrict__ vnext, const T* __restrict__ dot,
                            double* __restrict__ beta, int j, int write, long long nd) {
  const double b = sqrt(Tr<T>::re(dot[0]));
  if (blockIdx.x == 0 && threadIdx.x == 0) beta[j] = b;
  if (!write) return;
  const double inv = 1.0 / b;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nd;
       g += (long long)gridDim.x * blockDim.x)
    vnext[g] = scale(inv, w[g]);
}

// v0 / ||v0|| into V_0
template <class T>
__global__ void k_start(const T* __restrict__ v0, T* __restrict__ V0, const T* __restrict__ dot,
                        long long nd) {
  const double inv = 1.0 / sqrt(Tr<T>::re(dot[0]));
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nd;
       g += (long long)gridDim.x * blockDim.x)
    V0[g] = scale(inv, v0[g]);
}

// Number of eigenvalues of the symmetric tridiagonal T (diag a, off-diag b) below x
// (Sturm sequence of the LDL^T pivots of T - x I).
__device__ int sturm_count(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    if (q == 0.0) q = 1e-300;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Smallest and largest eigenvalue of T by multisection on the Sturm count (one warp:
// each step evaluates the count at 32 interior points and keeps the sub-interval where
// it reaches its target, shrinking the bracket 33-fold); writes out[0] = theta_min,
// out[1] = theta_max + |beta_k|.
__global__ void k_tridiag_bounds(const double* __restrict__ alpha, const double* __restrict__ beta,
                                 int k, double* __restrict__ out) {
  const int lane = threadIdx.x;
  if (lane >= 32) return;
  double lo = alpha[0], hi = alpha[0];
  for (int i = 0; i < k; ++i) {   // Gershgorin bracket
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < k ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  const double span = fmax(hi - lo, 1e-300);
  lo -= 1e-3 * span;
  hi += 1e-3 * span;
  double res[2];
  for (int which = 0; which < 2; ++which) {
    // which = 0: boundary of count 0 -> 1 (theta_min); which = 1: count k-1 -> k (theta_max)
    const int target = (which == 0) ? 1 : k;
    double l = lo, h = hi;
    for (int it = 0; it < 40; ++it) {
      const double x = l + (h - l) * (double)(lane + 1) / 33.0;
      // the points are nondecreasing in the lane, so the counts are too, even where x
      // rounds onto l or h
      const unsigned hit = __ballot_sync(0xffffffffu, sturm_count(alpha, beta, k, x) >= target);
      double nl = l, nh = h;
      if (hit) {
        const int j = __ffs(hit) - 1;   // first point at or past the boundary
        nh = l + (h - l) * (double)(j + 1) / 33.0;
        if (j > 0) nl = l + (h - l) * (double)j / 33.0;
      } else {
        nl = l + (h - l) * 32.0 / 33.0;
      }
      if (!(nl > l || nh < h)) break;   // no progress at FP64 resolution
      l = nl;
      h = nh;
    }
    res[which] = 0.5 * (l + h);
  }
  if (lane == 0) {
    out[0] = res[0];
    out[1] = res[1] + fabs(beta[k - 1]);
  }
}

template <class T>
sparc_status lanczos(sparc_ham* H, int ksteps, const T* v0, double* a0, double* b, cudaStream_t st) {
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  const size_t es = sizeof(T);
  const size_t vbytes = align256((size_t)nd * es);
  const size_t need = (size_t)(ksteps + 1) * vbytes + 2 * vbytes /*w, tmp*/ +
                      align256((size_t)std::max(1, H->nproj) * es) +
                      align256((size_t)RPARTS * 64 * es) + align256(128 * es) +
                      align256(256 * sizeof(double));
  if (!ensure_ws(ctx, need)) return fail(ctx, SPARC_ERR_OOM, "workspace allocation failed");
  char* p = (char*)ctx->ws;
  T* V = (T*)p;  // vectors spaced by vbytes
  p += (size_t)(ksteps + 1) * vbytes;
  T* w = (T*)p; p += vbytes;
  p += vbytes;  // spare vector
  T* gc = (T*)p; p += align256((size_t)std::max(1, H->nproj) * es);
  T* part = (T*)p; p += align256((size_t)RPARTS * 64 * es);
  T* dots = (T*)p; p += align256(128 * es);
  double* sc = (double*)p;    // alpha[0..63], beta[64..127], out[128..129]
  double* alpha = sc;
  double* beta = sc + 64;
  double* bounds = sc + 128;
  const long long vstride = (long long)(vbytes / es);
  auto Vi = [&](int i) { return V + (size_t)i * vstride; };
  const int EB = 256, EG = 2 * 152;
  // ||v0|| and V_0
  k_multidot_part<T><<<RPARTS, RB, 0, st>>>(v0, 1, 0, v0, nd, part);
  ++ctx->launches;
  k_multidot_final<T><<<1, 32, 0, st>>>(part, RPARTS, 1, dots);
  ++ctx->launches;
  k_start<T><<<EG, EB, 0, st>>>(v0, Vi(0), dots, nd);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "lanczos start");
  for (int j = 0; j < ksteps; ++j) {
    // w = H v_j  (single vector: interleaved width 1 equals plain layout)
    SPARC_CUDA(ctx, launch_nl_gather<T>(H, Vi(j), 1, 1, gc, st));
    SPARC_CUDA(ctx, launch_hpass<T>(H, Vi(j), nullptr, w, gc, 1, 1, 1.0, 0.0, 0.0, true, st));
    // alpha_j = Re(v_j^H w); w -= alpha_j v_j + beta_{j-1} v_{j-1}
    k_multidot_part<T><<<RPARTS, RB, 0, st>>>(Vi(j), 1, 0, w, nd, part);
    ++ctx->launches;
    k_multidot_final<T><<<1, 32, 0, st>>>(part, RPARTS, 1, dots);
    ++ctx->launches;
    k_three_term<T><<<EG, EB, 0, st>>>(w, Vi(j), j > 0 ? Vi(j - 1) : Vi(j), dots, alpha, beta, j, nd);
    ++ctx->launches;
    // full reorthogonalisation against v_0..v_j (the vectors are spaced by vstride)
    k_multidot_part<T><<<RPARTS, RB, 0, st>>>(V, j + 1, vstride, w, nd, part);
    ++ctx->launches;
    k_multidot_final<T><<<j + 1, 32, 0, st>>>(part, RPARTS, j + 1, dots);
    ++ctx->launches;
    k_reorth<T><<<EG, EB, 0, st>>>(w, V, j + 1, vstride, dots, nd);
    ++ctx->launches;
    // beta_j = ||w||, v_{j+1} = w / beta_j
    k_multidot_part<T><<<RPARTS, RB, 0, st>>>(w, 1, 0, w, nd, part);
    ++ctx->launches;
    k_multidot_final<T><<<1, 32, 0, st>>>(part, RPARTS, 1, dots);
    ++ctx->launches;
    k_normalise<T><<<EG, EB, 0, st>>>(w, j + 1 <= ksteps ? Vi(j + 1) : w, dots, beta, j,
                                      j + 1 < ksteps ? 1 : 0, nd);
    ++ctx->launches;
    SPARC_LAUNCH(ctx, "lanczos step");
  }
  k_tridiag_bounds<<<1, 32, 0, st>>>(alpha, beta, ksteps, bounds);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "lanczos bounds");
  double hb[2];
  SPARC_CUDA(ctx, cudaMemcpyAsync(hb, bounds, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  *a0 = hb[0];
  *b = hb[1];
  return SPARC_OK;
}

}  // namespace
}  // namespace sparc

using namespace sparc;

extern "C" sparc_status sparc_lanczos_bounds(sparc_ham* H, int ksteps, const void* v0, double* a0,
                                             double* b, void* stream) {
  if (!H) return SPARC_ERR_INVALID_ARG;
  if (ksteps < 2 || ksteps > 64) return fail(H->ctx, SPARC_ERR_INVALID_ARG, "ksteps must be in 2..64");
  if (!v0 || !a0 || !b) return fail(H->ctx, SPARC_ERR_INVALID_ARG, "null argument");
  SPARC_CUDA(H->ctx, cudaSetDevice(H->ctx->device));
  const sparc_dtype dt = H->gd.cplx ? SPARC_C128 : SPARC_F64;
  sparc_status s = ensure_vals(H, dt);
  if (s != SPARC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (H->gd.cplx) return lanczos<cf64>(H, ksteps, (const cf64*)v0, a0, b, st);
  return lanczos<double>(H, ksteps, (const double*)v0, a0, b, st);
}
