// Rayleigh-Ritz step of CheFSI (Section 3.4, Eqs. SubspaceGeneralizedEigenproblem
// and OrbitalTransformation): projections H~ = U^H H U and M~ = U^H U, Cholesky
// orthonormalisation M~ = L L^H, eigenproblem of C = L^-1 H~ L^-H by parallel
// cyclic Jacobi, and the rotation U <- U L^-H Q.
#include <math.h>

#include <algorithm>
#include <vector>

#include "rr.cuh"

namespace sparc {
namespace {

// ------------------------------------------------------------------ element conversions
__device__ __forceinline__ float cv(float*, float a) { return a; }
__device__ __forceinline__ float cv(float*, double a) { return (float)a; }
__device__ __forceinline__ double cv(double*, double a) { return a; }
__device__ __forceinline__ double cv(double*, float a) { return (double)a; }
__device__ __forceinline__ cf32 cv(cf32*, cf32 a) { return a; }
__device__ __forceinline__ cf32 cv(cf32*, cf64 a) { return {(float)a.x, (float)a.y}; }
__device__ __forceinline__ cf64 cv(cf64*, cf64 a) { return a; }
__device__ __forceinline__ cf64 cv(cf64*, cf32 a) { return {(double)a.x, (double)a.y}; }

template <class T> __device__ __forceinline__ T zero_of() { return Tr<T>::zero(); }

// ------------------------------------------------------------------ SIMT GEMM (split-K)
// C[kz] = alpha * op(A) op(B) over K-range kz, op(A): M x K, op(B): K x N, all
// column-major.  ACT: A is stored K x M and op(A) = A^H; BCT: B is stored N x K
// and op(B) = B^H.  TC is the multiply type; partial sums are flushed into the
// wide accumulator every KF k-tiles (FP32 products, FP64 running sum).
template <class TA, class TB, class TC, class TO, bool ACT, bool BCT>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, int K, const TA* __restrict__ A, long long lda, const TB* __restrict__ B,
       long long ldb, TO* __restrict__ C, long long ldc, long long cstride, int kchunk,
       double alpha) {
  using TW = typename Wide<TC>::W;
  constexpr int KF = (sizeof(typename Tr<TC>::R) == 4) ? 16 : 1 << 30;
  __shared__ TC As[16][65];
  __shared__ TC Bs[16][65];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TC acc[4][4];
  TW accw[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = zero_of<TC>(); accw[i][j] = zero_of<TW>(); }
  int tiles = 0;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = threadIdx.x + 256 * r;
      int mm, kk;
      if (ACT) { kk = idx % 16; mm = idx / 16; } else { mm = idx % 64; kk = idx / 64; }
      const int m = m0 + mm, k = k0 + kk;
      TC v = zero_of<TC>();
      if (m < M && k < kend) {
        if (ACT) v = Tr<TC>::conj(cv((TC*)nullptr, A[k + (long long)m * lda]));
        else v = cv((TC*)nullptr, A[m + (long long)k * lda]);
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = threadIdx.x + 256 * r;
      int nn, kk;
      if (BCT) { nn = idx % 64; kk = idx / 64; } else { kk = idx % 16; nn = idx / 16; }
      const int n = n0 + nn, k = k0 + kk;
      TC v = zero_of<TC>();
      if (n < N && k < kend) {
        if (BCT) v = Tr<TC>::conj(cv((TC*)nullptr, B[n + (long long)k * ldb]));
        else v = cv((TC*)nullptr, B[k + (long long)n * ldb]);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      TC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
    if (++tiles == KF) {
      tiles = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { accw[i][j] = add(accw[i][j], widen(acc[i][j])); acc[i][j] = zero_of<TC>(); }
    }
  }
  TO* Cz = C + (long long)blockIdx.z * cstride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        TW v = add(accw[i][j], widen(acc[i][j]));
        Cz[m + (long long)n * ldc] = narrow_to((TO*)nullptr, scale(alpha, v));
      }
    }
}

template <class TA, class TB, class TC, class TO, bool ACT, bool BCT>
cudaError_t gemm(sparc_ctx* ctx, int M, int N, int K, const TA* A, long long lda, const TB* B, long long ldb, TO* C,
                 long long ldc, int nsplit, long long cstride, double alpha, cudaStream_t st) {
  int kchunk = (int)(((long long)K + nsplit - 1) / nsplit);
  kchunk = (kchunk + 15) / 16 * 16;
  dim3 grid((unsigned)ceil_div(M, 64), (unsigned)ceil_div(N, 64), (unsigned)nsplit);
  k_gemm<TA, TB, TC, TO, ACT, BCT><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, cstride,
                                                        kchunk, alpha);
  ++ctx->launches;
  return cudaGetLastError();
}

// out = (S + S^H)/2 with S = sum_z part[z] (fixed order).
template <class TW>
__global__ void k_reduce_sym(const TW* __restrict__ part, int nsplit, long long pstride, int n,
                             TW* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  TW a = zero_of<TW>(), b = zero_of<TW>();
  for (int z = 0; z < nsplit; ++z) {
    a = add(a, part[z * pstride + i + (long long)j * n]);
    b = add(b, part[z * pstride + j + (long long)i * n]);
  }
  out[i + (long long)j * n] = scale(0.5, add(a, Tr<TW>::conj(b)));
}

// ------------------------------------------------------------------ Cholesky (one CTA)
// Lower factor M~ = L L^H in place; the strict upper part is zeroed.  A pivot
// that is not positive (below 1e-14 of its diagonal entry) latches
// STATUS_NOT_POSDEF and leaves the factor unfinished.
template <class TW>
__global__ void __launch_bounds__(1024) k_chol(TW* A, int n, int* status) {
  __shared__ double red[32];
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int j = 0; j < n; ++j) {
    double part = 0.0;
    for (int k = tid; k < j; k += nt) part += Tr<TW>::abs2(A[j + (long long)k * n]);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
      const double ajj = Tr<TW>::re(A[j + (long long)j * n]);
      const double d = ajj - s;
      // a pivot below 1e-14 of the diagonal entry is numerically zero
      if (!(d > 1e-14 * ajj) || !isfinite(d)) {
        bad = 1;
        atomicOr(status, STATUS_NOT_POSDEF);
      } else {
        A[j + (long long)j * n] = from_real<TW>(sqrt(d));
      }
    }
    __syncthreads();
    if (bad) return;
    const double ljj = Tr<TW>::re(A[j + (long long)j * n]);
    for (int i = j + 1 + tid; i < n; i += nt) {
      TW s = A[i + (long long)j * n];
      for (int k = 0; k < j; ++k) s = s - mul(A[i + (long long)k * n], Tr<TW>::conj(A[j + (long long)k * n]));
      A[i + (long long)j * n] = scale(1.0 / ljj, s);
    }
    __syncthreads();
  }
  for (long long t = tid; t < (long long)n * n; t += nt) {
    const int i = (int)(t % n), j = (int)(t / n);
    if (i < j) A[t] = zero_of<TW>();
  }
}

// Linv = L^-1 for lower-triangular L (one CTA, one thread per column).
template <class TW>
__global__ void __launch_bounds__(1024) k_trinv(const TW* __restrict__ L, TW* __restrict__ Li, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < j; ++i) Li[i + (long long)j * n] = zero_of<TW>();
    const double ljj = Tr<TW>::re(L[j + (long long)j * n]);
    Li[j + (long long)j * n] = from_real<TW>(1.0 / ljj);
    for (int i = j + 1; i < n; ++i) {
      TW s = zero_of<TW>();
      for (int k = j; k < i; ++k) s = fmac(s, L[i + (long long)k * n], Li[k + (long long)j * n]);
      Li[i + (long long)j * n] = scale(-1.0 / Tr<TW>::re(L[i + (long long)i * n]), s);
    }
  }
}

// ------------------------------------------------------------------ parallel cyclic Jacobi
// Round-robin ordering: in round r, position 0 holds index 0 and position i > 0
// holds 1 + (i - 1 + r) mod (npad - 1); pair P joins positions P and npad-1-P.
__device__ __forceinline__ int rr_player(int pos, int r, int npad) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (npad - 1);
}

// 2x2 unitary U (entries u[x][y], x,y in {p,q}) that annihilates A_pq:
// U = diag(1, e^{-i phi}) [[c, s], [-s, c]], e^{i phi} = A_pq/|A_pq|,
// t = sign(th)/(|th| + sqrt(th^2 + 1)), th = (A_qq - A_pp)/(2|A_pq|), c = 1/sqrt(1+t^2), s = t c.
template <class TW>
__device__ void jacobi_rot(const TW* A, int n, int p, int q, TW u[2][2]) {
  const TW one = from_real<TW>(1.0);
  u[0][0] = one; u[0][1] = zero_of<TW>(); u[1][0] = zero_of<TW>(); u[1][1] = one;
  if (p >= n || q >= n) return;
  const TW b = A[p + (long long)q * n];
  const double ab = sqrt(Tr<TW>::abs2(b));
  const double a = Tr<TW>::re(A[p + (long long)p * n]);
  const double d = Tr<TW>::re(A[q + (long long)q * n]);
  if (ab == 0.0 || ab < 1e-300) return;
  const double th = (d - a) / (2.0 * ab);
  const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
  const double c = 1.0 / sqrt(t * t + 1.0);
  const double s = t * c;
  const TW eph = Tr<TW>::conj(scale(1.0 / ab, b));   // e^{-i phi}
  u[0][0] = scale(c, one);
  u[0][1] = scale(s, one);
  u[1][0] = scale(-s, eph);
  u[1][1] = scale(c, eph);
}

template <class TW>
__global__ void __launch_bounds__(256)
k_jacobi_round(const TW* __restrict__ A, TW* __restrict__ An, TW* __restrict__ V, int n, int npad,
               int r) {
  const int half = npad / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nA = (long long)half * half;
  if (t < nA) {
    const int P = (int)(t % half), Q = (int)(t / half);
    const int ip[2] = {rr_player(P, r, npad), rr_player(npad - 1 - P, r, npad)};
    const int iq[2] = {rr_player(Q, r, npad), rr_player(npad - 1 - Q, r, npad)};
    TW up[2][2], uq[2][2];
    jacobi_rot(A, n, ip[0], ip[1], up);
    jacobi_rot(A, n, iq[0], iq[1], uq);
    TW a[2][2];
    for (int x = 0; x < 2; ++x)
      for (int y = 0; y < 2; ++y)
        a[x][y] = (ip[x] < n && iq[y] < n) ? A[ip[x] + (long long)iq[y] * n] : zero_of<TW>();
    for (int aa = 0; aa < 2; ++aa)
      for (int bb = 0; bb < 2; ++bb) {
        if (ip[aa] >= n || iq[bb] >= n) continue;
        TW s = zero_of<TW>();
        for (int x = 0; x < 2; ++x)
          for (int y = 0; y < 2; ++y)
            s = s + mul(Tr<TW>::conj(up[x][aa]), mul(a[x][y], uq[y][bb]));
        An[ip[aa] + (long long)iq[bb] * n] = s;
      }
  } else {
    const long long t2 = t - nA;
    if (t2 >= (long long)n * half) return;
    const int i = (int)(t2 % n), Q = (int)(t2 / n);
    const int iq[2] = {rr_player(Q, r, npad), rr_player(npad - 1 - Q, r, npad)};
    TW uq[2][2];
    jacobi_rot(A, n, iq[0], iq[1], uq);
    TW v[2];
    for (int y = 0; y < 2; ++y) v[y] = (iq[y] < n) ? V[i + (long long)iq[y] * n] : zero_of<TW>();
    for (int bb = 0; bb < 2; ++bb) {
      if (iq[bb] >= n) continue;
      TW s = zero_of<TW>();
      for (int y = 0; y < 2; ++y) s = fmac(s, v[y], uq[y][bb]);
      V[i + (long long)iq[bb] * n] = s;
    }
  }
}

template <class TW>
__global__ void k_identity(TW* V, int n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  V[t] = from_real<TW>((t % n == t / n) ? 1.0 : 0.0);
}

// out[0] = sum_{i != j} |A_ij|^2, out[1] = sum |A_ij|^2   (one CTA, fixed order)
template <class TW>
__global__ void __launch_bounds__(1024) k_offnorm(const TW* __restrict__ A, int n, double* out) {
  __shared__ double s0[1024], s1[1024];
  double off = 0.0, tot = 0.0;
  for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
    const double v = Tr<TW>::abs2(A[t]);
    tot += v;
    if (t % n != t / n) off += v;
  }
  s0[threadIdx.x] = off;
  s1[threadIdx.x] = tot;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { s0[threadIdx.x] += s0[threadIdx.x + s]; s1[threadIdx.x] += s1[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = s0[0]; out[1] = s1[0]; }
}

// Ascending order of the diagonal: eig[rank] = A_ii, Q[:, rank] = V[:, i]
// (ties broken by index, so the order is deterministic).
template <class TW>
__global__ void __launch_bounds__(1024) k_sort(const TW* __restrict__ A, const TW* __restrict__ V,
                                               int n, double* __restrict__ eig, TW* __restrict__ Q) {
  __shared__ int perm[1024];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = Tr<TW>::re(A[i + (long long)i * n]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = Tr<TW>::re(A[j + (long long)j * n]);
      if (lj < li || (lj == li && j < i)) ++rank;
    }
    perm[rank] = i;
    eig[rank] = li;
  }
  __syncthreads();
  for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
    const int row = (int)(t % n), col = (int)(t / n);
    Q[t] = V[row + (long long)perm[col] * n];
  }
}

template <class TW, class T>
__global__ void k_narrow(const TW* __restrict__ a, T* __restrict__ b, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = narrow_to((T*)nullptr, a[t]);
}

// ------------------------------------------------------------------ driver
template <class T, class TC>
sparc_status rayleigh_ritz(sparc_ham* H, T* U, int ns, long long ld, double* eig, cudaStream_t st) {
  using TW = typename Wide<T>::W;
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  const size_t es = sizeof(T), ew = sizeof(TW);
  const long long nn = (long long)ns * ns;
  const int tiles = ceil_div(ns, 64) * ceil_div(ns, 64);
  int nsplit = std::max(1, std::min(256, ceil_div(2 * 152, tiles)));
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, nd / 64));
  const size_t hub = align256((size_t)nd * ns * es);
  const size_t sm = align256((size_t)nn * ew);
  const size_t partb = align256((size_t)nsplit * nn * ew);
  const size_t extra = hub + 2 * partb + 10 * sm + align256(nn * es) + 256;
  BlockWs w;
  char* tail = nullptr;
  sparc_status s = block_ws(H, DtypeOf<T>::v, ns, extra, &w, &tail);
  if (s != SPARC_OK) return s;
  T* HU = (T*)tail; tail += hub;
  TW* partH = (TW*)tail; tail += partb;
  TW* partM = (TW*)tail; tail += partb;
  TW* Hs = (TW*)tail; tail += sm;
  TW* Ms = (TW*)tail; tail += sm;      // becomes L
  TW* Li = (TW*)tail; tail += sm;
  TW* T1 = (TW*)tail; tail += sm;
  TW* A0 = (TW*)tail; tail += sm;
  TW* A1 = (TW*)tail; tail += sm;
  TW* Vj = (TW*)tail; tail += sm;
  TW* Qs = (TW*)tail; tail += sm;
  TW* Yr = (TW*)tail; tail += sm;
  double* scal = (double*)tail; tail += sm;
  T* YrT = (T*)tail;

  // 1. HU = H U
  s = apply_block<T>(H, U, HU, ns, ld, st, w);
  if (s != SPARC_OK) return s;
  // 2. H~ = U^H (HU), M~ = U^H U (split-K partials, then fixed-order sum + symmetrisation)
  cudaEvent_t tg = timing_begin(ctx, st);
  SPARC_CUDA(ctx, (gemm<T, T, TC, TW, true, false>(ctx, ns, ns, (int)nd, U, ld, HU, nd, partH, ns, nsplit,
                                                   nn, 1.0, st)));
  SPARC_CUDA(ctx, (gemm<T, T, TC, TW, true, false>(ctx, ns, ns, (int)nd, U, ld, U, ld, partM, ns, nsplit,
                                                   nn, 1.0, st)));
  k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(partH, nsplit, nn, ns, Hs);
  ++ctx->launches;
  k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(partM, nsplit, nn, ns, Ms);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "gram");
  timing_end(ctx, TK_GRAM, tg, st);
  cudaEvent_t te = timing_begin(ctx, st);
  // 3. M~ = L L^H, Linv = L^-1
  k_chol<TW><<<1, 1024, 0, st>>>(Ms, ns, ctx->d_status);
  ++ctx->launches;
  k_trinv<TW><<<1, 1024, 0, st>>>(Ms, Li, ns);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "cholesky");
  int word = 0;
  SPARC_CUDA(ctx, cudaMemcpyAsync(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  if (word & STATUS_NOT_POSDEF) {
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
    return fail(ctx, SPARC_ERR_NOT_POSDEF, "M~ = U^H U is not positive definite");
  }
  // 4. C = Linv H~ Linv^H (symmetrised)
  SPARC_CUDA(ctx, (gemm<TW, TW, TW, TW, false, false>(ctx, ns, ns, ns, Li, ns, Hs, ns, T1, ns, 1, 0, 1.0, st)));
  SPARC_CUDA(ctx, (gemm<TW, TW, TW, TW, false, true>(ctx, ns, ns, ns, T1, ns, Li, ns, partH, ns, 1, 0, 1.0, st)));
  k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(partH, 1, nn, ns, A0);
  ++ctx->launches;
  // 5. Jacobi sweeps on C
  k_identity<TW><<<ceil_div(nn, 256), 256, 0, st>>>(Vj, ns);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "subspace matrix");
  const int npad = ns + (ns & 1);
  const long long nthr = (long long)(npad / 2) * (npad / 2) + (long long)ns * (npad / 2);
  TW* Acur = A0;
  TW* Anext = A1;
  bool converged = false;
  double hs[2];
  for (int sweep = 0; sweep < 40 && !converged; ++sweep) {
    for (int r = 0; r < npad - 1; ++r) {
      // copy-through of the entries no thread writes is not needed: every (P, Q)
      // block covers the whole matrix once per round
      k_jacobi_round<TW><<<ceil_div(nthr, 256), 256, 0, st>>>(Acur, Anext, Vj, ns, npad, r);
      ++ctx->launches;
      std::swap(Acur, Anext);
    }
    SPARC_LAUNCH(ctx, "jacobi round");
    k_offnorm<TW><<<1, 1024, 0, st>>>(Acur, ns, scal);
    ++ctx->launches;
    SPARC_CUDA(ctx, cudaMemcpyAsync(hs, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    converged = !(hs[0] > 1e-26 * hs[1]);
  }
  if (!converged) return fail(ctx, SPARC_ERR_NO_CONVERGENCE, "Jacobi sweep limit reached");
  // 6. ascending order, Ritz vectors of the pencil: Yr = Linv^H Q
  k_sort<TW><<<1, 1024, 0, st>>>(Acur, Vj, ns, eig, Qs);
  ++ctx->launches;
  SPARC_CUDA(ctx, (gemm<TW, TW, TW, TW, true, false>(ctx, ns, ns, ns, Li, ns, Qs, ns, Yr, ns, 1, 0, 1.0, st)));
  // 7. rotation U <- U Yr (into HU, then back into U)
  k_narrow<TW, T><<<ceil_div(nn, 256), 256, 0, st>>>(Yr, YrT, nn);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "ritz vectors");
  timing_end(ctx, TK_EIG, te, st);
  cudaEvent_t tr = timing_begin(ctx, st);
  SPARC_CUDA(ctx, (gemm<T, T, TC, T, false, false>(ctx, (int)nd, ns, ns, U, ld, YrT, ns, HU, nd, 1, 0, 1.0, st)));
  SPARC_CUDA(ctx, cudaMemcpy2DAsync(U, ld * es, HU, nd * es, nd * es, ns, cudaMemcpyDeviceToDevice, st));
  timing_end(ctx, TK_ROT, tr, st);
  return SPARC_OK;
}

}  // namespace
}  // namespace sparc

using namespace sparc;

extern "C" sparc_status sparc_rayleigh_ritz(sparc_ham* H, sparc_dtype dtype, void* U, int ns,
                                            int64_t ld, double* eig, int mode, void* stream) {
  if (!H) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H->ctx;
  if (ns < 2 || ns > 1024) return fail(ctx, SPARC_ERR_INVALID_ARG, "ns must be in 2..1024");
  if (!U || !eig) return fail(ctx, SPARC_ERR_INVALID_ARG, "null argument");
  if ((int)dtype < 0 || (int)dtype > 3) return fail(ctx, SPARC_ERR_INVALID_ARG, "unknown dtype");
  if (H->gd.cplx && (dtype == SPARC_F64 || dtype == SPARC_F32))
    return fail(ctx, SPARC_ERR_INVALID_ARG, "real dtype needs k = 0 (Gamma point)");
  if (ld < H->gd.nd) return fail(ctx, SPARC_ERR_INVALID_ARG, "ld must be >= Nd");
  if (H->gd.nd > 0x7fffffffLL) return fail(ctx, SPARC_ERR_INVALID_ARG, "grid too large");
  const bool wide = (dtype == SPARC_F64 || dtype == SPARC_C128);
  if (mode == SPARC_RR_FP64 && !wide)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "FP64 mode needs F64 or C128 data");
  if (mode == SPARC_RR_MIXED && wide)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "mixed mode needs F32 or C64 data");
  if (mode != SPARC_RR_FP64 && mode != SPARC_RR_MIXED)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "unknown mode");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  sparc_status s = ensure_vals(H, dtype);
  if (s != SPARC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case SPARC_F64: return rayleigh_ritz<double, double>(H, (double*)U, ns, ld, eig, st);
    case SPARC_F32: return rayleigh_ritz<float, float>(H, (float*)U, ns, ld, eig, st);
    case SPARC_C128: return rayleigh_ritz<cf64, cf64>(H, (cf64*)U, ns, ld, eig, st);
    case SPARC_C64: return rayleigh_ritz<cf32, cf32>(H, (cf32*)U, ns, ld, eig, st);
  }
  return SPARC_ERR_INVALID_ARG;
}
