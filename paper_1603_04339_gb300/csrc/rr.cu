// Rayleigh-Ritz step of CheFSI (Section 3.4, Eqs. SubspaceGeneralizedEigenproblem
// and OrbitalTransformation): projections H~ = U^H H U and M~ = U^H U, Cholesky
// orthonormalisation M~ = L L^H, eigenproblem of C = L^-1 H~ L^-H by parallel
// cyclic Jacobi, and the rotation U <- U L^-H Q.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <tuple>
#include <type_traits>
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
       long long ldb, TO* C, long long ldc, long long cstride, int kchunk,
       double alpha, double beta) {
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
        TW v = scale(alpha, add(accw[i][j], widen(acc[i][j])));
        if (beta != 0.0) v = add(v, scale(beta, widen(Cz[m + (long long)n * ldc])));
        Cz[m + (long long)n * ldc] = narrow_to((TO*)nullptr, v);
      }
    }
}

template <class TA, class TB, class TC, class TO, bool ACT, bool BCT>
cudaError_t gemm(sparc_ctx* ctx, int M, int N, int K, const TA* A, long long lda, const TB* B, long long ldb, TO* C,
                 long long ldc, int nsplit, long long cstride, double alpha, cudaStream_t st,
                 double beta = 0.0) {
  int kchunk = (int)(((long long)K + nsplit - 1) / nsplit);
  kchunk = (kchunk + 15) / 16 * 16;
  dim3 grid((unsigned)ceil_div(M, 64), (unsigned)ceil_div(N, 64), (unsigned)nsplit);
  k_gemm<TA, TB, TC, TO, ACT, BCT><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, cstride,
                                                        kchunk, alpha, beta);
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

// Diagonal block of the blocked Cholesky, FP64 or FP32 (TS), in shared memory (one
// CTA): the kb x kb block at A (leading dimension lda, lower part read) is factored
// right-looking, L is written back over the block (strict upper part zeroed), and
// L^-1 is formed in place (column-oriented, from the last column to the first)
// and written to Dk (leading dimension ldd).  A pivot at or below 1e-14 (FP64) or
// 1e-6 (FP32) of its original diagonal entry, or not finite, flags NOT_POSDEF.
template <class TS, int MB>
__global__ void __launch_bounds__(256) k_chol_blk(TS* A, long long lda, TS* Dk, long long ldd, int kb,
                                                  int* status) {
  constexpr TS PIVTOL = sizeof(TS) == 8 ? (TS)1e-14 : (TS)1e-6;
  __shared__ TS S[MB][MB + 1];
  __shared__ TS x[MB];
  __shared__ TS rdiag[MB];   // 1 / L_jj, one division per column (thread 0)
  __shared__ TS a0[MB];      // the block's diagonal before the factorisation
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    const TS v = i >= j ? A[i + (long long)j * lda] : (TS)0;
    S[i][j] = v;
    if (i == j) a0[i] = v;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      // S[j][j] holds a_jj minus the updates of the columns before j
      const TS d = S[j][j];
      const TS ajj = a0[j];
      if (!(d > PIVTOL * ajj) || !isfinite(d)) {
        bad = 1;
        atomicOr(status, STATUS_NOT_POSDEF);
      } else {
        S[j][j] = sqrt(d);
        rdiag[j] = (TS)1 / S[j][j];
      }
    }
    __syncthreads();
    if (bad) return;
    const TS inv = rdiag[j];
    for (int i = j + 1 + tid; i < kb; i += nt) S[i][j] *= inv;
    __syncthreads();
    // trailing lower triangle (i, c), j < c <= i: 16 x 16 thread tiles, no index division
    const int tx = tid & 15, ty = tid >> 4;
    for (int i = j + 1 + ty; i < kb; i += 16) {
      const TS lij = S[i][j];
      for (int c = j + 1 + tx; c <= i; c += 16) S[i][c] -= lij * S[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    A[i + (long long)j * lda] = i >= j ? S[i][j] : (TS)0;
  }
  __syncthreads();
  // in-place inverse: for j = kb-1 .. 0, column j below the diagonal becomes
  // -(1/L_jj) Linv[j+1:, j+1:] L[j+1:, j], using the already inverted trailing block
  __shared__ TS part[16][MB];
  for (int j = kb - 1; j >= 0; --j) {
    const TS ljj = rdiag[j];
    // x_i = sum_{k=j+1..i} Linv[i][k] L[k][j]: 16 partial sums per row over k, then a fixed-order sum
    const int tx = tid & 15, ty = tid >> 4;
    for (int i = j + 1 + ty; i < kb; i += 16) {
      TS s = 0;
      for (int k = j + 1 + tx; k <= i; k += 16) s += S[i][k] * S[k][j];
      part[tx][i] = s;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < kb; i += nt) {
      TS s = 0;
      for (int q = 0; q < 16; ++q) s += (j + 1 + q <= i) ? part[q][i] : (TS)0;
      x[i] = -ljj * s;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < kb; i += nt) S[i][j] = x[i];
    if (tid == 0) S[j][j] = ljj;
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    Dk[i + (long long)j * ldd] = i >= j ? S[i][j] : (TS)0;
  }
}

// The same for complex FP64 blocks (A = L L^H, Hermitian; kb <= 64), right-looking in
// dynamic shared memory (83,968 bytes): column j is scaled by the real 1 / L_jj, the
// trailing lower triangle updated with S_ic -= L_ij conj(L_cj), and L^-1 formed in place
// column by column from the last (X_jj = 1 / L_jj, X_ij = -(1 / L_jj) sum_{k=j+1..i}
// X_ik L_kj).  One launch per diagonal block, in place of the per-column kernels.
constexpr int CHOL_C_SMEM = (64 * 65 + 16 * 64 + 64) * (int)sizeof(cf64);
__global__ void __launch_bounds__(256) k_chol_blk_c(cf64* A, long long lda, cf64* Dk, long long ldd, int kb,
                                                    int* status) {
  extern __shared__ __align__(16) cf64 csm[];
  cf64(*S)[65] = reinterpret_cast<cf64(*)[65]>(csm);
  cf64(*part)[64] = reinterpret_cast<cf64(*)[64]>(csm + 64 * 65);
  cf64* x = csm + 64 * 65 + 16 * 64;
  __shared__ double rdiag[64];
  __shared__ double a0[64];
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    const cf64 v = i >= j ? A[i + (long long)j * lda] : cf64{0.0, 0.0};
    S[i][j] = v;
    if (i == j) a0[i] = v.x;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      const double d = S[j][j].x;   // a_jj minus the updates of the columns before j
      if (!(d > 1e-14 * a0[j]) || !isfinite(d)) {
        bad = 1;
        atomicOr(status, STATUS_NOT_POSDEF);
      } else {
        const double l = sqrt(d);
        S[j][j] = cf64{l, 0.0};
        rdiag[j] = 1.0 / l;
      }
    }
    __syncthreads();
    if (bad) return;
    const double inv = rdiag[j];
    for (int i = j + 1 + tid; i < kb; i += nt) S[i][j] = scale(inv, S[i][j]);
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    for (int i = j + 1 + ty; i < kb; i += 16) {
      const cf64 lij = S[i][j];
      for (int c = j + 1 + tx; c <= i; c += 16) S[i][c] = S[i][c] - lij * Tr<cf64>::conj(S[c][j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    A[i + (long long)j * lda] = i >= j ? S[i][j] : cf64{0.0, 0.0};
  }
  __syncthreads();
  for (int j = kb - 1; j >= 0; --j) {
    const double rj = rdiag[j];
    const int tx = tid & 15, ty = tid >> 4;
    for (int i = j + 1 + ty; i < kb; i += 16) {
      cf64 sacc{0.0, 0.0};
      for (int k = j + 1 + tx; k <= i; k += 16) sacc = sacc + S[i][k] * S[k][j];
      part[tx][i] = sacc;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < kb; i += nt) {
      cf64 sacc{0.0, 0.0};
      for (int q = 0; q < 16; ++q)
        if (j + 1 + q <= i) sacc = sacc + part[q][i];
      x[i] = scale(-rj, sacc);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < kb; i += nt) S[i][j] = x[i];
    if (tid == 0) S[j][j] = cf64{rj, 0.0};
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += nt) {
    const int i = e % kb, j = e / kb;
    Dk[i + (long long)j * ldd] = i >= j ? S[i][j] : cf64{0.0, 0.0};
  }
}

// The same for FP32 blocks of up to 64, left-looking with one thread per row: column j
// is L_jj = sqrt(a_jj - sum_{k<j} L_jk^2), L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj,
// two barriers per column; then thread j forms column j of L^-1 by forward
// substitution, X_jj = 1 / L_jj, X_ij = -(sum_{k=j}^{i-1} L_ik X_kj) / L_ii, with no
// barrier (each thread owns its column).  Same pivot rule as k_chol_blk<float>.
__global__ void __launch_bounds__(64) k_chol_blk_f32(float* A, long long lda, float* Dk, long long ldd, int kb,
                                                     int* status) {
  __shared__ float L[64][65];
  __shared__ float X[64][65];
  __shared__ float rd[64];   // 1 / L_jj
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  float ajj = 0.f;   // thread t: its original diagonal entry
  for (int k = 0; k < 64; ++k) {
    const float v = (t < kb && k <= t) ? A[t + (long long)k * lda] : 0.f;
    L[t][k] = v;
    if (k == t) ajj = v;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    float s0 = 0.f, s1 = 0.f;
    if (t >= j && t < kb) {
      int k = 0;
      for (; k + 1 < j; k += 2) {
        s0 = fmaf(L[t][k], L[j][k], s0);
        s1 = fmaf(L[t][k + 1], L[j][k + 1], s1);
      }
      if (k < j) s0 = fmaf(L[t][k], L[j][k], s0);
    }
    const float sv = (t >= j && t < kb) ? L[t][j] - (s0 + s1) : 0.f;
    if (t == j) {
      if (!(sv > 1e-6f * ajj) || !isfinite(sv)) {
        bad = 1;
        atomicOr(status, STATUS_NOT_POSDEF);
      } else {
        const float r = rsqrtf(sv);   // L_jj = sv r, 1 / L_jj = r (a few ulp)
        L[j][j] = sv * r;
        rd[j] = r;
      }
    }
    __syncthreads();
    if (bad) return;
    if (t > j && t < kb) L[t][j] = sv * rd[j];
    __syncthreads();
  }
  // column t of the inverse (multiplications by the stored reciprocals of the diagonal)
  if (t < kb) {
    for (int i = 0; i < t; ++i) X[i][t] = 0.f;
    X[t][t] = rd[t];
    for (int i = t + 1; i < kb; ++i) {
      float s0 = 0.f, s1 = 0.f;
      int k = t;
      for (; k + 1 < i; k += 2) {
        s0 = fmaf(L[i][k], X[k][t], s0);
        s1 = fmaf(L[i][k + 1], X[k + 1][t], s1);
      }
      if (k < i) s0 = fmaf(L[i][k], X[k][t], s0);
      X[i][t] = -(s0 + s1) * rd[i];
    }
  }
  __syncthreads();
  for (int e = t; e < kb * kb; e += 64) {
    const int i = e % kb, j = e / kb;
    A[i + (long long)j * lda] = i >= j ? L[i][j] : 0.f;
    Dk[i + (long long)j * ldd] = i >= j ? X[i][j] : 0.f;
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

// Rotation of pair (p, q): the 2x2 unitary U = diag(1, e^{-i phi}) [[c, s], [-s, c]]
// with e^{i phi} = A_pq/|A_pq|, t = sign(th)/(|th| + sqrt(th^2 + 1)),
// th = (A_qq - A_pp)/(2|A_pq|), c = 1/sqrt(1 + t^2), s = t c; it annihilates A_pq.
// Stored as (c, s, e^{-i phi}); indices >= n (the padding player) give the identity.
template <class TW>
struct Rot {
  typename Tr<TW>::R c, s;
  TW eph;
};

template <class TW>
__device__ Rot<TW> jacobi_rot(const TW* A, int n, int p, int q) {
  using R = typename Tr<TW>::R;
  Rot<TW> u;
  u.c = (R)1; u.s = (R)0; u.eph = from_real<TW>(1.0);
  if (p >= n || q >= n) return u;
  // the three entries are read together (one memory round trip, not two)
  const TW b = A[p + (long long)q * n];
  const R a = Tr<TW>::re(A[p + (long long)p * n]);
  const R d = Tr<TW>::re(A[q + (long long)q * n]);
  const R ab = sqrt(Tr<TW>::abs2(b));
  if (!(ab > (R)0)) return u;
  const R th = (d - a) / ((R)2 * ab);
  const R t = (th >= (R)0 ? (R)1 : (R)-1) / (fabs(th) + sqrt(th * th + (R)1));
  u.c = (R)1 / sqrt(t * t + (R)1);
  u.s = t * u.c;
  u.eph = Tr<TW>::conj(scale((R)1 / ab, b));
  return u;
}

// entry (x, y) of the 2x2 block of U for a pair: [[c, s], [-s eph, c eph]]
template <class TW>
__device__ __forceinline__ TW rot_entry(const Rot<TW>& u, int x, int y) {
  using R = typename Tr<TW>::R;
  if (x == 0) return from_real<TW>(y == 0 ? (double)u.c : (double)u.s);
  return scale(y == 0 ? -u.s : u.c, u.eph);
}

// One round of the parallel cyclic Jacobi method: A' = U^H A U (into An), V <- V U.
// CTAs [0, nta) update 16 x 16 tiles of 2x2 blocks (pair P, pair Q) of A; the
// remaining CTAs update 64 rows x 4 pairs of V.  Each CTA first computes the
// rotations of the pairs it touches into shared memory.
template <class TW>
__global__ void __launch_bounds__(256)
k_jacobi_round(const TW* __restrict__ A, TW* __restrict__ An, TW* __restrict__ V, int n, int npad,
               int r) {
  __shared__ Rot<TW> rp[16], rq[16];
  __shared__ int ip[16][2], iq[16][2];
  // rounds are chained by programmatic dependent launch: wait until the previous round's
  // grid has completed and its writes are visible (a no-op without such a dependency)
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const int half = npad / 2;
  const int tpa = (half + 15) / 16;           // pair tiles per side
  const int nta = tpa * tpa;
  const int tid = threadIdx.x;
  if ((int)blockIdx.x < nta) {
    const int P0 = (blockIdx.x % tpa) * 16, Q0 = (blockIdx.x / tpa) * 16;
    if (tid < 32) {
      const int k = tid % 16;
      const int Pp = (tid < 16 ? P0 : Q0) + k;
      int p = n, q = n;
      if (Pp < half) { p = rr_player(Pp, r, npad); q = rr_player(npad - 1 - Pp, r, npad); }
      const Rot<TW> u = jacobi_rot(A, n, p, q);
      if (tid < 16) { rp[k] = u; ip[k][0] = p; ip[k][1] = q; }
      else { rq[k] = u; iq[k][0] = p; iq[k][1] = q; }
    }
    __syncthreads();
    const int pl = tid % 16, ql = tid / 16;
    if (P0 + pl >= half || Q0 + ql >= half) return;
    const int i0 = ip[pl][0], i1 = ip[pl][1], j0 = iq[ql][0], j1 = iq[ql][1];
    const int ii[2] = {i0, i1}, jj[2] = {j0, j1};
    TW a[2][2];
    for (int x = 0; x < 2; ++x)
      for (int y = 0; y < 2; ++y)
        a[x][y] = (ii[x] < n && jj[y] < n) ? A[ii[x] + (long long)jj[y] * n] : zero_of<TW>();
    for (int aa = 0; aa < 2; ++aa)
      for (int bb = 0; bb < 2; ++bb) {
        if (ii[aa] >= n || jj[bb] >= n) continue;
        TW s = zero_of<TW>();
        for (int x = 0; x < 2; ++x)
          for (int y = 0; y < 2; ++y)
            s = s + mul(Tr<TW>::conj(rot_entry(rp[pl], x, aa)), mul(a[x][y], rot_entry(rq[ql], y, bb)));
        An[ii[aa] + (long long)jj[bb] * n] = s;
      }
  } else {
    const int vb = blockIdx.x - nta;
    const int rows = (n + 63) / 64;
    const int R0 = (vb % rows) * 64, Q0 = (vb / rows) * 4;
    if (tid < 4) {
      const int Qq = Q0 + tid;
      int p = n, q = n;
      if (Qq < half) { p = rr_player(Qq, r, npad); q = rr_player(npad - 1 - Qq, r, npad); }
      rq[tid] = jacobi_rot(A, n, p, q);
      iq[tid][0] = p; iq[tid][1] = q;
    }
    __syncthreads();
    const int i = R0 + tid % 64, ql = tid / 64;
    if (i >= n || Q0 + ql >= half) return;
    const int jj[2] = {iq[ql][0], iq[ql][1]};
    TW v[2];
    for (int y = 0; y < 2; ++y) v[y] = (jj[y] < n) ? V[i + (long long)jj[y] * n] : zero_of<TW>();
    for (int bb = 0; bb < 2; ++bb) {
      if (jj[bb] >= n) continue;
      TW s = zero_of<TW>();
      for (int y = 0; y < 2; ++y) s = fmac(s, v[y], rot_entry(rq[ql], y, bb));
      V[i + (long long)jj[bb] * n] = s;
    }
  }
}

// ------------------------------------------------------------------ block Jacobi (FP32)
// The parallel cyclic Jacobi method on index blocks of BJ (16 or 32): the npad/BJ blocks
// are paired round-robin (the scalar method's ordering on blocks), and a round rotates
// every pair's 2BJ x 2BJ subproblem A[I, I] (I = the pair's two blocks) by one inner
// cyclic sweep, accumulated into an orthogonal W_I, then applies all of them at once:
// A <- J^T A J and V <- V J with J = blockdiag(W_I).  A sweep is npad/BJ - 1 rounds
// instead of the scalar method's npad - 1, each two launches.
constexpr int BJ_MAX = 16;

// local index l of pair k's 2 BJ indices -> global index
template <int BJ>
__device__ __forceinline__ int bj_index(int l, int bp, int bq) { return l < BJ ? BJ * bp + l : BJ * bq + (l - BJ); }

// rotation of the pair (p, q) of pair subproblem S (local indices): the rotation of
// jacobi_rot (the angle theta in [-pi/4, pi/4] with tan 2 theta = 2b/d, d = S_qq - S_pp,
// b = S_pq), from the half-angle identities: cos 2 theta = |d| / r, sin 2 theta =
// sign(d) 2b / r with r = sqrt(d^2 + 4b^2), c^2 = (1 + cos 2 theta)/2 in [1/2, 1] (no
// cancellation), c = c^2 / sqrt(c^2), s = sin 2 theta / (2c).  Two dependent reciprocal
// square roots (the approximate ones, a few ulp) and no division: the rotation of an
// inner round is on the critical path of the pair solve.  Its small departure from
// orthogonality is removed afterwards by the Newton-Schulz step, and the eigenvalues come
// from FP64 Rayleigh quotients.  b = 0 gives the identity.  (n is a multiple of 2 BJ on
// this path, so every index of a pair subproblem is in range.)
template <int BJ>
__device__ __forceinline__ void bj_rot(const float (&S)[2 * BJ][2 * BJ + 1], int p, int q, float& c, float& sn) {
  const float b = S[p][q];
  const float d = S[q][q] - S[p][p];
  const float b2 = 2.f * b;
  const float rs = rsqrtf(fmaf(d, d, b2 * b2));
  const float cos2 = fabsf(d) * rs;
  const float sin2 = (d >= 0.f ? b2 : -b2) * rs;
  const float h = fmaf(0.5f, cos2, 0.5f);
  const float qh = rsqrtf(h);
  c = b != 0.f ? h * qh : 1.f;
  sn = b != 0.f ? 0.5f * sin2 * qh : 0.f;
}

// player of position x in round rr of the round-robin schedule of 2 BJ players
// (rr_player without the division: x - 1 + rr < 2 (2 BJ - 1))
template <int BJ>
__device__ __forceinline__ int bj_player(int x, int rr) {
  int v = x - 1 + rr;
  v = v >= 2 * BJ - 1 ? v - (2 * BJ - 1) : v;
  return x == 0 ? 0 : 1 + v;
}

// One cyclic sweep over the pair subproblem S (2BJ x 2BJ, in shared memory), its
// rotations accumulated into W (identity on entry) and stored as the pair's rotation
// Wbuf[k].  BJ^2 threads.  S and W are double-buffered: inner round rr reads buffer
// rr & 1 and writes the other, so a round needs one barrier.
template <int BJ>
__device__ __forceinline__ void bj_pair_sweep(float (&S)[2][2 * BJ][2 * BJ + 1], float (&W)[2][2 * BJ][2 * BJ + 1],
                                              float* __restrict__ Wbuf, int k) {
  const int t = threadIdx.x;
  // thread (x, y): the 2 x 2 block (pair x rows, pair y columns) of S and rows 2y, 2y+1
  // of W's pair-x columns.  Every thread computes the two rotations it needs from the
  // same entries (identical arithmetic, identical results), so a round is one read
  // phase and one write phase.
  const int x = t % BJ, y = t / BJ;
  for (int rr = 0; rr < 2 * BJ - 1; ++rr) {
    const int cb = rr & 1, nb = cb ^ 1;
    // the inner round-robin schedule: pair x of round rr is (i0, i1), pair y is (j0, j1)
    const int i0 = bj_player<BJ>(x, rr), i1 = bj_player<BJ>(2 * BJ - 1 - x, rr);
    const int j0 = bj_player<BJ>(y, rr), j1 = bj_player<BJ>(2 * BJ - 1 - y, rr);
    float cx, sx, cy, sy;
    bj_rot<BJ>(S[cb], i0, i1, cx, sx);
    bj_rot<BJ>(S[cb], j0, j1, cy, sy);
    const float a00 = S[cb][i0][j0], a01 = S[cb][i0][j1], a10 = S[cb][i1][j0], a11 = S[cb][i1][j1];
    const float w00 = W[cb][2 * y][i0], w01 = W[cb][2 * y][i1], w10 = W[cb][2 * y + 1][i0],
                w11 = W[cb][2 * y + 1][i1];
    // rows: [r0; r1] = [[c, -s], [s, c]] [a0; a1] (the rotation [[c, s], [-s, c]] transposed)
    const float b00 = cx * a00 - sx * a10, b01 = cx * a01 - sx * a11;
    const float b10 = sx * a00 + cx * a10, b11 = sx * a01 + cx * a11;
    // the threads' 2 x 2 blocks cover every entry of S and of W: the next buffers are
    // written whole
    S[nb][i0][j0] = cy * b00 - sy * b01;
    S[nb][i0][j1] = sy * b00 + cy * b01;
    S[nb][i1][j0] = cy * b10 - sy * b11;
    S[nb][i1][j1] = sy * b10 + cy * b11;
    // W <- W R (columns i0, i1)
    W[nb][2 * y][i0] = cx * w00 - sx * w01;
    W[nb][2 * y][i1] = sx * w00 + cx * w01;
    W[nb][2 * y + 1][i0] = cx * w10 - sx * w11;
    W[nb][2 * y + 1][i1] = sx * w10 + cx * w11;
    __syncthreads();
  }
  constexpr int fb = (2 * BJ - 1) & 1;   // the buffer of the last round's writes
  float* Wk = Wbuf + (size_t)k * 4 * BJ * BJ;
  for (int e = t; e < 4 * BJ * BJ; e += BJ * BJ) Wk[e] = W[fb][e % (2 * BJ)][e / (2 * BJ)];
  __syncthreads();
}

// One CTA (BJ^2 threads) per block pair: W = the product of the rotations of one cyclic
// sweep over the pair's 2BJ x 2BJ subproblem (rotations as jacobi_rot).
template <int BJ>
__global__ void __launch_bounds__(BJ * BJ) k_bj_pair(const float* __restrict__ A, float* __restrict__ Wbuf, int n,
                                                     int nbk, int r) {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  __shared__ float S[2][2 * BJ][2 * BJ + 1];
  __shared__ float W[2][2 * BJ][2 * BJ + 1];
  const int k = blockIdx.x;
  const int bp = rr_player(k, r, nbk), bq = rr_player(nbk - 1 - k, r, nbk);
  const int t = threadIdx.x;
  for (int e = t; e < 4 * BJ * BJ; e += BJ * BJ) {
    const int i = e % (2 * BJ), j = e / (2 * BJ);
    const int gi = bj_index<BJ>(i, bp, bq), gj = bj_index<BJ>(j, bp, bq);
    S[0][i][j] = A[gi + (long long)gj * n];
    W[0][i][j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  bj_pair_sweep<BJ>(S, W, Wbuf, k);
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Shared memory of k_bj_apply: X rows of 2BJ + 1 floats (its column reads vary the row
// across a warp); the operands in rows of 2BJ + 4, read as broadcast float4 (all lanes of
// a warp share the column group)
template <int BJ>
constexpr size_t bj_apply_smem() {
  return (size_t)(((2 * BJ) * (2 * BJ + 1) + 3) & ~3) * 4 + 3 * (size_t)(2 * BJ) * (2 * BJ + 4) * 4;
}

// A' = J^T A J (into An; part 0) or V <- V J (part 1) for J = blockdiag(W_k), 256 threads.
// Part 0: CTA (a, b), a <= b (np (np + 1) / 2 CTAs), computes the 2BJ x 2BJ block
// A'[I_a, I_b] = W_a^T A[I_a, I_b] W_b and stores it and its transpose A'[I_b, I_a] (A
// stays exactly symmetric).  Part 1: CTA (row block, k) the 2BJ-row block of V[:, I_k] W_k.
// Thread (i, column group): CPT entries (row i, CPT consecutive columns) of each product.
template <int BJ>
__global__ void __launch_bounds__(256) k_bj_apply(const float* __restrict__ A, float* __restrict__ An, float* V,
                                                  const float* __restrict__ Wbuf, int n, int nbk, int r, int part) {
  constexpr int NI = 2 * BJ, NW = 2 * BJ + 4, CPT = NI * NI / 256;
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  extern __shared__ __align__(16) float bj_sm[];
  float(*X)[NI + 1] = reinterpret_cast<float(*)[NI + 1]>(bj_sm);
  float(*Wl)[NW] = reinterpret_cast<float(*)[NW]>(bj_sm + ((NI * (NI + 1) + 3) & ~3));   // 16-byte aligned rows
  float(*Wr)[NW] = Wl + NI;
  float(*Tm)[NW] = Wr + NI;
  const int np = nbk / 2;
  const int t = threadIdx.x, bid = blockIdx.x;
  const int i = t % NI, j0 = (t / NI) * CPT;
  if (part == 0) {
    // bid = kb (kb + 1) / 2 + ka, ka <= kb
    int kb = (int)((sqrtf(8.f * (float)bid + 1.f) - 1.f) * 0.5f);
    while ((kb + 1) * (kb + 2) / 2 <= bid) ++kb;
    while (kb * (kb + 1) / 2 > bid) --kb;
    const int ka = bid - kb * (kb + 1) / 2;
    const int ap = rr_player(ka, r, nbk), aq = rr_player(nbk - 1 - ka, r, nbk);
    const int bp = rr_player(kb, r, nbk), bq = rr_player(nbk - 1 - kb, r, nbk);
    const float* Wa = Wbuf + (size_t)ka * NI * NI;
    const float* Wb = Wbuf + (size_t)kb * NI * NI;
    for (int e = t; e < NI * NI; e += 256) {
      const int ii = e % NI, jj = e / NI;
      X[ii][jj] = A[bj_index<BJ>(ii, ap, aq) + (long long)bj_index<BJ>(jj, bp, bq) * n];
      Wl[ii][jj] = Wa[e];
      Wr[ii][jj] = Wb[e];
    }
    __syncthreads();
    // T = X W_b, then W_a^T T; a warp covers consecutive rows of a column group, so its
    // stores into column-major A' coalesce
    float acc[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) acc[u] = 0.f;
#pragma unroll 8
    for (int l = 0; l < NI; ++l) {
      const float x = X[i][l];
#pragma unroll
      for (int u = 0; u < CPT; u += 4) {
        const float4 w = *reinterpret_cast<const float4*>(&Wr[l][j0 + u]);
        acc[u] = fmaf(x, w.x, acc[u]);
        acc[u + 1] = fmaf(x, w.y, acc[u + 1]);
        acc[u + 2] = fmaf(x, w.z, acc[u + 2]);
        acc[u + 3] = fmaf(x, w.w, acc[u + 3]);
      }
    }
#pragma unroll
    for (int u = 0; u < CPT; u += 4)
      *reinterpret_cast<float4*>(&Tm[i][j0 + u]) = make_float4(acc[u], acc[u + 1], acc[u + 2], acc[u + 3]);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CPT; ++u) acc[u] = 0.f;
#pragma unroll 8
    for (int l = 0; l < NI; ++l) {
      const float wl = Wl[l][i];
#pragma unroll
      for (int u = 0; u < CPT; u += 4) {
        const float4 tv = *reinterpret_cast<const float4*>(&Tm[l][j0 + u]);
        acc[u] = fmaf(wl, tv.x, acc[u]);
        acc[u + 1] = fmaf(wl, tv.y, acc[u + 1]);
        acc[u + 2] = fmaf(wl, tv.z, acc[u + 2]);
        acc[u + 3] = fmaf(wl, tv.w, acc[u + 3]);
      }
    }
    const int gi = bj_index<BJ>(i, ap, aq);
#pragma unroll
    for (int u = 0; u < CPT; ++u) An[gi + (long long)bj_index<BJ>(j0 + u, bp, bq) * n] = acc[u];
    if (ka != kb) {
      // the transpose through shared memory, so that a warp's stores cover 32 rows of a
      // column of A' (as the direct ones do)
      __syncthreads();
#pragma unroll
      for (int u = 0; u < CPT; ++u) Tm[i][j0 + u] = acc[u];
      __syncthreads();
      const int jj = t % NI, ig = (t / NI) * CPT;
      const int gj = bj_index<BJ>(jj, bp, bq);
#pragma unroll
      for (int u = 0; u < CPT; ++u) An[gj + (long long)bj_index<BJ>(ig + u, ap, aq) * n] = Tm[ig + u][jj];
    }
  } else {
    const int vb = bid;
    const int rows = n / NI;
    const int rb = vb % rows, k = vb / rows;
    const int bp = rr_player(k, r, nbk), bq = rr_player(nbk - 1 - k, r, nbk);
    const float* Wk = Wbuf + (size_t)k * NI * NI;
    for (int e = t; e < NI * NI; e += 256) {
      const int ii = e % NI, jj = e / NI;
      X[ii][jj] = V[rb * NI + ii + (long long)bj_index<BJ>(jj, bp, bq) * n];
      Wl[ii][jj] = Wk[e];
    }
    __syncthreads();
    const int gr = rb * NI + i;
    float acc[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) acc[u] = 0.f;
#pragma unroll 8
    for (int l = 0; l < NI; ++l) {
      const float x = X[i][l];
#pragma unroll
      for (int u = 0; u < CPT; u += 4) {
        const float4 w = *reinterpret_cast<const float4*>(&Wl[l][j0 + u]);
        acc[u] = fmaf(x, w.x, acc[u]);
        acc[u + 1] = fmaf(x, w.y, acc[u + 1]);
        acc[u + 2] = fmaf(x, w.z, acc[u + 2]);
        acc[u + 3] = fmaf(x, w.w, acc[u + 3]);
      }
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u) V[gr + (long long)bj_index<BJ>(j0 + u, bp, bq) * n] = acc[u];
  }
  __syncthreads();
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// out = in^T (n x n, column-major)
__global__ void k_transpose(const double* __restrict__ in, double* __restrict__ out, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  out[j + (long long)i * n] = in[e];
}

// out = in^H (n x n, column-major)
template <class TW>
__global__ void k_adjoint(const TW* __restrict__ in, TW* __restrict__ out, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  out[j + (long long)i * n] = Tr<TW>::conj(in[e]);
}

template <class TW>
__global__ void k_identity(TW* V, int n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  V[t] = from_real<TW>((t % n == t / n) ? 1.0 : 0.0);
}

// part[2 b], part[2 b + 1] = sums over column block b of the off-diagonal and all |A_ij|^2
// (one CTA per 8 columns, fixed order); k_offnorm_sum adds the blocks in order.
template <class TW>
__global__ void __launch_bounds__(256) k_offnorm(const TW* __restrict__ A, int n, double* part) {
  __shared__ double s0[256], s1[256];
  double off = 0.0, tot = 0.0;
  const int c0 = blockIdx.x * 8;
  for (int jj = 0; jj < 8; ++jj) {
    const int j = c0 + jj;
    if (j >= n) break;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = Tr<TW>::abs2(A[i + (long long)j * n]);
      tot += v;
      if (i != j) off += v;
    }
  }
  s0[threadIdx.x] = off;
  s1[threadIdx.x] = tot;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { s0[threadIdx.x] += s0[threadIdx.x + s]; s1[threadIdx.x] += s1[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
}

__global__ void k_offnorm_sum(const double* part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) { a += part[2 * i]; b += part[2 * i + 1]; }
  out[0] = a;
  out[1] = b;
}

// Ascending order of the diagonal: eig[rank] = A_ii, perm[rank] = i (ties broken by
// index, so the order is deterministic); vals != nullptr: sort by vals[i] instead of
// the diagonal of A.  Each CTA holds all n keys in shared memory (n <= 1024) as
// order-preserving 64-bit integers (integer compares: the FP64 ones run at the FP64
// rate) and ranks 128 of them.
__device__ __forceinline__ unsigned long long sort_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
template <class TW>
__global__ void __launch_bounds__(128) k_sort(const TW* __restrict__ A, const double* __restrict__ vals, int n,
                                              double* __restrict__ eig, int* __restrict__ perm) {
  __shared__ unsigned long long key[1024];
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    key[i] = sort_key(vals ? vals[i] : (double)Tr<TW>::re(A[i + (long long)i * n]));
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long ki = key[i];
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const unsigned long long kj = key[j];
    rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
  }
  perm[rank] = i;
  eig[rank] = vals ? vals[i] : (double)Tr<TW>::re(A[i + (long long)i * n]);
}

// Q[:, rank] = V[:, perm[rank]] (n x n), over the whole GPU
template <class TW>
__global__ void k_permute_cols(const TW* __restrict__ V, const int* __restrict__ perm, int n, TW* __restrict__ Q) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int row = (int)(t % n), col = (int)(t / n);
  Q[t] = V[row + (long long)perm[col] * n];
}

template <class TW, class T>
__global__ void k_narrow(const TW* __restrict__ a, T* __restrict__ b, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = narrow_to((T*)nullptr, a[t]);
}

// ------------------------------------------------------------------ blocked FP64 Cholesky pieces
constexpr int CB = 64;   // Cholesky / inverse block
// Largest max |E| of M~1 = I + E for the series factorisation of the mixed mode
// (the truncation errors are |E|^5 and below, under the FP64 rounding of the FP32
// products' corrections)
constexpr double EPS_SERIES = 1e-3;

// dst (M x N, ldd) = src (M x N, lds)
template <class TW>
__global__ void k_copy2d(const TW* __restrict__ src, long long lds, TW* __restrict__ dst, long long ldd,
                         int M, int N) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N) return;
  const int i = (int)(t % M), j = (int)(t / M);
  dst[i + (long long)j * ldd] = src[i + (long long)j * lds];
}

template <class TW>
__global__ void k_fill0(TW* a, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = zero_of<TW>();
}

// C = alpha * sum_z P[z] + beta * C  (M x N; partials packed with leading dimension M)
template <class TW>
__global__ void k_reduce_axpby(const TW* __restrict__ P, int nz, int M, int N, double alpha, double beta,
                               TW* C, long long ldc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N) return;
  const int i = (int)(t % M), j = (int)(t / M);
  TW v = zero_of<TW>();
  for (int z = 0; z < nz; ++z) v = add(v, P[(long long)z * M * N + t]);
  v = scale(alpha, v);
  if (beta != 0.0) v = add(v, scale(beta, C[i + (long long)j * ldc]));
  C[i + (long long)j * ldc] = v;
}

// lam[i] = Re(q_i^H z_i) / Re(q_i^H q_i)   (FP64 Rayleigh quotients, one column per thread)
template <class TW>
__global__ void k_rayleigh(const TW* __restrict__ Qm, const TW* __restrict__ Z, int n, double* lam) {
  // one warp per column: lanes over k (coalesced), partial sums reduced in a fixed order
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  double num = 0.0, den = 0.0;
  for (int k = lane; k < n; k += 32) {
    const TW q = Qm[k + (long long)i * n];
    num += Tr<TW>::re(mul(Tr<TW>::conj(q), Z[k + (long long)i * n]));
    den += Tr<TW>::abs2(q);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (lane == 0) lam[i] = num / den;
}

// G <- (3 I - G) / 2 (n x n): the Newton-Schulz factor from the Gram G = V^T V.
__global__ void k_ns_coef(double* G, int n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  G[t] = (i == j ? 1.5 : 0.0) - 0.5 * G[t];
}

// ------------------------------------------------------------------ mixed-mode orthonormalisation
// s_i = M_ii^(-1/2) and Mf = diag(s) M diag(s) in FP32 (unit diagonal): the diagonally
// scaled Gram whose FP32 Cholesky orthonormalises the filtered block.
__global__ void k_scale_unit(const double* __restrict__ M, int n, double* __restrict__ s, float* __restrict__ Mf,
                             int* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  const double di = M[i + (long long)i * n], dj = M[j + (long long)j * n];
  if (!(di > 0.0) || !(dj > 0.0) || !isfinite(di) || !isfinite(dj)) {
    if (i == j) {
      atomicOr(status, STATUS_NOT_POSDEF);
      s[i] = 0.0;
    }
    Mf[t] = 0.f;
    return;
  }
  const double si = rsqrt(di), sj = rsqrt(dj);
  if (i == j) s[i] = si;
  Mf[t] = (float)(M[t] * si * sj);
}

// T[i + j n] = s_i Li[j + i n] for j >= i, else 0: (diag(s) Li^T), the right factor
// U -> U diag(s) Li^T of the scaled Cholesky orthonormalisation (Li = L'^-1, lower).
__global__ void k_t1_scaled(const float* __restrict__ Li, const double* __restrict__ s, int n,
                            double* __restrict__ T) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  T[t] = j >= i ? s[i] * (double)Li[j + (long long)i * n] : 0.0;
}

// E = M - I and max |E_ij| (the bit pattern of a non-negative double, so that an
// integer maximum orders it; NaN orders above every finite value) into emax.
__global__ void __launch_bounds__(256) k_eminus(const double* __restrict__ M, int n, double* __restrict__ E,
                                                unsigned long long* emax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long m = 0ull;
  if (t < (long long)n * n) {
    const int i = (int)(t % n), j = (int)(t / n);
    const double v = M[t] - (i == j ? 1.0 : 0.0);
    E[t] = v;
    m = (unsigned long long)__double_as_longlong(fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
    m = q > m ? q : m;
  }
  __shared__ unsigned long long wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
    atomicMax(emax, m);
  }
}

// F = Phi(E - G): the strictly lower part of E - G plus half its diagonal, zero above
// (G may be null).  The lower-triangular F with (I + F)(I + F)^T = I + E is the fixed
// point F = Phi(E - F F^T).
__global__ void k_phi(const double* __restrict__ E, const double* __restrict__ G, int n, double* __restrict__ F) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  const double v = E[t] - (G ? G[t] : 0.0);
  F[t] = i > j ? v : (i == j ? 0.5 * v : 0.0);
}

// Y = I - X
__global__ void k_i_minus(const double* __restrict__ X, int n, double* __restrict__ Y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  Y[t] = (t % n == t / n ? 1.0 : 0.0) - X[t];
}

// A = sym(H) + P + P^T + sym(Q): C = (I + K) H (I + K)^T with P = K H, Q = P K^T.
__global__ void k_csum(const double* __restrict__ Hm, const double* __restrict__ P, const double* __restrict__ Q,
                       int n, double* __restrict__ A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  const long long tt = j + (long long)i * n;
  A[t] = 0.5 * (Hm[t] + Hm[tt]) + (P[t] + P[tt]) + 0.5 * (Q[t] + Q[tt]);
}

template <class TA, class TB>
__global__ void k_convert(const TA* __restrict__ a, TB* __restrict__ b, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = narrow_to((TB*)nullptr, widen(a[t]));
}

template <class T> struct Narrow;
template <> struct Narrow<double> { using N = float; };
template <> struct Narrow<cf64> { using N = cf32; };

// FP64 GEMM spread over the GPU: split K when the output has few tiles.
// C = alpha op(A) op(B) + beta C; `part` holds up to `cap` elements of partials.
template <class TW, bool ACT, bool BCT>
cudaError_t gemm64(sparc_ctx* ctx, int M, int N, int K, const TW* A, long long lda, const TW* B, long long ldb,
                   TW* C, long long ldc, double alpha, double beta, TW* part, long long cap, cudaStream_t st) {
  const int tiles = ceil_div(M, 64) * ceil_div(N, 64);
  int nz = std::max(1, std::min(ceil_div(2 * 152, tiles), K / 64));
  while (nz > 1 && (long long)nz * M * N > cap) --nz;
  if (nz == 1) return gemm<TW, TW, TW, TW, ACT, BCT>(ctx, M, N, K, A, lda, B, ldb, C, ldc, 1, 0, alpha, st, beta);
  cudaError_t e = gemm<TW, TW, TW, TW, ACT, BCT>(ctx, M, N, K, A, lda, B, ldb, part, M, nz, (long long)M * N, 1.0, st);
  if (e != cudaSuccess) return e;
  k_reduce_axpby<TW><<<ceil_div((long long)M * N, 256), 256, 0, st>>>(part, nz, M, N, alpha, beta, C, ldc);
  ++ctx->launches;
  return cudaGetLastError();
}

// C = alpha op(A) op(B) + beta C with FP32 products of FP64 operands (the small
// corrections of the mixed mode), split over K so that the GPU is filled: nz partials
// in `part` (at least nz M N doubles) summed in a fixed order by k_reduce_axpby.
template <bool ACT, bool BCT>
cudaError_t gemm_f32p(sparc_ctx* ctx, int M, int N, int K, const double* A, long long lda, const double* B,
                      long long ldb, double* C, long long ldc, double alpha, double beta, double* part, long long cap,
                      cudaStream_t st) {
  const int tiles = ceil_div(M, 64) * ceil_div(N, 64);
  int nz = std::max(1, std::min(ceil_div(2 * std::max(ctx->nsm, 1), tiles), K / 64));
  while (nz > 1 && (long long)nz * M * N > cap) --nz;
  if (nz == 1) return gemm<double, double, float, double, ACT, BCT>(ctx, M, N, K, A, lda, B, ldb, C, ldc, 1, 0, alpha,
                                                                   st, beta);
  cudaError_t e = gemm<double, double, float, double, ACT, BCT>(ctx, M, N, K, A, lda, B, ldb, part, M, nz,
                                                                (long long)M * N, 1.0, st);
  if (e != cudaSuccess) return e;
  k_reduce_axpby<double><<<ceil_div((long long)M * N, 256), 256, 0, st>>>(part, nz, M, N, alpha, beta, C, ldc);
  ++ctx->launches;
  return cudaGetLastError();
}

// C = A B (n x n, column-major, FP64) for an FP64 A and a B whose entries are FP32 values
// (the FP32 eigensolve's vectors), at the FP32 rate: with a = a_hi + a_lo (the FP32
// rounding of a and of its remainder), each product a b is a_hi b, formed exactly as
// p + e (p = fl(a_hi b), e = fma(a_hi, b, -p)), plus a_lo b (2^-24 of it, rounded), and
// the products are summed in float-float (TwoSum into hi, the errors into lo): relative
// error about 2^-44 instead of the FP64 GEMM's, at 1/6 of its time on this GPU.
// 32 x 32 output tiles of 256 threads, each 2 x 2 outputs; k-tiles of 16.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float p, float e) {
  const float s = hi + p;
  const float bp = s - hi;
  lo += ((hi - (s - bp)) + (p - bp)) + e;
  hi = s;
}
__global__ void __launch_bounds__(256) k_gemm_ff(const double* __restrict__ A, const double* __restrict__ B,
                                                 double* __restrict__ C, int n) {
  __shared__ float ah[16][33], al[16][33], bs[16][33];
  const int m0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  float hi[2][2] = {}, lo[2][2] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    for (int e = t; e < 512; e += 256) {
      const int mm = e % 32, kk = e / 32;   // A: consecutive threads, consecutive rows
      const int m = m0 + mm, k = k0 + kk;
      const double a = (m < n && k < n) ? A[m + (long long)k * n] : 0.0;
      const float h = (float)a;
      ah[kk][mm] = h;
      al[kk][mm] = (float)(a - (double)h);
      const int kb = e % 16, nb = e / 16;   // B: consecutive threads, consecutive k
      const int kg = k0 + kb, ng = n0 + nb;
      bs[kb][nb] = (kg < n && ng < n) ? (float)B[kg + (long long)ng * n] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float a0h = ah[kk][ty], a1h = ah[kk][ty + 16], a0l = al[kk][ty], a1l = al[kk][ty + 16];
      const float b0 = bs[kk][tx], b1 = bs[kk][tx + 16];
      const float ahs[2] = {a0h, a1h}, als[2] = {a0l, a1l}, bv[2] = {b0, b1};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float p = ahs[i] * bv[j];
          const float e = fmaf(ahs[i], bv[j], -p) + als[i] * bv[j];
          ff_add(hi[i][j], lo[i][j], p, e);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
      if (m < n && c < n) C[m + (long long)c * n] = (double)hi[i][j] + (double)lo[i][j];
    }
}

// Li's diagonal blocks (cb x cb, the last one ragged) from the block inverses Dinv.
template <class TW>
__global__ void k_copy_diag(const TW* __restrict__ Dinv, int cb, TW* __restrict__ Li, int n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int blk = (int)(t / ((long long)cb * cb)), r = (int)(t % ((long long)cb * cb));
  const int i = r % cb, j = r / cb;
  const int gi = blk * cb + i, gj = blk * cb + j;
  if (gi < n && gj < n) Li[gi + (long long)gj * n] = Dinv[(size_t)blk * cb * cb + i + (size_t)j * cb];
}

// Blocked right-looking Cholesky of the n x n Hermitian A (lower factor in place)
// and L^-1 into Li; Dinv receives the inverted diagonal blocks.
template <class TW>
sparc_status chol_inverse(sparc_ctx* ctx, TW* A, TW* Li, int n, TW* Dinv, TW* tmp, TW* part, long long cap,
                          cudaStream_t st) {
  const int nbk = ceil_div(n, CB);
  for (int kblk = 0; kblk < nbk; ++kblk) {
    const int k0 = kblk * CB, kb = std::min(CB, n - k0);
    TW* Dk = Dinv + (size_t)kblk * CB * CB;
    TW* Akk = A + k0 + (long long)k0 * n;
    // diagonal block: contiguous copy, one-CTA factor and inverse, copies back
    if constexpr (std::is_same<TW, float>::value) {
      // factor and invert the block in shared memory, one launch
      k_chol_blk_f32<<<1, 64, 0, st>>>(Akk, n, Dk, CB, kb, ctx->d_status);
      ctx->launches += 1;
    } else if constexpr (std::is_same<TW, double>::value) {
      k_chol_blk<TW, CB><<<1, 256, 0, st>>>(Akk, n, Dk, CB, kb, ctx->d_status);
      ctx->launches += 1;
    } else if constexpr (std::is_same<TW, cf64>::value) {
      SPARC_CUDA(ctx, cudaFuncSetAttribute(k_chol_blk_c, cudaFuncAttributeMaxDynamicSharedMemorySize, CHOL_C_SMEM));
      k_chol_blk_c<<<1, 256, CHOL_C_SMEM, st>>>(Akk, n, Dk, CB, kb, ctx->d_status);
      ctx->launches += 1;
    } else {
      TW* blk = part;                     // kb x kb, leading dimension kb
      TW* blki = part + (size_t)CB * CB;  // its inverse
      k_copy2d<TW><<<ceil_div((long long)kb * kb, 256), 256, 0, st>>>(Akk, n, blk, kb, kb, kb);
      k_chol<TW><<<1, 1024, 0, st>>>(blk, kb, ctx->d_status);
      k_trinv<TW><<<1, 1024, 0, st>>>(blk, blki, kb);
      k_copy2d<TW><<<ceil_div((long long)kb * kb, 256), 256, 0, st>>>(blk, kb, Akk, n, kb, kb);
      k_copy2d<TW><<<ceil_div((long long)kb * kb, 256), 256, 0, st>>>(blki, kb, Dk, CB, kb, kb);
      ctx->launches += 5;
    }
    SPARC_LAUNCH(ctx, "cholesky block");
    const int m2 = n - k0 - kb;
    if (m2 > 0) {
      TW* A21 = A + (k0 + kb) + (long long)k0 * n;
      if constexpr (std::is_same<TW, float>::value) {
        // A21 <- T = A21 L_kk^-H in place (one 64-column tile: each CTA reads its rows of
        // A21 whole before it writes them); A22 -= T T^H
        SPARC_CUDA(ctx, (gemm<TW, TW, TW, TW, false, true>(ctx, m2, kb, kb, A21, n, Dk, CB, A21, n, 1, 0, 1.0, st)));
        SPARC_CUDA(ctx, (gemm64<TW, false, true>(ctx, m2, m2, kb, A21, n, A21, n,
                                                 A + (k0 + kb) + (long long)(k0 + kb) * n, n, -1.0, 1.0, part, cap,
                                                 st)));
      } else {
        // T = A21 L_kk^-H ; A22 -= T T^H ; A21 = T
        SPARC_CUDA(ctx, (gemm64<TW, false, true>(ctx, m2, kb, kb, A21, n, Dk, CB, tmp, m2, 1.0, 0.0, part, cap, st)));
        SPARC_CUDA(ctx, (gemm64<TW, false, true>(ctx, m2, m2, kb, tmp, m2, tmp, m2,
                                                 A + (k0 + kb) + (long long)(k0 + kb) * n, n, -1.0, 1.0, part, cap,
                                                 st)));
        k_copy2d<TW><<<ceil_div((long long)m2 * kb, 256), 256, 0, st>>>(tmp, m2, A21, n, m2, kb);
        ++ctx->launches;
      }
    }
  }
  k_fill0<TW><<<ceil_div((long long)n * n, 256), 256, 0, st>>>(Li, (long long)n * n);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "inverse init");
  if constexpr (std::is_same<TW, float>::value) {
    // L^-1 by recursive doubling: its diagonal blocks are the Dinv blocks; at width w the
    // off-diagonal block of each pair of consecutive w-ranges a, b is
    // Li[b, a] = -Li[b, b] L[b, a] Li[a, a].  The pairs of one width are independent and
    // run on up to four streams (branches of the captured graph), each with its own part
    // of tmp and of the split-K scratch: a chain of 3 widths x 2 GEMMs at n = 512 instead
    // of 8 block rows x 3 launches.
    k_copy_diag<TW><<<ceil_div((long long)nbk * CB * CB, 256), 256, 0, st>>>(Dinv, CB, Li, n);
    ++ctx->launches;
    for (int b = 0; b < 3; ++b)
      if (!ctx->aux_stream[b]) SPARC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream[b], cudaStreamNonBlocking));
    cudaEvent_t ev[5] = {};
    for (cudaEvent_t& e : ev) SPARC_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t le = cudaSuccess;
    for (int w = CB; w < n && le == cudaSuccess; w *= 2) {
      const int npairs = ceil_div(n - w, 2 * w);   // pairs with a non-empty b range
      const int nbr = std::min(4, npairs);
      le = cudaEventRecord(ev[0], st);   // fork
      for (int br = 1; br < nbr && le == cudaSuccess; ++br) le = cudaStreamWaitEvent(ctx->aux_stream[br - 1], ev[0], 0);
      for (int pr = 0; pr < npairs && le == cudaSuccess; ++pr) {
        const int a0 = 2 * w * pr, b0 = a0 + w, wb = std::min(w, n - b0);
        cudaStream_t bs = (pr % nbr) == 0 ? st : ctx->aux_stream[(pr % nbr) - 1];
        TW* tp = tmp + (size_t)(pr % nbr) * w * w;
        TW* pp = part + (size_t)(pr % nbr) * (cap / nbr);
        le = gemm64<TW, false, false>(ctx, wb, w, w, A + b0 + (long long)a0 * n, n, Li + a0 + (long long)a0 * n, n, tp,
                                      wb, 1.0, 0.0, pp, cap / nbr, bs);
        if (le == cudaSuccess)
          le = gemm64<TW, false, false>(ctx, wb, w, wb, Li + b0 + (long long)b0 * n, n, tp, wb,
                                        Li + b0 + (long long)a0 * n, n, -1.0, 0.0, pp, cap / nbr, bs);
      }
      for (int br = 1; br < nbr && le == cudaSuccess; ++br) {   // join
        le = cudaEventRecord(ev[br], ctx->aux_stream[br - 1]);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(st, ev[br], 0);
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    SPARC_CUDA(ctx, le);
    SPARC_LAUNCH(ctx, "triangular inverse");
    return SPARC_OK;
  }
  // L^-1 by block rows: Li_ij = -Dinv_i (sum_{k<i} L_ik Li_kj)
  for (int iblk = 0; iblk < nbk; ++iblk) {
    const int i0 = iblk * CB, ib = std::min(CB, n - i0);
    TW* Di = Dinv + (size_t)iblk * CB * CB;
    k_copy2d<TW><<<ceil_div((long long)ib * ib, 256), 256, 0, st>>>(Di, CB, Li + i0 + (long long)i0 * n, n, ib, ib);
    ++ctx->launches;
    if (i0 > 0) {
      SPARC_CUDA(ctx, (gemm64<TW, false, false>(ctx, ib, i0, i0, A + i0, n, Li, n, tmp, ib, 1.0, 0.0, part, cap, st)));
      SPARC_CUDA(ctx, (gemm64<TW, false, false>(ctx, ib, i0, ib, Di, CB, tmp, ib, Li + i0, n, -1.0, 0.0, part, cap, st)));
    }
  }
  SPARC_LAUNCH(ctx, "triangular inverse");
  return SPARC_OK;
}

// Parallel cyclic Jacobi on the n x n Hermitian A (ping-pong A0/A1, eigenvectors in V),
// one sweep per replay of a captured CUDA graph (one graph from each buffer: a sweep
// has an odd number of rounds), until off(A)^2 <= tol |A|^2 or off(A) stagnates at the
// rounding floor of the element type.
// Whether the block Jacobi method takes an n x n problem of element type TJ.
template <class TJ>
constexpr bool bj_type() { return std::is_same<TJ, float>::value; }
// Block size of the block method for an n x n problem: 16 where n is a multiple of 32
// (at least two block pairs); 0: the scalar method.  (Blocks of 32 were measured 2x
// slower at n = 512: the 64 x 64 inner sweep's 63 rounds on 1024 threads dominate.)
inline int bj_size(int n) { return (n % 32 == 0 && n >= 64) ? 16 : 0; }

template <class TJ>
sparc_status jacobi(sparc_ctx* ctx, TJ* A0, TJ* A1, TJ* V, int n, double tol, int max_sweeps, double* scal,
                    TJ** result, int* sweeps_out, cudaStream_t st, float* Wbuf = nullptr) {
  const int bjs = (bj_type<TJ>() && Wbuf != nullptr) ? bj_size(n) : 0;
  const bool blockj = bjs > 0;
  const int npad = n + (n & 1);
  const int half = npad / 2;
  const int nblocks = ((half + 15) / 16) * ((half + 15) / 16) + ((n + 63) / 64) * ((half + 3) / 4);
  const int nbk = blockj ? n / bjs : 0, npair = nbk / 2;
  // one sweep per graph: npad - 1 scalar rounds, or nbk - 1 block rounds of two launches
  const int rounds = blockj ? nbk - 1 : npad - 1;
  if (!ctx->cap_stream) {
    SPARC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  }
  if (blockj && !ctx->cap_stream2) {
    SPARC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  }
  // the sweep graph that starts from buffer par (0: A0, 1: A1); its result lands in the other
  auto sweep_graph = [&](int par, cudaGraphExec_t* out) -> sparc_status {
  const auto key = std::make_tuple((int)sizeof(TJ) * 2 + (int)Tr<TJ>::cplx + 64 * bjs + 4096 * par, n,
                                   (void*)A0, (void*)A1, (void*)V);
  cudaGraphExec_t ge = nullptr;
  auto it = ctx->graphs.find(key);
  if (it != ctx->graphs.end()) {
    ge = it->second;
  } else {
    cudaGraph_t g = nullptr;
    SPARC_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    TJ* a = par ? A1 : A0;
    TJ* b = par ? A0 : A1;
    // each round may begin launching while the previous one finishes (programmatic
    // dependent launch); it waits for that round's results before it reads A or V
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->cap_stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t le = cudaSuccess;
    // block method: the V updates run on a second branch (cap_stream2), beside the next
    // round's pair solves, which use few SMs; the rotations are double-buffered (round r
    // in Wbuf half r & 1), and the pair solve of round r + 2 waits for the V update of r
    cudaEvent_t evp = nullptr, evv[2] = {nullptr, nullptr};
    if (blockj) {
      le = cudaEventCreateWithFlags(&evp, cudaEventDisableTiming);
      if (le == cudaSuccess) le = cudaEventCreateWithFlags(&evv[0], cudaEventDisableTiming);
      if (le == cudaSuccess) le = cudaEventCreateWithFlags(&evv[1], cudaEventDisableTiming);
    }
    const size_t wh = (size_t)npair * 4 * 16 * 16;   // floats of one round's rotations
    for (int r = 0; r < rounds && le == cudaSuccess; ++r) {
      if (blockj) {
        if constexpr (bj_type<TJ>()) {
          cudaLaunchConfig_t c1 = cfg, c2 = cfg, c3 = cfg;
          c1.gridDim = dim3((unsigned)npair);
          c1.blockDim = dim3((unsigned)(bjs * bjs));
          c2.gridDim = dim3((unsigned)(npair * (npair + 1) / 2));
          c2.dynamicSmemBytes = bj_apply_smem<16>();
          c3.gridDim = dim3((unsigned)((n / (2 * bjs)) * npair));
          c3.dynamicSmemBytes = bj_apply_smem<16>();
          c3.stream = ctx->cap_stream2;
          const int rb = r % (nbk - 1);
          float* Wr = Wbuf + (r & 1) * wh;
          if (r >= 2) le = cudaStreamWaitEvent(ctx->cap_stream, evv[r & 1], 0);
          if (le == cudaSuccess) le = cudaLaunchKernelEx(&c1, k_bj_pair<16>, (const float*)a, Wr, n, nbk, rb);
          if (le == cudaSuccess) le = cudaEventRecord(evp, ctx->cap_stream);
          if (le == cudaSuccess)
            le = cudaLaunchKernelEx(&c2, k_bj_apply<16>, (const float*)a, (float*)b, (float*)V, (const float*)Wr, n,
                                    nbk, rb, 0);
          if (le == cudaSuccess) le = cudaStreamWaitEvent(ctx->cap_stream2, evp, 0);
          if (le == cudaSuccess)
            le = cudaLaunchKernelEx(&c3, k_bj_apply<16>, (const float*)a, (float*)b, (float*)V, (const float*)Wr, n,
                                    nbk, rb, 1);
          if (le == cudaSuccess) le = cudaEventRecord(evv[r & 1], ctx->cap_stream2);
        }
      } else {
        le = cudaLaunchKernelEx(&cfg, k_jacobi_round<TJ>, (const TJ*)a, b, V, n, npad, r % (npad - 1));
      }
      std::swap(a, b);
    }
    // join the V branch
    if (blockj && le == cudaSuccess) le = cudaStreamWaitEvent(ctx->cap_stream, evv[(rounds - 1) & 1], 0);
    if (evp) cudaEventDestroy(evp);
    for (cudaEvent_t ev : evv)
      if (ev) cudaEventDestroy(ev);
    if (le != cudaSuccess) {
      cudaStreamEndCapture(ctx->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, le, "jacobi round launch");
    }
    SPARC_CUDA(ctx, cudaStreamEndCapture(ctx->cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    SPARC_CUDA(ctx, e);
    ctx->graphs[key] = ge;
  }
  *out = ge;
  return SPARC_OK;
  };
  cudaGraphExec_t ges[2];
  for (int par = 0; par < 2; ++par) {
    const sparc_status s = sweep_graph(par, &ges[par]);
    if (s != SPARC_OK) return s;
  }
  double hs[2];
  double prev_off = -1.0;
  int sweeps = 0;
  bool converged = false;
  cudaEvent_t tj = timing_begin(ctx, st);
  int ahead = 1;   // sweeps before the next test
  while (sweeps < max_sweeps && !converged) {
    for (int a = 0; a < ahead && sweeps < max_sweeps; ++a) {
      SPARC_CUDA(ctx, cudaGraphLaunch(ges[sweeps & 1], st));
      ctx->launches += blockj ? 3 * rounds : rounds;
      ++ctx->graph_launches;
      ++sweeps;
    }
    const int nbo = ceil_div(n, 8);
    k_offnorm<TJ><<<nbo, 256, 0, st>>>((sweeps & 1) ? A1 : A0, n, scal + 2);
    k_offnorm_sum<<<1, 32, 0, st>>>(scal + 2, nbo, scal);
    ctx->launches += 2;
    SPARC_CUDA(ctx, cudaMemcpyAsync(hs, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    // converged, or stagnated at the rounding floor of the element type (Jacobi
    // converges quadratically, so from the fourth sweep on a sweep that leaves off(A)^2
    // above 0.7 of its previous value is at the floor)
    converged = !(hs[0] > tol * hs[1]) || (sweeps >= 4 && prev_off >= 0.0 && hs[0] > 0.7 * prev_off);
    prev_off = hs[0];
    // far from convergence the next sweeps cannot reach the tolerance (Jacobi at best
    // squares off(A)^2 / |A|^2 per sweep, and tol <= 1e-10): test again after 3 sweeps
    // above 1e-1, after 2 above 1e-3, else after each
    const double rel = hs[1] > 0.0 ? hs[0] / hs[1] : 0.0;
    ahead = rel > 1e-1 ? 3 : (rel > 1e-3 ? 2 : 1);
  }
  timing_end(ctx, TK_JAC, tj, st);
  *result = (sweeps & 1) ? A1 : A0;   // each sweep moves the matrix to the other buffer
  *sweeps_out = sweeps;
  if (!converged) return fail(ctx, SPARC_ERR_NO_CONVERGENCE, "Jacobi sweep limit reached");
  return SPARC_OK;
}

// ------------------------------------------------------------------ driver
// Run `launches` (a chain of small launches with fixed sizes and buffers) on st: captured
// once per key into a CUDA graph held by the context and replayed after that, so that the
// chain costs one host launch; issued directly with the synchronous debug check.
template <class F>
static sparc_status replay(sparc_ctx* ctx, const std::tuple<int, int, void*, void*, void*>& key, cudaStream_t st,
                           F&& launches) {
  if (sync_check()) return launches(st);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (!ctx->cap_stream) SPARC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const long long l0 = ctx->launches;
    SPARC_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const sparc_status s = launches(ctx->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->graph_kernels[key] = ctx->launches - l0;
    ctx->launches = l0;
    if (s != SPARC_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    SPARC_CUDA(ctx, ec);
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    SPARC_CUDA(ctx, ei);
    it = ctx->graphs.emplace(key, ge).first;
  }
  SPARC_CUDA(ctx, cudaGraphLaunch(it->second, st));
  ctx->launches += ctx->graph_kernels[key];
  ++ctx->graph_launches;
  return SPARC_OK;
}

template <class T, class TC>
sparc_status rayleigh_ritz(sparc_ham* H, T* U, int ns, long long ld, double* eig, bool mixed, cudaStream_t st) {
  using TW = typename Wide<T>::W;
  using TS = typename Narrow<TW>::N;
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  const size_t es = sizeof(T), ew = sizeof(TW);
  const long long nn = (long long)ns * ns;
  const int tiles = ceil_div(ns, 64) * ceil_div(ns, 64);
  int nsplit = std::max(1, std::min(256, ceil_div(2 * 152, tiles)));
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, nd / 64));
  const size_t hub = align256((size_t)nd * ns * es);
  const size_t sm = align256((size_t)nn * ew);
  // split-K partials; also the diagonal-block scratch of the Cholesky (2 * CB * CB)
  const size_t partb = align256((size_t)std::max<long long>(std::max<long long>(nsplit, 8) * nn, 2LL * CB * CB) * ew);
  const int nbk = ceil_div(ns, CB);
  const size_t dinvb = align256((size_t)nbk * CB * CB * ew);
  constexpr bool TCP = std::is_same<T, float>::value;   // FP32 data: tensor-core Grams and rotation
  constexpr bool TCC = std::is_same<T, cf32>::value;    // complex64 data: the same, on the real views
  const size_t tcb = TCP   ? align256(std::max(tc::gram_scratch_bytes(ctx, ns, nd), tc::rot_scratch_bytes(ns)))
                     : TCC ? align256(std::max(tc::cgram_scratch_bytes(ctx, ns, nd), tc::rot_scratch_bytes(ns, true)))
                           : 0;
  const size_t w1b = (TCP || TCC) ? hub : 0;   // U1, the orthonormalised basis
  const size_t jbb = TCC ? hub : 0;            // i B, the second operand of a complex Gram's imaginary part
  const size_t gsb = apply_scratch_bytes(H, DtypeOf<T>::v, ns);   // projection scratch of the H-apply
  // rotations of the block Jacobi rounds (FP32 subproblems of the mixed mode)
  // (block size b: ns / b / 2 pairs of 4 b^2 floats, that is 2 b ns floats, twice: the
  // rotations of two consecutive rounds)
  const size_t wjb = (bj_type<TS>() && bj_size(ns) > 0) ? align256((size_t)4 * BJ_MAX * ns * sizeof(float)) : 0;
  const size_t extra = hub + 2 * partb + 10 * sm + dinvb + align256(nn * es) + 3 * align256(nn * sizeof(TS)) +
                       2 * align256(ns * sizeof(double)) + tcb + w1b + jbb + gsb + wjb + 256;
  BlockWs w;
  char* tail = nullptr;
  sparc_status s = block_ws(H, DtypeOf<T>::v, ns, extra, &w, &tail);
  if (s != SPARC_OK) return s;
  if (gsb) { w.gs = tail; tail += gsb; }
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
  TW* Dinv = (TW*)tail; tail += dinvb;
  T* YrT = (T*)tail; tail += align256(nn * es);
  TS* S0 = (TS*)tail; tail += align256(nn * sizeof(TS));
  TS* S1 = (TS*)tail; tail += align256(nn * sizeof(TS));
  TS* SV = (TS*)tail; tail += align256(nn * sizeof(TS));
  double* lam = (double*)tail; tail += align256(ns * sizeof(double));
  double* eigw = (double*)tail; tail += align256(ns * sizeof(double));   // sorted Ritz values (graph-owned)
  // the block Jacobi's rotations ahead of the tensor-core scratch, whose size depends on
  // Nd: every buffer a cached graph uses sits at an offset fixed by those in its key
  float* Wjb = wjb ? (float*)tail : nullptr; tail += wjb;
  void* tcs = tail; tail += tcb;
  T* JB = (T*)tail; tail += jbb;
  T* W1 = (T*)tail;
  const long long pcap = (long long)(partb / ew);

  T* Ub = U;            // basis of the Rayleigh-Ritz pass
  long long ldb = ld;
  cudaEvent_t tg = nullptr;
  if constexpr (TCP) {
    // FP32 data: orthonormalise first (Cholesky-QR, U1 = U L^-T), then Rayleigh-Ritz in
    // the basis U1 with H U1 applied to it.  The filtered block is ill-conditioned
    // (kappa(M~) grows like the square of the filter's gain T_m), and one Cholesky of
    // M~ amplifies the Gram's rounding by kappa; in the basis U1 the pencil has M~1 ~ I.
    // Both bases span the same subspace (Eq. SubspaceGeneralizedEigenproblem).
    tg = timing_begin(ctx, st);
    SPARC_CUDA(ctx, tc::gram(ctx, U, ld, U, ld, nd, ns, Ms, tcs, st, false, true));
    SPARC_LAUNCH(ctx, "gram M0");
    timing_end(ctx, TK_GRAM, tg, st);
    cudaEvent_t t0 = timing_begin(ctx, st);
    cudaEvent_t to = timing_begin(ctx, st);
    // FP32 Cholesky of the diagonally scaled Gram, D^-1/2 M~ D^-1/2 = L' L'^T (unit
    // diagonal), U1 = U D^-1/2 L'^-T.  How closely U1 comes out orthonormal is all its
    // rounding decides: the Gram of U1 below measures what is left and the second
    // factorisation removes it.  A failed FP32 factorisation falls back to FP64.
    float* M32 = S0;
    float* Li32 = S1;
    int w0 = 0;
    if (ctx->inject_fp64_ortho >= 2) {
      w0 = STATUS_NOT_POSDEF;   // injected: as if the FP32 factorisation had failed
    } else {
      // the scaling and the blocked factorisation and inverse: a chain of small launches,
      // captured once per size and workspace into a CUDA graph and replayed (eagerly with
      // the synchronous debug check)
      auto factor = [&](cudaStream_t fs) -> sparc_status {
        k_scale_unit<<<ceil_div(nn, 256), 256, 0, fs>>>((const double*)Ms, ns, lam, M32, ctx->d_status);
        ++ctx->launches;
        return chol_inverse<float>(ctx, M32, Li32, ns, (float*)Dinv, SV, (float*)partH, 2 * pcap, fs);
      };
      s = replay(ctx, std::make_tuple(1 << 20, ns, (void*)Ms, (void*)M32, (void*)Li32), st, factor);
      if (s != SPARC_OK) return s;
      SPARC_CUDA(ctx, cudaMemcpyAsync(&w0, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    }
    if (w0 & STATUS_NOT_POSDEF) {
      cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
      s = chol_inverse<TW>(ctx, Ms, Li, ns, Dinv, T1, partH, pcap, st);
      if (s != SPARC_OK) return s;
      SPARC_CUDA(ctx, cudaMemcpyAsync(&w0, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      SPARC_CUDA(ctx, cudaStreamSynchronize(st));
      if (w0 & STATUS_NOT_POSDEF) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
        return fail(ctx, SPARC_ERR_NOT_POSDEF, "M~ = U^H U is not positive definite");
      }
      k_transpose<<<ceil_div(nn, 256), 256, 0, st>>>((const double*)Li, (double*)T1, ns);
    } else {
      k_t1_scaled<<<ceil_div(nn, 256), 256, 0, st>>>(Li32, lam, ns, (double*)T1);
    }
    ++ctx->launches;
    timing_end(ctx, TK_ORTHO, to, st);
    timing_end(ctx, TK_EIG, t0, st);
    cudaEvent_t t1 = timing_begin(ctx, st);
    SPARC_CUDA(ctx, tc::rotate(ctx, U, ld, (const double*)T1, nd, ns, W1, nd, tcs, st, true));   // U1 (T1 upper triangular)
    SPARC_LAUNCH(ctx, "orthonormalise");
    timing_end(ctx, TK_ROT, t1, st);
    Ub = W1;
    ldb = nd;
  }
  if constexpr (TCC) {
    // complex64 data: the same first orthonormalisation, U1 = U L^-H, with the Gram and
    // the rotation on the tensor cores and the factorisation of M~ = L L^H in FP64
    tg = timing_begin(ctx, st);
    SPARC_CUDA(ctx, tc::cgram(ctx, U, ld, U, ld, nd, ns, Ms, JB, tcs, st, true));
    SPARC_LAUNCH(ctx, "gram M0");
    timing_end(ctx, TK_GRAM, tg, st);
    cudaEvent_t t0 = timing_begin(ctx, st);
    cudaEvent_t to = timing_begin(ctx, st);
    s = chol_inverse<TW>(ctx, Ms, Li, ns, Dinv, T1, partH, pcap, st);
    if (s != SPARC_OK) return s;
    int w0 = 0;
    SPARC_CUDA(ctx, cudaMemcpyAsync(&w0, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    if (w0 & STATUS_NOT_POSDEF) {
      cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
      return fail(ctx, SPARC_ERR_NOT_POSDEF, "M~ = U^H U is not positive definite");
    }
    k_adjoint<TW><<<ceil_div(nn, 256), 256, 0, st>>>(Li, T1, ns);   // L^-H, upper triangular
    ++ctx->launches;
    timing_end(ctx, TK_ORTHO, to, st);
    timing_end(ctx, TK_EIG, t0, st);
    cudaEvent_t t1 = timing_begin(ctx, st);
    SPARC_CUDA(ctx, tc::crotate(ctx, U, ld, T1, nd, ns, W1, nd, tcs, st));
    SPARC_LAUNCH(ctx, "orthonormalise");
    timing_end(ctx, TK_ROT, t1, st);
    Ub = W1;
    ldb = nd;
  }
  // 1. HU = H U (U1 for FP32 and complex64 data)
  s = apply_block<T>(H, Ub, HU, ns, ldb, st, w);
  if (s != SPARC_OK) return s;
  // 2. H~ = U^H (HU), M~ = U^H U (split-K partials, then fixed-order sum + symmetrisation)
  tg = timing_begin(ctx, st);
  if constexpr (TCP) {
    SPARC_CUDA(ctx, tc::gram(ctx, Ub, nd, HU, nd, nd, ns, Hs, tcs, st));
    SPARC_LAUNCH(ctx, "gram H");
    SPARC_CUDA(ctx, tc::gram(ctx, Ub, nd, Ub, nd, nd, ns, Ms, tcs, st));
    SPARC_LAUNCH(ctx, "gram M");
  } else if constexpr (TCC) {
    SPARC_CUDA(ctx, tc::cgram(ctx, Ub, nd, HU, nd, nd, ns, Hs, JB, tcs, st));
    SPARC_LAUNCH(ctx, "gram H");
    SPARC_CUDA(ctx, tc::cgram(ctx, Ub, nd, Ub, nd, nd, ns, Ms, JB, tcs, st));
    SPARC_LAUNCH(ctx, "gram M");
  } else {
    SPARC_CUDA(ctx, (gemm<T, T, TC, TW, true, false>(ctx, ns, ns, (int)nd, U, ld, HU, nd, partH, ns, nsplit,
                                                     nn, 1.0, st)));
    SPARC_LAUNCH(ctx, "gram H");
    SPARC_CUDA(ctx, (gemm<T, T, TC, TW, true, false>(ctx, ns, ns, (int)nd, U, ld, U, ld, partM, ns, nsplit,
                                                     nn, 1.0, st)));
    SPARC_LAUNCH(ctx, "gram M");
    k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(partH, nsplit, nn, ns, Hs);
    ++ctx->launches;
    k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(partM, nsplit, nn, ns, Ms);
    ++ctx->launches;
    SPARC_LAUNCH(ctx, "gram");
  }
  timing_end(ctx, TK_GRAM, tg, st);
  cudaEvent_t te = timing_begin(ctx, st);
  cudaEvent_t tser = timing_begin(ctx, st);
  // In the orthonormalised basis M~1 = I + E with E of the order of the FP32 rounding
  // of the first factorisation.  Where max |E| <= EPS_SERIES its factor and inverse
  // are short series in E (below) whose small products run in FP32; otherwise the
  // blocked FP64 factorisation.
  bool series = false;
  if constexpr (TCP) {
    unsigned long long* emax = (unsigned long long*)scal;
    SPARC_CUDA(ctx, cudaMemsetAsync(emax, 0, sizeof(unsigned long long), st));
    k_eminus<<<ceil_div(nn, 256), 256, 0, st>>>((const double*)Ms, ns, (double*)A1, emax);
    ++ctx->launches;
    unsigned long long eb = 0;
    SPARC_CUDA(ctx, cudaMemcpyAsync(&eb, emax, sizeof(eb), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    double e;
    std::memcpy(&e, &eb, sizeof(e));
    series = e <= EPS_SERIES && ctx->inject_fp64_ortho == 0;
    ctx->last_ortho_err = e;
  }
  TW* Kc = Li;   // series: K = (I + F)^-1 - I, Linv = I + K
  if constexpr (TCP) {
    if (series) {
      // the series' chain of small launches, replayed from a CUDA graph
      auto series_launches = [&](cudaStream_t fs) -> sparc_status {
        double* E = (double*)A1;
        double* F = (double*)Vj;
        double* G = (double*)Qs;
        // 3'. F lower triangular with (I + F)(I + F)^T = I + E: F = Phi(E - F F^T),
        // iterated from F = Phi(E); each pass gains a power of |E| (|E|^5 after four)
        k_phi<<<ceil_div(nn, 256), 256, 0, fs>>>(E, nullptr, ns, F);
        ++ctx->launches;
        for (int it = 0; it < 3; ++it) {
          SPARC_CUDA(ctx, (gemm_f32p<false, true>(ctx, ns, ns, ns, F, ns, F, ns, G, ns, 1.0, 0.0, (double*)partH, pcap,
                                                  fs)));
          k_phi<<<ceil_div(nn, 256), 256, 0, fs>>>(E, G, ns, F);
          ++ctx->launches;
        }
        // K = (I + F)^-1 - I = -F (I - F (I - F (I - F))), error |F|^5
        double* Ta = (double*)Yr;
        double* Tb = (double*)T1;
        k_i_minus<<<ceil_div(nn, 256), 256, 0, fs>>>(F, ns, Ta);
        ++ctx->launches;
        for (int it = 0; it < 2; ++it) {
          k_identity<double><<<ceil_div(nn, 256), 256, 0, fs>>>(Tb, ns);
          ++ctx->launches;
          SPARC_CUDA(ctx, (gemm_f32p<false, false>(ctx, ns, ns, ns, F, ns, Ta, ns, Tb, ns, -1.0, 1.0, (double*)partH,
                                                   pcap, fs)));
          std::swap(Ta, Tb);
        }
        SPARC_CUDA(ctx, (gemm_f32p<false, false>(ctx, ns, ns, ns, F, ns, Ta, ns, (double*)Kc, ns, -1.0, 0.0,
                                                 (double*)partH, pcap, fs)));
        // 4'. C = (I + K) H~ (I + K)^T = H~ + P + P^T + P K^T with P = K H~; the
        // corrections are O(|K| |H~|), so their FP32 products are FP64-accurate in C
        double* P = (double*)T1;
        double* Q = (double*)Yr;
        SPARC_CUDA(ctx, (gemm_f32p<false, false>(ctx, ns, ns, ns, (const double*)Kc, ns, (const double*)Hs, ns, P, ns,
                                                 1.0, 0.0, (double*)partH, pcap, fs)));
        SPARC_CUDA(ctx, (gemm_f32p<false, true>(ctx, ns, ns, ns, P, ns, (const double*)Kc, ns, Q, ns, 1.0, 0.0,
                                                (double*)partH, pcap, fs)));
        k_csum<<<ceil_div(nn, 256), 256, 0, fs>>>((const double*)Hs, P, Q, ns, (double*)A0);
        ++ctx->launches;
        return SPARC_OK;
      };
      s = replay(ctx, std::make_tuple(1 << 21, ns, (void*)A1, (void*)Vj, (void*)Qs), st, series_launches);
      if (s != SPARC_OK) return s;
    }
  }
  if (!series) {
    // 3. M~ = L L^H (blocked, FP64) and Linv = L^-1
    s = chol_inverse<TW>(ctx, Ms, Li, ns, Dinv, T1, partH, pcap, st);
    if (s != SPARC_OK) return s;
    int word = 0;
    SPARC_CUDA(ctx, cudaMemcpyAsync(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    if (word & STATUS_NOT_POSDEF) {
      cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
      return fail(ctx, SPARC_ERR_NOT_POSDEF, "M~ = U^H U is not positive definite");
    }
    // 4. C = Linv H~ Linv^H (symmetrised) into A0
    SPARC_CUDA(ctx, (gemm64<TW, false, false>(ctx, ns, ns, ns, Li, ns, Hs, ns, T1, ns, 1.0, 0.0, partH, pcap, st)));
    SPARC_CUDA(ctx, (gemm64<TW, false, true>(ctx, ns, ns, ns, T1, ns, Li, ns, Yr, ns, 1.0, 0.0, partH, pcap, st)));
    k_reduce_sym<TW><<<ceil_div(nn, 256), 256, 0, st>>>(Yr, 1, nn, ns, A0);
    ++ctx->launches;
  }
  timing_end(ctx, TK_SERIES, tser, st);
  int sweeps = 0;
  cudaEvent_t tritz = nullptr;
  if (!mixed) {
    // 5a. FP64 Jacobi on C; eigenvalues from the converged diagonal
    k_identity<TW><<<ceil_div(nn, 256), 256, 0, st>>>(Vj, ns);
    ++ctx->launches;
    SPARC_LAUNCH(ctx, "subspace matrix");
    TW* Ares = nullptr;
    s = jacobi<TW>(ctx, A0, A1, Vj, ns, 1e-26, 40, scal, &Ares, &sweeps, st);
    if (s != SPARC_OK) return s;
    k_sort<TW><<<ceil_div(ns, 128), 128, 0, st>>>(Ares, nullptr, ns, eig, (int*)scal);
    k_permute_cols<TW><<<ceil_div(nn, 256), 256, 0, st>>>(Vj, (const int*)scal, ns, Qs);
    ctx->launches += 2;
  } else {
    // 5b. FP32 Jacobi on C for the eigenvectors, FP64 Rayleigh quotients for the eigenvalues
    k_convert<TW, TS><<<ceil_div(nn, 256), 256, 0, st>>>(A0, S0, nn);
    ++ctx->launches;
    k_identity<TS><<<ceil_div(nn, 256), 256, 0, st>>>(SV, ns);
    ++ctx->launches;
    SPARC_LAUNCH(ctx, "subspace matrix");
    TS* Sres = nullptr;
    s = jacobi<TS>(ctx, S0, S1, SV, ns, 1e-10, 40, scal, &Sres, &sweeps, st, Wjb);
    if (s != SPARC_OK) return s;
    tritz = timing_begin(ctx, st);
    // FP32 Jacobi vectors are orthonormal to about (rotations per vector) x u32; one
    // Newton-Schulz step, V <- V (3 I - V^H V) / 2, squares that error
    // the Ritz pairs' chain of launches (FP32 data: replayed from a CUDA graph)
    auto ritz = [&](cudaStream_t fs) -> sparc_status {
      if constexpr (TCP) {
        // real data: the step on the tensor cores (compensated TF32 Gram with FP64 sums,
        // 3xTF32 product): V ends orthonormal to about 1e-7, below the FP32 rounding of
        // the orbitals it rotates
        SPARC_CUDA(ctx, tc::gram(ctx, (const float*)SV, ns, (const float*)SV, ns, ns, ns, (double*)T1, tcs, fs));
        k_ns_coef<<<ceil_div(nn, 256), 256, 0, fs>>>((double*)T1, ns);
        ++ctx->launches;
        SPARC_CUDA(ctx, tc::rotate(ctx, (const float*)SV, ns, (const double*)T1, ns, ns, (float*)S1, ns, tcs, fs));
        k_convert<TS, TW><<<ceil_div(nn, 256), 256, 0, fs>>>(S1, Vj, nn);
        ++ctx->launches;
        // C V with FP32-exact V: float-float products and sums at the FP32 rate
        k_gemm_ff<<<dim3((unsigned)ceil_div(ns, 32), (unsigned)ceil_div(ns, 32)), 256, 0, fs>>>(
            (const double*)A0, (const double*)Vj, (double*)T1, ns);
        ++ctx->launches;
      } else {
        k_convert<TS, TW><<<ceil_div(nn, 256), 256, 0, fs>>>(SV, A1, nn);
        ++ctx->launches;
        SPARC_CUDA(ctx, (gemm64<TW, true, false>(ctx, ns, ns, ns, A1, ns, A1, ns, T1, ns, 1.0, 0.0, partH, pcap, fs)));
        SPARC_CUDA(ctx, cudaMemcpyAsync(Vj, A1, nn * sizeof(TW), cudaMemcpyDeviceToDevice, fs));
        SPARC_CUDA(ctx, (gemm64<TW, false, false>(ctx, ns, ns, ns, A1, ns, T1, ns, Vj, ns, -0.5, 1.5, partH, pcap, fs)));
        SPARC_CUDA(ctx, (gemm64<TW, false, false>(ctx, ns, ns, ns, A0, ns, Vj, ns, T1, ns, 1.0, 0.0, partH, pcap, fs)));
      }
      k_rayleigh<TW><<<ceil_div(ns, 8), 256, 0, fs>>>(Vj, T1, ns, lam);
      ++ctx->launches;
      k_sort<TW><<<ceil_div(ns, 128), 128, 0, fs>>>(nullptr, lam, ns, eigw, (int*)scal);
      k_permute_cols<TW><<<ceil_div(nn, 256), 256, 0, fs>>>(Vj, (const int*)scal, ns, Qs);
      ctx->launches += 2;
      return SPARC_OK;
    };
    if constexpr (TCP) s = replay(ctx, std::make_tuple(1 << 22, ns, (void*)SV, (void*)eigw, (void*)Qs), st, ritz);
    else s = ritz(st);
    if (s != SPARC_OK) return s;
    // the caller's eig outside the graph, so that the graph's key holds no caller buffer
    SPARC_CUDA(ctx, cudaMemcpyAsync(eig, eigw, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  timing_end(ctx, TK_RITZ, tritz, st);
  ctx->last_sweeps = sweeps;
  // 6. Ritz vectors of the pencil: Yr = Linv^H Q (series: Q + K^T Q)
  if (series) {
    SPARC_CUDA(ctx, cudaMemcpyAsync(Yr, Qs, nn * sizeof(TW), cudaMemcpyDeviceToDevice, st));
    if constexpr (TCP)
      SPARC_CUDA(ctx, (gemm_f32p<true, false>(ctx, ns, ns, ns, (const double*)Kc, ns, (const double*)Qs, ns,
                                              (double*)Yr, ns, 1.0, 1.0, (double*)partH, pcap, st)));
  } else {
    SPARC_CUDA(ctx, (gemm64<TW, true, false>(ctx, ns, ns, ns, Li, ns, Qs, ns, Yr, ns, 1.0, 0.0, partH, pcap, st)));
  }
  // 7. rotation U <- U Yr (into HU, then back into U)
  if constexpr (!TCP && !TCC) {
    k_narrow<TW, T><<<ceil_div(nn, 256), 256, 0, st>>>(Yr, YrT, nn);
    ++ctx->launches;
  }
  SPARC_LAUNCH(ctx, "ritz vectors");
  timing_end(ctx, TK_EIG, te, st);
  cudaEvent_t tr = timing_begin(ctx, st);
  if constexpr (TCP) {
    SPARC_CUDA(ctx, tc::rotate(ctx, Ub, ldb, Yr, nd, ns, U, ld, tcs, st));   // U1 -> U
  } else if constexpr (TCC) {
    SPARC_CUDA(ctx, tc::crotate(ctx, Ub, ldb, Yr, nd, ns, U, ld, tcs, st));  // U1 -> U
  } else {
    SPARC_CUDA(ctx, (gemm<T, T, TC, T, false, false>(ctx, (int)nd, ns, ns, U, ld, YrT, ns, HU, nd, 1, 0, 1.0, st)));
    SPARC_CUDA(ctx, cudaMemcpy2DAsync(U, ld * es, HU, nd * es, nd * es, ns, cudaMemcpyDeviceToDevice, st));
  }
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
    case SPARC_F64: return rayleigh_ritz<double, double>(H, (double*)U, ns, ld, eig, false, st);
    case SPARC_F32: return rayleigh_ritz<float, float>(H, (float*)U, ns, ld, eig, true, st);
    case SPARC_C128: return rayleigh_ritz<cf64, cf64>(H, (cf64*)U, ns, ld, eig, false, st);
    case SPARC_C64: return rayleigh_ritz<cf32, cf32>(H, (cf32*)U, ns, ld, eig, true, st);
  }
  return SPARC_ERR_INVALID_ARG;
}
