// H-apply / Chebyshev-recurrence pass, nonlocal projection (gather) and the
// layout transposes between the column-major ABI layout and the
// orbital-interleaved layout the kernels work in.
//
// Interleaved layout: B[blk][g][lane], lane = orbital within a block of `nbl`
// orbitals (nbl = NB = 8 for blocks of orbitals, 1 for single vectors).  The 8
// orbitals of one grid node are one contiguous 32-byte sector (FP32), the
// projector values of a node are shared by its 8 lanes, and every node-index
// computation is shared by those lanes.
#include <type_traits>

#include "ham.cuh"

namespace sparc {

namespace {

template <class T>
__device__ __forceinline__ T ldg(const T* p) { return *p; }
template <>
__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ cf64 ldg(const cf64* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ cf32 ldg(const cf32* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// One output element of  Yout = alpha * ((H - shift) Yin) + beta * Yprev.
// H = -1/2 nabla_h^2 (Eq. FD:Laplacian, Bloch-periodic wrap) + V_eff
//   + sum_p chi~_p gc_p (Eq. NonlocalPS:FD; gc = gamma h^3 chi~^H Yin from the gather).
// DIFF selects the difference form sum_p c_p ((f_{+p} - f_0) + (f_{-p} - f_0)), which
// uses sum_p w_p = -w_0 to drop the centre weight: constants are annihilated
// exactly and rounding stays relative to the local variation of f, so FP32
// weights do not shift the spectrum.  The filter passes use the direct form.
template <class T, int NBL, bool DIFF>
__global__ void __launch_bounds__(256)
k_hpass(GridDev gd, const T* __restrict__ Yin, const T* Yprev, T* Yout,
        const typename Tr<T>::R* __restrict__ veff, const int* __restrict__ pt_ptr,
        const int* __restrict__ pt_p, const T* __restrict__ pt_val, const T* __restrict__ gc,
        int nblk, typename Tr<T>::R alpha, typename Tr<T>::R shift, typename Tr<T>::R beta) {
  using R = typename Tr<T>::R;
  using C = typename Tr<T>::C;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = (int)(t % NBL);
  const long long g = t / NBL;
  if (g >= gd.nd) return;
  const int blk = blockIdx.y;
  const size_t base = (size_t)blk * gd.nd * NBL;
  const T* Y = Yin + base;
  const int n1 = gd.n1, n2 = gd.n2, n3 = gd.n3;
  const int i = (int)(g % n1);
  const int j = (int)((g / n1) % n2);
  const int k = (int)(g / ((long long)n1 * n2));
  const long long sx = NBL, sy = (long long)n1 * NBL, sz = (long long)n1 * n2 * NBL;
  const T* yc = Y + g * NBL + lane;
  const T f0 = ldg(yc);
  R c0 = veff[g] - shift;
  if (!DIFF) c0 += (R)(2.0 * (gd.coef[0][0] + gd.coef[1][0] + gd.coef[2][0]));
  T acc = scale(c0, f0);
  C phx{(R)gd.ph_re[0], (R)gd.ph_im[0]}, phy{(R)gd.ph_re[1], (R)gd.ph_im[1]},
      phz{(R)gd.ph_re[2], (R)gd.ph_im[2]};
  C phxm{phx.x, -phx.y}, phym{phy.x, -phy.y}, phzm{phz.x, -phz.y};
  // x
  for (int p = 1; p <= gd.no; ++p) {
    int ip = i + p, im = i - p;
    T a, b;
    if (ip < n1) a = ldg(yc + p * sx);
    else { a = ldg(yc + (long long)(ip - n1 - i) * sx); if constexpr (Tr<T>::cplx) a = Tr<T>::mulc(a, phx); }
    if (im >= 0) b = ldg(yc - p * sx);
    else { b = ldg(yc + (long long)(im + n1 - i) * sx); if constexpr (Tr<T>::cplx) b = Tr<T>::mulc(b, phxm); }
    if (DIFF) acc = axpy(acc, (R)gd.coef[0][p], add(a - f0, b - f0));
    else acc = axpy(acc, (R)gd.coef[0][p], add(a, b));
  }
  // y
  for (int p = 1; p <= gd.no; ++p) {
    int jp = j + p, jm = j - p;
    T a, b;
    if (jp < n2) a = ldg(yc + p * sy);
    else { a = ldg(yc + (long long)(jp - n2 - j) * sy); if constexpr (Tr<T>::cplx) a = Tr<T>::mulc(a, phy); }
    if (jm >= 0) b = ldg(yc - p * sy);
    else { b = ldg(yc + (long long)(jm + n2 - j) * sy); if constexpr (Tr<T>::cplx) b = Tr<T>::mulc(b, phym); }
    if (DIFF) acc = axpy(acc, (R)gd.coef[1][p], add(a - f0, b - f0));
    else acc = axpy(acc, (R)gd.coef[1][p], add(a, b));
  }
  // z
  for (int p = 1; p <= gd.no; ++p) {
    int kp = k + p, km = k - p;
    T a, b;
    if (kp < n3) a = ldg(yc + p * sz);
    else { a = ldg(yc + (long long)(kp - n3 - k) * sz); if constexpr (Tr<T>::cplx) a = Tr<T>::mulc(a, phz); }
    if (km >= 0) b = ldg(yc - p * sz);
    else { b = ldg(yc + (long long)(km + n3 - k) * sz); if constexpr (Tr<T>::cplx) b = Tr<T>::mulc(b, phzm); }
    if (DIFF) acc = axpy(acc, (R)gd.coef[2][p], add(a - f0, b - f0));
    else acc = axpy(acc, (R)gd.coef[2][p], add(a, b));
  }
  // nonlocal scatter: sum over the projectors whose box holds node g
  if (pt_ptr != nullptr) {
    const int e1 = pt_ptr[g + 1];
    for (int e = pt_ptr[g]; e < e1; ++e) {
      const int p = pt_p[e];
      acc = fmac(acc, ldg(pt_val + e), ldg(gc + ((size_t)p * nblk + blk) * NBL + lane));
    }
  }
  T out = scale(alpha, acc);
  const size_t o = base + (size_t)g * NBL + lane;
  if (Yprev != nullptr) out = axpy(out, beta, Yprev[o]);
  Yout[o] = out;
}

// gc[p][blk][lane] = gamma_p * dv * sum_{e in box p} conj(chi~_p[e]) * Y[blk][g_e][lane]
// (trapezoidal rule, Eq. IntApprox; projection of Eq. NonlocalPS:FD).  One CTA
// per (projector, block); deterministic two-level reduction, no atomics.
template <class T, int NBL>
__global__ void __launch_bounds__(256)
k_nl_gather(const T* __restrict__ Y, long long nd, const long long* __restrict__ p_off,
            const int* __restrict__ p_g, const T* __restrict__ p_val,
            const typename Tr<T>::R* __restrict__ gamma, typename Tr<T>::R dv, T* __restrict__ gc,
            int nblk) {
  constexpr int G = 256 / NBL;
  __shared__ T sm[256];
  const int p = blockIdx.x, blk = blockIdx.y;
  const int lane = threadIdx.x % NBL, grp = threadIdx.x / NBL;
  const T* Yb = Y + (size_t)blk * nd * NBL;
  T acc = Tr<T>::zero();
  const long long e1 = p_off[p + 1];
  for (long long e = p_off[p] + grp; e < e1; e += G)
    acc = fmacj(acc, ldg(p_val + e), ldg(Yb + (size_t)p_g[e] * NBL + lane));
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = G / 2; s >= 1; s >>= 1) {
    if (grp < s) sm[threadIdx.x] = add(sm[threadIdx.x], sm[threadIdx.x + s * NBL]);
    __syncthreads();
  }
  if (grp == 0) gc[((size_t)p * nblk + blk) * NBL + lane] = scale(gamma[p] * dv, sm[lane]);
}

// Column-major X (Nd x ns, ld) -> B[blk][g][NB]; lanes past ns are zero.
// One CTA moves 32 nodes x NB orbitals: coalesced reads along g per orbital,
// one contiguous 32*NB-element write.
template <class T>
__global__ void __launch_bounds__(256) k_to_blocks(const T* __restrict__ X, long long ld, int ns,
                                                   T* __restrict__ B, long long nd) {
  __shared__ T tile[NB][33];
  const long long g0 = (long long)blockIdx.x * 32;
  const int blk = blockIdx.y;
  const int o = threadIdx.y, x = threadIdx.x;   // blockDim = (32, NB)
  const int n = blk * NB + o;
  const long long g = g0 + x;
  tile[o][x] = (n < ns && g < nd) ? X[g + (long long)n * ld] : Tr<T>::zero();
  __syncthreads();
  const int t = threadIdx.y * 32 + threadIdx.x;
  const int p = t / NB, l = t % NB;
  if (g0 + p < nd) B[((size_t)blk * nd + g0 + p) * NB + l] = tile[l][p];
}

template <class T>
__global__ void __launch_bounds__(256) k_from_blocks(const T* __restrict__ B, long long nd,
                                                     T* __restrict__ X, long long ld, int ns) {
  __shared__ T tile[NB][33];
  const long long g0 = (long long)blockIdx.x * 32;
  const int blk = blockIdx.y;
  const int t = threadIdx.y * 32 + threadIdx.x;
  const int p = t / NB, l = t % NB;
  if (g0 + p < nd) tile[l][p] = B[((size_t)blk * nd + g0 + p) * NB + l];
  __syncthreads();
  const int o = threadIdx.y, x = threadIdx.x;
  const int n = blk * NB + o;
  const long long g = g0 + x;
  if (n < ns && g < nd) X[g + (long long)n * ld] = tile[o][x];
}

// The same moves, a CTA per (rows of one block): the nodes form rows of n1, and the
// block holds each row as n1 + 2 pad nodes, x' = x + pad, where x' < pad and
// x' >= n1 + pad repeat the other end of the row (the periodic wrap in x; pad = 0 for
// the plain layout).  Thread (x', part) moves the 16 bytes of 16 / sizeof(T)
// orbitals of node x' in every row of the CTA: reads along a row are coalesced per
// orbital, writes contiguous; orbitals past ns read as zero.  nd = nrows n1.
// Complex data are Bloch-periodic (Section 3.1): a ghost node x = x' - pad outside
// [0, n1) holds its image's value times ph^t, t = floor(x / n1), ph = exp(i k_x L_x).
template <class T>
__global__ void __launch_bounds__(1024) k_to_blocks_rows(const T* __restrict__ X, long long ld, int ns,
                                                        T* __restrict__ B, int n1, int pad, long long nrows,
                                                        int rpc, cf32 ph) {
  constexpr int EPT = 16 / (int)sizeof(T), TPN = NB / EPT;
  const int n1p = n1 + 2 * pad;
  const int t = threadIdx.x;
  if (t >= TPN * n1p) return;
  const int xp = t / TPN, part = t % TPN;
  const int xs = ((xp - pad) % n1 + n1) % n1;
  // phase of this thread's node: 1 inside the row, ph (right ghosts) or conj(ph) (left)
  const cf32 gph = xp < pad ? cf32{ph.x, -ph.y} : (xp >= n1 + pad ? ph : cf32{1.f, 0.f});
  const int blk = blockIdx.y;
  const int c0 = blk * NB + part * EPT;
  const long long r0 = (long long)blockIdx.x * rpc, r1 = min(nrows, r0 + rpc);
  T* Bb = B + (size_t)blk * nrows * n1p * NB + part * EPT;
#pragma unroll 4
  for (long long r = r0; r < r1; ++r) {
    const long long g = r * n1 + xs;
    union { T v[EPT]; uint4 u; } w;
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      w.v[e] = c0 + e < ns ? X[g + (long long)(c0 + e) * ld] : Tr<T>::zero();
    if constexpr (std::is_same<T, cf32>::value) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) w.v[e] = w.v[e] * gph;
    }
    *reinterpret_cast<uint4*>(Bb + (size_t)(r * n1p + xp) * NB) = w.u;
  }
}

template <class T>
__global__ void __launch_bounds__(1024) k_from_blocks_rows(const T* __restrict__ B, int n1, int pad,
                                                          long long nrows, int rpc, T* __restrict__ X,
                                                          long long ld, int ns) {
  constexpr int EPT = 16 / (int)sizeof(T), TPN = NB / EPT;
  const int n1p = n1 + 2 * pad;
  const int t = threadIdx.x;
  if (t >= TPN * n1) return;
  const int x = t / TPN, part = t % TPN;
  const int blk = blockIdx.y;
  const int c0 = blk * NB + part * EPT;
  const long long r0 = (long long)blockIdx.x * rpc, r1 = min(nrows, r0 + rpc);
  const T* Bb = B + (size_t)blk * nrows * n1p * NB + part * EPT;
#pragma unroll 4
  for (long long r = r0; r < r1; ++r) {
    const long long g = r * n1 + x;
    union { T v[EPT]; uint4 u; } w;
    w.u = *reinterpret_cast<const uint4*>(Bb + (size_t)(r * n1p + x + pad) * NB);
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (c0 + e < ns) X[g + (long long)(c0 + e) * ld] = w.v[e];
  }
}

template <class T>
const typename Tr<T>::R* veff_of(const sparc_ham* H);
template <> const double* veff_of<double>(const sparc_ham* H) { return H->d_veff; }
template <> const double* veff_of<cf64>(const sparc_ham* H) { return H->d_veff; }
template <> const float* veff_of<float>(const sparc_ham* H) { return H->d_veff32; }
template <> const float* veff_of<cf32>(const sparc_ham* H) { return H->d_veff32; }

template <class T>
const typename Tr<T>::R* gamma_of(const sparc_ham* H);
template <> const double* gamma_of<double>(const sparc_ham* H) { return H->d_gamma; }
template <> const double* gamma_of<cf64>(const sparc_ham* H) { return H->d_gamma; }
template <> const float* gamma_of<float>(const sparc_ham* H) { return H->d_gamma32; }
template <> const float* gamma_of<cf32>(const sparc_ham* H) { return H->d_gamma32; }

}  // namespace

// Rows per CTA of the row kernels: about 16 KB moved per CTA.
template <class T>
static int rows_per_cta(int n1p) {
  return std::max(1, (int)(16384 / ((size_t)n1p * NB * sizeof(T))));
}

template <class T>
cudaError_t launch_to_blocks_rows(const T* X, long long ld, int ns, T* B, long long nd, int n1, int pad,
                                  int nblk, cudaStream_t st, cf32 ph) {
  constexpr int TPN = NB / (16 / (int)sizeof(T));
  const int n1p = n1 + 2 * pad;
  if (TPN * n1p > 1024 || n1 <= 0 || nd % n1 != 0) return cudaErrorInvalidValue;
  const long long nrows = nd / n1;
  const int rpc = rows_per_cta<T>(n1p);
  dim3 grid((unsigned)ceil_div(nrows, (long long)rpc), (unsigned)nblk);
  k_to_blocks_rows<T><<<grid, (unsigned)ceil_div(TPN * n1p, 32) * 32, 0, st>>>(X, ld, ns, B, n1, pad, nrows, rpc,
                                                                                 ph);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_from_blocks_rows(const T* B, long long nd, int n1, int pad, int nblk, T* X, long long ld,
                                    int ns, cudaStream_t st) {
  constexpr int TPN = NB / (16 / (int)sizeof(T));
  const int n1p = n1 + 2 * pad;
  if (TPN * n1p > 1024 || n1 <= 0 || nd % n1 != 0) return cudaErrorInvalidValue;
  const long long nrows = nd / n1;
  const int rpc = rows_per_cta<T>(n1p);
  dim3 grid((unsigned)ceil_div(nrows, (long long)rpc), (unsigned)nblk);
  k_from_blocks_rows<T><<<grid, (unsigned)ceil_div(TPN * n1, 32) * 32, 0, st>>>(B, n1, pad, nrows, rpc, X, ld, ns);
  return cudaGetLastError();
}

// The plain layout [blk][g][NB] as rows of 128 nodes (the last one ragged).
template <class T>
cudaError_t launch_to_blocks(const T* X, long long ld, int ns, T* B, long long nd, int nblk,
                             cudaStream_t st) {
  if (nd % 128 != 0) {
    dim3 grid((unsigned)ceil_div(nd, 32), (unsigned)nblk), block(32, NB);
    k_to_blocks<T><<<grid, block, 0, st>>>(X, ld, ns, B, nd);
    return cudaGetLastError();
  }
  return launch_to_blocks_rows<T>(X, ld, ns, B, nd, 128, 0, nblk, st);
}

template <class T>
cudaError_t launch_from_blocks(const T* B, long long nd, int nblk, T* X, long long ld, int ns,
                               cudaStream_t st) {
  if (nd % 128 != 0) {
    dim3 grid((unsigned)ceil_div(nd, 32), (unsigned)nblk), block(32, NB);
    k_from_blocks<T><<<grid, block, 0, st>>>(B, nd, X, ld, ns);
    return cudaGetLastError();
  }
  return launch_from_blocks_rows<T>(B, nd, 128, 0, nblk, X, ld, ns, st);
}

template <class T>
cudaError_t launch_nl_gather(const sparc_ham* H, const T* Y, int nbl, int nblk, T* gc,
                             cudaStream_t st) {
  if (H->nproj == 0) return cudaSuccess;
  using R = typename Tr<T>::R;
  const T* pv = reinterpret_cast<const T*>(H->d_p_val[DtypeOf<T>::v]);
  const R dv = (R)(H->grid.h[0] * H->grid.h[1] * H->grid.h[2]);
  dim3 grid((unsigned)H->nproj, (unsigned)nblk);
  cudaEvent_t t0 = timing_begin(H->ctx, st);
  if (nbl == NB)
    k_nl_gather<T, NB><<<grid, 256, 0, st>>>(Y, H->gd.nd, H->d_p_off, H->d_p_g, pv, gamma_of<T>(H),
                                             dv, gc, nblk);
  else
    k_nl_gather<T, 1><<<grid, 256, 0, st>>>(Y, H->gd.nd, H->d_p_off, H->d_p_g, pv, gamma_of<T>(H),
                                            dv, gc, nblk);
  ++H->ctx->launches;
  timing_end(H->ctx, TK_GATHER, t0, st);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_hpass(const sparc_ham* H, const T* Yin, const T* Yprev, T* Yout, const T* gc,
                         int nbl, int nblk, double alpha, double shift, double beta, bool diff,
                         cudaStream_t st) {
  using R = typename Tr<T>::R;
  const T* ptv = H->nproj ? reinterpret_cast<const T*>(H->d_pt_val[DtypeOf<T>::v]) : nullptr;
  const int* ptr = H->nproj ? H->d_pt_ptr : nullptr;
  long long threads = H->gd.nd * nbl;
  dim3 grid((unsigned)ceil_div(threads, 256), (unsigned)nblk);
  cudaEvent_t t0 = timing_begin(H->ctx, st);
#define SPARC_HPASS(NBL_, D_)                                                                  \
  k_hpass<T, NBL_, D_><<<grid, 256, 0, st>>>(H->gd, Yin, Yprev, Yout, veff_of<T>(H), ptr,      \
                                             H->d_pt_p, ptv, gc, nblk, (R)alpha, (R)shift,    \
                                             (R)beta)
  if (nbl == NB) {
    if (diff) SPARC_HPASS(NB, true); else SPARC_HPASS(NB, false);
  } else {
    if (diff) SPARC_HPASS(1, true); else SPARC_HPASS(1, false);
  }
#undef SPARC_HPASS
  ++H->ctx->launches;
  timing_end(H->ctx, TK_HPASS, t0, st);
  return cudaGetLastError();
}

#define SPARC_INST(T)                                                                          \
  template cudaError_t launch_to_blocks_rows<T>(const T*, long long, int, T*, long long, int, int, \
                                                int, cudaStream_t, cf32);                      \
  template cudaError_t launch_from_blocks_rows<T>(const T*, long long, int, int, int, T*,      \
                                                  long long, int, cudaStream_t);               \
  template cudaError_t launch_to_blocks<T>(const T*, long long, int, T*, long long, int,       \
                                           cudaStream_t);                                      \
  template cudaError_t launch_from_blocks<T>(const T*, long long, int, T*, long long, int,     \
                                             cudaStream_t);                                    \
  template cudaError_t launch_nl_gather<T>(const sparc_ham*, const T*, int, int, T*,           \
                                           cudaStream_t);                                      \
  template cudaError_t launch_hpass<T>(const sparc_ham*, const T*, const T*, T*, const T*, int,\
                                       int, double, double, double, bool, cudaStream_t);
SPARC_INST(double)
SPARC_INST(float)
SPARC_INST(cf64)
SPARC_INST(cf32)

}  // namespace sparc
