// Learned initial density (project-added; the paper starts from the superposition
// of atomic densities): atom-centred Gaussian descriptors of the grid nodes and a
// 3-layer ReLU perceptron 16 -> 128 -> 128 -> 1, trained with the mean-squared
// error and Adam, all in these kernels.
//
// Training kernel: persistent CTAs (one per SM) take tiles of 64 points; a tile's
// forward pass keeps both hidden layers in shared memory, its backward pass
// reuses them in place, and the weight gradients accumulate in registers across
// the CTA's tiles.  Per-CTA partial gradients are reduced in a fixed order in
// FP64, so a gradient is reproducible bit for bit.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ham.cuh"

namespace sparc {
namespace mlp {

constexpr int NF = 16, NH = 128, TP = 64, THR = 256;
constexpr int NPAR = NF * NH + NH + NH * NH + NH + NH + 1;
constexpr int PW = NH + 4;   // row pitch (floats) of the [.][NH] shared arrays: rows stay 16-byte aligned
// offsets of the flat parameter vector [W1, b1, W2, b2, w3, b3]
constexpr int OW1 = 0, OB1 = OW1 + NF * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
static_assert(OB3 + 1 == NPAR, "parameter layout");

struct Smem {
  float W1[NF][NH];
  float b1[NH], b2[NH], w3[NH];
  float W2[NH][PW];     // W2[i][j]
  float W2T[NH][PW];    // W2[j][i] (the backward product with W2^T)
  float X[TP][NF];
  float A1[TP][PW];     // relu(z1), later dL/dz1
  float A2[TP][PW];     // relu(z2), later dL/dz2
  float t[TP], dy[TP];
  float b3;
  double red[THR / 32];
};

static_assert(sizeof(Smem) <= 227 * 1024, "shared memory of one CTA");

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Parameters into shared memory (both orientations of W2).
__device__ void load_params(Smem& s, const float* __restrict__ th) {
  for (int e = threadIdx.x; e < NF * NH; e += THR) s.W1[e / NH][e % NH] = th[OW1 + e];
  for (int e = threadIdx.x; e < NH * NH; e += THR) {
    const float w = th[OW2 + e];
    s.W2[e / NH][e % NH] = w;
    s.W2T[e % NH][e / NH] = w;
  }
  for (int e = threadIdx.x; e < NH; e += THR) {
    s.b1[e] = th[OB1 + e];
    s.b2[e] = th[OB2 + e];
    s.w3[e] = th[OW3 + e];
  }
  if (threadIdx.x == 0) s.b3 = th[OB3];
}

// Points [p0, p0 + TP) of the batch (point p is row idx[p] of D and t, or row p without
// idx) into s.X (and targets into s.t); rows past np are zero.  A row index outside
// [0, nrows) is not read: the point counts as zero and the status word records it.
__device__ void load_tile(Smem& s, const float* __restrict__ D, const float* __restrict__ tgt,
                          const long long* __restrict__ idx, long long p0, long long np, long long nrows,
                          int* status) {
  for (int e = threadIdx.x; e < TP * NF; e += THR) {
    const int r = e / NF, f = e % NF;
    const long long p = p0 + r;
    float v = 0.f;
    if (p < np) {
      const long long row = idx ? idx[p] : p;
      if (row >= 0 && row < nrows) v = D[row * NF + f];
      else if (f == 0) atomicOr(status, STATUS_BAD_INDEX);
    }
    s.X[r][f] = v;
  }
  if (tgt)
    for (int r = threadIdx.x; r < TP; r += THR) {
      const long long p = p0 + r;
      const long long row = p < np ? (idx ? idx[p] : p) : -1;
      s.t[r] = (row >= 0 && row < nrows) ? tgt[row] : 0.f;
    }
}

// A1 = relu(X W1 + b1), A2 = relu(A1 W2 + b2) for the tile (thread: 4 points x 8 units).
__device__ void hidden_layers(Smem& s) {
  const int pr = (threadIdx.x / 16) * 4, jc = (threadIdx.x % 16) * 8;
  float acc[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = s.b1[jc + c];
#pragma unroll 4
  for (int k = 0; k < NF; ++k) {
    const float4 w0 = ld4(&s.W1[k][jc]), w1 = ld4(&s.W1[k][jc + 4]);
    const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float x = s.X[pr + r][k];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(x, w[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s.A1[pr + r][jc + c] = fmaxf(acc[r][c], 0.f);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = s.b2[jc + c];
#pragma unroll 4
  for (int k = 0; k < NH; ++k) {
    const float4 w0 = ld4(&s.W2[k][jc]), w1 = ld4(&s.W2[k][jc + 4]);
    const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float a = s.A1[pr + r][k];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a, w[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s.A2[pr + r][jc + c] = fmaxf(acc[r][c], 0.f);
  __syncthreads();
}

// y of the tile's point tid/4 (all four lanes of the group return it).
__device__ float output(Smem& s) {
  const int p = threadIdx.x / 4, q = threadIdx.x % 4;
  float v = 0.f;
#pragma unroll 8
  for (int j = q * 32; j < q * 32 + 32; ++j) v = fmaf(s.A2[p][j], s.w3[j], v);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v + s.b3;
}

__global__ void __launch_bounds__(THR, 1)
k_mlp_forward(const float* __restrict__ th, const float* __restrict__ D, long long np, float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& s = *reinterpret_cast<Smem*>(smraw);
  load_params(s, th);
  for (long long p0 = (long long)blockIdx.x * TP; p0 < np; p0 += (long long)gridDim.x * TP) {
    __syncthreads();
    load_tile(s, D, nullptr, nullptr, p0, np, np, nullptr);
    __syncthreads();
    hidden_layers(s);
    const float v = output(s);
    const long long p = p0 + threadIdx.x / 4;
    if (threadIdx.x % 4 == 0 && p < np) y[p] = v;
  }
}

// Per-CTA partial gradient of sum_p (y_p - t_p)^2 / N into part[cta][NPAR] and the
// partial loss sum_p (y_p - t_p)^2 into lpart[cta].
__global__ void __launch_bounds__(THR, 1)
k_mlp_grad(const float* __restrict__ th, const float* __restrict__ D, const float* __restrict__ tgt,
           const long long* __restrict__ idx, long long np, long long nrows, int* status, float* __restrict__ part,
           double* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& s = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x;
  load_params(s, th);
  const float inv_n = 1.0f / (float)np;
  // register accumulators: gW2 (8 x 8 block), gW1 (8 units of one feature),
  // gb1/gb2/gw3 (thread j < NH), gb3 and the loss
  const int gi = (tid / 16) * 8, gj = (tid % 16) * 8;   // gW2 block
  const int f1 = tid / 16, u1 = (tid % 16) * 8;          // gW1 row f1, units u1..u1+7
  float gW2[8][8], gW1[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    gW1[a] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) gW2[a][c] = 0.f;
  }
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
  double loss = 0.0;
  for (long long p0 = (long long)blockIdx.x * TP; p0 < np; p0 += (long long)gridDim.x * TP) {
    __syncthreads();
    load_tile(s, D, tgt, idx, p0, np, nrows, status);
    __syncthreads();
    hidden_layers(s);
    // output and dL/dy = 2 (y - t) / N (zero for padding rows)
    {
      const float v = output(s);
      const int p = tid / 4;
      if (tid % 4 == 0) {
        const bool ok = p0 + p < np;
        const float r = ok ? v - s.t[p] : 0.f;
        s.dy[p] = 2.f * r * inv_n;
        loss += (double)r * (double)r;
      }
    }
    __syncthreads();
    if (tid < NH) {
      float a = 0.f, c = 0.f;
      for (int p = 0; p < TP; ++p) a = fmaf(s.A2[p][tid], s.dy[p], a);
      gw3 += a;
      if (tid == 0) {
        for (int p = 0; p < TP; ++p) c += s.dy[p];
        gb3 += c;
      }
    }
    __syncthreads();
    // dL/dz2 = dy w3 [a2 > 0], in place of A2
    {
      const int pr = (tid / 16) * 4, jc = (tid % 16) * 8;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float a = s.A2[pr + r][jc + c];
          s.A2[pr + r][jc + c] = a > 0.f ? s.dy[pr + r] * s.w3[jc + c] : 0.f;
        }
    }
    __syncthreads();
    // gW2 += A1^T dZ2, gb2 += sum_p dZ2
#pragma unroll 2
    for (int p = 0; p < TP; ++p) {
      const float4 a0 = ld4(&s.A1[p][gi]), a1 = ld4(&s.A1[p][gi + 4]);
      const float4 d0 = ld4(&s.A2[p][gj]), d1 = ld4(&s.A2[p][gj + 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) gW2[a][c] = fmaf(av[a], dv[c], gW2[a][c]);
    }
    if (tid < NH) {
      float c = 0.f;
      for (int p = 0; p < TP; ++p) c += s.A2[p][tid];
      gb2 += c;
    }
    // dL/da1 = dZ2 W2^T (thread: 4 points x 8 units), masked by [a1 > 0]
    float dA[4][8];
    {
      const int pr = (tid / 16) * 4, ic = (tid % 16) * 8;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) dA[r][c] = 0.f;
#pragma unroll 4
      for (int j = 0; j < NH; ++j) {
        const float4 w0 = ld4(&s.W2T[j][ic]), w1 = ld4(&s.W2T[j][ic + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float d = s.A2[pr + r][j];
#pragma unroll
          for (int c = 0; c < 8; ++c) dA[r][c] = fmaf(d, w[c], dA[r][c]);
        }
      }
    }
    __syncthreads();   // every read of A1 (gW2) is done
    {
      const int pr = (tid / 16) * 4, ic = (tid % 16) * 8;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float a = s.A1[pr + r][ic + c];
          s.A1[pr + r][ic + c] = a > 0.f ? dA[r][c] : 0.f;
        }
    }
    __syncthreads();
    // gW1 += X^T dZ1, gb1 += sum_p dZ1
#pragma unroll 4
    for (int p = 0; p < TP; ++p) {
      const float x = s.X[p][f1];
      const float4 d0 = ld4(&s.A1[p][u1]), d1 = ld4(&s.A1[p][u1 + 4]);
      const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
      for (int c = 0; c < 8; ++c) gW1[c] = fmaf(x, dv[c], gW1[c]);
    }
    if (tid < NH) {
      float c = 0.f;
      for (int p = 0; p < TP; ++p) c += s.A1[p][tid];
      gb1 += c;
    }
  }
  // partial gradient of this CTA
  float* g = part + (size_t)blockIdx.x * NPAR;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) g[OW2 + (gi + a) * NH + gj + c] = gW2[a][c];
#pragma unroll
  for (int c = 0; c < 8; ++c) g[OW1 + f1 * NH + u1 + c] = gW1[c];
  if (tid < NH) {
    g[OB1 + tid] = gb1;
    g[OB2 + tid] = gb2;
    g[OW3 + tid] = gw3;
  }
  if (tid == 0) g[OB3] = gb3;
  // loss: warp shuffles, then the warps in order
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (tid % 32 == 0) s.red[tid / 32] = loss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < THR / 32; ++w) t += s.red[w];
    lpart[blockIdx.x] = t;
  }
}

// grad[i] = sum over CTAs of part[c][i] (FP64, fixed order); loss = sum lpart / N.
__global__ void k_mlp_reduce(const float* __restrict__ part, const double* __restrict__ lpart, int ncta,
                             long long np, float* __restrict__ grad, double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPAR) {
    double v = 0.0;
    for (int c = 0; c < ncta; ++c) v += (double)part[(size_t)c * NPAR + i];
    grad[i] = (float)v;
  }
  if (i == 0) {
    double l = 0.0;
    for (int c = 0; c < ncta; ++c) l += lpart[c];
    *loss = l / (double)np;
  }
}

// Adam (Kingma and Ba): m, v moments, bias corrections c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPAR) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Per-axis image sums g[(a * NF + k) * natom + J][x] = sum_{t=-1..1}
// exp(-(x_a - R_Ja - t L_a)^2 / s_k^2), x over the nodes of axis a (padded to nmax).
__global__ void k_desc_axis(int n0, int n1, int n2, double h0, double h1, double h2, const double* __restrict__ R,
                            int natom, const double* __restrict__ s, int nmax, double* __restrict__ g) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = 3LL * NF * natom * nmax;
  if (e >= tot) return;
  const int x = (int)(e % nmax);
  const int J = (int)((e / nmax) % natom);
  const int k = (int)((e / ((long long)nmax * natom)) % NF);
  const int a = (int)(e / ((long long)nmax * natom * NF));
  const int n = a == 0 ? n0 : a == 1 ? n1 : n2;
  const double h = a == 0 ? h0 : a == 1 ? h1 : h2;
  double v = 0.0;
  if (x < n) {
    const double L = n * h;
    const double xa = -0.5 * L + x * h - R[3 * J + a];
    const double sk2 = s[k] * s[k];
    for (int t = -1; t <= 1; ++t) {
      const double d = xa - t * L;
      v += exp(-d * d / sk2);
    }
  }
  g[e] = v;
}

// D[node][k] = sum_J gx gy gz (FP64 sum, stored FP32).
__global__ void k_desc(int n0, int n1, int n2, int natom, int nmax, const double* __restrict__ g,
                       float* __restrict__ D) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nd = (long long)n0 * n1 * n2;
  if (node >= nd) return;
  const int i = (int)(node % n0), j = (int)((node / n0) % n1), l = (int)(node / ((long long)n0 * n1));
  for (int k = 0; k < NF; ++k) {
    const double* gx = g + ((size_t)(0 * NF + k) * natom) * nmax;
    const double* gy = g + ((size_t)(1 * NF + k) * natom) * nmax;
    const double* gz = g + ((size_t)(2 * NF + k) * natom) * nmax;
    double v = 0.0;
    for (int J = 0; J < natom; ++J) v += gx[(size_t)J * nmax + i] * gy[(size_t)J * nmax + j] * gz[(size_t)J * nmax + l];
    D[node * NF + k] = (float)v;
  }
}

}  // namespace mlp
}  // namespace sparc

using namespace sparc;
using namespace sparc::mlp;

struct sparc_mlp {
  sparc_ctx* ctx = nullptr;
  int device = 0;
  float *d_theta = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr, *d_part = nullptr;
  double *d_lpart = nullptr, *d_loss = nullptr;
  int ncta = 0;
  long long step = 0;
};

static void free_mlp(sparc_mlp* M) {
  cudaFree(M->d_theta);
  cudaFree(M->d_m);
  cudaFree(M->d_v);
  cudaFree(M->d_grad);
  cudaFree(M->d_part);
  cudaFree(M->d_lpart);
  cudaFree(M->d_loss);
}

static sparc_status launch_grad(sparc_mlp* M, const float* D, const float* t, const long long* idx, long long np,
                                long long nrows, cudaStream_t st) {
  const size_t smem = sizeof(Smem);
  SPARC_CUDA(M->ctx, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ncta = (int)std::min<long long>(M->ncta, (np + TP - 1) / TP);
  k_mlp_grad<<<ncta, THR, smem, st>>>(M->d_theta, D, t, idx, np, nrows, M->ctx->d_status, M->d_part, M->d_lpart);
  k_mlp_reduce<<<(NPAR + 255) / 256, 256, 0, st>>>(M->d_part, M->d_lpart, ncta, np, M->d_grad, M->d_loss);
  M->ctx->launches += 2;
  SPARC_LAUNCH(M->ctx, "mlp gradient");
  return SPARC_OK;
}

extern "C" {

sparc_status sparc_mlp_create(sparc_ctx* ctx, const float* theta, sparc_mlp** out) {
  if (!ctx || !theta || !out) return SPARC_ERR_INVALID_ARG;
  *out = nullptr;
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  sparc_mlp* M = new (std::nothrow) sparc_mlp();
  if (!M) return fail(ctx, SPARC_ERR_OOM, "mlp allocation failed");
  M->ctx = ctx;
  M->device = ctx->device;
  M->ncta = std::max(1, ctx->nsm);
  const size_t pb = NPAR * sizeof(float);
  bool ok = cudaMalloc(&M->d_theta, pb) == cudaSuccess && cudaMalloc(&M->d_m, pb) == cudaSuccess &&
            cudaMalloc(&M->d_v, pb) == cudaSuccess && cudaMalloc(&M->d_grad, pb) == cudaSuccess &&
            cudaMalloc(&M->d_part, pb * M->ncta) == cudaSuccess &&
            cudaMalloc(&M->d_lpart, M->ncta * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&M->d_loss, sizeof(double)) == cudaSuccess;
  ok = ok && cudaMemcpy(M->d_theta, theta, pb, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(M->d_m, 0, pb) == cudaSuccess && cudaMemset(M->d_v, 0, pb) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_mlp(M);
    delete M;
    return fail(ctx, SPARC_ERR_OOM, "mlp device allocation failed");
  }
  *out = M;
  return SPARC_OK;
}

sparc_status sparc_mlp_params(sparc_mlp* M, float* theta_host, int set) {
  if (!M || !theta_host) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(M->ctx, cudaSetDevice(M->ctx->device));
  const size_t pb = NPAR * sizeof(float);
  if (set) {
    SPARC_CUDA(M->ctx, cudaDeviceSynchronize());
    SPARC_CUDA(M->ctx, cudaMemcpy(M->d_theta, theta_host, pb, cudaMemcpyHostToDevice));
    SPARC_CUDA(M->ctx, cudaMemset(M->d_m, 0, pb));
    SPARC_CUDA(M->ctx, cudaMemset(M->d_v, 0, pb));
    M->step = 0;
  } else {
    SPARC_CUDA(M->ctx, cudaDeviceSynchronize());
    SPARC_CUDA(M->ctx, cudaMemcpy(theta_host, M->d_theta, pb, cudaMemcpyDeviceToHost));
  }
  return SPARC_OK;
}

sparc_status sparc_mlp_descriptors(sparc_ctx* ctx, const int* n, const double* h, int natom, const double* R,
                                   const double* widths, float* D, void* stream) {
  if (!ctx || !n || !h || !R || !widths || !D || natom < 1) return SPARC_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (n[a] < 1 || !(h[a] > 0.0)) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_mlp_descriptors: bad grid");
  for (int k = 0; k < NF; ++k)
    if (!(widths[k] > 0.0)) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_mlp_descriptors: widths must be > 0");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int nmax = std::max(n[0], std::max(n[1], n[2]));
  const size_t gsz = (size_t)3 * NF * natom * nmax;
  const size_t need = align_up(gsz * sizeof(double)) + align_up((size_t)3 * natom * sizeof(double)) +
                      align_up(NF * sizeof(double));
  if (!ensure_ws(ctx, need)) return fail(ctx, SPARC_ERR_OOM, "workspace allocation failed");
  char* p = (char*)ctx->ws;
  double* g = (double*)p;
  double* dR = (double*)(p + align_up(gsz * sizeof(double)));
  double* ds = (double*)(p + align_up(gsz * sizeof(double)) + align_up((size_t)3 * natom * sizeof(double)));
  SPARC_CUDA(ctx, cudaMemcpyAsync(dR, R, 3 * natom * sizeof(double), cudaMemcpyHostToDevice, st));
  SPARC_CUDA(ctx, cudaMemcpyAsync(ds, widths, NF * sizeof(double), cudaMemcpyHostToDevice, st));
  k_desc_axis<<<(unsigned)((gsz + 255) / 256), 256, 0, st>>>(n[0], n[1], n[2], h[0], h[1], h[2], dR, natom, ds,
                                                             nmax, g);
  const long long nd = (long long)n[0] * n[1] * n[2];
  k_desc<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(n[0], n[1], n[2], natom, nmax, g, D);
  ctx->launches += 2;
  SPARC_LAUNCH(ctx, "descriptors");
  // the host arrays were staged by cudaMemcpyAsync from pageable memory: finish before returning
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  return SPARC_OK;
}

sparc_status sparc_mlp_forward(sparc_mlp* M, const float* D, int64_t np, float* y, void* stream) {
  if (!M || !D || !y || np < 1) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(M->ctx, cudaSetDevice(M->ctx->device));
  const size_t smem = sizeof(Smem);
  SPARC_CUDA(M->ctx, cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ncta = (int)std::min<long long>(M->ncta, (np + TP - 1) / TP);
  k_mlp_forward<<<ncta, THR, smem, (cudaStream_t)stream>>>(M->d_theta, D, np, y);
  ++M->ctx->launches;
  SPARC_LAUNCH(M->ctx, "mlp forward");
  return SPARC_OK;
}

sparc_status sparc_mlp_grad(sparc_mlp* M, const float* D, const float* t, int64_t nrows, const int64_t* idx,
                            int64_t np, float* grad, double* loss, void* stream) {
  if (!M || !D || !t || np < 1 || nrows < 1 || (!idx && np > nrows)) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(M->ctx, cudaSetDevice(M->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  sparc_status s = launch_grad(M, D, t, (const long long*)idx, np, nrows, st);
  if (s != SPARC_OK) return s;
  if (grad) SPARC_CUDA(M->ctx, cudaMemcpyAsync(grad, M->d_grad, NPAR * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (loss) {
    SPARC_CUDA(M->ctx, cudaMemcpyAsync(loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(M->ctx, cudaStreamSynchronize(st));
  }
  return SPARC_OK;
}

sparc_status sparc_mlp_train_step(sparc_mlp* M, const float* D, const float* t, int64_t nrows, const int64_t* idx,
                                  int64_t np, float lr, double* loss, void* stream) {
  if (!M || !D || !t || np < 1 || nrows < 1 || (!idx && np > nrows) || !(lr > 0.f)) return SPARC_ERR_INVALID_ARG;
  SPARC_CUDA(M->ctx, cudaSetDevice(M->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  sparc_status s = launch_grad(M, D, t, (const long long*)idx, np, nrows, st);
  if (s != SPARC_OK) return s;
  const double b1 = 0.9, b2 = 0.999;
  ++M->step;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)M->step)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)M->step)));
  k_adam<<<(NPAR + 255) / 256, 256, 0, st>>>(M->d_theta, M->d_grad, M->d_m, M->d_v, lr, (float)b1, (float)b2, c1, c2,
                                              1e-8f);
  ++M->ctx->launches;
  SPARC_LAUNCH(M->ctx, "adam");
  if (loss) {
    SPARC_CUDA(M->ctx, cudaMemcpyAsync(loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(M->ctx, cudaStreamSynchronize(st));
  }
  return SPARC_OK;
}

void sparc_mlp_destroy(sparc_mlp* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  cudaDeviceSynchronize();
  free_mlp(M);
  delete M;
}

}  // extern "C"
