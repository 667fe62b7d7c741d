// Shared device/host helpers of libsparc: scalar traits for the four element
// types, complex arithmetic, launch-error plumbing and the internal context.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sparc.h"

namespace sparc {

// ----------------------------------------------------------------- complex types
struct cf32 { float x, y; };
struct cf64 { double x, y; };

__host__ __device__ __forceinline__ cf32 operator+(cf32 a, cf32 b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cf32 operator-(cf32 a, cf32 b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cf32 operator*(cf32 a, cf32 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ __forceinline__ cf32 operator*(float s, cf32 a) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ cf64 operator+(cf64 a, cf64 b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cf64 operator-(cf64 a, cf64 b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cf64 operator*(cf64 a, cf64 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ __forceinline__ cf64 operator*(double s, cf64 a) { return {s * a.x, s * a.y}; }

// Scalar traits: R is the real type of the scalar T, C the complex type of the
// same precision (the phase factors of Bloch-periodic wrap are of type C).
template <class T> struct Tr;
template <> struct Tr<double> {
  using R = double; using C = cf64; static constexpr bool cplx = false;
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double conj(double a) { return a; }
  __host__ __device__ static double re(double a) { return a; }
  __host__ __device__ static double abs2(double a) { return a * a; }
  __host__ __device__ static double mulc(double a, cf64 ph) { return a * ph.x; }   // real path: phase is 1
  __host__ __device__ static double fromc(cf64 a) { return a.x; }
};
template <> struct Tr<float> {
  using R = float; using C = cf32; static constexpr bool cplx = false;
  __host__ __device__ static float zero() { return 0.f; }
  __host__ __device__ static float conj(float a) { return a; }
  __host__ __device__ static float re(float a) { return a; }
  __host__ __device__ static float abs2(float a) { return a * a; }
  __host__ __device__ static float mulc(float a, cf32 ph) { return a * ph.x; }
  __host__ __device__ static float fromc(cf32 a) { return a.x; }
};
template <> struct Tr<cf64> {
  using R = double; using C = cf64; static constexpr bool cplx = true;
  __host__ __device__ static cf64 zero() { return {0.0, 0.0}; }
  __host__ __device__ static cf64 conj(cf64 a) { return {a.x, -a.y}; }
  __host__ __device__ static double re(cf64 a) { return a.x; }
  __host__ __device__ static double abs2(cf64 a) { return a.x * a.x + a.y * a.y; }
  __host__ __device__ static cf64 mulc(cf64 a, cf64 ph) { return a * ph; }
  __host__ __device__ static cf64 fromc(cf64 a) { return a; }
};
template <> struct Tr<cf32> {
  using R = float; using C = cf32; static constexpr bool cplx = true;
  __host__ __device__ static cf32 zero() { return {0.f, 0.f}; }
  __host__ __device__ static cf32 conj(cf32 a) { return {a.x, -a.y}; }
  __host__ __device__ static float re(cf32 a) { return a.x; }
  __host__ __device__ static float abs2(cf32 a) { return a.x * a.x + a.y * a.y; }
  __host__ __device__ static cf32 mulc(cf32 a, cf32 ph) { return a * ph; }
  __host__ __device__ static cf32 fromc(cf32 a) { return a; }
};

// a*b for a real or complex scalar times a real or complex scalar of the same family.
__host__ __device__ __forceinline__ double mul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ float mul(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ cf64 mul(cf64 a, cf64 b) { return a * b; }
__host__ __device__ __forceinline__ cf32 mul(cf32 a, cf32 b) { return a * b; }
__host__ __device__ __forceinline__ double scale(double s, double a) { return s * a; }
__host__ __device__ __forceinline__ float scale(float s, float a) { return s * a; }
__host__ __device__ __forceinline__ cf64 scale(double s, cf64 a) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ cf32 scale(float s, cf32 a) { return {s * a.x, s * a.y}; }
// a + s*b
__host__ __device__ __forceinline__ double axpy(double a, double s, double b) { return fma(s, b, a); }
__host__ __device__ __forceinline__ float axpy(float a, float s, float b) { return fmaf(s, b, a); }
__host__ __device__ __forceinline__ cf64 axpy(cf64 a, double s, cf64 b) { return {fma(s, b.x, a.x), fma(s, b.y, a.y)}; }
__host__ __device__ __forceinline__ cf32 axpy(cf32 a, float s, cf32 b) { return {fmaf(s, b.x, a.x), fmaf(s, b.y, a.y)}; }
// a + b*c (all same type)
__host__ __device__ __forceinline__ double fmac(double a, double b, double c) { return fma(b, c, a); }
__host__ __device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(b, c, a); }
__host__ __device__ __forceinline__ cf64 fmac(cf64 a, cf64 b, cf64 c) {
  return {fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y))};
}
__host__ __device__ __forceinline__ cf32 fmac(cf32 a, cf32 b, cf32 c) {
  return {fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y))};
}
// a + conj(b)*c
__host__ __device__ __forceinline__ double fmacj(double a, double b, double c) { return fma(b, c, a); }
__host__ __device__ __forceinline__ float fmacj(float a, float b, float c) { return fmaf(b, c, a); }
__host__ __device__ __forceinline__ cf64 fmacj(cf64 a, cf64 b, cf64 c) {
  return {fma(b.x, c.x, fma(b.y, c.y, a.x)), fma(b.x, c.y, fma(-b.y, c.x, a.y))};
}
__host__ __device__ __forceinline__ cf32 fmacj(cf32 a, cf32 b, cf32 c) {
  return {fmaf(b.x, c.x, fmaf(b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(-b.y, c.x, a.y))};
}
__host__ __device__ __forceinline__ double add(double a, double b) { return a + b; }
__host__ __device__ __forceinline__ float add(float a, float b) { return a + b; }
__host__ __device__ __forceinline__ cf64 add(cf64 a, cf64 b) { return a + b; }
__host__ __device__ __forceinline__ cf32 add(cf32 a, cf32 b) { return a + b; }

// Widening conversions used where FP32 data meets FP64 accumulators.
__host__ __device__ __forceinline__ double widen(float a) { return (double)a; }
__host__ __device__ __forceinline__ double widen(double a) { return a; }
__host__ __device__ __forceinline__ cf64 widen(cf32 a) { return {(double)a.x, (double)a.y}; }
__host__ __device__ __forceinline__ cf64 widen(cf64 a) { return a; }

// The scalar with real part r and zero imaginary part.
template <class T> __host__ __device__ __forceinline__ T from_real(double r);
template <> __host__ __device__ __forceinline__ double from_real<double>(double r) { return r; }
template <> __host__ __device__ __forceinline__ float from_real<float>(double r) { return (float)r; }
template <> __host__ __device__ __forceinline__ cf64 from_real<cf64>(double r) { return {r, 0.0}; }
template <> __host__ __device__ __forceinline__ cf32 from_real<cf32>(double r) { return {(float)r, 0.f}; }

// sparc_dtype of an element type.
template <class T> struct DtypeOf;
template <> struct DtypeOf<double> { static constexpr sparc_dtype v = SPARC_F64; };
template <> struct DtypeOf<float> { static constexpr sparc_dtype v = SPARC_F32; };
template <> struct DtypeOf<cf64> { static constexpr sparc_dtype v = SPARC_C128; };
template <> struct DtypeOf<cf32> { static constexpr sparc_dtype v = SPARC_C64; };

template <class T> struct Wide;
template <> struct Wide<float> { using W = double; };
template <> struct Wide<double> { using W = double; };
template <> struct Wide<cf32> { using W = cf64; };
template <> struct Wide<cf64> { using W = cf64; };

__host__ __device__ __forceinline__ float narrow_to(float*, double a) { return (float)a; }
__host__ __device__ __forceinline__ double narrow_to(double*, double a) { return a; }
__host__ __device__ __forceinline__ cf32 narrow_to(cf32*, cf64 a) { return {(float)a.x, (float)a.y}; }
__host__ __device__ __forceinline__ cf64 narrow_to(cf64*, cf64 a) { return a; }

// ----------------------------------------------------------------- device status word
// Bits latched by kernels; read and cleared by sparc_sync().
enum : int {
  STATUS_NOT_POSDEF = 1,
  STATUS_TIMEOUT = 2,
  STATUS_NO_CONVERGENCE = 4,
  STATUS_BAD_INDEX = 8,
};

// ----------------------------------------------------------------- geometry passed to kernels
constexpr int MAX_FD = 8;
constexpr int NB = 8;         // orbitals per interleaved block (8 lanes share a grid node)

struct GridDev {
  int n1, n2, n3;
  int no;                     // FD radius n_o
  long long nd;               // n1*n2*n3
  double coef[3][MAX_FD + 1]; // -1/2 * w_{p,s}  (w from Eq. weightsLap), p = 0..no
  double ph_re[3], ph_im[3];  // exp(i k_s L_s): Bloch phase picked up across the upper face
  int cplx;                   // k != 0
};

}  // namespace sparc

// ----------------------------------------------------------------- internal objects
struct sparc_ctx {
  int device = 0;
  int nsm = 152;                   // multiprocessors of the device
  std::string last_error;
  int* d_status = nullptr;         // device status word
  // growable workspace arena
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // kernel timing: event pairs per timed kernel class
  static constexpr int NTIMED = 10;
  long long launches = 0;          // kernels launched by this context (instrumentation)
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[NTIMED];
  std::vector<cudaEvent_t> ev_pool;
  // captured Jacobi sweeps, keyed by (element kind, n, buffers)
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_stream2 = nullptr;   // the second branch of a captured graph (block Jacobi V updates)
  cudaStream_t aux_stream[3] = {};       // branches of the FP32 triangular inverse
  std::map<std::tuple<int, int, void*, void*, void*>, cudaGraphExec_t> graphs;
  std::map<std::tuple<int, int, void*, void*, void*>, long long> graph_kernels;   // kernels per replay
  int last_sweeps = 0;
  double last_ortho_err = -1.0;   // max |U1^T U1 - I| of the last mixed Rayleigh-Ritz (-1: none)
  // the last k-point batch filter, captured as one graph: its arguments and executable
  struct KBatchGraph {
    std::vector<const void*> H;
    int m = 0, ns = 0, nkg = 0, nbk = 0;
    long long ld = 0;
    const void* X = nullptr;
    void* Y = nullptr;
    void* ws = nullptr;
    std::vector<double> a, b, a0;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
  } kbg;
  long long graph_launches = 0;    // graph launches of this context (instrumentation)
  // filter launch configuration chosen by sparc_autotune_filter, keyed by (dtype, Nd,
  // ns, number of k-points): units (blocks of NB orbitals) per launch + TUNE_SHAPE x the
  // FP32 pass tile shape
  std::map<std::tuple<int, long long, int, int>, int> tuned;
  // failure injection (sparc_debug_inject)
  int inject_alloc_fail = 0;        // workspace growths still to fail
  long long inject_wait_limit = 0;  // clocks of the TMA pass's bounded waits (0: default)
  int inject_stall = -1;            // step at which the next TMA pass stops producing
  int inject_cg_max = 0;            // Poisson CG iteration cap (0: default)
  int inject_fp64_ortho = 0;        // mixed RR: 1 second, 2 both orthonormalisations in FP64
};

namespace sparc {

struct Workspace;
bool ensure_ws(sparc_ctx* ctx, size_t bytes);

// Set the context's error string and return `st`.
sparc_status fail(sparc_ctx* ctx, sparc_status st, const std::string& msg);
sparc_status cuda_fail(sparc_ctx* ctx, cudaError_t e, const char* where);

#define SPARC_CUDA(ctx, call)                                   \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::sparc::cuda_fail(ctx, e_, #call); \
  } while (0)

// Debug aid: with SPARC_SYNC_CHECK=1 in the environment every checkpoint also
// synchronises the device, so that an asynchronous fault is reported at the
// stage that caused it.
bool sync_check();

#define SPARC_LAUNCH(ctx, what)                                                  \
  do {                                                                           \
    cudaError_t e_ = cudaGetLastError();                                         \
    if (e_ == cudaSuccess && ::sparc::sync_check()) e_ = cudaDeviceSynchronize(); \
    if (e_ != cudaSuccess) return ::sparc::cuda_fail(ctx, e_, what);             \
  } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// A tuned filter configuration packs units per launch (below TUNE_SHAPE) and the
// FP32 pass tile shape (its multiple of TUNE_SHAPE).
constexpr int TUNE_SHAPE = 1 << 20;

// Timing hooks: bracket a launch with events on `st` while timing is enabled.
// TK_ORTHO, TK_SERIES, TK_RITZ: parts of TK_EIG (mixed Rayleigh-Ritz): the first
// orthonormalisation's factorisation, the second factorisation with the reduction of H~,
// and the Ritz pairs after the sweeps (Newton-Schulz step, Rayleigh quotients, order)
enum TimedKernel { TK_HPASS = 0, TK_GATHER = 1, TK_GRAM = 2, TK_EIG = 3, TK_ROT = 4, TK_JAC = 5, TK_FPASS = 6,
                   TK_ORTHO = 7, TK_SERIES = 8, TK_RITZ = 9 };
cudaEvent_t timing_begin(sparc_ctx* ctx, cudaStream_t st);
void timing_end(sparc_ctx* ctx, int which, cudaEvent_t begin, cudaStream_t st);

}  // namespace sparc
