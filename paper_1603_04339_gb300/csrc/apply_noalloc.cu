// sparc_apply_H_noalloc: Y = H X with no device allocation in the call.
//
// Some callers cannot call cudaMalloc at the point where they need H X:
// applications whose device memory is owned by another allocator or pool that
// must not be bypassed (a framework's caching allocator, a fixed memory budget),
// and latency-bound loops that may not block on the driver's allocator, which
// can synchronise the device.  sparc_apply_H grows the context workspace on
// demand; this variant instead works in a fixed scratch array that lives in
// the library image itself (a file-scope __device__ array), so the only
// memory it touches is the caller's X and Y, the Hamiltonian's own arrays and
// that array.
//
// The scratch array is SPARC_NOALLOC_SCRATCH_BYTES (32 MiB) on every GPU that
// loads the library, held until the process exits.  Every call on a device
// shares it: calls that overlap on the GPU (other streams, other contexts,
// other threads) race on it and must be serialised by the caller.  Each call
// writes every scratch byte it reads before reading it (block copy of X,
// projector coefficients, H-pass output), so nothing has to start at zero and
// what a previous call left behind is never used.
#include <mutex>

#include "rr.cuh"

// The fixed scratch array (one copy per device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPARC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on `device` (which must be current).
// cudaGetSymbolAddress runs once per device, on the first call there; in host
// code the array's name is only a host-side stand-in, so kernels get this address.
// The address is kept for the life of the process (stale after cudaDeviceReset).
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (g_scratch_dev[device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[device] = p;
  }
  *out = g_scratch_dev[device];
  return cudaSuccess;
}

template <class T>
sparc_status apply_static(sparc_ham* H, const T* X, T* Y, int ns, long long ld, cudaStream_t st,
                          char* base, size_t bb) {
  using namespace sparc;
  const int nblk = ceil_div(ns, NB);
  T* b0 = (T*)base;
  T* b1 = (T*)(base + bb);
  T* gc = (T*)(base + 2 * bb);
  SPARC_CUDA(H->ctx, launch_to_blocks<T>(X, ld, ns, b0, H->gd.nd, nblk, st));
  ++H->ctx->launches;
  SPARC_CUDA(H->ctx, launch_nl_gather<T>(H, b0, NB, nblk, gc, st));
  SPARC_CUDA(H->ctx, launch_hpass<T>(H, b0, nullptr, b1, gc, NB, nblk, 1.0, 0.0, 0.0, true, st));
  SPARC_CUDA(H->ctx, launch_from_blocks<T>(b1, H->gd.nd, nblk, Y, ld, ns, st));
  ++H->ctx->launches;
  return SPARC_OK;
}

}  // namespace

using namespace sparc;

extern "C" sparc_status sparc_apply_H_noalloc(sparc_ham* H, sparc_dtype dtype, const void* X,
                                              void* Y, int ns, int64_t ld, void* stream) {
  if (!H) return SPARC_ERR_INVALID_ARG;
  sparc_ctx* ctx = H->ctx;
  if ((int)dtype < 0 || (int)dtype > 3) return fail(ctx, SPARC_ERR_INVALID_ARG, "unknown dtype");
  if (H->gd.cplx && (dtype == SPARC_F64 || dtype == SPARC_F32))
    return fail(ctx, SPARC_ERR_INVALID_ARG, "real dtype needs k = 0 (Gamma point)");
  if (ns < 1) return fail(ctx, SPARC_ERR_INVALID_ARG, "ns must be >= 1");
  if (ld < H->gd.nd) return fail(ctx, SPARC_ERR_INVALID_ARG, "ld must be >= Nd");
  if (X == nullptr || Y == nullptr) return fail(ctx, SPARC_ERR_INVALID_ARG, "null X or Y");
  const size_t es = dtype_size(dtype);
  const char* x0 = (const char*)X;
  const char* y0 = (const char*)Y;
  const size_t span = ((size_t)(ns - 1) * (size_t)ld + (size_t)H->gd.nd) * es;
  if (x0 < y0 + span && y0 < x0 + span) return fail(ctx, SPARC_ERR_INVALID_ARG, "X and Y overlap");
  // projector values in this precision are uploaded by the allocating entry points
  if (H->nproj > 0 && (H->d_p_val[dtype] == nullptr || H->d_pt_val[dtype] == nullptr))
    return fail(ctx, SPARC_ERR_INVALID_ARG,
                "projector values for this dtype are not on the device yet: call sparc_apply_H "
                "once with this dtype and this Hamiltonian first");
  const int nblk = ceil_div(ns, NB);
  const size_t bb = align256((size_t)nblk * H->gd.nd * NB * es);
  const size_t gb = align256((size_t)(H->nproj > 0 ? H->nproj : 1) * nblk * NB * es);
  if (2 * bb + gb > (size_t)SPARC_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, SPARC_ERR_INVALID_ARG,
                "problem too large for the fixed scratch of sparc_apply_H_noalloc: needs " +
                    std::to_string(2 * bb + gb) + " bytes, limit " +
                    std::to_string((size_t)SPARC_NOALLOC_SCRATCH_BYTES) +
                    " (2 * ceil(ns/8)*8*Nd + nproj*ceil(ns/8)*8 elements)");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  void* base = nullptr;
  SPARC_CUDA(ctx, scratch_address(ctx->device, &base));
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case SPARC_F64:
      return apply_static<double>(H, (const double*)X, (double*)Y, ns, ld, st, (char*)base, bb);
    case SPARC_F32:
      return apply_static<float>(H, (const float*)X, (float*)Y, ns, ld, st, (char*)base, bb);
    case SPARC_C128:
      return apply_static<cf64>(H, (const cf64*)X, (cf64*)Y, ns, ld, st, (char*)base, bb);
    case SPARC_C64:
      return apply_static<cf32>(H, (const cf32*)X, (cf32*)Y, ns, ld, st, (char*)base, bb);
  }
  return SPARC_ERR_INVALID_ARG;
}
