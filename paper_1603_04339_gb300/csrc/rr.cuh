// Internal interfaces shared by the API, Lanczos and Rayleigh-Ritz translation units.
#pragma once

#include "ham.cuh"

namespace sparc {

struct BlockWs {
  void* b0;   // interleaved block buffer
  void* b1;   // interleaved block buffer
  void* gc;   // projector coefficients [nproj][nblk][NB]
  char* tail; // first byte after the block workspace (start of the caller's extra bytes)
  void* gs = nullptr;   // projection scratch of the tiled FP32 H-apply (null: the generic kernels)
};
// Bytes of projection scratch the tiled FP32 H-apply needs for ns orbitals (0 where it
// does not apply).
size_t apply_scratch_bytes(sparc_ham* H, sparc_dtype dt, int ns);

sparc_status ensure_vals(sparc_ham* H, sparc_dtype dt);
sparc_status check_block_args(sparc_ham* H, sparc_dtype dt, const void* X, const void* Y, int ns,
                              int64_t ld);
// Carve the block workspace plus `extra` bytes (returned through *tail, 256-aligned).
sparc_status block_ws(sparc_ham* H, sparc_dtype dt, int ns, size_t extra, BlockWs* w, char** tail);
template <class T>
sparc_status apply_block(sparc_ham* H, const T* X, T* Y, int ns, long long ld, cudaStream_t st,
                         const BlockWs& w);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of workspace one filter call of (H, dtype, ns) needs; with `base`, also lay
// the block workspace out there.
size_t filter_ws(sparc_ham* H, sparc_dtype dt, int ns, char* base, BlockWs* w);
// The filter on a caller-laid-out workspace (arguments already checked).
sparc_status filter_run(sparc_ham* H, sparc_dtype dtype, int m, double a, double b, double a0, const void* X,
                        void* Y, int ns, long long ld, cudaStream_t st, const BlockWs& w);

// Tensor-core (tcgen05, 3xTF32) products of FP32 orbitals (tc_gemm.cu).
namespace tc {
// G = A^T B (ns x ns, FP64, symmetrised) for column-major nd x ns FP32 A, B.
size_t gram_scratch_bytes(const sparc_ctx* ctx, int ns, long long nd);
// anti: G is antisymmetric (tiles below the diagonal are minus the transposes);
// fast: longer FP32 accumulation chunks (sums of like-signed products about 6e-7 low
// instead of 2.5e-7), where FP32 accuracy is enough.
cudaError_t gram(sparc_ctx* ctx, const float* A, long long lda, const float* B, long long ldb, long long nd, int ns,
                 double* G, void* scratch, cudaStream_t st, bool anti = false, bool fast = false);
// G = A^H B (ns x ns, complex FP64, Hermitian) for column-major nd x ns complex64 A, B,
// from two real Grams of the real views; JB: nd x ns complex64 scratch (i B).
size_t cgram_scratch_bytes(const sparc_ctx* ctx, int ns, long long nd);
cudaError_t cgram(sparc_ctx* ctx, const cf32* A, long long lda, const cf32* B, long long ldb, long long nd, int ns,
                  cf64* G, cf32* JB, void* scratch, cudaStream_t st, bool fast = false);
// C = U Yr (nd x ns, FP32) for column-major FP32 U and FP64 ns x ns Yr; C must not overlap U.
size_t rot_scratch_bytes(int ns, bool cplx = false);
cudaError_t rotate(sparc_ctx* ctx, const float* U, long long ldu, const double* Yr, long long nd, int ns, float* C,
                   long long ldc, void* scratch, cudaStream_t st, bool upper = false);
// The same for complex64 U, C and complex FP64 Yr (one real rotation with 2 ns values of k).
cudaError_t crotate(sparc_ctx* ctx, const cf32* U, long long ldu, const cf64* Yr, long long nd, int ns, cf32* C,
                    long long ldc, void* scratch, cudaStream_t st);
}  // namespace tc

}  // namespace sparc
