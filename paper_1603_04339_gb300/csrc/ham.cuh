// Internal representation of H(k) on the device and the kernel entry points
// shared between the translation units of libsparc.
#pragma once

#include "common.cuh"

struct sparc_ham {
  sparc_ctx* ctx = nullptr;
  int device = 0;                // the context's device (sparc_ham_destroy does not read ctx)
  sparc_grid grid{};
  sparc::GridDev gd{};
  double* d_veff = nullptr;      // [Nd]
  float* d_veff32 = nullptr;     // [Nd]
  int nproj = 0;
  double* d_gamma = nullptr;     // [nproj]
  float* d_gamma32 = nullptr;
  // Projector-major list (gather): entries p_off[p] .. p_off[p+1] hold the grid
  // node and the value chi~_p[g] (Bloch phase of the image included).
  long long n_ent = 0;
  long long* d_p_off = nullptr;  // [nproj+1]
  int* d_p_g = nullptr;          // [n_ent]
  // Node-major list (scatter): entries pt_ptr[g] .. pt_ptr[g+1] hold (p, chi~_p[g]).
  int* d_pt_ptr = nullptr;       // [Nd+1]
  int* d_pt_p = nullptr;         // [n_ent]
  // chi~ values converted to each element type (indexed by sparc_dtype), built
  // on first use; host copies of the exact values are kept for that.
  void* d_p_val[4] = {nullptr, nullptr, nullptr, nullptr};   // [n_ent], projector-major
  void* d_pt_val[4] = {nullptr, nullptr, nullptr, nullptr};  // [n_ent], node-major
  std::vector<double> h_p_re, h_p_im, h_pt_re, h_pt_im;
  void* fast = nullptr;          // sparc::fast::Tables* (tiled FP32 kernels)
};

namespace sparc {

// Element size of a dtype.
inline size_t dtype_size(sparc_dtype d) {
  switch (d) {
    case SPARC_F64: return 8;
    case SPARC_F32: return 4;
    case SPARC_C128: return 16;
    case SPARC_C64: return 8;
  }
  return 0;
}

// Launchers implemented in hpass.cu (templated on the element type).
template <class T>
cudaError_t launch_to_blocks(const T* X, long long ld, int ns, T* B, long long nd, int nblk,
                             cudaStream_t st);
template <class T>
cudaError_t launch_from_blocks(const T* B, long long nd, int nblk, T* X, long long ld, int ns,
                               cudaStream_t st);
// The same between X and a row layout: nd = rows x n1 nodes, each row held as n1 + 2 pad
// nodes in the blocks (pad ghost nodes at either end repeat the other end of the row;
// for complex data times the Bloch factor ph = exp(i k_x L_x) on the right, conj(ph) on
// the left).
template <class T>
cudaError_t launch_to_blocks_rows(const T* X, long long ld, int ns, T* B, long long nd, int n1, int pad,
                                  int nblk, cudaStream_t st, cf32 ph = cf32{1.f, 0.f});
template <class T>
cudaError_t launch_from_blocks_rows(const T* B, long long nd, int n1, int pad, int nblk, T* X, long long ld,
                                    int ns, cudaStream_t st);
// gc[p][blk][lane] = gamma_p * h1h2h3 * sum_g conj(chi~_p[g]) Y[blk][g][lane]
template <class T>
cudaError_t launch_nl_gather(const sparc_ham* H, const T* Y, int nbl, int nblk, T* gc,
                             cudaStream_t st);
// Yout = alpha*((H - shift) Yin) + beta*Yprev   (Yprev may alias Yout, or be null);
// diff: Laplacian in difference form (exact on constants; used for plain H-applies)
template <class T>
cudaError_t launch_hpass(const sparc_ham* H, const T* Yin, const T* Yprev, T* Yout, const T* gc,
                         int nbl, int nblk, double alpha, double shift, double beta, bool diff,
                         cudaStream_t st);

}  // namespace sparc
