// Tables and launchers of the tiled FP32 / complex64 H-pass (hpass_fast.cu).
#pragma once

#include "ham.cuh"

namespace sparc {
namespace fast {

constexpr int R = 6;                  // FD radius of the tiled kernel (the paper's n_o = 6)
constexpr int TX = 16;                // x extent of a CTA tile
constexpr int ZC = 13;                // z-range of a CTA (one turn of the 13-deep queue)
constexpr int THREADS = 512;
constexpr int MAXI = 96;              // projector-box pieces a CTA can hold in shared memory
constexpr int MAXSTEP = 2048;         // (z, rows, x-run, piece) activations a CTA can hold
// per element type: x-consecutive nodes per thread and y extent of a CTA tile
// (the register queue holds 13 * RX values, which bounds RX for complex data)
template <class T> struct Shape;
template <> struct Shape<float> { static constexpr int RX = 4, TY = 16; };
template <> struct Shape<cf32> { static constexpr int RX = 2, TY = 8; };

// One axis-aligned piece of a projector group's box inside the grid: every
// node of the piece lies in the same periodic image, so its Bloch phase is one
// constant.  Box-local index of grid node (x, y, z) of the piece:
//   (x - gx0 + bx0) + nbx * ((y - gy0 + by0) + nby * (z - gz0 + bz0)).
struct SubBox {
  int gx0, gx1, gy0, gy1, gz0, gz1;
  int bx0, by0, bz0;
  int nbx, nby;
  int grp;
  long long chi4_off;   // group's first box node in chi4 (units of 4 projector values)
  float ph_re, ph_im;   // exp(-i k.(t L)) of this piece
};

// Up to four projectors sharing one box (s, p_x, p_y, p_z of one atom).
struct Group {
  int proj[4];          // projector indices, -1 where absent
  int sb0, sb1;         // sub-box range
};

// Per kernel tile shape (0: FP32 16x16, 1: complex64 16x8, 2: FP32 16x8 for
// 256-thread CTAs, two per SM): for every CTA
// (tile, z-chunk) the pieces that touch it, and per z the CTA-local indices
// of the pieces active in that plane.
struct Layout {
  int tiles_x = 0, tiles_y = 0, nchunk = 0;
  int max_items = 0, max_steps = 0;
  int* d_cptr = nullptr;      // [cta + 1] into d_citems
  int* d_citems = nullptr;    // sub-box ids
  int* d_sptr = nullptr;      // [((cta * ZC + k) * row groups + rg) * x-runs + xr] into d_sslots
  int* d_sslots = nullptr;    // CTA-local indices of the pieces touching those nodes at z
};

struct Tables {
  int ngrp = 0, nsb = 0;
  Group* d_grp = nullptr;
  SubBox* d_sb = nullptr;
  float* d_chi4 = nullptr;    // [box nodes][4], zero where a group has < 4 projectors
  Layout lay[3];
  unsigned long long geom = 0;   // hash of the grid, groups and piece geometry (not phases)
};

// k-points of one batched complex launch.  The Hamiltonians of a batch share the
// grid and the projector geometry (boxes, groups, per-CTA lists); each k keeps its
// own piece phases, projector values, V_eff and Bloch phases of the faces.
constexpr int KMAX = 32;
struct KSlot {
  const SubBox* sb;       // pieces with this k's phases (geometry as the batch's first H)
  const float4* chi4;
  const float* veff;
  const float* gamma;
  long long ubase;        // block-buffer unit of this slot's first block
  float phx_r, phx_i, phy_r, phy_i, phz_r, phz_i;   // exp(i k_s L_s)
  float alpha, shift, beta;                          // recurrence coefficients of this k
};
// A launch covers the units ubase(kk) + j for kk < nk, j < nbk.
struct KSlots {
  KSlot s[KMAX];
  int nk, nbk;
};
// Fill the per-k fields of a slot from H (not ubase, alpha, shift, beta).
void kslot(const sparc_ham* H, KSlot& s);
// Hash of the geometry the batched kernels take from the first Hamiltonian: equal
// hashes (with equal grids) mean one launch may serve several of them.
unsigned long long geometry_hash(const sparc_ham* H);

// Host: build the tables from the projector boxes (called by sparc_ham_create).
sparc_status build_tables(sparc_ham* H, const sparc_nonlocal* nl);
void free_tables(Tables& t);

// FP32 pass tile shapes: 0 = 16 x 16 nodes, 512 threads, one CTA per SM;
// 1 = 16 x 8 nodes, 256 threads, two CTAs per SM.
constexpr int NSHAPE_F32 = 2;
// launch_pass<float> shape for a plain H-apply: 16 x 16 tiles, stencil in difference form
constexpr int SHAPE_DIFF = 16;
bool shape_usable(const sparc_ham* H, int shape);
// Whether the tiled kernel handles this Hamiltonian (radius 6, FP32 element types).
bool usable(const sparc_ham* H);
// Work items (tile x z-chunk) of one block of orbitals for the element type T.
template <class T>
int items_per_block(const sparc_ham* H, int shape = 0);

// gc[p][blk][lane] for the blocks [blk0, blk0 + nb) (gamma_p h^3 chi~_p^H Y);
// `scratch` holds gather_scratch_bytes(H, nb, sizeof(T)) bytes of per-slab partial sums.
size_t gather_scratch_bytes(const sparc_ham* H, int nb, size_t esize);
template <class T>
cudaError_t launch_gather(const sparc_ham* H, const T* Y, int nblk_total, int blk0, int nb, T* gc,
                          T* scratch, cudaStream_t st);
// Yout = alpha (H - shift) Yin + beta Yprev for blocks [blk0, blk0 + nb).
template <class T>
cudaError_t launch_pass(const sparc_ham* H, const T* Yin, const T* Yprev, T* Yout, const T* gc,
                        int nblk_total, int blk0, int nb, double alpha, double shift, double beta,
                        cudaStream_t st, int shape = 0);

// Complex64, batched over k: the same two steps for the units of `ks`; `gc` and
// the block buffers hold nunit_total units ([unit][Nd][NB] and [p][unit][NB]);
// geometry and launch shape from H0.
cudaError_t launch_gather_k(const sparc_ham* H0, const cf32* Y, long long nunit_total, const KSlots& ks,
                            cf32* gc, cf32* scratch, cudaStream_t st);
cudaError_t launch_pass_k(const sparc_ham* H0, const cf32* Yin, const cf32* Yprev, cf32* Yout, const cf32* gc,
                          long long nunit_total, const KSlots& ks, cudaStream_t st);

}  // namespace fast
}  // namespace sparc
