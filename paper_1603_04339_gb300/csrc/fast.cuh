// Tables and launchers of the tiled FP32 / complex64 H-pass (hpass_fast.cu).
#pragma once

#include <array>
#include <vector>

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

// Tables of the TMA-fed passes (hpass_tma.cu): per tile column (16 x 16 (x, y) tile,
// all z) the projector slots that meet it, and per (tile, plane) a record of the A
// fragments of the projector term for each of the 16 warps of a CTA.  A slot is a
// projector group (atom box); for complex (k-point) Hamiltonians it is a group in one
// periodic image t = (tx, ty, tz) of the cell, so that its Bloch factor exp(-i k.(t L))
// is one constant that the kernel folds into the slot's coefficients.
constexpr int TMA_MAXG = 64;                 // projector slots per tile column, at most
constexpr unsigned TMA_REC_MAX = 36352;      // bytes of one plane's record, at most
constexpr int TMA_MAXTY = 16;                // tile rows (n2 <= 256)
constexpr int TMA_MAXSEG = 4;                // y segments of one halo frame
constexpr int TMA_NMAPS = 8;                 // distinct segment heights
constexpr unsigned TMA_REC_MAX_C = 30080;    // complex pass: bytes of one plane's record, at most
constexpr int TMA_MAXTILE_C = 256;           // complex pass: tile columns, at most
struct TmaTables {
  bool ok = false;            // built: the grid and projectors fit the kernel's limits
  bool cplx = false;          // slots split by periodic image (complex Hamiltonian)
  int zl = 0, nchunk = 0, tiles_x = 0, tiles_y = 0;   // zl = n3, nchunk = 1 (per launch: see the launcher)
  int max_rec = 0;
  // The halo frame of tile row ty, rows y = 16 ty - 6 .. 16 ty + 21 wrapped into [0, n2),
  // as up to TMA_MAXSEG runs of consecutive y: run j starts at y = yseg[ty][j][0], lands
  // at frame row yseg[ty][j][1] and has the height map_h[yseg[ty][j][2]] (-1: no run).
  int nmaps = 0;
  int map_h[TMA_NMAPS] = {};
  // work items of one block (FP32: one per tile) or unit (complex: tile | half << 16 |
  // dual mode << 17 per entry; full tiles twice, narrow tiles once as dual items)
  int nts = 0;
  int tsmap[2 * TMA_MAXTILE_C] = {};
  int yseg[TMA_MAXTY][TMA_MAXSEG][3] = {};
  int* d_cproj = nullptr;     // [tile][TMA_MAXG][4] projector index of (group slot, s/px/py/pz), -1 if none
  int* d_cng = nullptr;       // [tile] slots of the tile column
  int* d_cimg = nullptr;      // [tile][TMA_MAXG] image of the slot: (tx+1) | (ty+1) << 2 | (tz+1) << 4
  unsigned long long rec_hash = 0;   // hash of the record values (projector values at the nodes)
  int* d_rec = nullptr;       // [tile * n3 + z] record offsets in 16-byte units (+ one end entry)
  void* d_stream = nullptr;   // the records
  size_t stream_bytes = 0;
};

// The same tables on the host, before upload.
struct TmaHost {
  TmaTables dims;                 // zl, nchunk, tiles, max_rec (no device pointers)
  std::vector<int> cproj, cng, rec, cimg;
  std::vector<uint32_t> words;    // the records
};

struct Tables {
  TmaTables tma;              // folded slots: the FP32 pass (real Hamiltonians)
  TmaTables tmac;             // slots split by image: the complex64 pass
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
// Host: the TMA pass tables from the projector groups, their boxes (lo[3], n[3]) and
// box values chi4 ([box node][4]); leaves T->tma.ok false where the kernel does not apply.
sparc_status build_tma_tables(sparc_ham* H, Tables* T, const std::vector<Group>& grps,
                              const std::vector<std::array<int, 6>>& gbox, const std::vector<float>& chi4);
void free_tma_tables(TmaTables& M);
bool tma_frame_segments(int n2, TmaTables& M);
// images: one slot per (group, periodic image) instead of one per group.
bool tma_host_tables(const int n[3], const std::vector<Group>& grps, const std::vector<std::array<int, 6>>& gbox,
                     const std::vector<float>& chi4, TmaHost& out, bool images = false);
// Whether the TMA-fed FP32 pass applies to H (Gamma point, radius 6, n1 % 4 == 0,
// n1 >= 2R, the table limits).
bool tma_usable(const sparc_ham* H);
// Whether the TMA-fed complex64 pass applies to H (any k; as above, and every halo-frame
// row within one cell of the grid in y).
bool tma_usable_c(const sparc_ham* H);
// The TMA pass works on an x-padded block layout: every (y, z) row holds R ghost nodes
// on each side, copies of the other end of the row (periodic wrap):
//   B[blk][z][y][x'][NB], x' = x + R in [0, n1 + 2R); x' < R holds x = n1 - R + x',
//   x' >= n1 + R holds x = x' - n1 - R.
long long padded_nd(const sparc_ham* H);
cudaError_t launch_to_blocks_px(const sparc_ham* H, const float* X, long long ld, int ns, float* B, int nblk,
                                cudaStream_t st);
cudaError_t launch_from_blocks_px(const sparc_ham* H, const float* B, int nblk, float* X, long long ld, int ns,
                                  cudaStream_t st);
// Complex64: ghost nodes hold the Bloch image, x' < R: conj(ph_x) Y(x + n1), x' >= n1 + R:
// ph_x Y(x - n1), ph_x = exp(i k_x L_x).
cudaError_t launch_to_blocks_px(const sparc_ham* H, const cf32* X, long long ld, int ns, cf32* B, int nblk,
                                cudaStream_t st);
cudaError_t launch_from_blocks_px(const sparc_ham* H, const cf32* B, int nblk, cf32* X, long long ld, int ns,
                                  cudaStream_t st);
// The TMA-fed FP32 pass: Yout = alpha (H - shift) Yin + beta Yprev for blocks [blk0, blk0 + nb)
// of x-padded buffers (Yout's ghost nodes are written too).
cudaError_t launch_pass_tma(const sparc_ham* H, const float* Yin, const float* Yprev, float* Yout, const float* gc,
                            int nblk_total, int blk0, int nb, double alpha, double shift, double beta,
                            cudaStream_t st);
// Whether the complex TMA pass of H0 may serve H in one batched launch: the same grid,
// projector slots and record values (the per-k phases, V_eff and gamma may differ).
bool tma_batch_compatible(const sparc_ham* H0, const sparc_ham* H);
// Work items of one block (FP32) or unit (complex: two half-units) per z-chunk.
int tma_items_per_unit(const sparc_ham* H);

// FP32 pass tile shapes: 0 = 16 x 16 nodes, 512 threads, one CTA per SM;
// 1 = 16 x 8 nodes, 256 threads, two CTAs per SM; 2 = the TMA-fed pass (16 x 16
// tiles, z-chunks, one producer and 16 consumer warps), the default where it applies.
constexpr int NSHAPE_F32 = 3;
constexpr int SHAPE_TMA = 2;
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
// padded: Y is in the x-padded layout of the TMA passes.
template <class T>
cudaError_t launch_gather(const sparc_ham* H, const T* Y, int nblk_total, int blk0, int nb, T* gc,
                          T* scratch, cudaStream_t st, bool padded = false);
// Yout = alpha (H - shift) Yin + beta Yprev for blocks [blk0, blk0 + nb).
template <class T>
cudaError_t launch_pass(const sparc_ham* H, const T* Yin, const T* Yprev, T* Yout, const T* gc,
                        int nblk_total, int blk0, int nb, double alpha, double shift, double beta,
                        cudaStream_t st, int shape = 0);

// Complex64, batched over k: the same two steps for the units of `ks`; `gc` and
// the block buffers hold nunit_total units ([unit][Nd][NB] and [p][unit][NB]);
// geometry and launch shape from H0.
// nblk_k: blocks of one k in total (fixes the summation order); padded: Y in the x-padded
// layout of the TMA passes.
cudaError_t launch_gather_k(const sparc_ham* H0, const cf32* Y, long long nunit_total, const KSlots& ks, int nblk_k,
                            cf32* gc, cf32* scratch, cudaStream_t st, bool padded = false);
cudaError_t launch_pass_k(const sparc_ham* H0, const cf32* Yin, const cf32* Yprev, cf32* Yout, const cf32* gc,
                          long long nunit_total, const KSlots& ks, cudaStream_t st);
// The TMA-fed complex64 pass over the units of `ks` in x-padded buffers (hpass_tma.cu);
// every H of the batch passes tma_batch_compatible with H0.  Uses alpha, shift, beta,
// veff and the face phases of the slots.
cudaError_t launch_pass_tma_k(const sparc_ham* H0, const cf32* Yin, const cf32* Yprev, cf32* Yout, const cf32* gc,
                              long long nunit_total, const KSlots& ks, cudaStream_t st);

}  // namespace fast
}  // namespace sparc
