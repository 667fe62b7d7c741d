// FP32 H-pass of the Chebyshev filter, fed by the tensor memory accelerator (TMA).
//
// One launch applies one filter degree (the three-term recurrence of Eq. ChebFilter)
//     Yout = alpha (H - shift) Yin + beta Yprev
// to the blocks [blk0, blk0 + nb) of the interleaved layout B[blk][z][y][x'][8 orbitals],
// x-padded: each (y, z) row carries R ghost nodes at either end that repeat the other
// end of the row, so that an x-halo never wraps (the pass writes them with the row),
// with H = -1/2 lap_h (twelfth-order FD Laplacian, Eq. FD:Laplacian, weights
// Eq. weightsLap) + V_eff + the Kleinman-Bylander projector term of Eq. NonlocalPS:FD,
// at the Gamma point (real orbitals, periodic wrap).  Yprev may be null (first degree)
// or alias Yout (the recurrence runs in place).
//
// Work: persistent CTAs loop over items = (16 x 16 (x, y) tile, z-chunk of up to 32
// planes, block).  The item's planes z' = zs-6 .. ze+5 pass through a ring of three
// shared-memory stages:
//   * the last warp, before each of its steps, fills the stage two steps ahead (the
//     producer role): for a plane of the chunk, the tile with its 6-node halo (28 x 28
//     nodes: one cp.async.bulk.tensor box, split along y into up to three boxes where
//     the rows wrap around the periodic y faces; the x wrap is in the ghost nodes),
//     the tile's V_eff (tensor box), the projector
//     fragment record of the plane (bulk copy) and, for the output plane z'-6, the
//     tile's Yprev (tensor box); for the six planes on either side of the chunk only
//     the tile's own 16 x 16 nodes (tensor box).  Completion is counted in bytes on
//     the stage's "full" mbarrier; the consumers release a stage on its "empty" one.
//   * all 16 warps consume: each thread owns the nodes (x, y) and (x, y+1) of the tile
//     and one orbital pair (a float2).  The z part of the stencil is a scatter: plane
//     z' adds c_|d| f(z') to the accumulators of the outputs z'+d, d = -6..6, kept
//     in a ring of 13 registers that the unrolled step loop renames; the x and y
//     parts, (c_0 + V - shift) f and the projector term go to the output z' itself;
//     the output z'-6 is then complete and is written as alpha acc + beta Yprev.
//   * the projector term sum_p chi_p(node) gc_p(orbital) runs on mma.sync m16n8k8
//     TF32 products (3xTF32: about FP32 accuracy).  The host precomputes for every
//     warp and plane the A fragments (chi of two projector groups of one atom box
//     each at the warp's 16 nodes, zero outside the boxes), so the kernel does no
//     index or bounds arithmetic for them; B (gc = gamma h^3 chi^T Y, split into TF32
//     high and low parts) is staged in shared memory per item.
// Every mbarrier wait is bounded: one that runs out latches STATUS_TIMEOUT in the
// device status word and the kernel goes on, so it cannot hang.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "fast.cuh"
#include "ptx.cuh"

namespace sparc {
namespace fast {
namespace tma {

constexpr int MAXG = TMA_MAXG;
constexpr int TT = 16;                   // tile edge in x and y
constexpr int FR = TT + 2 * R;           // 28: tile plus halo
constexpr int ZLMAX = 128;               // output planes per z-chunk, at most
constexpr int NCW = 16;                  // warps; the last one also produces
constexpr int NTHR = NCW * 32;
constexpr uint32_t FRAME_B = FR * FR * NB * 4;   // 25088
constexpr uint32_t TILE_B = TT * TT * NB * 4;    // 8192
constexpr uint32_t V_B = TT * TT * 4;            // 1024
constexpr uint32_t GCS_B = (MAXG + 1) * 32 * 4;  // coefficients of one item (half): float[MAXG + 1][32]
constexpr uint32_t CPJ_B = MAXG * 4 * 4;         // projector indices of one item: int[MAXG][4]
constexpr int RECN = ZLMAX + 4;                  // record offsets of one item (nz + 1 used), 16-byte multiple

// Shared-memory layout of a CTA: a ring of NBUF stages, each a halo frame (or the tile of
// a boundary plane), the Yprev tile, V_eff and the plane's record; then per-item tables,
// filled ahead by cp.async: coefficients gc of the item's slots (two items), their
// projector indices (two items), record offsets (three items); then the mbarriers.
// FP32: three stages, the producer two steps ahead.  Complex: two stages, the producer one
// step ahead, each with room for both halves of a unit (the dual items of narrow tiles:
// frames, tiles and Yprev of half 1 after those of half 0; coefficients of both halves).
template <bool CX>
struct Lay {
  static constexpr int NBUF = CX ? 2 : 3;             // stages in the ring
  static constexpr int DIST = CX ? 1 : 2;             // steps the producer runs ahead (< NBUF)
  static constexpr int NH = CX ? 2 : 1;               // halves a stage holds
  static constexpr uint32_t REC = CX ? TMA_REC_MAX_C : TMA_REC_MAX;
  static constexpr uint32_t OFF_YP = NH * FRAME_B;
  static constexpr uint32_t OFF_V = OFF_YP + NH * TILE_B;
  static constexpr uint32_t OFF_REC = OFF_V + V_B;
  static constexpr uint32_t STAGE_B = OFF_REC + REC;
  static constexpr uint32_t OFF_GCS = NBUF * STAGE_B;
  static constexpr uint32_t GCS_ITEM = NH * GCS_B;
  static constexpr uint32_t OFF_CPJ = OFF_GCS + 2 * GCS_ITEM;
  static constexpr uint32_t OFF_RECS = OFF_CPJ + 2 * CPJ_B;
  static constexpr uint32_t OFF_BAR = OFF_RECS + 3 * RECN * 4;
  static constexpr uint32_t SMEM_B = OFF_BAR + 2 * NBUF * 8;
  static_assert(OFF_BAR % 8 == 0, "mbarrier alignment");
  static_assert(STAGE_B % 128 == 0 && OFF_REC % 128 == 0 && OFF_YP % 128 == 0 && FRAME_B % 128 == 0,
                "stage alignment");
  static_assert(SMEM_B <= 232448, "shared memory of one CTA");
};

// Node origin (xa, ya) of warp w's 8 x 2 nodes in a tile, and the half of the unit it
// computes in a dual item: mode 0, a full tile (2 x 8 warps); mode 1, a tile of at most 8
// valid columns (x-dual: even warps half 0, odd warps half 1, both at x 0..7); mode 2, a
// tile of more than 8 valid columns and at most 8 valid rows (y-dual: warps 0..7 half 0,
// warps 8..15 half 1, both at y 0..7).
__host__ __device__ __forceinline__ void warp_origin(int md, int w, int& xa, int& ya, int& wh) {
  if (md == 1) { xa = 0; ya = 2 * (w >> 1); wh = w & 1; }
  else if (md == 2) { xa = 8 * (w & 1); ya = 2 * ((w >> 1) & 3); wh = w >> 3; }
  else { xa = 8 * (w & 1); ya = 2 * (w >> 1); wh = 0; }
}

// --------------------------------------------------------------------------- host tables

static int cover(int c, int lo, int nb, int n) {   // box-local index of coordinate c, or -1
  int u = (c - lo) % n;
  if (u < 0) u += n;
  return u < nb ? u : -1;
}
// Box-local index of grid coordinate c in periodic image t (the box node lo + u lies at
// grid node lo + u - t n), or -1.
static int cover_img(int c, int t, int lo, int nb, int n) {
  const int u = c + t * n - lo;
  return (u >= 0 && u < nb) ? u : -1;
}
static int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

}  // namespace tma

// The tables on the host: false where the grid or the projectors exceed the kernel's
// limits (slots per CTA, record size, images beyond the neighbouring cells).
bool tma_host_tables(const int n[3], const std::vector<Group>& grps, const std::vector<std::array<int, 6>>& gbox,
                     const std::vector<float>& chi4, TmaHost& out, bool images) {
  using namespace tma;
  TmaTables& M = out.dims;
  std::vector<int>& cproj = out.cproj;
  std::vector<int>& cng = out.cng;
  std::vector<int>& rec = out.rec;
  std::vector<int>& cimg = out.cimg;
  std::vector<uint32_t>& words = out.words;
  const uint32_t rec_max = images ? TMA_REC_MAX_C : TMA_REC_MAX;
  // tables per tile column (all z); the z-chunking of the work is chosen per launch
  M.nchunk = 1;
  M.zl = n[2];
  M.tiles_x = ceil_div(n[0], TT);
  M.tiles_y = ceil_div(n[1], TT);
  const int ncta = M.tiles_x * M.tiles_y;
  const int ngrp = (int)grps.size();
  std::vector<long long> off4(ngrp);
  {
    long long o = 0;
    for (int g = 0; g < ngrp; ++g) {
      off4[g] = o;
      o += (long long)gbox[g][3] * gbox[g][4] * gbox[g][5];
    }
  }
  cproj.assign((size_t)ncta * MAXG * 4, -1);
  cimg.assign((size_t)ncta * MAXG, 1 | (1 << 2) | (1 << 4));   // image (0, 0, 0)
  cng.assign(ncta, 0);
  rec.assign((size_t)ncta * M.zl + 1, 0);
  words.clear();
  words.reserve(1 << 20);
  int max_rec = 0;
  for (int cta = 0; cta < ncta; ++cta) {
    const int tile = cta;
    const int x0 = (tile % M.tiles_x) * TT, y0 = (tile / M.tiles_x) * TT;
    const int zs = 0, nz = n[2];
    const int xe = std::min(n[0], x0 + TT), ye = std::min(n[1], y0 + TT);
    // complex tables: a narrow tile runs as dual items (both halves of a unit)
    const int md = !images ? 0 : (xe - x0 <= 8 ? 1 : (ye - y0 <= 8 ? 2 : 0));
    // the slots that meet the tile over the chunk's planes: the atom boxes (projector
    // groups), with images split (one slot per image whose nodes meet the tile)
    std::vector<int> loc, limg;
    std::vector<std::array<int, TT>> ux, uy;
    std::vector<std::vector<int>> uz;
    for (int G = 0; G < ngrp; ++G) {
      const int* lo = &gbox[G][0];
      const int* nb = &gbox[G][3];
      // candidate images per axis: all of them (folded, t = 0 stands for every image)
      // or each image of the unwrapped box [lo, lo + nb)
      int t0[3], t1[3];
      for (int ax = 0; ax < 3; ++ax) {
        t0[ax] = images ? floordiv(lo[ax], n[ax]) : 0;
        t1[ax] = images ? floordiv(lo[ax] + nb[ax] - 1, n[ax]) : 0;
        if (t0[ax] < -1 || t1[ax] > 1) return false;   // images beyond the neighbouring cells
      }
      auto cov = [&](int c, int t, int ax) {
        return images ? cover_img(c, t, lo[ax], nb[ax], n[ax]) : cover(c, lo[ax], nb[ax], n[ax]);
      };
      for (int tz = t0[2]; tz <= t1[2]; ++tz) {
        std::vector<int> cz(nz);
        bool hz = false;
        for (int k = 0; k < nz; ++k) {
          cz[k] = cov(zs + k, tz, 2);
          hz |= cz[k] >= 0;
        }
        if (!hz) continue;
        for (int ty = t0[1]; ty <= t1[1]; ++ty) {
          std::array<int, TT> cy;
          bool hy = false;
          for (int i = 0; i < TT; ++i) {
            cy[i] = (y0 + i < ye) ? cov(y0 + i, ty, 1) : -1;
            hy |= cy[i] >= 0;
          }
          if (!hy) continue;
          for (int tx = t0[0]; tx <= t1[0]; ++tx) {
            std::array<int, TT> cx;
            bool hx = false;
            for (int i = 0; i < TT; ++i) {
              cx[i] = (x0 + i < xe) ? cov(x0 + i, tx, 0) : -1;
              hx |= cx[i] >= 0;
            }
            if (!hx) continue;
            loc.push_back(G);
            limg.push_back((tx + 1) | ((ty + 1) << 2) | ((tz + 1) << 4));
            ux.push_back(cx);
            uy.push_back(cy);
            uz.push_back(cz);
          }
        }
      }
    }
    if ((int)loc.size() > MAXG) return false;   // too many slots per tile column: the other kernels run
    cng[cta] = (int)loc.size();
    for (size_t g = 0; g < loc.size(); ++g) {
      for (int l = 0; l < 4; ++l) cproj[((size_t)cta * MAXG + g) * 4 + l] = grps[loc[g]].proj[l];
      cimg[(size_t)cta * MAXG + g] = limg[g];
    }
    for (int k = 0; k < M.zl; ++k) {
      rec[(size_t)cta * M.zl + k] = (int)(words.size() / 4);
      if (k >= nz) continue;
      // per warp: the local boxes active at its 16 nodes, in pairs (one mma round each)
      std::vector<int> hdr(32, 0), ids;
      std::vector<std::vector<int>> act(NCW);
      for (int w = 0; w < NCW; ++w) {
        int xa, ya, wh;
        warp_origin(md, w, xa, ya, wh);
        for (size_t g = 0; g < loc.size(); ++g) {
          if (uz[g][k] < 0) continue;
          if (uy[g][ya] < 0 && uy[g][ya + 1] < 0) continue;
          bool hx = false;
          for (int i = 0; i < 8; ++i) hx |= ux[g][xa + i] >= 0;
          if (hx) act[w].push_back((int)g);
        }
        hdr[w] = (int)ids.size();
        for (size_t j = 0; j < act[w].size(); j += 2) {
          const int g0 = act[w][j], g1 = (j + 1 < act[w].size()) ? act[w][j + 1] : MAXG;
          ids.push_back(g0 | (g1 << 16));
        }
      }
      const int nr = (int)ids.size();
      hdr[NCW] = nr;
      const int nid = (nr + 3) & ~3;
      const int bytes = 128 + 4 * nid + 512 * nr;
      max_rec = std::max(max_rec, bytes);
      if (bytes > (int)rec_max) return false;   // record too large for a stage
      for (int v : hdr) words.push_back((uint32_t)v);
      for (int j = 0; j < nid; ++j) words.push_back(j < nr ? (uint32_t)ids[j] : 0u);
      for (int w = 0; w < NCW; ++w) {
        int xa, ya, wh;
        warp_origin(md, w, xa, ya, wh);
        for (size_t j = 0; j < act[w].size(); j += 2) {
          const int gg[2] = {act[w][j], (j + 1 < act[w].size()) ? act[w][j + 1] : -1};
          for (int lane = 0; lane < 32; ++lane) {
            const int gq = lane >> 2, cq = lane & 3;
            float v[4] = {0.f, 0.f, 0.f, 0.f};   // (g0, node A), (g0, node B), (g1, A), (g1, B)
            for (int h = 0; h < 2; ++h) {
              const int g = gg[h];
              if (g < 0) continue;
              const int G = loc[g];
              const int bx = ux[g][xa + gq];
              const int bz = uz[g][k];
              for (int r = 0; r < 2; ++r) {
                const int by = uy[g][ya + r];
                if (bx < 0 || by < 0 || bz < 0) continue;
                const long long e = off4[G] + bx + (long long)gbox[G][3] * (by + (long long)gbox[G][4] * bz);
                v[2 * h + r] = chi4[(size_t)e * 4 + cq];
              }
            }
            for (int c = 0; c < 4; ++c) {
              uint32_t u;
              std::memcpy(&u, &v[c], 4);
              words.push_back(u);
            }
          }
        }
      }
    }
  }
  rec[(size_t)ncta * M.zl] = (int)(words.size() / 4);
  if (words.size() / 4 >= (size_t)INT32_MAX) return false;
  M.max_rec = max_rec;
  // the work items of one unit: (tile, half) for full tiles, (tile, dual mode) for narrow
  // ones (complex tables); one per tile for the FP32 tables
  M.nts = 0;
  if (images) {
    if (ncta > TMA_MAXTILE_C) return false;
    for (int t = 0; t < ncta; ++t) {
      const int x0 = (t % M.tiles_x) * TT, y0 = (t / M.tiles_x) * TT;
      const int md = n[0] - x0 <= 8 ? 1 : (n[1] - y0 <= 8 ? 2 : 0);
      if (md == 0) {
        M.tsmap[M.nts++] = t;
        M.tsmap[M.nts++] = t | (1 << 16);
      } else {
        M.tsmap[M.nts++] = t | (md << 17);
      }
    }
  } else {
    M.nts = ncta;
  }
  return true;
}

// The y runs of every tile row's halo frame and the distinct run heights (one tensor
// map each); false if the grid needs more than the kernel's limits.
bool tma_frame_segments(int n2, TmaTables& M) {
  using namespace tma;
  if (M.tiles_y > TMA_MAXTY) return false;
  M.nmaps = 0;
  for (int ty = 0; ty < M.tiles_y; ++ty) {
    for (int j = 0; j < TMA_MAXSEG; ++j) M.yseg[ty][j][0] = M.yseg[ty][j][1] = M.yseg[ty][j][2] = -1;
    int r = 0, j = 0;
    while (r < FR) {
      if (j == TMA_MAXSEG) return false;
      int y = (ty * TT - R + r) % n2;
      if (y < 0) y += n2;
      const int hgt = std::min(FR - r, n2 - y);
      int mi = 0;
      while (mi < M.nmaps && M.map_h[mi] != hgt) ++mi;
      if (mi == M.nmaps) {
        if (M.nmaps == TMA_NMAPS) return false;
        M.map_h[M.nmaps++] = hgt;
      }
      M.yseg[ty][j][0] = y;
      M.yseg[ty][j][1] = r;
      M.yseg[ty][j][2] = mi;
      r += hgt;
      ++j;
    }
  }
  return true;
}

// One table set: folded slots (images = false, the FP32 pass at the Gamma point) or
// slots split by periodic image (the complex pass); M.ok stays false where the grid or
// the projectors exceed the kernel's limits.
static sparc_status build_tma_set(sparc_ham* H, TmaTables& M, const std::vector<Group>& grps,
                                  const std::vector<std::array<int, 6>>& gbox, const std::vector<float>& chi4,
                                  bool images) {
  using namespace tma;
  M = TmaTables();
  const int n[3] = {H->gd.n1, H->gd.n2, H->gd.n3};
  // not this kernel's case: another radius; V_eff rows not 16-byte multiples; rows
  // shorter than their two ghost runs; planes that a z-chunk's halo would wrap twice
  if (H->gd.no != R || n[0] % 4 != 0 || n[0] < 2 * R || n[2] <= R) return SPARC_OK;
  if (images) {
    // the complex pass applies one Bloch factor per halo-frame row: every frame row
    // y = 16 ty - 6 .. 16 ty + 21 lies within one cell of [0, n2)
    if (n[1] <= R) return SPARC_OK;
    for (int y0 = 0; y0 < n[1]; y0 += TT)
      if (y0 + TT + R - 1 >= 2 * n[1]) return SPARC_OK;
  }
  TmaHost h;
  if (!tma_host_tables(n, grps, gbox, chi4, h, images)) return SPARC_OK;
  if (!tma_frame_segments(n[1], h.dims)) return SPARC_OK;
  M = h.dims;
  M.cplx = images;
  const std::vector<int>& cproj = h.cproj;
  const std::vector<int>& cng = h.cng;
  const std::vector<int>& rec = h.rec;
  const std::vector<int>& cimg = h.cimg;
  const std::vector<uint32_t>& words = h.words;
  {
    // FNV-1a over everything a launch takes from the tables (the batched complex pass
    // serves several Hamiltonians with the tables of one)
    unsigned long long hsh = 1469598103934665603ULL;
    auto mix = [&](const void* p, size_t bytes) {
      const unsigned char* c = (const unsigned char*)p;
      for (size_t i = 0; i < bytes; ++i) { hsh ^= c[i]; hsh *= 1099511628211ULL; }
    };
    mix(n, sizeof(int) * 3);
    mix(cproj.data(), cproj.size() * sizeof(int));
    mix(cimg.data(), cimg.size() * sizeof(int));
    mix(cng.data(), cng.size() * sizeof(int));
    mix(rec.data(), rec.size() * sizeof(int));
    mix(words.data(), words.size() * sizeof(uint32_t));
    M.rec_hash = hsh;
  }
  auto up = [&](void** d, const void* h, size_t bytes) -> bool {
    if (cudaMalloc(d, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    return bytes == 0 || cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up((void**)&M.d_cproj, cproj.data(), cproj.size() * sizeof(int)) ||
      !up((void**)&M.d_cimg, cimg.data(), cimg.size() * sizeof(int)) ||
      !up((void**)&M.d_cng, cng.data(), cng.size() * sizeof(int)) ||
      !up((void**)&M.d_rec, rec.data(), rec.size() * sizeof(int)) ||
      !up(&M.d_stream, words.data(), words.size() * sizeof(uint32_t))) {
    cudaGetLastError();
    free_tma_tables(M);
    return fail(H->ctx, SPARC_ERR_OOM, "TMA pass table allocation failed");
  }
  M.stream_bytes = words.size() * sizeof(uint32_t);
  M.ok = true;
  return SPARC_OK;
}

// A real Hamiltonian gets both sets (FP32 filters take the folded one; complex64 filters
// the split one, which a k-point batch shares with the complex Hamiltonians); a complex
// one the split set only.
sparc_status build_tma_tables(sparc_ham* H, Tables* T, const std::vector<Group>& grps,
                              const std::vector<std::array<int, 6>>& gbox, const std::vector<float>& chi4) {
  T->tma = TmaTables();
  if (!H->gd.cplx) {
    const sparc_status s = build_tma_set(H, T->tma, grps, gbox, chi4, false);
    if (s != SPARC_OK) return s;
  }
  return build_tma_set(H, T->tmac, grps, gbox, chi4, true);
}

void free_tma_tables(TmaTables& M) {
  void* ps[] = {M.d_cproj, M.d_cimg, M.d_cng, M.d_rec, M.d_stream};
  for (void* p : ps)
    if (p) cudaFree(p);
  M = TmaTables();
}

bool tma_usable(const sparc_ham* H) {
  const Tables* T = (const Tables*)H->fast;
  return T != nullptr && T->tma.ok && usable(H);
}

bool tma_usable_c(const sparc_ham* H) {
  const Tables* T = (const Tables*)H->fast;
  return T != nullptr && T->tmac.ok && usable(H);
}

int tma_items_per_unit(const sparc_ham* H) { return ((const Tables*)H->fast)->tmac.nts; }

bool tma_batch_compatible(const sparc_ham* H0, const sparc_ham* H) {
  if (!tma_usable_c(H0) || !tma_usable_c(H)) return false;
  const TmaTables& A = ((const Tables*)H0->fast)->tmac;
  const TmaTables& B = ((const Tables*)H->fast)->tmac;
  return A.rec_hash == B.rec_hash && A.stream_bytes == B.stream_bytes && H0->gd.n1 == H->gd.n1 &&
         H0->gd.n2 == H->gd.n2 && H0->gd.n3 == H->gd.n3;
}

namespace tma {

// --------------------------------------------------------------------------- device code

struct Args {
  int n1, n2, n3, tiles_x, ntiles, nchunk, zl;
  int n1p;                   // padded row length n1 + 2R
  int blk0, nblk_total, nitems;
  long long ndp;             // nodes per block of the padded layout
  int yseg[TMA_MAXTY][TMA_MAXSEG][3];   // y runs of the halo frames (src y, frame row, map)
  float2 cx2[R + 1], cy2[R + 1], cz2[R + 1];
  float c0s;                 // sum of the centre coefficients minus the shift
  float2 alpha2, beta2;
  const float* yin;
  const float* yprev;        // null on the first degree
  float* yout;
  const float* gc;           // [p][blk][NB]
  const int* cproj;          // [tile][MAXG][4]
  const int* cng;            // [tile]
  const int* rec;            // [tile * n3 + z] record offsets, 16-byte units
  const unsigned char* stream;
  const int* cimg;           // [tile][MAXG] slot images (complex pass)
  int* status;
  long long wait_limit;      // SM clocks of a bounded wait
  int stall;                 // failure injection: the producer stops at this step (-1: off)
};

__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
          "r"(ptx::saddr(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(ptx::saddr(bar))
      : "memory");
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* m, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(ptx::saddr(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(ptx::saddr(bar))
      : "memory");
}
// L2 cache policies: evict_last for data every block re-reads (the projector records),
// evict_first for data read once (Yprev).
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          ptx::saddr(dst)),
      "l"(src), "r"(bytes), "r"(ptx::saddr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma4_hint(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, uint64_t* bar,
                                          uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::
          "r"(ptx::saddr(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(ptx::saddr(bar)), "l"(pol)
      : "memory");
}

// The tensor maps of a launch: halo-frame runs of each height, the tile of Yin and of
// Yprev (16 x 16 nodes, padded layout) and V_eff (one per k of a complex launch).
template <bool CX>
struct MapsT {
  CUtensorMap frame[TMA_NMAPS];
  CUtensorMap tile_in, tile_prev;
  CUtensorMap veff[CX ? KMAX : 1];
};

// Per-k fields of a complex launch: it covers the units ubase[kk] + j, j < nbk, kk < nk,
// each as two halves of four complex orbitals (items are half-units).
struct KArgs {
  int nk, nbk;
  int nts;                          // work items of one unit per z-chunk
  int tsmap[2 * TMA_MAXTILE_C];     // tile | half << 16 | dual mode << 17 of each
  long long ubase[KMAX];
  float2 alpha2[KMAX], beta2[KMAX];
  float c0s[KMAX];
  float2 phx[KMAX], phy[KMAX], phz[KMAX];   // exp(i k_s L_s)
};
struct KArgsNone {
  int unused;
};
template <bool CX>
using KArgsT = typename std::conditional<CX, KArgs, KArgsNone>::type;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
// ph^t for t in {-1, 0, 1}
__device__ __forceinline__ float2 face(float2 ph, int t) {
  return t == 0 ? make_float2(1.f, 0.f) : (t > 0 ? ph : conj2(ph));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::saddr(b)) : "memory");
}


__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(float (&d)[4], float a0, float a1, float a2, float a3, float b0, float b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(__float_as_uint(a0)), "r"(__float_as_uint(a1)), "r"(__float_as_uint(a2)), "r"(__float_as_uint(a3)),
        "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}

// A work item: tile column, z-chunk and block (FP32) or unit part (complex: half h of
// unit blk, or both halves for a dual item of mode md > 0; kk the k slot).
struct Item {
  int tile, chunk, tx0, ty0, zs, nz;
  int blk, h, md, kk;
};
template <bool CX>
__device__ __forceinline__ Item decode(const Args& a, const KArgsT<CX>& ka, int item) {
  Item it;
  int u;
  if constexpr (CX) {
    const int e = ka.tsmap[item % ka.nts];
    const int rest = item / ka.nts;
    it.chunk = rest % a.nchunk;
    u = rest / a.nchunk;
    it.tile = e & 0xFFFF;
    it.h = (e >> 16) & 1;
    it.md = e >> 17;
    it.kk = u / ka.nbk;
    it.blk = (int)(ka.ubase[it.kk] + u % ka.nbk);
  } else {
    it.tile = item % a.ntiles;
    const int rest = item / a.ntiles;
    it.chunk = rest % a.nchunk;
    u = rest / a.nchunk;
    it.h = 0;
    it.md = 0;
    it.kk = 0;
    it.blk = a.blk0 + u;
  }
  it.tx0 = (it.tile % a.tiles_x) * TT;
  it.ty0 = (it.tile / a.tiles_x) * TT;
  it.zs = it.chunk * a.zl;
  it.nz = min(a.zl, a.n3 - it.zs);
  return it;
}

// The producer role: fill the stage of step (item, s) of this CTA (all 32 lanes of the
// last warp call it).  recs: the record offsets of the item's planes (16-byte units,
// entries 0 .. nz).  Returns false if the wait for the stage to be free ran out; once
// a wait has run out (wait == false) no further waits are made, so that a broken
// pipeline ends the kernel quickly instead of timing out at every step.  A dual item
// loads the frames (tiles) and Yprev tiles of both halves.
template <bool CX>
__device__ __forceinline__ bool produce(const Args& a, const MapsT<CX>& mp, unsigned char* smem, uint64_t* bars,
                                       const Item& it, int s, int g, const int* recs, bool wait) {
  using L = Lay<CX>;
  const int lane = threadIdx.x & 31;
  const int blk = it.blk;
  const int c0 = CX ? 8 * it.h : 0;   // first float of the node's half (complex: 16 floats a node)
  const int nh = (CX && it.md) ? 2 : 1;
  const int slot = g % L::NBUF;
  unsigned char* st = smem + (size_t)slot * L::STAGE_B;
  uint64_t* full = bars + slot;
  uint64_t* empty = bars + L::NBUF + slot;
  bool ok = true;
  if (a.stall >= 0 && g >= a.stall) return true;   // injected stall: from this step of the CTA on, nothing is issued
  if (wait && g >= L::NBUF && !ptx::mbar_wait_lim(empty, (uint32_t)((g / L::NBUF) - 1) & 1u, a.wait_limit)) ok = false;
  const int p = it.zs - R + s;
  int zw = p;
  if (zw < 0) zw += a.n3;
  else if (zw >= a.n3) zw -= a.n3;
  const bool comp = s >= R && s < R + it.nz;
  const bool yp = a.yprev != nullptr && s >= 2 * R;
  const int k = comp ? s - R : 0;
  const int o0 = recs[k];
  const uint32_t rbytes = comp ? 16u * (uint32_t)(recs[k + 1] - o0) : 0u;
  const uint32_t bytes = (comp ? nh * FRAME_B + V_B + rbytes : nh * TILE_B) + (yp ? nh * TILE_B : 0u);
  if (lane == 0) ptx::mbar_arrive_expect_tx(full, bytes);
  __syncwarp();
  const int zc = blk * a.n3 + zw;
  if (comp) {
    // halo frame: padded columns tx0 .. tx0+27 (nodes x = tx0-6 .. tx0+21), one box per y
    // run; lanes 4 .. 7 the frame of half 1 of a dual item
    if (lane < TMA_MAXSEG * nh) {
      const int hh = lane / TMA_MAXSEG;
      const int* sg = a.yseg[it.ty0 / TT][lane % TMA_MAXSEG];
      if (sg[2] >= 0)
        tma4(st + hh * FRAME_B + (size_t)sg[1] * FR * NB * 4, &mp.frame[sg[2]], c0 + 8 * hh, it.tx0, sg[0], zc,
             full);
    }
    if (lane == 29) tma3(st + L::OFF_V, &mp.veff[CX ? it.kk : 0], it.tx0, it.ty0, zw, full);
    if (lane == 30) bulk_g2s_hint(st + L::OFF_REC, a.stream + 16 * (size_t)o0, rbytes, full, policy_evict_last());
  } else if (lane < nh) {
    tma4(st + lane * FRAME_B, &mp.tile_in, c0 + 8 * lane, it.tx0 + R, it.ty0, zc, full);
  }
  if (yp && lane >= 32 - nh) {
    const int hh = 31 - lane;
    tma4_hint(st + L::OFF_YP + hh * TILE_B, &mp.tile_prev, c0 + 8 * hh, it.tx0 + R, it.ty0, blk * a.n3 + (p - R), full,
              policy_evict_first());
  }
  return ok;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  // 4-byte asynchronous copy; an invalid source copies nothing and zero-fills dst
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(ptx::saddr(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asynchronous per-item staging by all threads: the record offsets (entries 0 .. nz) and
// the projector indices of an item (tile column), or its coefficients gc (projector
// indices read from cpj, zero for absent projectors).
template <bool CX>
__device__ __forceinline__ void stage_recs(const Args& a, const KArgsT<CX>& ka, int item, int* dst) {
  const int t = threadIdx.x;
  if (item < a.nitems && t <= ZLMAX) {
    const Item it = decode<CX>(a, ka, item);
    if (t <= it.nz) cp_async4(dst + t, a.rec + (size_t)it.tile * a.n3 + it.zs + t, true);
  }
}
template <bool CX>
__device__ __forceinline__ void stage_cproj(const Args& a, const KArgsT<CX>& ka, int item, int* dst) {
  if (item >= a.nitems) return;
  const Item it = decode<CX>(a, ka, item);
  for (int i = threadIdx.x; i < MAXG * 4; i += NTHR) cp_async4(dst + i, a.cproj + (size_t)it.tile * MAXG * 4 + i, true);
}
// Complex: B column n = lane >> 2 of a slot is component n & 1 (re, im) of orbital
// 4 h + (n >> 1); a dual item stages both halves (half 1 GCS_B bytes after half 0); the
// Bloch factor of the slot is applied after the copies landed (phase_gc).
template <bool CX>
__device__ __forceinline__ void stage_gc(const Args& a, const KArgsT<CX>& ka, int item, const int* cpj, float* dst) {
  if (item >= a.nitems) return;
  const Item it = decode<CX>(a, ka, item);
  const int nh = (CX && it.md) ? 2 : 1;
  for (int idx = threadIdx.x; idx < nh * MAXG * 32; idx += NTHR) {
    const int hl = idx / (MAXG * 32), i = idx - hl * (MAXG * 32);
    const int l = i & 31;
    const int pp = cpj[(i >> 5) * 4 + (l & 3)];
    const size_t row = ((size_t)(pp < 0 ? 0 : pp) * a.nblk_total + it.blk) * NB;
    const float* src =
        CX ? a.gc + (row + 4 * (it.h + hl) + (l >> 3)) * 2 + ((l >> 2) & 1) : a.gc + row + (l >> 2);
    cp_async4(dst + hl * (GCS_B / 4) + i, src, pp >= 0);
  }
}

// The Bloch factors of an item's slots, folded into its staged coefficients: slot g in
// periodic image t gets exp(-i k.(t L)) = prod_s ph_s^(-t_s) (the factor of the image's
// projector values at the grid nodes, Eq. NonlocalPS:FD); (re, im) of (slot, orbital c,
// projector k) sit at lanes 8 c + k and 8 c + 4 + k; both halves of a dual item.
__device__ __forceinline__ void phase_gc(const Args& a, const KArgs& ka, const Item& it, float* gcs) {
  const float2 px = ka.phx[it.kk], py = ka.phy[it.kk], pz = ka.phz[it.kk];
  const int nh = it.md ? 2 : 1;
  for (int q = threadIdx.x; q < nh * MAXG * 16; q += NTHR) {
    const int hl = q / (MAXG * 16), r = q - hl * (MAXG * 16);
    const int g = r >> 4, c = (r >> 2) & 3, k = r & 3;
    const int code = __ldg(a.cimg + (size_t)it.tile * MAXG + g);
    const float2 ph = cmul(cmul(face(px, 1 - (code & 3)), face(py, 1 - ((code >> 2) & 3))), face(pz, 1 - (code >> 4)));
    float* v = gcs + hl * (GCS_B / 4) + g * 32 + 8 * c + k;
    const float re = v[0], im = v[4];
    v[0] = ph.x * re - ph.y * im;
    v[4] = ph.x * im + ph.y * re;
  }
}

// Ring position I of a step of plane z': the output z' gets d (its x/y/centre/projector
// part); plane z' feeds c_|d| f to the outputs z' + d, d = -6..6 (slot (I + 7 + d) mod 13;
// the output z'+6 opens in slot I); e receives the completed output z'-6 (slot I + 1).
template <int I>
__device__ __forceinline__ void zstep(float2 (&acc)[13][2], const float2* cz2, float2 f0, float2 f1, float2 d0,
                                      float2 d1, float2& e0, float2& e1) {
  acc[(I + 7) % 13][0] = __fadd2_rn(acc[(I + 7) % 13][0], d0);
  acc[(I + 7) % 13][1] = __fadd2_rn(acc[(I + 7) % 13][1], d1);
#pragma unroll
  for (int d = 1; d < R; ++d) {
    acc[(I + 7 + d) % 13][0] = __ffma2_rn(cz2[d], f0, acc[(I + 7 + d) % 13][0]);
    acc[(I + 7 + d) % 13][1] = __ffma2_rn(cz2[d], f1, acc[(I + 7 + d) % 13][1]);
  }
  acc[I][0] = __fmul2_rn(cz2[R], f0);
  acc[I][1] = __fmul2_rn(cz2[R], f1);
#pragma unroll
  for (int d = 1; d <= R; ++d) {
    acc[(I + 7 - d) % 13][0] = __ffma2_rn(cz2[d], f0, acc[(I + 7 - d) % 13][0]);
    acc[(I + 7 - d) % 13][1] = __ffma2_rn(cz2[d], f1, acc[(I + 7 - d) % 13][1]);
  }
  e0 = acc[(I + 1) % 13][0];
  e1 = acc[(I + 1) % 13][1];
}

// CX: complex64 units (16 floats a node), taken as half-units of four complex orbitals
// (one float2 each), so that the frames, stencil and projector products are those of the
// FP32 pass; the Bloch factors enter at the periodic faces (Section 3.1): x in the ghost
// nodes the epilogue writes, y on the frame rows that crossed a face, z on the halo planes
// that crossed one, and in the projector slots' coefficients (phase_gc).
template <bool CX>
__global__ void __launch_bounds__(NTHR, 1)
k_pass_tma(const __grid_constant__ MapsT<CX> mp, const __grid_constant__ Args a,
           const __grid_constant__ KArgsT<CX> ka) {
  using L = Lay<CX>;
  constexpr int NF = CX ? 2 * NB : NB;   // floats per node of the block buffers
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < L::NBUF; ++b) {
      ptx::mbar_init(bars + b, 1);
      ptx::mbar_init(bars + L::NBUF + b, NCW);
    }
    ptx::mbar_init_fence();
  }
  int* recs = reinterpret_cast<int*>(smem + L::OFF_RECS);
  int* cpj = reinterpret_cast<int*>(smem + L::OFF_CPJ);
  float* gcsb = reinterpret_cast<float*>(smem + L::OFF_GCS);
  // tables of the first two items (record offsets, projector indices), then the
  // coefficients of the first item; the zero slot MAXG of every coefficient buffer
  stage_recs<CX>(a, ka, blockIdx.x, recs);
  stage_recs<CX>(a, ka, blockIdx.x + gridDim.x, recs + RECN);
  stage_cproj<CX>(a, ka, blockIdx.x, cpj);
  stage_cproj<CX>(a, ka, blockIdx.x + gridDim.x, cpj + MAXG * 4);
  if (tid < 64 * L::NH) gcsb[(tid >> 5) * (GCS_B / 4) + MAXG * 32 + (tid & 31)] = 0.f;
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  stage_gc<CX>(a, ka, blockIdx.x, cpj, gcsb);
  cp_async_commit();
  __syncthreads();
  const bool producer = warp == NCW - 1;
  bool ok = true;
  // producer cursor: the step DIST ahead of the consumers (item, step, steps of the item, local item index)
  // (complex: the item decoded once per item, its per-k fields coming from the parameter
  // space; FP32: decoded at every step, a few integer operations)
  int pitem = blockIdx.x, ps = 0, pli = 0;
  Item pit;
  if constexpr (CX) pit = decode<CX>(a, ka, pitem < a.nitems ? pitem : 0);
  int pS = pitem < a.nitems ? decode<CX>(a, ka, pitem).nz + 2 * R : 0;
  auto produce_next = [&](int gp) {
    if (pitem >= a.nitems) return;
    if constexpr (CX) ok &= produce<CX>(a, mp, smem, bars, pit, ps, gp, recs + (pli % 3) * RECN, ok);
    else ok &= produce<CX>(a, mp, smem, bars, decode<CX>(a, ka, pitem), ps, gp, recs + (pli % 3) * RECN, ok);
    if (++ps == pS) {
      ps = 0;
      ++pli;
      pitem += gridDim.x;
      if (pitem < a.nitems) {
        if constexpr (CX) pit = decode<CX>(a, ka, pitem);
      }
      pS = pitem < a.nitems ? (CX ? pit.nz : decode<CX>(a, ka, pitem).nz) + 2 * R : 0;
    }
  };
  if (producer)
    for (int gp = 0; gp < L::DIST; ++gp) produce_next(gp);

  // ---- every warp consumes
  const int gq = lane >> 2, op = lane & 3;
  const size_t plane = (size_t)a.n1p * a.n2 * NF;   // one z-plane of a padded block
  int g = 0, li = 0;
  int cslot = 0;          // g mod NBUF
  uint32_t cphase = 0;    // parity of (g / NBUF)
  float2 acc[13][2];
#pragma unroll
  for (int i = 0; i < 13; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x, ++li) {
    const Item it = decode<CX>(a, ka, item);
    const int blk = it.blk;
    // The item's coefficients (gc of its boxes, B-fragment order: lane = 4 orbital +
    // projector; slot MAXG is zero) were copied at the previous item's start.  Wait for
    // this thread's copies, then let every warp finish the previous item; then start the
    // copies of the next item's coefficients and of the tables of the item after it, into
    // the buffers the previous item has left.
    cp_async_wait_all();
    __syncthreads();
    if constexpr (CX) {
      phase_gc(a, ka, it, gcsb + (li & 1) * (L::GCS_ITEM / 4));
      __syncthreads();
    }
    stage_gc<CX>(a, ka, item + gridDim.x, cpj + ((li + 1) & 1) * MAXG * 4, gcsb + ((li + 1) & 1) * (L::GCS_ITEM / 4));
    stage_cproj<CX>(a, ka, item + 2 * gridDim.x, cpj + (li & 1) * MAXG * 4);
    stage_recs<CX>(a, ka, item + 2 * gridDim.x, recs + ((li + 2) % 3) * RECN);
    cp_async_commit();
    // this warp's nodes (x, y), (x, y + 1) with x = tx0 + xl + gq, y = ty0 + yl, and the
    // half it computes (a dual item's warps split between the halves)
    int xl, yl, wh;
    warp_origin(CX ? it.md : 0, warp, xl, yl, wh);
    xl += gq;
    const int fo = wh * (FRAME_B / 4) + ((yl + R) * FR + xl + R) * NB + 2 * op;   // frame offset of node 0 (floats)
    const int to = wh * (FRAME_B / 4) + (yl * TT + xl) * NB + 2 * op;             // tile offset of node 0
    const int tp = wh * (TILE_B / 4) + (yl * TT + xl) * NB + 2 * op;              // Yprev tile offset of node 0
    const int vo = yl * TT + xl;
    const float* gcs = gcsb + (li & 1) * (L::GCS_ITEM / 4) + wh * (GCS_B / 4);
    const int gx = it.tx0 + xl, gy = it.ty0 + yl;
    const bool v0 = gx < a.n1 && gy < a.n2, v1 = gx < a.n1 && gy + 1 < a.n2;
    float* outp =
        a.yout + ((size_t)blk * a.ndp + (size_t)gy * a.n1p + gx + R) * NF + (CX ? 8 * (it.h + wh) : 0) + 2 * op;
    // ghost copies: nodes x < R repeat at x' = x + n1 + R, nodes x >= n1 - R at x' = x - n1 + R
    const long long gofs = gx < R ? (long long)a.n1 * NF : (gx >= a.n1 - R ? -(long long)a.n1 * NF : 0);
    // recurrence coefficients; complex: per k, with the Bloch factors of the faces
    float2 alpha2, beta2, gph = make_float2(1.f, 0.f), phy = make_float2(1.f, 0.f);
    float c0s;
    int nlo = 0, rhi = 2 * R + 2;   // column entries r < nlo lie below y = 0, r >= rhi at y >= n2
    if constexpr (CX) {
      alpha2 = ka.alpha2[it.kk];
      beta2 = ka.beta2[it.kk];
      c0s = ka.c0s[it.kk];
      const float2 px = ka.phx[it.kk];
      gph = gx < R ? px : conj2(px);   // the ghost of x < R lies at x + n1: ph_x; of x >= n1 - R at x - n1
      phy = ka.phy[it.kk];
      const int yb = it.ty0 + yl - R;   // y of column entry 0
      nlo = max(0, -yb);
      rhi = min(2 * R + 2, a.n2 - yb);
    } else {
      alpha2 = a.alpha2;
      beta2 = a.beta2;
      c0s = a.c0s;
    }
    const int S = it.nz + 2 * R;
    int ring = 0;   // s mod 13: the accumulator of output z'+d sits in slot (ring + 7 + d) mod 13
    for (int s = 0; s < S; ++s) {
      if (producer) produce_next(g + L::DIST);
      const int slot = cslot;
      const unsigned char* st = smem + (size_t)slot * L::STAGE_B;
      if (ok && !ptx::mbar_test(bars + slot, cphase) && !ptx::mbar_wait_lim(bars + slot, cphase, a.wait_limit))
        ok = false;
      const float* F = reinterpret_cast<const float*>(st);
      const bool comp = s >= R && s < R + it.nz;
      float2 f0, f1, d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);
      if (comp) {
        // y column of rows yl-6 .. yl+7 at the thread's x; rows 6 and 7 are its nodes
        float2 col[2 * R + 2];
#pragma unroll
        for (int r = 0; r < 2 * R + 2; ++r) col[r] = lds2(F + fo + (r - R) * FR * NB);
        if constexpr (CX) {
          // rows of the frame that crossed a y face: the image's value times ph_y^t
          if (nlo > 0 || rhi < 2 * R + 2) {
#pragma unroll
            for (int r = 0; r < 2 * R + 2; ++r) {
              if (r == R || r == R + 1) continue;   // the thread's own nodes never cross
              if (r < nlo) col[r] = cmul(col[r], conj2(phy));
              else if (r >= rhi) col[r] = cmul(col[r], phy);
            }
          }
        }
        f0 = col[R];
        f1 = col[R + 1];
        float2 ys0 = __fmul2_rn(a.cy2[1], __fadd2_rn(col[R + 1], col[R - 1]));
        float2 ys1 = __fmul2_rn(a.cy2[1], __fadd2_rn(col[R + 2], col[R]));
#pragma unroll
        for (int q = 2; q <= R; ++q) {
          ys0 = __ffma2_rn(a.cy2[q], __fadd2_rn(col[R + q], col[R - q]), ys0);
          ys1 = __ffma2_rn(a.cy2[q], __fadd2_rn(col[R + 1 + q], col[R + 1 - q]), ys1);
        }
        float2 xs0, xs1;
        {
          float2 w[2 * R + 1];
#pragma unroll
          for (int q = 0; q <= 2 * R; ++q) w[q] = (q == R) ? f0 : lds2(F + fo + (q - R) * NB);
          xs0 = __fmul2_rn(a.cx2[1], __fadd2_rn(w[R + 1], w[R - 1]));
#pragma unroll
          for (int q = 2; q <= R; ++q) xs0 = __ffma2_rn(a.cx2[q], __fadd2_rn(w[R + q], w[R - q]), xs0);
        }
        {
          float2 w[2 * R + 1];
#pragma unroll
          for (int q = 0; q <= 2 * R; ++q) w[q] = (q == R) ? f1 : lds2(F + fo + FR * NB + (q - R) * NB);
          xs1 = __fmul2_rn(a.cx2[1], __fadd2_rn(w[R + 1], w[R - 1]));
#pragma unroll
          for (int q = 2; q <= R; ++q) xs1 = __ffma2_rn(a.cx2[q], __fadd2_rn(w[R + q], w[R - q]), xs1);
        }
        const float* Vs = reinterpret_cast<const float*>(st + L::OFF_V);
        const float2 cen0 = __fmul2_rn(f2(c0s + Vs[vo]), f0);
        const float2 cen1 = __fmul2_rn(f2(c0s + Vs[vo + TT]), f1);
        // projector term on the tensor cores (3xTF32); the three products of a round go to
        // three accumulators, so that consecutive mma.sync do not wait on each other
        float nl[4] = {0.f, 0.f, 0.f, 0.f}, nla[4] = {0.f, 0.f, 0.f, 0.f}, nlb[4] = {0.f, 0.f, 0.f, 0.f};
        {
          const int* hdr = reinterpret_cast<const int*>(st + L::OFF_REC);
          const int r0 = hdr[warp], r1 = hdr[warp + 1], nr = hdr[NCW];
          const int* ids = hdr + 32;
          const float4* A = reinterpret_cast<const float4*>(st + L::OFF_REC + 128 + 4 * ((nr + 3) & ~3));
          for (int r = r0; r < r1; ++r) {
            const int id = ids[r];
            const float4 av = A[r * 32 + lane];
            const float bv0 = gcs[(id & 0xFFFF) * 32 + lane], bv1 = gcs[(id >> 16) * 32 + lane];
            const float2 bh = make_float2(tf32_hi(bv0), tf32_hi(bv1));
            const float2 bl = __ffma2_rn(f2(-1.f), bh, make_float2(bv0, bv1));
            const float2 b0 = make_float2(bh.x, bl.x), b1 = make_float2(bh.y, bl.y);
            const float h0 = tf32_hi(av.x), h1 = tf32_hi(av.y), h2 = tf32_hi(av.z), h3 = tf32_hi(av.w);
            // low parts a - hi (exact: hi holds the leading bits of a)
            const float2 l01 = __ffma2_rn(f2(-1.f), make_float2(h0, h1), make_float2(av.x, av.y));
            const float2 l23 = __ffma2_rn(f2(-1.f), make_float2(h2, h3), make_float2(av.z, av.w));
            mma_tf32(nla, l01.x, l01.y, l23.x, l23.y, b0.x, b1.x);
            mma_tf32(nlb, h0, h1, h2, h3, b0.y, b1.y);
            mma_tf32(nl, h0, h1, h2, h3, b0.x, b1.x);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) nl[c] += nla[c] + nlb[c];
        }
        d0 = __fadd2_rn(__fadd2_rn(cen0, xs0), __fadd2_rn(ys0, make_float2(nl[0], nl[1])));
        d1 = __fadd2_rn(__fadd2_rn(cen1, xs1), __fadd2_rn(ys1, make_float2(nl[2], nl[3])));
      } else {
        f0 = lds2(F + to);
        f1 = lds2(F + to + TT * NB);
        if constexpr (CX) {
          // a halo plane that crossed a z face: ph_z^t
          const int p = it.zs - R + s;
          if (p < 0 || p >= a.n3) {
            const float2 pz = p < 0 ? conj2(ka.phz[it.kk]) : ka.phz[it.kk];
            f0 = cmul(f0, pz);
            f1 = cmul(f1, pz);
          }
        }
      }
      // z part and the output z' itself, in the ring position's specialisation (only
      // this part depends on the ring position, so the step body exists once)
      float2 e0, e1;
      switch (ring) {
        case 0: zstep<0>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 1: zstep<1>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 2: zstep<2>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 3: zstep<3>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 4: zstep<4>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 5: zstep<5>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 6: zstep<6>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 7: zstep<7>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 8: zstep<8>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 9: zstep<9>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 10: zstep<10>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        case 11: zstep<11>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
        default: zstep<12>(acc, a.cz2, f0, f1, d0, d1, e0, e1); break;
      }
      // output z'-6 is complete: recurrence epilogue
      if (s >= 2 * R) {
        float2 r0 = __fmul2_rn(alpha2, e0);
        float2 r1 = __fmul2_rn(alpha2, e1);
        if (a.yprev != nullptr) {
          const float* P = reinterpret_cast<const float*>(st + L::OFF_YP);
          r0 = __ffma2_rn(beta2, lds2(P + tp), r0);
          r1 = __ffma2_rn(beta2, lds2(P + tp + TT * NB), r1);
        }
        float* o = outp + (size_t)(it.zs + s - 2 * R) * plane;
        if (v0) *reinterpret_cast<float2*>(o) = r0;
        if (v1) *reinterpret_cast<float2*>(o + (size_t)a.n1p * NF) = r1;
        if (gofs != 0) {
          if constexpr (CX) {
            r0 = cmul(r0, gph);
            r1 = cmul(r1, gph);
          }
          if (v0) *reinterpret_cast<float2*>(o + gofs) = r0;
          if (v1) *reinterpret_cast<float2*>(o + (size_t)a.n1p * NF + gofs) = r1;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + L::NBUF + slot);
      ++g;
      if (++cslot == L::NBUF) { cslot = 0; cphase ^= 1u; }
      ring = ring == 12 ? 0 : ring + 1;
    }
  }
  if (!ok && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
}

// --------------------------------------------------------------------------- launcher

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  });
  return fn;
}

}  // namespace tma

long long padded_nd(const sparc_ham* H) { return (long long)(H->gd.n1 + 2 * R) * H->gd.n2 * H->gd.n3; }

namespace tma {

// Tensor map of an x-padded block buffer of nf floats a node (8: FP32 block; 16:
// complex64 unit): dims (nf, n1 + 2R, n2, n3 * nblk), box (8, bx, by, 1).
static bool map_blocks(CUtensorMap* m, const float* base, int nf, int n1p, int n2, int n3, long long nblk, int bx,
                       int by) {
  const cuuint64_t dims[4] = {(cuuint64_t)nf, (cuuint64_t)n1p, (cuuint64_t)n2, (cuuint64_t)n3 * nblk};
  const cuuint64_t strides[3] = {(cuuint64_t)nf * 4, (cuuint64_t)n1p * nf * 4, (cuuint64_t)n1p * n2 * nf * 4};
  const cuuint32_t box[4] = {(cuuint32_t)NB, (cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool map_veff(CUtensorMap* m, const float* veff, int n1, int n2, int n3) {
  const cuuint64_t dims[3] = {(cuuint64_t)n1, (cuuint64_t)n2, (cuuint64_t)n3};
  const cuuint64_t strides[2] = {(cuuint64_t)n1 * 4, (cuuint64_t)n1 * n2 * 4};
  const cuuint32_t box[3] = {TT, TT, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)veff, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One launch over nunits work units (FP32 blocks blk0 .. blk0 + nunits - 1, or the complex
// units of ks); the per-launch fields of Args and the maps of the geometry of H.
template <bool CX>
static cudaError_t launch_tma(const sparc_ham* H, const float* Yin, const float* Yprev, float* Yout, const float* gc,
                              long long nblk_total, int blk0, int nunits, double alpha, double shift, double beta,
                              KArgsT<CX>& ka, const KSlots* ks, cudaStream_t st) {
  const Tables* Tb = (const Tables*)H->fast;
  const TmaTables& M = CX ? Tb->tmac : Tb->tma;
  if (!M.ok || M.cplx != CX || encoder() == nullptr) return cudaErrorNotSupported;
  constexpr int NF = CX ? 2 * NB : NB;
  const int n1 = H->gd.n1, n2 = H->gd.n2, n3 = H->gd.n3, n1p = n1 + 2 * R;
  MapsT<CX> mp;
  for (int i = 0; i < M.nmaps; ++i)
    if (!map_blocks(&mp.frame[i], Yin, NF, n1p, n2, n3, nblk_total, FR, M.map_h[i])) return cudaErrorInvalidValue;
  for (int i = M.nmaps; i < TMA_NMAPS; ++i) mp.frame[i] = mp.frame[0];
  if (!map_blocks(&mp.tile_in, Yin, NF, n1p, n2, n3, nblk_total, TT, TT) ||
      !map_blocks(&mp.tile_prev, Yprev ? Yprev : Yin, NF, n1p, n2, n3, nblk_total, TT, TT))
    return cudaErrorInvalidValue;
  if constexpr (CX) {
    for (int kk = 0; kk < KMAX; ++kk)
      if (kk < ks->nk ? !map_veff(&mp.veff[kk], ks->s[kk].veff, n1, n2, n3) : false) return cudaErrorInvalidValue;
    for (int kk = ks->nk; kk < KMAX; ++kk) mp.veff[kk] = mp.veff[0];
  } else {
    if (!map_veff(&mp.veff[0], H->d_veff32, n1, n2, n3)) return cudaErrorInvalidValue;
  }
  Args a;
  a.n1 = n1; a.n2 = n2; a.n3 = n3;
  a.n1p = n1p;
  a.tiles_x = M.tiles_x;
  a.ntiles = M.tiles_x * M.tiles_y;
  // z-chunks per tile column: whole columns (twelve boundary planes per column) unless
  // the launch would then have fewer than two items per multiprocessor; chunks of at
  // least 16 planes and at most ZLMAX
  const int nsm = std::max(H->ctx->nsm, 1);
  const int per_unit = CX ? M.nts : a.ntiles;   // items of one unit per z-chunk
  if constexpr (CX) {
    ka.nts = M.nts;
    std::memcpy(ka.tsmap, M.tsmap, sizeof(ka.tsmap));
  }
  int nchunk = ceil_div(n3, ZLMAX);
  while ((long long)per_unit * nchunk * nunits < 2 * nsm && n3 / (nchunk + 1) >= 16) ++nchunk;
  a.nchunk = nchunk;
  a.zl = ceil_div(n3, nchunk);
  a.blk0 = blk0;
  a.nblk_total = (int)nblk_total;
  const long long nitems = (long long)per_unit * nchunk * nunits;
  if (nitems >= INT32_MAX || nblk_total >= INT32_MAX) return cudaErrorInvalidValue;
  a.nitems = (int)nitems;
  a.ndp = padded_nd(H);
  std::memcpy(a.yseg, M.yseg, sizeof(a.yseg));
  for (int p = 0; p <= R; ++p) {
    const float cx = (float)H->gd.coef[0][p], cy = (float)H->gd.coef[1][p], cz = (float)H->gd.coef[2][p];
    a.cx2[p] = make_float2(cx, cx);
    a.cy2[p] = make_float2(cy, cy);
    a.cz2[p] = make_float2(cz, cz);
  }
  const double csum = 2.0 * (H->gd.coef[0][0] + H->gd.coef[1][0] + H->gd.coef[2][0]);
  a.c0s = (float)csum - (float)shift;
  a.alpha2 = make_float2((float)alpha, (float)alpha);
  a.beta2 = make_float2((float)beta, (float)beta);
  a.yin = Yin;
  a.yprev = Yprev;
  a.yout = Yout;
  a.gc = gc;
  a.cproj = M.d_cproj;
  a.cng = M.d_cng;
  a.rec = M.d_rec;
  a.stream = (const unsigned char*)M.d_stream;
  a.cimg = M.d_cimg;
  a.status = H->ctx->d_status;
  a.wait_limit = H->ctx->inject_wait_limit > 0 ? H->ctx->inject_wait_limit : (1LL << 32);
  a.stall = H->ctx->inject_stall;
  H->ctx->inject_stall = -1;   // one launch
  cudaError_t e =
      cudaFuncSetAttribute(k_pass_tma<CX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay<CX>::SMEM_B);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(a.nitems, nsm);
  cudaEvent_t t0 = timing_begin(H->ctx, st);
  k_pass_tma<CX><<<grid, NTHR, Lay<CX>::SMEM_B, st>>>(mp, a, ka);
  ++H->ctx->launches;
  timing_end(H->ctx, TK_FPASS, t0, st);
  return cudaGetLastError();
}

}  // namespace tma

cudaError_t launch_to_blocks_px(const sparc_ham* H, const float* X, long long ld, int ns, float* B, int nblk,
                                cudaStream_t st) {
  return launch_to_blocks_rows<float>(X, ld, ns, B, H->gd.nd, H->gd.n1, R, nblk, st);
}

cudaError_t launch_from_blocks_px(const sparc_ham* H, const float* B, int nblk, float* X, long long ld, int ns,
                                  cudaStream_t st) {
  return launch_from_blocks_rows<float>(B, H->gd.nd, H->gd.n1, R, nblk, X, ld, ns, st);
}

cudaError_t launch_to_blocks_px(const sparc_ham* H, const cf32* X, long long ld, int ns, cf32* B, int nblk,
                                cudaStream_t st) {
  const cf32 ph{(float)H->gd.ph_re[0], (float)H->gd.ph_im[0]};
  return launch_to_blocks_rows<cf32>(X, ld, ns, B, H->gd.nd, H->gd.n1, R, nblk, st, ph);
}

cudaError_t launch_from_blocks_px(const sparc_ham* H, const cf32* B, int nblk, cf32* X, long long ld, int ns,
                                  cudaStream_t st) {
  return launch_from_blocks_rows<cf32>(B, H->gd.nd, H->gd.n1, R, nblk, X, ld, ns, st);
}

cudaError_t launch_pass_tma(const sparc_ham* H, const float* Yin, const float* Yprev, float* Yout, const float* gc,
                            int nblk_total, int blk0, int nb, double alpha, double shift, double beta,
                            cudaStream_t st) {
  tma::KArgsNone none{0};
  return tma::launch_tma<false>(H, Yin, Yprev, Yout, gc, nblk_total, blk0, nb, alpha, shift, beta, none, nullptr, st);
}

cudaError_t launch_pass_tma_k(const sparc_ham* H0, const cf32* Yin, const cf32* Yprev, cf32* Yout, const cf32* gc,
                              long long nunit_total, const KSlots& ks, cudaStream_t st) {
  using namespace tma;
  if (ks.nk < 1 || ks.nk > KMAX || ks.nbk < 1) return cudaErrorInvalidValue;
  KArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.nk = ks.nk;
  ka.nbk = ks.nbk;
  const double csum = 2.0 * (H0->gd.coef[0][0] + H0->gd.coef[1][0] + H0->gd.coef[2][0]);
  for (int kk = 0; kk < ks.nk; ++kk) {
    const KSlot& S = ks.s[kk];
    ka.ubase[kk] = S.ubase;
    ka.alpha2[kk] = make_float2(S.alpha, S.alpha);
    ka.beta2[kk] = make_float2(S.beta, S.beta);
    ka.c0s[kk] = (float)csum - S.shift;
    ka.phx[kk] = make_float2(S.phx_r, S.phx_i);
    ka.phy[kk] = make_float2(S.phy_r, S.phy_i);
    ka.phz[kk] = make_float2(S.phz_r, S.phz_i);
  }
  return launch_tma<true>(H0, (const float*)Yin, (const float*)Yprev, (float*)Yout, (const float*)gc, nunit_total,
                          0, ks.nk * ks.nbk, 0.0, 0.0, 0.0, ka, &ks, st);
}

}  // namespace fast
}  // namespace sparc
