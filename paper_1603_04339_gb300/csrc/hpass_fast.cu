// Tiled H-pass for FP32 and complex64 blocks (radius-6 FD stencil, the paper's
// twelfth order), and the projection of the nonlocal operator by projector group.
//
// Pass kernels (k_pass_f2 for FP32, k_pass_c2 for complex64): persistent CTAs of
// 512 threads loop over items = (x-y tile, 13-plane z-chunk, block of NB = 8
// orbitals); FP32 tiles are 16 x 16 nodes, complex64 tiles 16 x 8.
//   * each thread owns 2 x-consecutive nodes x one float2 (an orbital pair, or the
//     (re, im) of one complex orbital) and keeps their values at z-6 .. z+6 in a
//     register queue; the z loop is unrolled over the chunk, so the queue rotates
//     by renaming;
//   * the (x, y) plane at z with its 6-node halo is staged in shared memory: owned
//     nodes from the queues, the halo by cp.async from L2 with periodic wrap (and,
//     for complex data, the Bloch phase of the face crossed); triple-buffered, one
//     barrier per plane;
//   * stencil terms are packed FFMA2/FADD2 with one partial sum per axis;
//   * the nonlocal term sum_p chi~_p gc_p is added from the projector pieces active
//     at (tile, z, rows) (precomputed lists), 4 projectors per piece; FP32 runs it
//     on m16n8k8 TF32 fragments;
//   * the Chebyshev recurrence is the epilogue: Yout = alpha (H - shift) Yin + beta Yprev.
#include <algorithm>
#include <array>
#include <map>
#include <tuple>
#include <vector>

#include "fast.cuh"

namespace sparc {
namespace fast {

// --------------------------------------------------------------------------- host tables

void free_tables(Tables& t) {
  free_tma_tables(t.tma);
  free_tma_tables(t.tmac);
  void* ps[] = {t.d_grp, t.d_sb, t.d_chi4};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (Layout& L : t.lay) {
    void* qs[] = {L.d_cptr, L.d_citems, L.d_sptr, L.d_sslots};
    for (void* p : qs)
      if (p) cudaFree(p);
  }
  t = Tables();
}

static long long fdiv(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

sparc_status build_tables(sparc_ham* H, const sparc_nonlocal* nl) {
  sparc_ctx* ctx = H->ctx;
  Tables* T = new Tables();
  H->fast = T;
  const int n[3] = {H->gd.n1, H->gd.n2, H->gd.n3};
  const double L[3] = {H->grid.n[0] * H->grid.h[0], H->grid.n[1] * H->grid.h[1],
                       H->grid.n[2] * H->grid.h[2]};
  const int np = nl ? nl->nproj : 0;
  // group projectors with identical boxes, in order, at most four per group
  std::vector<Group> grps;
  std::vector<std::array<int, 6>> gbox;
  std::map<std::array<int, 6>, int> open;   // box -> index of the group being filled
  for (int p = 0; p < np; ++p) {
    std::array<int, 6> key{nl->box_lo[3 * p], nl->box_lo[3 * p + 1], nl->box_lo[3 * p + 2],
                           nl->box_n[3 * p], nl->box_n[3 * p + 1], nl->box_n[3 * p + 2]};
    auto it = open.find(key);
    int gi;
    if (it == open.end() || [&] { Group& g = grps[it->second]; return g.proj[3] >= 0; }()) {
      Group g;
      g.proj[0] = g.proj[1] = g.proj[2] = g.proj[3] = -1;
      g.sb0 = g.sb1 = 0;
      grps.push_back(g);
      gbox.push_back(key);
      gi = (int)grps.size() - 1;
      open[key] = gi;
    } else {
      gi = it->second;
    }
    Group& g = grps[gi];
    for (int s = 0; s < 4; ++s)
      if (g.proj[s] < 0) { g.proj[s] = p; break; }
  }
  // box values [node][4] and the periodic pieces of every box
  std::vector<float> chi4;
  std::vector<SubBox> sbs;
  long long off4 = 0;
  for (size_t gi = 0; gi < grps.size(); ++gi) {
    Group& g = grps[gi];
    const int* lo = &gbox[gi][0];
    const int* nb = &gbox[gi][3];
    const long long sz = (long long)nb[0] * nb[1] * nb[2];
    chi4.resize((size_t)(off4 + sz) * 4, 0.0f);
    for (int s = 0; s < 4; ++s) {
      const int p = g.proj[s];
      if (p < 0) continue;
      for (long long e = 0; e < sz; ++e) chi4[(size_t)(off4 + e) * 4 + s] = (float)nl->chi[nl->chi_off[p] + e];
    }
    // per axis: pieces [q0, q1) of the unwrapped box with one image index t each
    std::vector<std::array<long long, 3>> piece[3];
    for (int a = 0; a < 3; ++a) {
      long long q = lo[a];
      const long long qe = (long long)lo[a] + nb[a];
      while (q < qe) {
        const long long t = fdiv(q, n[a]);
        const long long q1 = std::min(qe, (t + 1) * n[a]);
        piece[a].push_back({q, q1, t});
        q = q1;
      }
    }
    g.sb0 = (int)sbs.size();
    for (auto& pz : piece[2])
      for (auto& py : piece[1])
        for (auto& px : piece[0]) {
          SubBox b;
          b.gx0 = (int)(px[0] - px[2] * n[0]); b.gx1 = (int)(px[1] - px[2] * n[0]);
          b.gy0 = (int)(py[0] - py[2] * n[1]); b.gy1 = (int)(py[1] - py[2] * n[1]);
          b.gz0 = (int)(pz[0] - pz[2] * n[2]); b.gz1 = (int)(pz[1] - pz[2] * n[2]);
          b.bx0 = (int)(px[0] - lo[0]); b.by0 = (int)(py[0] - lo[1]); b.bz0 = (int)(pz[0] - lo[2]);
          b.nbx = nb[0]; b.nby = nb[1];
          b.grp = (int)gi;
          b.chi4_off = off4;
          const double kt = H->grid.k[0] * L[0] * (double)px[2] + H->grid.k[1] * L[1] * (double)py[2] +
                            H->grid.k[2] * L[2] * (double)pz[2];
          b.ph_re = (float)cos(kt);
          b.ph_im = (float)(-sin(kt));
          sbs.push_back(b);
        }
    g.sb1 = (int)sbs.size();
    off4 += sz;
  }
  // FNV-1a over what the batched kernels share between Hamiltonians
  {
    unsigned long long hsh = 1469598103934665603ULL;
    auto mix = [&](long long v) {
      for (int i = 0; i < 8; ++i) { hsh ^= (unsigned long long)((v >> (8 * i)) & 0xFF); hsh *= 1099511628211ULL; }
    };
    for (int a = 0; a < 3; ++a) mix(n[a]);
    mix(off4);
    for (const Group& g : grps) { for (int s = 0; s < 4; ++s) mix(g.proj[s]); mix(g.sb0); mix(g.sb1); }
    for (const SubBox& b : sbs) {
      const int f[12] = {b.gx0, b.gx1, b.gy0, b.gy1, b.gz0, b.gz1, b.bx0, b.by0, b.bz0, b.nbx, b.nby, b.grp};
      for (int v : f) mix(v);
      mix(b.chi4_off);
    }
    T->geom = hsh;
  }
  // per kernel tile shape: CTA item lists and per-z active slots
  T->ngrp = (int)grps.size();
  T->nsb = (int)sbs.size();
  for (int si = 0; si < 3; ++si) {
    Layout& Lo = T->lay[si];
    const int TYk = (si == 0) ? Shape<float>::TY : (si == 1) ? Shape<cf32>::TY : 8;
    Lo.tiles_x = ceil_div(n[0], TX);
    Lo.tiles_y = ceil_div(n[1], TYk);
    Lo.nchunk = ceil_div(n[2], ZC);
    const int nct = Lo.tiles_x * Lo.tiles_y * Lo.nchunk;
    std::vector<std::vector<int>> items(nct);
    for (int i = 0; i < (int)sbs.size(); ++i) {
      const SubBox& b = sbs[i];
      for (int ty = 0; ty < Lo.tiles_y; ++ty) {
        const int y0 = ty * TYk, y1 = std::min(n[1], y0 + TYk);
        if (b.gy1 <= y0 || b.gy0 >= y1) continue;
        for (int tx = 0; tx < Lo.tiles_x; ++tx) {
          const int x0 = tx * TX, x1 = std::min(n[0], x0 + TX);
          if (b.gx1 <= x0 || b.gx0 >= x1) continue;
          for (int c = 0; c < Lo.nchunk; ++c) {
            const int z0 = c * ZC, z1 = std::min(n[2], z0 + ZC);
            if (b.gz1 <= z0 || b.gz0 >= z1) continue;
            items[(ty * Lo.tiles_x + tx) * Lo.nchunk + c].push_back(i);
          }
        }
      }
    }
    // per (CTA, z, row group): CTA-local indices of the pieces that touch those rows;
    // a row group is the rows one warp covers (8 for FP32, 4 for complex64)
    const int rgh = (si == 1) ? 4 : 8;
    const int nrg = TYk / rgh;
    const int xrw = (si == 1) ? TX : 2;          // x extent of a list (FP32: one warp's x-run)
    const int nxr = TX / xrw;
    std::vector<int> cptr(nct + 1, 0), citems, sptr((size_t)nct * ZC * nrg * nxr + 1, 0), sslots;
    Lo.max_items = 0;
    Lo.max_steps = 0;
    for (int c = 0; c < nct; ++c) {
      const auto& it = items[c];
      Lo.max_items = std::max(Lo.max_items, (int)it.size());
      cptr[c + 1] = cptr[c] + (int)it.size();
      citems.insert(citems.end(), it.begin(), it.end());
      const int tile = c / Lo.nchunk;
      const int x0 = (tile % Lo.tiles_x) * TX, x1 = std::min(n[0], x0 + TX);
      const int y0t = (tile / Lo.tiles_x) * TYk;
      const int z0 = (c % Lo.nchunk) * ZC;
      const int first = (int)sslots.size();
      for (int k = 0; k < ZC; ++k)
        for (int rg = 0; rg < nrg; ++rg)
          for (int xq = 0; xq < nxr; ++xq) {
            sptr[(((size_t)c * ZC + k) * nrg + rg) * nxr + xq] = (int)sslots.size();
            const int z = z0 + k;
            const int y0 = y0t + rgh * rg, y1 = std::min(n[1], y0 + rgh);
            const int xa = x0 + xq * xrw, xb = std::min(x1, xa + xrw);
            if (z < n[2] && y0 < y1 && xa < xb)
              for (int j = 0; j < (int)it.size(); ++j) {
                const SubBox& b = sbs[it[j]];
                if (b.gz0 <= z && z < b.gz1 && b.gy0 < y1 && b.gy1 > y0 && b.gx0 < xb && b.gx1 > xa)
                  sslots.push_back(j);
              }
          }
      Lo.max_steps = std::max(Lo.max_steps, (int)sslots.size() - first);
    }
    sptr[(size_t)nct * ZC * nrg * nxr] = (int)sslots.size();
    auto up = [&](void** d, const void* h, size_t bytes) -> bool {
      if (cudaMalloc(d, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
      return bytes == 0 || cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up((void**)&Lo.d_cptr, cptr.data(), cptr.size() * sizeof(int)) ||
        !up((void**)&Lo.d_citems, citems.data(), citems.size() * sizeof(int)) ||
        !up((void**)&Lo.d_sptr, sptr.data(), sptr.size() * sizeof(int)) ||
        !up((void**)&Lo.d_sslots, sslots.data(), sslots.size() * sizeof(int))) {
      cudaGetLastError();
      return fail(ctx, SPARC_ERR_OOM, "projector table allocation failed");
    }
  }
  auto up = [&](void** d, const void* h, size_t bytes) -> bool {
    if (cudaMalloc(d, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    return bytes == 0 || cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up((void**)&T->d_grp, grps.data(), grps.size() * sizeof(Group)) ||
      !up((void**)&T->d_sb, sbs.data(), sbs.size() * sizeof(SubBox)) ||
      !up((void**)&T->d_chi4, chi4.data(), chi4.size() * sizeof(float))) {
    cudaGetLastError();
    return fail(ctx, SPARC_ERR_OOM, "projector table allocation failed");
  }
  return build_tma_tables(H, T, grps, gbox, chi4);
}

unsigned long long geometry_hash(const sparc_ham* H) {
  const Tables* T = (const Tables*)H->fast;
  return T ? T->geom : 0ULL;
}

void kslot(const sparc_ham* H, KSlot& s) {
  const Tables* T = (const Tables*)H->fast;
  s.sb = T->d_sb;
  s.chi4 = (const float4*)T->d_chi4;
  s.veff = H->d_veff32;
  s.gamma = H->d_gamma32;
  s.phx_r = (float)H->gd.ph_re[0]; s.phx_i = (float)H->gd.ph_im[0];
  s.phy_r = (float)H->gd.ph_re[1]; s.phy_i = (float)H->gd.ph_im[1];
  s.phz_r = (float)H->gd.ph_re[2]; s.phz_i = (float)H->gd.ph_im[2];
}

bool shape_usable(const sparc_ham* H, int shape) {
  const Tables* T = (const Tables*)H->fast;
  if (!usable(H) || shape < 0 || shape >= NSHAPE_F32) return false;
  if (shape == SHAPE_TMA) return tma_usable(H);
  return shape == 0 || (T->lay[2].max_items <= MAXI && T->lay[2].max_steps <= MAXSTEP);
}

bool usable(const sparc_ham* H) {
  const Tables* T = (const Tables*)H->fast;
  return T != nullptr && H->gd.no == R && T->lay[0].max_items <= MAXI && T->lay[1].max_items <= MAXI &&
         T->lay[0].max_steps <= MAXSTEP && T->lay[1].max_steps <= MAXSTEP;
}

// --------------------------------------------------------------------------- device helpers

template <class T> struct FT;
template <> struct FT<float> {
  static constexpr bool cplx = false;
  __device__ static float zero() { return 0.f; }
};
template <> struct FT<cf32> {
  static constexpr bool cplx = true;
  __device__ static cf32 zero() { return {0.f, 0.f}; }
};

__device__ __forceinline__ float fld(const float* p) { return __ldg(p); }
__device__ __forceinline__ cf32 fld(const cf32* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// Wrap g into [0, n) and return the number of cells crossed.
__device__ __forceinline__ int wrap(int& g, int n) {
  int t = 0;
  while (g >= n) { g -= n; ++t; }
  while (g < 0) { g += n; --t; }
  return t;
}

// Asynchronous global -> shared copies (completion tracked per thread by groups).
__device__ __forceinline__ void cp16(void* sm, const void* gm) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp4(void* sm, const void* gm) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

struct PassArgs {
  long long nd;
  int n1, n2, n3;
  int tiles_x, nchunk, blk0, nblk_total;
  float cx[R + 1], cy[R + 1], cz[R + 1];
  float c0;                       // centre Laplacian coefficient (sum of -w_0 over axes)
  float phx_r, phx_i, phy_r, phy_i, phz_r, phz_i;   // exp(i k_s L_s)
  float alpha, shift, beta;
  float2 cx2[R + 1], cy2[R + 1], cz2[R + 1], alpha2, beta2;   // the same, as packed pairs
  const float* veff;
  const int* cptr;
  const int* citems;
  const int* sptr;
  const int* sslots;
  const SubBox* sb;
  const Group* grp;
  const float4* chi4;
};

// Compact form of a projector-box piece for the scatter: chi4 row of grid row
// (y, z) starts at base + sy * y + sz * z (index of grid x = 0).
struct __align__(16) Piece {
  int gy0, gy1, gx0, gx1;
  int base, sy, sz, pad0;
  float ph_re, ph_im, pad1, pad2;
};

constexpr int PX = TX + 2 * R;
constexpr int RP = PX * NB + 8;     // row pitch in elements: rows of a warp land 8 banks apart
template <class T, int TYv = Shape<T>::TY> struct Smem {
  static constexpr int TY = TYv, PY = TYv + 2 * R;
  static constexpr int NRG = TY / (sizeof(T) == 4 ? 8 : 4);   // row groups of the z lists
  static constexpr int NXR = (sizeof(T) == 4) ? 8 : 1;         // x-runs of the z lists
  static constexpr int NL = ZC * NRG * NXR;                    // lists per CTA
  static constexpr size_t planes = 3 * (size_t)PY * RP * sizeof(T);
  static constexpr size_t yprev = 3 * (size_t)TY * TX * NB * sizeof(T);
  static constexpr size_t vb = 3 * (size_t)TY * TX * sizeof(float);
  static constexpr size_t desc = (size_t)MAXI * sizeof(Piece);
  static constexpr size_t gcs = (size_t)MAXI * 4 * NB * sizeof(T);
  static constexpr size_t steps = (size_t)(NL + 1 + MAXSTEP) * sizeof(int);
  static constexpr size_t total = planes + yprev + vb + desc + gcs + steps;
};

// ---------------------------------------------------------------------------
// FP32 pass with orbital pairs: each thread owns 2 x-consecutive nodes x 2
// orbitals (a float2), so every stencil term is one packed FFMA2/FADD2 and every
// shared-memory neighbour read is one 64-bit load.  A warp covers 8 rows x 4
// orbital pairs at one x-run.  CTAs are persistent: they loop over (tile,
// z-chunk, block) items, so the last wave is not partly empty.
constexpr int RX2 = 2;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += A B for one m16n8k8 TF32 tile in three products (a_hi b_hi + a_hi b_lo +
// a_lo b_hi, hi = the value with its low 13 mantissa bits cleared): about 21 bits,
// close to an FP32 product.  a: the thread's 4 A-fragment values, b: its 2 B values.
__device__ __forceinline__ void mma_tf32x3(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float hi = __uint_as_float(__float_as_uint(a[i]) & 0xFFFFE000u);
    ah[i] = __float_as_uint(hi);
    al[i] = __float_as_uint(a[i] - hi);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float hi = __uint_as_float(__float_as_uint(b[i]) & 0xFFFFE000u);
    bh[i] = __float_as_uint(hi);
    bl[i] = __float_as_uint(b[i] - hi);
  }
  mma_tf32_16x8x8(d, al, bh);
  mma_tf32_16x8x8(d, ah, bl);
  mma_tf32_16x8x8(d, ah, bh);
}

// TYT: tile rows (16 or 8); NT: threads (TYT * 32, two orbital pairs x 2 x-nodes each).
// DIFF: the stencil in difference form sum_p c_p ((f_{+p} - f_0) + (f_{-p} - f_0)) plus
// (V - shift) f_0, whose FP32 rounding stays relative to the differences rather than
// to |c_0| f_0 (the form a plain H-apply for the Rayleigh-Ritz projections needs).
template <int TYT, int NT, bool DIFF = false>
__global__ void __launch_bounds__(NT, 512 / NT)
k_pass_f2(PassArgs a, const float* __restrict__ Yin, const float* Yprev, float* Yout,
          const float* __restrict__ gc, int nitems) {
  constexpr int Q = 2 * R + 1;
  constexpr int PY = TYT + 2 * R;
  using SM = Smem<float, TYT>;
  static_assert(NT == TYT * 32, "two x-nodes x one orbital pair per thread");
  constexpr int CH = 2;                                  // 16-byte chunks per node (8 floats)
  constexpr int NHC = (PX * PY * CH + NT - 1) / NT;
  constexpr int NPC = (TX * TYT * CH + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* planes = reinterpret_cast<float*>(smraw);
  float* yps = reinterpret_cast<float*>(smraw + SM::planes);
  float* vbs = reinterpret_cast<float*>(smraw + SM::planes + SM::yprev);
  Piece* desc = reinterpret_cast<Piece*>(smraw + SM::planes + SM::yprev + SM::vb);
  float* gcs = reinterpret_cast<float*>(smraw + SM::planes + SM::yprev + SM::vb +
                                        SM::desc);
  int* steps = reinterpret_cast<int*>(smraw + SM::planes + SM::yprev + SM::vb +
                                      SM::desc + SM::gcs);
  const int t = threadIdx.x;
  const int op = t % 4;                  // orbital pair
  const int r8 = (t / 4) % 8;            // row within the warp
  const int xr = (t / 32) % (TX / RX2);  // x-run
  const int yg = t / 256;                // row group (0, 1)
  const int yl = yg * 8 + r8, xl0 = xr * RX2;
  const int o2 = 2 * op;
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const long long plane_el = (long long)n1 * n2 * NB;
  const int ntiles = a.tiles_x * ((n2 + TYT - 1) / TYT);
  constexpr int NRG = SM::NRG, NXR = SM::NXR, NL = SM::NL;
  static_assert(NRG == TYT / 8 && NXR == TX / RX2, "one list per warp");

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % ntiles;
    const int chunk = (item / ntiles) % a.nchunk;
    const int bi = item / (ntiles * a.nchunk);
    const int cta = tile * a.nchunk + chunk;
    const int tx0 = (tile % a.tiles_x) * TX, ty0 = (tile / a.tiles_x) * TYT;
    const int zs = chunk * ZC;
    const int ze = min(zs + ZC, n3);
    const int blk = a.blk0 + bi;
    const size_t boff = (size_t)blk * a.nd * NB;
    const float* Y = Yin + boff;
    const int gy = ty0 + yl;
    const bool vy = gy < n2;
    const int txv = min(TX, n1 - tx0), tyv = min(TYT, n2 - ty0);
    bool vr[RX2];
#pragma unroll
    for (int r = 0; r < RX2; ++r) vr[r] = vy && (tx0 + xl0 + r < n1);

    // ---- item tables
    const int it0 = __ldg(a.cptr + cta), nit = __ldg(a.cptr + cta + 1) - it0;
    for (int i = t; i < nit; i += NT) {
      const SubBox b = a.sb[__ldg(a.citems + it0 + i)];
      Piece pc;
      pc.gy0 = b.gy0; pc.gy1 = b.gy1; pc.gx0 = b.gx0; pc.gx1 = b.gx1;
      pc.sy = b.nbx;
      pc.sz = b.nbx * b.nby;
      pc.base = (int)b.chi4_off + b.bx0 - b.gx0 + b.nbx * (b.by0 - b.gy0) + pc.sz * (b.bz0 - b.gz0);
      pc.ph_re = b.ph_re; pc.ph_im = b.ph_im;
      desc[i] = pc;
      for (int l = 0; l < 4; ++l) {
        const int p = a.grp[b.grp].proj[l];
        for (int oo = 0; oo < NB; ++oo)
          gcs[(i * 4 + l) * NB + oo] = (p >= 0) ? gc[((size_t)p * a.nblk_total + blk) * NB + oo] : 0.f;
      }
    }
    const size_t sb0 = (size_t)cta * NL;
    const int s0 = __ldg(a.sptr + sb0);
    for (int k = t; k <= NL; k += NT) steps[k] = __ldg(a.sptr + sb0 + k) - s0;
    const int nst = __ldg(a.sptr + sb0 + NL) - s0;
    for (int k = t; k < nst; k += NT) steps[NL + 1 + k] = __ldg(a.sslots + s0 + k);

    // ---- copy descriptors
    int hs[NHC], hg[NHC];
#pragma unroll
    for (int i = 0; i < NHC; ++i) {
      const int idx = t + i * NT;
      hs[i] = -1; hg[i] = 0;
      if (idx < PX * PY * CH) {
        const int pnt = idx / CH, ch = idx % CH;
        const int sx = pnt % PX, sy = pnt / PX;
        const int lx = sx - R, ly = sy - R;
        if (!(lx >= 0 && lx < txv && ly >= 0 && ly < tyv)) {
          int gxw = tx0 + lx, gyw = ty0 + ly;
          wrap(gxw, n1);
          wrap(gyw, n2);
          hs[i] = sy * RP + sx * NB + ch * 4;
          hg[i] = (gyw * n1 + gxw) * NB + ch * 4;
        }
      }
    }
    int ps[NPC], pg[NPC];
#pragma unroll
    for (int i = 0; i < NPC; ++i) {
      const int idx = t + i * NT;
      ps[i] = -1; pg[i] = 0;
      if (idx < TX * TYT * CH) {
        const int node = idx / CH, ch = idx % CH;
        const int lx = node % TX, ly = node / TX;
        if (lx < txv && ly < tyv) {
          ps[i] = node * NB + ch * 4;
          pg[i] = ((ty0 + ly) * n1 + tx0 + lx) * NB + ch * 4;
        }
      }
    }
    const int vlx = t % TX, vly = t / TX;
    const bool vv = t < TX * TYT && vlx < txv && vly < tyv;
    const int vgo = (ty0 + vly) * n1 + tx0 + vlx;

    float2 q[Q][RX2];
    auto load_z = [&](int zz, float2* dst) {
      int zw = zz;
      wrap(zw, n3);
      const float* src = Y + (size_t)zw * plane_el + ((size_t)gy * n1 + tx0 + xl0) * NB + o2;
#pragma unroll
      for (int r = 0; r < RX2; ++r)
        dst[r] = vr[r] ? __ldg(reinterpret_cast<const float2*>(src + r * NB)) : make_float2(0.f, 0.f);
    };
#pragma unroll
    for (int i = 0; i < Q; ++i) load_z(zs - R + i, q[i]);

    auto issue = [&](int zz, int b) {
      int zw = zz;
      wrap(zw, n3);
      float* P = planes + (size_t)b * PY * RP;
      const float* Yz = Y + (size_t)zw * plane_el;
#pragma unroll
      for (int i = 0; i < NHC; ++i)
        if (hs[i] >= 0) cp16(P + hs[i], Yz + hg[i]);
      if (vv) cp4(vbs + (size_t)b * TYT * TX + t, a.veff + (size_t)zw * n1 * n2 + vgo);
      if (Yprev != nullptr) {
        float* Pp = yps + (size_t)b * TYT * TX * NB;
        const float* Yp = Yprev + boff + (size_t)zw * plane_el;
#pragma unroll
        for (int i = 0; i < NPC; ++i)
          if (ps[i] >= 0) cp16(Pp + ps[i], Yp + pg[i]);
      }
    };
    auto own = [&](const float2* vals, int b) {
      float* P = planes + (size_t)b * PY * RP;
#pragma unroll
      for (int r = 0; r < RX2; ++r)
        if (vr[r]) *reinterpret_cast<float2*>(P + (yl + R) * RP + (xl0 + r + R) * NB + o2) = vals[r];
    };

    issue(zs, 0);
    cp_commit();
    if (zs + 1 < ze) issue(zs + 1, 1);
    cp_commit();
    own(q[R], 0);
    cp_wait1();
    __syncthreads();

    // the z loop is unrolled over the 13 planes of a chunk, so the register queue
    // rotates by renaming: plane z + d sits in q[(sidx + R + d) % Q]
#pragma unroll
    for (int sidx = 0; sidx < ZC; ++sidx) {
      const int z = zs + sidx;
      if (z < ze) {   // uniform over the CTA; no break, so the loop unrolls completely
      const int b = sidx % 3;
      const float* P = planes + (size_t)b * PY * RP;
      float2 acc[RX2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (vy) {
        const float* row = P + (yl + R) * RP + o2;
        float2 w[RX2 + 2 * R];
#pragma unroll
        for (int i = 0; i < RX2 + 2 * R; ++i) w[i] = lds2(row + (xl0 + i) * NB);
        const float* V = vbs + (size_t)b * TYT * TX + yl * TX + xl0;
#pragma unroll
        for (int r = 0; r < RX2; ++r) {
          // one partial sum per axis: three short dependency chains instead of one long one
          const float2 xc = q[(sidx + R) % Q][r];
          float2 sx = __fmul2_rn(f2((DIFF ? 0.f : a.c0) + V[r] - a.shift), xc);
          float2 sy = make_float2(0.f, 0.f), sz = make_float2(0.f, 0.f);
          const float* col = P + (xl0 + r + R) * NB + o2;
          const float2 m1 = f2(-1.f);
#pragma unroll
          for (int p = 1; p <= R; ++p) {
            const float2 u = lds2(col + (yl + R + p) * RP);
            const float2 d = lds2(col + (yl + R - p) * RP);
            const float2 qu = q[(sidx + R + p) % Q][r], qd = q[(sidx + R - p) % Q][r];
            if constexpr (DIFF) {   // f - f0 is one rounding (exact when f and f0 are close)
              sx = __ffma2_rn(a.cx2[p], __fadd2_rn(__ffma2_rn(m1, xc, w[R + r + p]), __ffma2_rn(m1, xc, w[R + r - p])), sx);
              sy = __ffma2_rn(a.cy2[p], __fadd2_rn(__ffma2_rn(m1, xc, u), __ffma2_rn(m1, xc, d)), sy);
              sz = __ffma2_rn(a.cz2[p], __fadd2_rn(__ffma2_rn(m1, xc, qu), __ffma2_rn(m1, xc, qd)), sz);
            } else {
              sx = __ffma2_rn(a.cx2[p], __fadd2_rn(w[R + r + p], w[R + r - p]), sx);
              sy = __ffma2_rn(a.cy2[p], __fadd2_rn(u, d), sy);
              sz = __ffma2_rn(a.cz2[p], __fadd2_rn(qu, qd), sz);
            }
          }
          acc[r] = __fadd2_rn(sx, __fadd2_rn(sy, sz));
        }
      }
      // nonlocal scatter on the tensor cores: for the warp's 16 nodes (8 rows x 2
      // columns) x 8 orbitals, sum_p chi_p(node) gc_p(orbital) over the pieces active at
      // z is a 16 x 8 x (4 per piece) product.  The m16n8k8 fragments match the thread
      // layout (row groupID = the thread's row, threadID_in_group = its orbital pair),
      // so two pieces (K = 8) per mma.sync, in 3xTF32 for FP32 accuracy, accumulate
      // into nl, which is added to the stencil sum in FP32.
      {
        const int li = (sidx * NRG + yg) * NXR + xr;
        const int ea = steps[li], eb = steps[li + 1];
        const int x0r = tx0 + xl0;
        const int cq = op, gq = r8;   // threadID_in_group, groupID
        float nl[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = ea; e < eb; e += 2) {
          float av[4], bv[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            av[2 * h] = av[2 * h + 1] = 0.f;
            bv[h] = 0.f;
            if (e + h < eb) {
              const int it = steps[NL + 1 + e + h];
              const int4 pa = *reinterpret_cast<const int4*>(&desc[it].gy0);   // gy0 gy1 gx0 gx1
              const int4 pb = *reinterpret_cast<const int4*>(&desc[it].base);  // base sy sz -
              const bool rok = vy && gy >= pa.x && gy < pa.y;
              const int rowoff = pb.x + pb.y * gy + pb.z * z;
#pragma unroll
              for (int r = 0; r < RX2; ++r) {
                const int gx = x0r + r;
                if (rok && gx >= pa.z && gx < pa.w) av[2 * h + r] = __ldg(reinterpret_cast<const float*>(a.chi4) + (size_t)(rowoff + gx) * 4 + cq);
              }
              bv[h] = gcs[(it * 4 + cq) * NB + gq];
            }
          }
          mma_tf32x3(nl, av, bv);
        }
        acc[0] = __fadd2_rn(acc[0], make_float2(nl[0], nl[1]));
        acc[1] = __fadd2_rn(acc[1], make_float2(nl[2], nl[3]));
      }
      if (vy) {
        // recurrence epilogue
        const float* Pp = yps + (size_t)b * TYT * TX * NB + (yl * TX + xl0) * NB + o2;
        float* out = Yout + boff + (size_t)z * plane_el + ((size_t)gy * n1 + tx0 + xl0) * NB + o2;
#pragma unroll
        for (int r = 0; r < RX2; ++r) {
          if (!vr[r]) continue;
          float2 v = __fmul2_rn(a.alpha2, acc[r]);
          if (Yprev) v = __ffma2_rn(a.beta2, lds2(Pp + r * NB), v);
          *reinterpret_cast<float2*>(out + r * NB) = v;
        }
      }
      if (z + 1 < ze) own(q[(sidx + R + 1) % Q], (sidx + 1) % 3);
      if (z + 2 < ze) issue(z + 2, (sidx + 2) % 3);
      cp_commit();
      load_z(z + R + 1, q[sidx % Q]);   // plane z - R is no longer needed
      cp_wait1();
      __syncthreads();
      }
    }
  }
}

// Complex64 pass in the form of the FP32 one: a cf32 value is a float2 (re, im) and
// the stencil, V_eff and recurrence coefficients are real, so every stencil term is
// one packed FFMA2/FADD2 on (re, im).  Each thread owns 2 x-consecutive nodes x one
// orbital; a warp covers 4 rows x 8 orbitals at one x-run; the 13-plane z queue
// rotates by renaming in the unrolled z loop; CTAs are persistent over (tile,
// z-chunk, k-point unit) items.  Values that cross a face pick up the Bloch phase
// of that face: the z queue when it loads a wrapped plane, the staged halo after
// its copy lands (the x/y face crossings are encoded in the copy descriptors).
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// exp(i k L t) for a face crossing t in {-1, 0, 1} from exp(i k L) = (pr, pi)
__device__ __forceinline__ float2 face_phase(float pr, float pi, int t) {
  return t == 0 ? make_float2(1.f, 0.f) : make_float2(pr, t > 0 ? pi : -pi);
}

__global__ void __launch_bounds__(THREADS, 1)
k_pass_c2(PassArgs a, const __grid_constant__ KSlots ks, const cf32* __restrict__ Yin, const cf32* Yprev,
          cf32* Yout, const cf32* __restrict__ gc, int nitems) {
  constexpr int Q = 2 * R + 1;
  constexpr int TYC = Shape<cf32>::TY;
  constexpr int PY = TYC + 2 * R;
  constexpr int CH = NB * (int)sizeof(cf32) / 16;         // 16-byte chunks per node (4)
  constexpr int NHC = (PX * PY * CH + THREADS - 1) / THREADS;
  constexpr int NPC = (TX * TYC * CH + THREADS - 1) / THREADS;
  constexpr int NRG = Smem<cf32>::NRG, NL = Smem<cf32>::NL;
  static_assert(NRG == TYC / 4 && Smem<cf32>::NXR == 1, "one list per row group");
  static_assert((TX / RX2) * 4 * NB * NRG == THREADS, "thread layout");
  extern __shared__ __align__(16) unsigned char smraw[];
  cf32* planes = reinterpret_cast<cf32*>(smraw);
  cf32* yps = reinterpret_cast<cf32*>(smraw + Smem<cf32>::planes);
  float* vbs = reinterpret_cast<float*>(smraw + Smem<cf32>::planes + Smem<cf32>::yprev);
  Piece* desc = reinterpret_cast<Piece*>(smraw + Smem<cf32>::planes + Smem<cf32>::yprev + Smem<cf32>::vb);
  cf32* gcs = reinterpret_cast<cf32*>(smraw + Smem<cf32>::planes + Smem<cf32>::yprev + Smem<cf32>::vb +
                                      Smem<cf32>::desc);
  int* steps = reinterpret_cast<int*>(smraw + Smem<cf32>::planes + Smem<cf32>::yprev + Smem<cf32>::vb +
                                      Smem<cf32>::desc + Smem<cf32>::gcs);
  const int t = threadIdx.x;
  const int o = t % NB;                  // orbital
  const int r4 = (t / NB) % 4;           // row within the warp
  const int xr = (t / 32) % (TX / RX2);  // x-run
  const int yg = t / 256;                // row group (0, 1)
  const int yl = yg * 4 + r4, xl0 = xr * RX2;
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const long long plane_el = (long long)n1 * n2 * NB;
  const int ntiles = a.tiles_x * ((n2 + TYC - 1) / TYC);
  auto ld2 = [](const cf32* p) { return *reinterpret_cast<const float2*>(p); };

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % ntiles;
    const int chunk = (item / ntiles) % a.nchunk;
    const int j = item / (ntiles * a.nchunk);
    const KSlot& S = ks.s[j / ks.nbk];
    const long long blk = S.ubase + j % ks.nbk;
    const int cta = tile * a.nchunk + chunk;
    const int tx0 = (tile % a.tiles_x) * TX, ty0 = (tile / a.tiles_x) * TYC;
    const int zs = chunk * ZC;
    const int ze = min(zs + ZC, n3);
    const size_t boff = (size_t)blk * a.nd * NB;
    const cf32* Y = Yin + boff;
    const int gy = ty0 + yl;
    const bool vy = gy < n2;
    const int txv = min(TX, n1 - tx0), tyv = min(TYC, n2 - ty0);
    bool vr[RX2];
#pragma unroll
    for (int r = 0; r < RX2; ++r) vr[r] = vy && (tx0 + xl0 + r < n1);
    const float2 alpha2 = make_float2(S.alpha, S.alpha), beta2 = make_float2(S.beta, S.beta);

    // ---- item tables (the previous item's readers finished at its last barrier)
    const int it0 = __ldg(a.cptr + cta), nit = __ldg(a.cptr + cta + 1) - it0;
    for (int i = t; i < nit; i += THREADS) {
      const SubBox b = S.sb[__ldg(a.citems + it0 + i)];
      Piece pc;
      pc.gy0 = b.gy0; pc.gy1 = b.gy1; pc.gx0 = b.gx0; pc.gx1 = b.gx1;
      pc.sy = b.nbx;
      pc.sz = b.nbx * b.nby;
      pc.base = (int)b.chi4_off + b.bx0 - b.gx0 + b.nbx * (b.by0 - b.gy0) + pc.sz * (b.bz0 - b.gz0);
      pc.ph_re = b.ph_re; pc.ph_im = b.ph_im;
      desc[i] = pc;
      // the piece's Bloch phase folded into its coefficients: ph * gc
      for (int l = 0; l < 4; ++l) {
        const int p = a.grp[b.grp].proj[l];
        for (int oo = 0; oo < NB; ++oo) {
          const cf32 g = (p >= 0) ? gc[((size_t)p * a.nblk_total + blk) * NB + oo] : cf32{0.f, 0.f};
          gcs[(i * 4 + l) * NB + oo] = cf32{b.ph_re * g.x - b.ph_im * g.y, b.ph_re * g.y + b.ph_im * g.x};
        }
      }
    }
    const size_t sb0 = (size_t)cta * NL;
    const int s0 = __ldg(a.sptr + sb0);
    for (int k = t; k <= NL; k += THREADS) steps[k] = __ldg(a.sptr + sb0 + k) - s0;
    const int nst = __ldg(a.sptr + sb0 + NL) - s0;
    for (int k = t; k < nst; k += THREADS) steps[NL + 1 + k] = __ldg(a.sslots + s0 + k);

    // ---- copy descriptors: hs = smem element offset | (face crossings (tx+1) + 3 (ty+1)) << 20
    int hs[NHC], hg[NHC];
#pragma unroll
    for (int i = 0; i < NHC; ++i) {
      const int idx = t + i * THREADS;
      hs[i] = -1; hg[i] = 0;
      if (idx < PX * PY * CH) {
        const int pnt = idx / CH, ch = idx % CH;
        const int sx = pnt % PX, sy = pnt / PX;
        const int lx = sx - R, ly = sy - R;
        if (!(lx >= 0 && lx < txv && ly >= 0 && ly < tyv)) {
          int gxw = tx0 + lx, gyw = ty0 + ly;
          const int cx = wrap(gxw, n1), cy = wrap(gyw, n2);
          hs[i] = (sy * RP + sx * NB + ch * 2) | (((cx + 1) + 3 * (cy + 1)) << 20);
          hg[i] = (gyw * n1 + gxw) * NB + ch * 2;
        }
      }
    }
    int ps[NPC], pg[NPC];
#pragma unroll
    for (int i = 0; i < NPC; ++i) {
      const int idx = t + i * THREADS;
      ps[i] = -1; pg[i] = 0;
      if (idx < TX * TYC * CH) {
        const int node = idx / CH, ch = idx % CH;
        const int lx = node % TX, ly = node / TX;
        if (lx < txv && ly < tyv) {
          ps[i] = node * NB + ch * 2;
          pg[i] = ((ty0 + ly) * n1 + tx0 + lx) * NB + ch * 2;
        }
      }
    }
    const int vlx = t % TX, vly = t / TX;
    const bool vv = t < TX * TYC && vlx < txv && vly < tyv;
    const int vgo = (ty0 + vly) * n1 + tx0 + vlx;

    float2 q[Q][RX2];
    auto load_z = [&](int zz, float2* dst) {
      int zw = zz;
      const int cz = wrap(zw, n3);
      const float2 ph = face_phase(S.phz_r, S.phz_i, cz);
      const cf32* src = Y + (size_t)zw * plane_el + ((size_t)gy * n1 + tx0 + xl0) * NB + o;
#pragma unroll
      for (int r = 0; r < RX2; ++r) {
        const float2 v = vr[r] ? __ldg(reinterpret_cast<const float2*>(src + r * NB)) : make_float2(0.f, 0.f);
        dst[r] = cz ? cmul2(v, ph) : v;
      }
    };
#pragma unroll
    for (int i = 0; i < Q; ++i) load_z(zs - R + i, q[i]);

    auto issue = [&](int zz, int b) {
      int zw = zz;
      wrap(zw, n3);
      cf32* P = planes + (size_t)b * PY * RP;
      const cf32* Yz = Y + (size_t)zw * plane_el;
#pragma unroll
      for (int i = 0; i < NHC; ++i)
        if (hs[i] >= 0) cp16(P + (hs[i] & 0xFFFFF), Yz + hg[i]);
      if (vv) cp4(vbs + (size_t)b * TYC * TX + t, S.veff + (size_t)zw * n1 * n2 + vgo);
      if (Yprev != nullptr) {
        cf32* Pp = yps + (size_t)b * TYC * TX * NB;
        const cf32* Yp = Yprev + boff + (size_t)zw * plane_el;
#pragma unroll
        for (int i = 0; i < NPC; ++i)
          if (ps[i] >= 0) cp16(Pp + ps[i], Yp + pg[i]);
      }
    };
    // Bloch phase of the halo chunks this thread copied (after they landed)
    auto fixup = [&](int zz, int b) {
      int zw = zz;
      const int cz = wrap(zw, n3);
      const float2 pz = face_phase(S.phz_r, S.phz_i, cz);
      cf32* P = planes + (size_t)b * PY * RP;
#pragma unroll
      for (int i = 0; i < NHC; ++i) {
        const int hw = hs[i] >> 20;
        if (hs[i] < 0 || (hw == 4 && cz == 0)) continue;
        const float2 ph = cmul2(cmul2(face_phase(S.phx_r, S.phx_i, hw % 3 - 1), face_phase(S.phy_r, S.phy_i, hw / 3 - 1)), pz);
        float4* c = reinterpret_cast<float4*>(P + (hs[i] & 0xFFFFF));
        const float4 v = *c;
        const float2 v0 = cmul2(make_float2(v.x, v.y), ph), v1 = cmul2(make_float2(v.z, v.w), ph);
        *c = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    };
    auto own = [&](const float2* vals, int b) {
      cf32* P = planes + (size_t)b * PY * RP;
#pragma unroll
      for (int r = 0; r < RX2; ++r)
        if (vr[r]) *reinterpret_cast<float2*>(P + (yl + R) * RP + (xl0 + r + R) * NB + o) = vals[r];
    };

    issue(zs, 0);
    cp_commit();
    if (zs + 1 < ze) issue(zs + 1, 1);
    cp_commit();
    own(q[R], 0);
    cp_wait1();
    fixup(zs, 0);
    __syncthreads();

#pragma unroll
    for (int sidx = 0; sidx < ZC; ++sidx) {
      const int z = zs + sidx;
      if (z < ze) {   // uniform over the CTA; no break, so the loop unrolls completely
      const int b = sidx % 3;
      const cf32* P = planes + (size_t)b * PY * RP;
      float2 acc[RX2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (vy) {
        const cf32* row = P + (yl + R) * RP + o;
        float2 w[RX2 + 2 * R];
#pragma unroll
        for (int i = 0; i < RX2 + 2 * R; ++i) w[i] = ld2(row + (xl0 + i) * NB);
        const float* V = vbs + (size_t)b * TYC * TX + yl * TX + xl0;
#pragma unroll
        for (int r = 0; r < RX2; ++r) {
          float2 sx = __fmul2_rn(f2(a.c0 + V[r] - S.shift), q[(sidx + R) % Q][r]);
          float2 sy = make_float2(0.f, 0.f), sz = make_float2(0.f, 0.f);
          const cf32* col = P + (xl0 + r + R) * NB + o;
#pragma unroll
          for (int p = 1; p <= R; ++p) {
            const float2 u = ld2(col + (yl + R + p) * RP);
            const float2 d = ld2(col + (yl + R - p) * RP);
            sx = __ffma2_rn(a.cx2[p], __fadd2_rn(w[R + r + p], w[R + r - p]), sx);
            sy = __ffma2_rn(a.cy2[p], __fadd2_rn(u, d), sy);
            sz = __ffma2_rn(a.cz2[p], __fadd2_rn(q[(sidx + R + p) % Q][r], q[(sidx + R - p) % Q][r]), sz);
          }
          acc[r] = __fadd2_rn(sx, __fadd2_rn(sy, sz));
        }
        // nonlocal: sum over the pieces active at (z, this row group) of
        // sum_l chi_l(node) (phase gc_l)(orbital)
        const int ea = steps[sidx * NRG + yg], eb = steps[sidx * NRG + yg + 1];
        const int x0r = tx0 + xl0;
        for (int e = ea; e < eb; ++e) {
          const int it = steps[NL + 1 + e];
          const int4 pa = *reinterpret_cast<const int4*>(&desc[it].gy0);   // gy0 gy1 gx0 gx1
          if (gy < pa.x || gy >= pa.y) continue;
          const int4 pb = *reinterpret_cast<const int4*>(&desc[it].base);  // base sy sz -
          const float2 g0 = ld2(gcs + (it * 4 + 0) * NB + o), g1 = ld2(gcs + (it * 4 + 1) * NB + o);
          const float2 g2 = ld2(gcs + (it * 4 + 2) * NB + o), g3 = ld2(gcs + (it * 4 + 3) * NB + o);
          const int rowoff = pb.x + pb.y * gy + pb.z * z;
#pragma unroll
          for (int r = 0; r < RX2; ++r) {
            const int gx = x0r + r;
            if (gx < pa.z || gx >= pa.w) continue;
            const float4 c4 = __ldg(S.chi4 + rowoff + gx);
            acc[r] = __ffma2_rn(f2(c4.x), g0, acc[r]);
            acc[r] = __ffma2_rn(f2(c4.y), g1, acc[r]);
            acc[r] = __ffma2_rn(f2(c4.z), g2, acc[r]);
            acc[r] = __ffma2_rn(f2(c4.w), g3, acc[r]);
          }
        }
        // recurrence epilogue
        const cf32* Pp = yps + (size_t)b * TYC * TX * NB + (yl * TX + xl0) * NB + o;
        cf32* out = Yout + boff + (size_t)z * plane_el + ((size_t)gy * n1 + tx0 + xl0) * NB + o;
#pragma unroll
        for (int r = 0; r < RX2; ++r) {
          if (!vr[r]) continue;
          float2 v = __fmul2_rn(alpha2, acc[r]);
          if (Yprev) v = __ffma2_rn(beta2, ld2(Pp + r * NB), v);
          *reinterpret_cast<float2*>(out + r * NB) = v;
        }
      }
      if (z + 1 < ze) own(q[(sidx + R + 1) % Q], (sidx + 1) % 3);
      if (z + 2 < ze) issue(z + 2, (sidx + 2) % 3);
      cp_commit();
      load_z(z + R + 1, q[sidx % Q]);   // plane z - R is no longer needed
      cp_wait1();
      if (z + 1 < ze) fixup(z + 1, (sidx + 1) % 3);
      __syncthreads();
      }
    }
  }
}

// s[b][l] += sum over this lane's nodes ix = xi, xi+4, .. < wx of chi_l(ix) Y_b(ix).
// The row is taken in chunks of 4 NXS nodes; every load of a chunk is issued
// before its first multiply, so a warp has (1 + NBM) NXS loads in flight.
template <class T, int NBM, int NXS>
__device__ __forceinline__ void gather_row(T (&s)[NBM][4], const float4* __restrict__ c, const T* __restrict__ y0,
                                           size_t bstride, int wx, int xi, int nbv) {
  for (int x0 = 0; x0 < wx; x0 += 4 * NXS) {
    float4 c4[NXS];
    T y[NXS][NBM];
#pragma unroll
    for (int u = 0; u < NXS; ++u) {
      const int ix = x0 + xi + 4 * u;
      const bool ok = ix < wx;
      c4[u] = ok ? __ldg(c + ix) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int b = 0; b < NBM; ++b)
        y[u][b] = (ok && b < nbv) ? fld(y0 + b * bstride + (size_t)ix * NB) : FT<T>::zero();
    }
#pragma unroll
    for (int u = 0; u < NXS; ++u)
#pragma unroll
      for (int b = 0; b < NBM; ++b) {
        if constexpr (FT<T>::cplx) {   // (re, im) packed: one FFMA2 per projector
          const float2 yv = make_float2(y[u][b].x, y[u][b].y);
          const float cl[4] = {c4[u].x, c4[u].y, c4[u].z, c4[u].w};
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const float2 r = __ffma2_rn(make_float2(cl[l], cl[l]), yv, make_float2(s[b][l].x, s[b][l].y));
            s[b][l].x = r.x;
            s[b][l].y = r.y;
          }
        } else {
          s[b][0] = fmaf(c4[u].x, y[u][b], s[b][0]); s[b][1] = fmaf(c4[u].y, y[u][b], s[b][1]);
          s[b][2] = fmaf(c4[u].z, y[u][b], s[b][2]); s[b][3] = fmaf(c4[u].w, y[u][b], s[b][3]);
        }
      }
  }
}

// Projection by row slabs: CTA (group g, slab s, octet q) sums conj(chi~) Y over
// the box rows r of group g with r % nslab == s, for the blocks q*NBM .. q*NBM+NBM-1.
// A warp takes one box row at a time; lane = xi * 8 + o covers 4 x-consecutive
// nodes x 8 orbital lanes, so one load of a block is 4 contiguous 32-byte node
// groups and the chi values of those 4 nodes are read once for all NBM blocks.
// The row sums of a piece carry its constant phase; partial sums are reduced
// over xi by shuffles and over the 8 warps in shared memory, in a fixed order.
// Grid z runs over (k slot, octet of its nbk blocks); an octet never spans two k.
// part[((g * nslab + s) * 4 + l) * (nk * nbk * NB) + (kk * nbk + bi) * NB + lane] gets the CTA sum.
template <class T, int NBM>
__global__ void __launch_bounds__(256, 2)
k_gather_rows(const T* __restrict__ Y, long long nd, int rowp, int xoff, int n2, const Group* __restrict__ grp,
              const __grid_constant__ KSlots ks, T* __restrict__ part, int noct, int nslab) {
  __shared__ T red[8][NBM][4][NB];
  const int gi = blockIdx.x, sl = blockIdx.y;
  const int kk = blockIdx.z / noct, q = blockIdx.z % noct;
  const KSlot& S = ks.s[kk];
  const SubBox* __restrict__ sbs = S.sb;
  const float4* __restrict__ chi4 = S.chi4;
  const int nb = ks.nbk;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int o = lane % NB, xi = lane / NB;
  const int nbv = min(NBM, nb - q * NBM);   // valid blocks of this octet (uniform per CTA)
  const T* Yb = Y + (size_t)(S.ubase + q * NBM) * nd * NB + o;
  const size_t bstride = (size_t)nd * NB;
  const Group G = grp[gi];
  T acc[NBM][4];
#pragma unroll
  for (int b = 0; b < NBM; ++b)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[b][l] = FT<T>::zero();
  int rbase = 0;
  for (int sbi = G.sb0; sbi < G.sb1; ++sbi) {
    const SubBox sb = sbs[sbi];
    const int wx = sb.gx1 - sb.gx0, wy = sb.gy1 - sb.gy0, wz = sb.gz1 - sb.gz0;
    const int rows = wy * wz;
    const int first = (sl - rbase % nslab + nslab) % nslab;
    for (int row = first + warp * nslab; row < rows; row += 8 * nslab) {
      const int iy = row % wy, iz = row / wy;
      const long long yrow = ((long long)(sb.gz0 + iz) * n2 + (sb.gy0 + iy)) * rowp + sb.gx0 + xoff;
      const long long crow =
          sb.chi4_off + sb.bx0 + (long long)sb.nbx * ((sb.by0 + iy) + (long long)sb.nby * (sb.bz0 + iz));
      if constexpr (FT<T>::cplx) {
        T s[NBM][4];
#pragma unroll
        for (int b = 0; b < NBM; ++b)
#pragma unroll
          for (int l = 0; l < 4; ++l) s[b][l] = FT<T>::zero();
        gather_row<T, NBM, FT<T>::cplx ? 3 : 5>(s, chi4 + crow, Yb + (size_t)yrow * NB, bstride, wx, xi, nbv);
#pragma unroll
        for (int b = 0; b < NBM; ++b)
#pragma unroll
          for (int l = 0; l < 4; ++l) {   // conj(phase) of this piece
            acc[b][l].x += sb.ph_re * s[b][l].x + sb.ph_im * s[b][l].y;
            acc[b][l].y += sb.ph_re * s[b][l].y - sb.ph_im * s[b][l].x;
          }
      } else {
        // real data: k = 0, every phase is 1; accumulate in place
        gather_row<T, NBM, 5>(acc, chi4 + crow, Yb + (size_t)yrow * NB, bstride, wx, xi, nbv);
      }
    }
    rbase += rows;
  }
  // reduce over the 4 x-lanes (xi) of each orbital lane: fixed butterfly order
#pragma unroll
  for (int b = 0; b < NBM; ++b)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if constexpr (FT<T>::cplx) {
        acc[b][l].x += __shfl_xor_sync(0xffffffffu, acc[b][l].x, 8);
        acc[b][l].y += __shfl_xor_sync(0xffffffffu, acc[b][l].y, 8);
        acc[b][l].x += __shfl_xor_sync(0xffffffffu, acc[b][l].x, 16);
        acc[b][l].y += __shfl_xor_sync(0xffffffffu, acc[b][l].y, 16);
      } else {
        acc[b][l] += __shfl_xor_sync(0xffffffffu, acc[b][l], 8);
        acc[b][l] += __shfl_xor_sync(0xffffffffu, acc[b][l], 16);
      }
    }
  if (xi == 0) {
#pragma unroll
    for (int b = 0; b < NBM; ++b)
#pragma unroll
      for (int l = 0; l < 4; ++l) red[warp][b][l][o] = acc[b][l];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NBM * 4 * NB; t += blockDim.x) {   // fixed order over warps
    const int oo = t % NB, l = (t / NB) % 4, b = t / (4 * NB);
    if (b >= nbv) continue;
    T v = red[0][b][l][oo];
    for (int w2 = 1; w2 < 8; ++w2) {
      if constexpr (FT<T>::cplx) { v.x += red[w2][b][l][oo].x; v.y += red[w2][b][l][oo].y; }
      else v += red[w2][b][l][oo];
    }
    const int bi = kk * nb + q * NBM + b;
    part[((size_t)(gi * nslab + sl) * 4 + l) * ((size_t)ks.nk * nb * NB) + (size_t)bi * NB + oo] = v;
  }
}

// FP32 projection with pairs of blocks packed in float2 (one FFMA2 per projector and
// node serves two blocks); same row slabs, lane layout and fixed-order reductions as
// k_gather_rows.  NB2 pairs = 2 NB2 blocks per CTA (grid z covers the rest).
template <int NB2>
__device__ __forceinline__ void gather_row_f2(float2 (&s)[NB2][4], const float4* __restrict__ c,
                                              const float* __restrict__ y0, size_t bstride, int wx, int xi,
                                              int nbv) {
  constexpr int NXS = 5;
  for (int x0 = 0; x0 < wx; x0 += 4 * NXS) {
    float4 c4[NXS];
    float2 y[NXS][NB2];
#pragma unroll
    for (int u = 0; u < NXS; ++u) {
      const int ix = x0 + xi + 4 * u;
      const bool ok = ix < wx;
      c4[u] = ok ? __ldg(c + ix) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NB2; ++j) {
        const float* p = y0 + (size_t)(2 * j) * bstride + (size_t)ix * NB;
        y[u][j].x = (ok && 2 * j < nbv) ? __ldg(p) : 0.f;
        y[u][j].y = (ok && 2 * j + 1 < nbv) ? __ldg(p + bstride) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < NXS; ++u)
#pragma unroll
      for (int j = 0; j < NB2; ++j) {
        s[j][0] = __ffma2_rn(f2(c4[u].x), y[u][j], s[j][0]);
        s[j][1] = __ffma2_rn(f2(c4[u].y), y[u][j], s[j][1]);
        s[j][2] = __ffma2_rn(f2(c4[u].z), y[u][j], s[j][2]);
        s[j][3] = __ffma2_rn(f2(c4[u].w), y[u][j], s[j][3]);
      }
  }
}

// rowp, xoff: row length and x offset of the block buffer (n1 and 0, or n1 + 12 and 6
// for the x-padded layout of the TMA pass); nd: nodes per block of that layout.
template <int NB2>
__global__ void __launch_bounds__(256, 2)
k_gather_rows_f2(const float* __restrict__ Y, long long nd, int rowp, int xoff, int n2, const Group* __restrict__ grp,
                 const SubBox* __restrict__ sbs, const float4* __restrict__ chi4, float* __restrict__ part,
                 int blk0, int nb, int nslab) {
  constexpr int NBM = 2 * NB2;
  __shared__ float red[8][NBM][4][NB];
  const int gi = blockIdx.x, sl = blockIdx.y, q = blockIdx.z;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int o = lane % NB, xi = lane / NB;
  const int nbv = min(NBM, nb - q * NBM);
  const float* Yb = Y + (size_t)(blk0 + q * NBM) * nd * NB + o;
  const size_t bstride = (size_t)nd * NB;
  const Group G = grp[gi];
  float2 acc[NB2][4];
#pragma unroll
  for (int j = 0; j < NB2; ++j)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[j][l] = make_float2(0.f, 0.f);
  int rbase = 0;
  for (int sbi = G.sb0; sbi < G.sb1; ++sbi) {
    const SubBox sb = sbs[sbi];
    const int wx = sb.gx1 - sb.gx0, wy = sb.gy1 - sb.gy0, wz = sb.gz1 - sb.gz0;
    const int rows = wy * wz;
    const int first = (sl - rbase % nslab + nslab) % nslab;
    for (int row = first + warp * nslab; row < rows; row += 8 * nslab) {
      const int iy = row % wy, iz = row / wy;
      const long long yrow = ((long long)(sb.gz0 + iz) * n2 + (sb.gy0 + iy)) * rowp + sb.gx0 + xoff;
      const long long crow =
          sb.chi4_off + sb.bx0 + (long long)sb.nbx * ((sb.by0 + iy) + (long long)sb.nby * (sb.bz0 + iz));
      // real data: k = 0, every phase is 1; accumulate in place
      gather_row_f2<NB2>(acc, chi4 + crow, Yb + (size_t)yrow * NB, bstride, wx, xi, nbv);
    }
    rbase += rows;
  }
#pragma unroll
  for (int j = 0; j < NB2; ++j)
#pragma unroll
    for (int l = 0; l < 4; ++l) {   // over the 4 x-lanes: fixed butterfly order
      acc[j][l].x += __shfl_xor_sync(0xffffffffu, acc[j][l].x, 8);
      acc[j][l].y += __shfl_xor_sync(0xffffffffu, acc[j][l].y, 8);
      acc[j][l].x += __shfl_xor_sync(0xffffffffu, acc[j][l].x, 16);
      acc[j][l].y += __shfl_xor_sync(0xffffffffu, acc[j][l].y, 16);
    }
  if (xi == 0) {
#pragma unroll
    for (int j = 0; j < NB2; ++j)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        red[warp][2 * j][l][o] = acc[j][l].x;
        red[warp][2 * j + 1][l][o] = acc[j][l].y;
      }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NBM * 4 * NB; t += blockDim.x) {   // fixed order over warps
    const int oo = t % NB, l = (t / NB) % 4, b = t / (4 * NB);
    if (b >= nbv) continue;
    float v = red[0][b][l][oo];
    for (int w2 = 1; w2 < 8; ++w2) v += red[w2][b][l][oo];
    const int bi = q * NBM + b;
    part[((size_t)(gi * nslab + sl) * 4 + l) * ((size_t)nb * NB) + bi * NB + oo] = v;
  }
}

// gc[p][blk][lane] = gamma_p h^3 sum_s part[g][s][l][bi][lane] (fixed order over slabs)
template <class T>
__global__ void k_gather_sum(const T* __restrict__ part, const Group* __restrict__ grp,
                             const float* __restrict__ gamma, float dv, T* __restrict__ gc, int ngrp,
                             int nslab, int nblk_total, int blk0, int nb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = 4LL * nb * NB;
  if (t >= (long long)ngrp * per) return;
  const int gi = (int)(t / per);
  const int rem = (int)(t % per);
  const int l = rem / (nb * NB), bi = (rem / NB) % nb, o = rem % NB;
  const int p = grp[gi].proj[l];
  if (p < 0) return;
  T v = FT<T>::zero();
  for (int s = 0; s < nslab; ++s) {
    const T x = part[((size_t)(gi * nslab + s) * 4 + l) * ((size_t)nb * NB) + bi * NB + o];
    if constexpr (FT<T>::cplx) { v.x += x.x; v.y += x.y; }
    else v += x;
  }
  const float f = gamma[p] * dv;
  if constexpr (FT<T>::cplx) v = cf32{f * v.x, f * v.y};
  else v = f * v;
  gc[((size_t)p * nblk_total + blk0 + bi) * NB + o] = v;
}

// The same for the units of a k batch: gamma per k, unit ubase(kk) + bi.
__global__ void k_gather_sum_k(const cf32* __restrict__ part, const Group* __restrict__ grp,
                               const __grid_constant__ KSlots ks, float dv, cf32* __restrict__ gc, int ngrp,
                               int nslab, long long nunit_total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = ks.nk * ks.nbk;
  const long long per = 4LL * nu * NB;
  if (t >= (long long)ngrp * per) return;
  const int gi = (int)(t / per);
  const int rem = (int)(t % per);
  const int l = rem / (nu * NB), uu = (rem / NB) % nu, o = rem % NB;
  const int p = grp[gi].proj[l];
  if (p < 0) return;
  const KSlot& S = ks.s[uu / ks.nbk];
  float vx = 0.f, vy = 0.f;
  for (int s = 0; s < nslab; ++s) {
    const cf32 x = part[((size_t)(gi * nslab + s) * 4 + l) * ((size_t)nu * NB) + (size_t)uu * NB + o];
    vx += x.x;
    vy += x.y;
  }
  const float f = S.gamma[p] * dv;
  gc[((size_t)p * nunit_total + S.ubase + uu % ks.nbk) * NB + o] = cf32{f * vx, f * vy};
}

// --------------------------------------------------------------------------- launchers

constexpr int NSLAB_MAX = 16;
constexpr int GATHER_OCT_C = 4;   // complex64 blocks per projection CTA
// Complex64: row slabs per projector group such that the blocks of one k give about six
// CTAs per SM (at most 16).  From the k's block count, not the launch's units, so that a
// batch over k and the per-k filter sum in the same order.
static int gather_slabs(const sparc_ham* H, int nblk_k) {
  const Tables* Tb = (const Tables*)H->fast;
  const int want = 6 * H->ctx->nsm;
  const int octs = std::max(1, ceil_div(nblk_k, GATHER_OCT_C));
  return std::max(1, std::min(NSLAB_MAX, ceil_div(want, std::max(1, Tb->ngrp) * octs)));
}
// FP32: slabs from the total block count (8 blocks per CTA at most), not the blocks of
// one launch, so that every grouping of the same filter sums in the same order.
static int gather_slabs_f2(const sparc_ham* H, int nblk_total) {
  const Tables* Tb = (const Tables*)H->fast;
  const int want = 6 * H->ctx->nsm;
  const int octs = std::max(1, ceil_div(nblk_total, 8));
  return std::max(1, std::min(NSLAB_MAX, ceil_div(want, std::max(1, Tb->ngrp) * octs)));
}

size_t gather_scratch_bytes(const sparc_ham* H, int nb, size_t esize) {
  const Tables* Tb = (const Tables*)H->fast;
  return (size_t)std::max(1, Tb->ngrp) * NSLAB_MAX * 4 * nb * NB * esize;
}

cudaError_t launch_gather_k(const sparc_ham* H0, const cf32* Y, long long nunit_total, const KSlots& ks, int nblk_k,
                            cf32* gc, cf32* scratch, cudaStream_t st, bool padded) {
  const Tables* Tb = (const Tables*)H0->fast;
  if (H0->nproj == 0 || Tb->ngrp == 0) return cudaSuccess;
  const float dv = (float)(H0->grid.h[0] * H0->grid.h[1] * H0->grid.h[2]);
  const int nslab = gather_slabs(H0, nblk_k);
  cudaEvent_t t0 = timing_begin(H0->ctx, st);
  constexpr int NBM = GATHER_OCT_C;
  const int noct = ceil_div(ks.nbk, NBM);
  const dim3 grid((unsigned)Tb->ngrp, (unsigned)nslab, (unsigned)(ks.nk * noct));
  const int rowp = padded ? H0->gd.n1 + 2 * R : H0->gd.n1;
  const long long ndl = (long long)rowp * H0->gd.n2 * H0->gd.n3;
  k_gather_rows<cf32, NBM><<<grid, 256, 0, st>>>(Y, ndl, rowp, padded ? R : 0, H0->gd.n2, Tb->d_grp, ks, scratch,
                                                 noct, nslab);
  const long long tot = (long long)Tb->ngrp * 4 * ks.nk * ks.nbk * NB;
  k_gather_sum_k<<<ceil_div(tot, 256), 256, 0, st>>>(scratch, Tb->d_grp, ks, dv, gc, Tb->ngrp, nslab,
                                                      nunit_total);
  H0->ctx->launches += 2;
  timing_end(H0->ctx, TK_GATHER, t0, st);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_gather(const sparc_ham* H, const T* Y, int nblk_total, int blk0, int nb, T* gc,
                          T* scratch, cudaStream_t st, bool padded) {
  const Tables* Tb = (const Tables*)H->fast;
  if (H->nproj == 0 || Tb->ngrp == 0) return cudaSuccess;
  if constexpr (FT<T>::cplx) {
    KSlots ks;
    ks.nk = 1;
    ks.nbk = nb;
    kslot(H, ks.s[0]);
    ks.s[0].ubase = blk0;
    ks.s[0].alpha = ks.s[0].shift = ks.s[0].beta = 0.f;
    return launch_gather_k(H, Y, nblk_total, ks, nblk_total, gc, scratch, st, padded);
  } else {
    const float dv = (float)(H->grid.h[0] * H->grid.h[1] * H->grid.h[2]);
    const int nslab = gather_slabs_f2(H, nblk_total);
    cudaEvent_t t0 = timing_begin(H->ctx, st);
    // pairs of blocks per CTA: as many as the group has, at most 4 pairs
    const int nb2 = std::min(4, (nb + 1) / 2);
    const dim3 grid((unsigned)Tb->ngrp, (unsigned)nslab, (unsigned)ceil_div(nb, 2 * nb2));
    const int rowp = padded ? H->gd.n1 + 2 * R : H->gd.n1;
    const long long ndl = (long long)rowp * H->gd.n2 * H->gd.n3;
    auto go = [&](auto kern) {
      kern<<<grid, 256, 0, st>>>(Y, ndl, rowp, padded ? R : 0, H->gd.n2, Tb->d_grp, Tb->d_sb,
                                 (const float4*)Tb->d_chi4, scratch, blk0, nb, nslab);
    };
    switch (nb2) {
      case 1: go(k_gather_rows_f2<1>); break;
      case 2: go(k_gather_rows_f2<2>); break;
      case 3: go(k_gather_rows_f2<3>); break;
      default: go(k_gather_rows_f2<4>); break;
    }
    const long long tot = (long long)Tb->ngrp * 4 * nb * NB;
    k_gather_sum<T><<<ceil_div(tot, 256), 256, 0, st>>>(scratch, Tb->d_grp, H->d_gamma32, dv, gc, Tb->ngrp,
                                                        nslab, nblk_total, blk0, nb);
    H->ctx->launches += 2;
    timing_end(H->ctx, TK_GATHER, t0, st);
    return cudaGetLastError();
  }
}

// Geometry and stencil fields of the pass arguments (shared by every k of a batch).
static PassArgs pass_args(const sparc_ham* H, const Layout& Lo) {
  PassArgs a;
  a.nd = H->gd.nd;
  a.n1 = H->gd.n1; a.n2 = H->gd.n2; a.n3 = H->gd.n3;
  a.tiles_x = Lo.tiles_x;
  a.nchunk = Lo.nchunk;
  a.blk0 = 0;
  a.nblk_total = 0;
  for (int p = 0; p <= R; ++p) {
    a.cx[p] = (float)H->gd.coef[0][p];
    a.cy[p] = (float)H->gd.coef[1][p];
    a.cz[p] = (float)H->gd.coef[2][p];
  }
  a.c0 = (float)(2.0 * (H->gd.coef[0][0] + H->gd.coef[1][0] + H->gd.coef[2][0]));
  a.phx_r = (float)H->gd.ph_re[0]; a.phx_i = (float)H->gd.ph_im[0];
  a.phy_r = (float)H->gd.ph_re[1]; a.phy_i = (float)H->gd.ph_im[1];
  a.phz_r = (float)H->gd.ph_re[2]; a.phz_i = (float)H->gd.ph_im[2];
  a.alpha = a.shift = a.beta = 0.f;
  for (int p = 0; p <= R; ++p) {
    a.cx2[p] = make_float2(a.cx[p], a.cx[p]);
    a.cy2[p] = make_float2(a.cy[p], a.cy[p]);
    a.cz2[p] = make_float2(a.cz[p], a.cz[p]);
  }
  a.alpha2 = a.beta2 = make_float2(0.f, 0.f);
  a.veff = H->d_veff32;
  const Tables* Tb = (const Tables*)H->fast;
  a.cptr = Lo.d_cptr; a.citems = Lo.d_citems; a.sptr = Lo.d_sptr; a.sslots = Lo.d_sslots;
  a.sb = Tb->d_sb; a.grp = Tb->d_grp;
  a.chi4 = (const float4*)Tb->d_chi4;
  return a;
}

cudaError_t launch_pass_k(const sparc_ham* H0, const cf32* Yin, const cf32* Yprev, cf32* Yout, const cf32* gc,
                          long long nunit_total, const KSlots& ks, cudaStream_t st) {
  const Tables* Tb = (const Tables*)H0->fast;
  const Layout& Lo = Tb->lay[1];
  PassArgs a = pass_args(H0, Lo);
  a.nblk_total = (int)nunit_total;
  const size_t smem = Smem<cf32>::total;
  cudaError_t e = cudaFuncSetAttribute(k_pass_c2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // persistent CTAs over (tile, chunk, unit) items
  const int nitems = Lo.tiles_x * Lo.tiles_y * Lo.nchunk * ks.nk * ks.nbk;
  cudaEvent_t t0 = timing_begin(H0->ctx, st);
  k_pass_c2<<<std::min(nitems, std::max(H0->ctx->nsm, 1)), THREADS, smem, st>>>(a, ks, Yin, Yprev, Yout, gc, nitems);
  ++H0->ctx->launches;
  timing_end(H0->ctx, TK_FPASS, t0, st);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_pass(const sparc_ham* H, const T* Yin, const T* Yprev, T* Yout, const T* gc,
                        int nblk_total, int blk0, int nb, double alpha, double shift, double beta,
                        cudaStream_t st, int shape) {
  if constexpr (FT<T>::cplx) {
    KSlots ks;
    ks.nk = 1;
    ks.nbk = nb;
    kslot(H, ks.s[0]);
    ks.s[0].ubase = blk0;
    ks.s[0].alpha = (float)alpha; ks.s[0].shift = (float)shift; ks.s[0].beta = (float)beta;
    return launch_pass_k(H, Yin, Yprev, Yout, gc, nblk_total, ks, st);
  } else {
    const Tables* Tb = (const Tables*)H->fast;
    const bool half = shape == 1 && shape_usable(H, 1);
    const bool diff = shape == SHAPE_DIFF;
    const Layout& Lo = Tb->lay[half ? 2 : 0];
    PassArgs a = pass_args(H, Lo);
    a.blk0 = blk0;
    a.nblk_total = nblk_total;
    a.alpha = (float)alpha; a.shift = (float)shift; a.beta = (float)beta;
    a.alpha2 = make_float2(a.alpha, a.alpha);
    a.beta2 = make_float2(a.beta, a.beta);
    // persistent CTAs over (tile, chunk, block) items
    const int nitems = Lo.tiles_x * Lo.tiles_y * Lo.nchunk * nb;
    const int nsm = std::max(H->ctx->nsm, 1);
    cudaEvent_t t0 = nullptr;
    if (half) {
      constexpr size_t smem = Smem<float, 8>::total;
      cudaError_t e = cudaFuncSetAttribute(k_pass_f2<8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      t0 = timing_begin(H->ctx, st);
      k_pass_f2<8, 256><<<std::min(nitems, 2 * nsm), 256, smem, st>>>(a, Yin, Yprev, Yout, gc, nitems);
    } else if (diff) {
      constexpr size_t smem = Smem<float, 16>::total;
      cudaError_t e =
          cudaFuncSetAttribute(k_pass_f2<16, 512, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      t0 = timing_begin(H->ctx, st);
      k_pass_f2<16, 512, true><<<std::min(nitems, nsm), 512, smem, st>>>(a, Yin, Yprev, Yout, gc, nitems);
    } else {
      constexpr size_t smem = Smem<float, 16>::total;
      cudaError_t e = cudaFuncSetAttribute(k_pass_f2<16, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      t0 = timing_begin(H->ctx, st);
      k_pass_f2<16, 512><<<std::min(nitems, nsm), 512, smem, st>>>(a, Yin, Yprev, Yout, gc, nitems);
    }
    ++H->ctx->launches;
    timing_end(H->ctx, diff ? TK_HPASS : TK_FPASS, t0, st);   // the plain H-apply is not a filter pass
    return cudaGetLastError();
  }
}

template <class T>
int items_per_block(const sparc_ham* H, int shape) {
  const int li = FT<T>::cplx ? 1 : (shape == 1 && shape_usable(H, 1)) ? 2 : 0;
  const Layout& Lo = ((const Tables*)H->fast)->lay[li];
  return Lo.tiles_x * Lo.tiles_y * Lo.nchunk;
}
template int items_per_block<float>(const sparc_ham*, int);
template int items_per_block<cf32>(const sparc_ham*, int);

template cudaError_t launch_gather<float>(const sparc_ham*, const float*, int, int, int, float*, float*, cudaStream_t,
                                          bool);
template cudaError_t launch_gather<cf32>(const sparc_ham*, const cf32*, int, int, int, cf32*, cf32*, cudaStream_t,
                                         bool);
template cudaError_t launch_pass<float>(const sparc_ham*, const float*, const float*, float*, const float*,
                                        int, int, int, double, double, double, cudaStream_t, int);
template cudaError_t launch_pass<cf32>(const sparc_ham*, const cf32*, const cf32*, cf32*, const cf32*,
                                       int, int, int, double, double, double, cudaStream_t, int);

}  // namespace fast
}  // namespace sparc
