// Tensor-core products of Rayleigh-Ritz for FP32 and complex64 orbitals (Section 3.4: the
// projections of Eq. SubspaceGeneralizedEigenproblem and the rotation of Eq.
// OrbitalTransformation) on sm_103a.
//
// tcgen05.mma kind::tf32 with the accumulator in tensor memory (TMEM).  Operands
// are staged in shared memory in the canonical K-major layout with the 128-byte
// swizzle (rows of 32 FP32 values, 8-row groups 1024 bytes apart).  Products
// are error-compensated ("3xTF32"):
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
// where a_hi is a rounded to the nearest TF32 value (10 stored mantissa bits) and
// a_lo = a - a_hi exactly; a_lo b_lo (relative size 2^-22; over a sum of squares a
// bias of about 4e-8) is dropped in the rotation and kept in the Grams (four
// products), whose sums decide the Ritz values.
//
// Gram  G = A^T B (Ns x Ns, FP64): one CTA per (upper-triangular 128 x 128 tile
//   pair, split of the Nd range); the CTA accumulates 2^gsh k-tiles at a time in
//   TMEM (FP32; a_hi b_hi and the cross terms in separate accumulators) and adds
//   each chunk in FP64 to its own partial; a second kernel
//   sums the splits in a fixed order and mirrors the tiles, so the result is
//   deterministic.
// Rotation  C = U Yr (Nd x Ns): one CTA per (128 grid rows, 256 columns); Yr is
//   split and swizzled once into its shared-memory images, U is split and
//   transposed to K-major on its way into shared memory.
// Complex64 orbitals (k-points, Section 3.3) take the same kernels on their real
// views: a column of nd complex values is a column of 2 nd FP32 values (real and
// imaginary parts interleaved along the grid index).  For columns u, v with real
// views r(u), r(v), and i v = (-Im v, Re v) interleaved the same way,
//   Re(u^H v) = r(u) . r(v),   Im(u^H v) = -r(u) . r(i v),
// so a complex Gram is two real Grams of 2 nd rows (the second of an antisymmetric
// matrix), and the rotation U Q = r(U) Re Q + r(i U) Im Q is one real rotation with
// 2 Ns values of k, the i U half formed as U is loaded.  Four real products per
// complex one, all on the tensor cores.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "ptx.cuh"
#include "rr.cuh"

namespace sparc {
namespace tc {
namespace {

constexpr int BM = 128;        // MMA M: rows of D = TMEM lanes
constexpr int BK = 32;         // k-tile: 32 FP32 values = one 128-byte swizzled row
constexpr int THREADS = 256;   // rotation CTA
constexpr int GTHREADS = 512;  // Gram CTA: 16 warps split, swizzle and stage the operands
constexpr int GN = 128;        // Gram tile N
constexpr int GST = 3;         // Gram pipeline stages
// Gram k-tiles per FP32 accumulation chunk, 2^gsh: 2 (64 grid points), or 8 (256)
// where the Gram only has to be good to FP32 accuracy (the first orthonormalisation,
// which the second corrects).  The tensor core's FP32 accumulation rounds toward zero:
// a sum of like-signed products (each diagonal entry of M~, most of H~'s, columns
// close to parallel) comes out low, by 6e-7 of itself over chunks of 8 k-tiles (32
// MMAs, measured) against 2.5e-7 over chunks of 2.  A bias the same for every entry of
// M~ and H~ would leave the Ritz values alone, but it is not (H~'s sums are partly of
// mixed sign): on the 64^3 cell the mixed Ritz values were 7.6e-7 Ha from the FP64
// path's with chunks of 8 (and a truncated split), 1.7e-7 with chunks of 2.
constexpr int GCH_ACC_LOG = 1;    // 2 k-tiles
constexpr int GCH_FAST_LOG = 3;   // 8 k-tiles
constexpr int RN = 256;        // rotation tile N
constexpr int RST = 2;         // rotation pipeline stages
constexpr int TILE_A = BM * BK * 4;   // 16 KB: one 128-row operand image
constexpr int GSTAGE = 4 * TILE_A;    // A_hi, A_lo, B_hi, B_lo
constexpr int RSTAGE = 2 * TILE_A + 2 * (RN * BK * 4);
constexpr int GSMEM = GST * GSTAGE + 1024;
constexpr int RSMEM = RST * RSTAGE + 1024;

// ------------------------------------------------------------------ PTX wrappers
using ptx::mbar_init;
using ptx::mbar_wait;
using ptx::saddr;
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {   // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {     // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// arrive once on `bar` when every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
// thread l of the warp reads TMEM lane (lane field of taddr) + l, 32 consecutive columns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// two loads of 16 consecutive columns (at taddr0 and taddr1), one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr0, uint32_t taddr1, float (&v)[16], float (&w)[16]) {
  uint32_t r[16], u[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr0));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
               : "r"(taddr1));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) { v[i] = __uint_as_float(r[i]); w[i] = __uint_as_float(u[i]); }
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B
// apart (stride byte offset), descriptor version 1, base offset 0 (operand images
// start on 1024-byte boundaries; the start address advances 32 B per K = 8 step).
__device__ __forceinline__ uint64_t desc_k128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// byte offset of 16-byte chunk c (0..7) of row r in a swizzled operand image
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// x = hi + lo: hi is x rounded to the nearest TF32 value (10 stored mantissa bits;
// on the magnitude bits: add half a unit of the last kept bit, clear the 13 bits
// below; ties, one x in 2^13, go away from zero), lo = x - hi exactly (|lo| <= 2^-11
// |x|, up to 12 significant bits, of either sign).  The tensor core reads lo to 11
// significant bits, truncating at most one, so the product's error is about 2^-22 of
// it and, lo being as often negative as positive, without bias.  (Truncating x to hi
// instead leaves lo with the sign of x: the dropped parts of every square then add
// up, about 2e-7 low over a sum of squares.)
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}
__device__ __forceinline__ void split4(float4 x, float4& hi, float4& lo) {
  split(x.x, hi.x, lo.x); split(x.y, hi.y, lo.y); split(x.z, hi.z, lo.z); split(x.w, hi.w, lo.w);
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}

// Issue the MMAs of one k-tile (4 K-steps x 3 products, x 4 with LOLO): a_hi b_hi
// into d, the small products into ds (ds == d accumulates them all together).  The
// tensor core's FP32 accumulation rounds each addition, so keeping the small terms
// apart from the large one, and the chunks short, bounds the accumulated rounding.
template <bool LOLO = false>
__device__ __forceinline__ void mma_ktile(uint32_t d, uint32_t ds, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, uint32_t idesc, bool overwrite) {
#pragma unroll
  for (int kk = 0; kk < BK / 8; ++kk) {
    const uint64_t ah = desc_k128(a_hi + kk * 32), al = desc_k128(a_lo + kk * 32);
    const uint64_t bh = desc_k128(b_hi + kk * 32), bl = desc_k128(b_lo + kk * 32);
    const bool first = overwrite && kk == 0;
    mma_tf32(d, ah, bh, idesc, first ? 0u : 1u);
    mma_tf32(ds, ah, bl, idesc, (first && ds != d) ? 0u : 1u);
    mma_tf32(ds, al, bh, idesc, 1u);
    if (LOLO) mma_tf32(ds, al, bl, idesc, 1u);
  }
}

// ------------------------------------------------------------------ Gram
// Load one k-tile (rows i0..i0+127 of A^T and j0..j0+127 of B^T, grid points
// g0..g0+31) into registers: thread t holds 16-byte chunks f = t + GTHREADS q,
// row f / 8, chunk f % 8.  Out-of-range rows or points read as zero.
constexpr int GQ = BM * 8 / GTHREADS;   // chunks per thread and operand
template <bool VEC>
__device__ __forceinline__ void gram_load(const float* __restrict__ X, long long ldx, int r0, int ns, long long nd,
                                          long long g0, float4 (&v)[GQ]) {
#pragma unroll
  for (int q = 0; q < GQ; ++q) {
    const int f = threadIdx.x + GTHREADS * q;
    const int r = f >> 3, c = f & 7;
    const long long g = g0 + 4 * c;
    const bool rok = r0 + r < ns;
    const float* p = X + (long long)(r0 + r) * ldx + g;
    if (VEC) {
      v[q] = (rok && g < nd) ? __ldg((const float4*)p) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      v[q].x = (rok && g + 0 < nd) ? __ldg(p + 0) : 0.f;
      v[q].y = (rok && g + 1 < nd) ? __ldg(p + 1) : 0.f;
      v[q].z = (rok && g + 2 < nd) ? __ldg(p + 2) : 0.f;
      v[q].w = (rok && g + 3 < nd) ? __ldg(p + 3) : 0.f;
    }
  }
}
__device__ __forceinline__ void gram_store(uint8_t* hi, uint8_t* lo, const float4 (&v)[GQ]) {
#pragma unroll
  for (int q = 0; q < GQ; ++q) {
    const int f = threadIdx.x + GTHREADS * q;
    const uint32_t off = swz(f >> 3, f & 7);
    float4 h, l;
    split4(v[q], h, l);
    *(float4*)(hi + off) = h;
    *(float4*)(lo + off) = l;
  }
}

// part[(blockIdx.x * nsplit + split)][j][i] = sum over this CTA's grid points of
// A[g][ti*128 + i] B[g][tj*128 + j]  (tile pair blockIdx.x = (ti <= tj), split = blockIdx.y)
template <bool VEC>
__global__ void __launch_bounds__(GTHREADS, 1)
k_gram_tc(const float* __restrict__ A, long long lda, const float* __restrict__ B, long long ldb, long long nd,
          int ns, int nt, int nsplit, double* __restrict__ part, int* status, int gsh) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar[GST];
  __shared__ uint32_t tmem_base;
  const uint32_t raw = saddr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  int pr = blockIdx.x, ti = 0;
  while (pr >= nt - ti) { pr -= nt - ti; ++ti; }
  const int tj = ti + pr;
  const int sp = blockIdx.y;
  const long long nkt_all = (nd + BK - 1) / BK;
  const long long kt0 = nkt_all * sp / nsplit;
  const int nkt = (int)(nkt_all * (sp + 1) / nsplit - kt0);
  double* P = part + (size_t)(blockIdx.x * nsplit + sp) * (BM * GN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nkt <= 0) {   // empty split: a zero partial
    for (int e = threadIdx.x; e < BM * GN; e += GTHREADS) P[e] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < GST; ++s) mbar_init(&bar[s], 1);
    ptx::mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * GN);   // D (a_hi b_hi) and Ds (cross terms)
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t IDESC = idesc_tf32(BM, GN);
  const int i0 = ti * BM, j0 = tj * GN;
  float4 ca[GQ], cb[GQ], na[GQ], nb[GQ];
  gram_load<VEC>(A, lda, i0, ns, nd, kt0 * BK, ca);
  gram_load<VEC>(B, ldb, j0, ns, nd, kt0 * BK, cb);
  const int gm = (1 << gsh) - 1;   // a chunk is 2^gsh k-tiles
  bool first_flush = true, aborted = false;
  int last = -1;
  for (int t = 0; t < nkt; ++t) {
    const int s = t % GST;
    if (t + 1 < nkt) {
      gram_load<VEC>(A, lda, i0, ns, nd, (kt0 + t + 1) * BK, na);
      gram_load<VEC>(B, ldb, j0, ns, nd, (kt0 + t + 1) * BK, nb);
    }
    bool ok = true;
    if (t >= GST) ok = mbar_wait(&bar[s], (uint32_t)((t / GST) - 1) & 1u);   // MMAs of tile t - GST done
    uint8_t* st = sm + s * GSTAGE;
    gram_store(st, st + TILE_A, ca);
    gram_store(st + 2 * TILE_A, st + 3 * TILE_A, cb);
    proxy_fence();
    if (__syncthreads_or(!ok)) { aborted = true; break; }
    if (threadIdx.x == 0) {
      tc_after();
      const uint32_t b0 = saddr(st);
      mma_ktile<true>(tmem, tmem + GN, b0, b0 + TILE_A, b0 + 2 * TILE_A, b0 + 3 * TILE_A, IDESC, (t & gm) == 0);
      mma_commit(&bar[s]);
    }
    last = t;
#pragma unroll
    for (int q = 0; q < GQ; ++q) { ca[q] = na[q]; cb[q] = nb[q]; }
    if ((t & gm) == gm || t == nkt - 1) {
      // drain the FP32 chunk in TMEM into the FP64 partial
      ok = mbar_wait(&bar[s], (uint32_t)(t / GST) & 1u);
      tc_after();
      const int row = 32 * (warp & 3) + lane;
      const int c0 = (warp >> 2) * (GN * 4 / (GTHREADS / 32));   // warps 4q..4q+3 drain columns 32q..
#pragma unroll
      for (int h = 0; h < GN * 4 / GTHREADS; ++h) {
        float v[32], vs[32];
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 32 * h);
        tmem_ld32(ta, v);
        tmem_ld32(ta + GN, vs);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          double* p = P + (size_t)(c0 + 32 * h + c) * BM + row;
          const double x = (double)v[c] + (double)vs[c];
          *p = first_flush ? x : *p + x;
        }
      }
      first_flush = false;
      tc_before();
      if (__syncthreads_or(!ok)) { aborted = true; break; }
    }
  }
  if (aborted) {
    if (threadIdx.x == 0) {
      atomicOr(status, STATUS_TIMEOUT);
      if (last >= 0) mbar_wait(&bar[last % GST], (uint32_t)(last / GST) & 1u);
    }
    tc_before();
    __syncthreads();
  }
  tc_after();
  if (warp == 0) tmem_free(tmem, 2 * GN);
}

// ------------------------------------------------------------------ Gram, TMA-fed
// The same partials from a CTA of 16 warps fed by the tensor memory accelerator:
//   * loads: each k-tile of A and B (32 grid points x 128 columns, K-major: the
//     columns are contiguous in the grid index) arrives by cp.async.bulk.tensor in the
//     128-byte swizzle the MMA reads, into a ring of NH slots (four k-tiles in flight);
//   * warps 0..14 split each landed tile in place into its TF32 high part and the
//     remainder, whose images go to a ring of NL slots (a slot is free once the MMAs of
//     the k-tile NL before are done); all 16 warps, every 2^gsh k-tiles, drain the finished FP32 TMEM
//     chunk into float-float accumulators in registers (TwoSum: the GPU's FP64 rate
//     would make FP64 adds the bottleneck);
//   * the 16 MMAs of a k-tile (four products) go into one of two TMEM accumulator pairs,
//     alternating per chunk, so that a chunk drains while the next accumulates.
// Lane 0 of warp 15 issues the loads and the MMAs, as non-blocking steps in a loop that
// also drains that warp's share of each completed chunk; it splits no tiles, so an MMA
// goes out as soon as the last splitting warp arrives.  Every wait is bounded; one that
// runs out latches STATUS_TIMEOUT and raises the CTA's abort flag, and the CTA winds
// down (in-flight copies and MMAs waited for, with bounds) before it frees its TMEM.
constexpr int TTHREADS = 512;
constexpr int NCTL = 15;                       // the control warp; warps 0 .. NCTL-1 split tiles
constexpr int TST = 5;                         // NH: slots of landed (then high-part) images
constexpr int TLO = 2;                         // NL: slots of low-part images
constexpr int TSTAGE = 2 * TILE_A;             // A, B (32 KB)
constexpr int TSMEM = (TST + TLO) * TSTAGE + 1024;

__device__ __forceinline__ void tma2(uint32_t dst, const CUtensorMap* m, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst), "l"(m), "r"(c0), "r"(c1), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ void arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

struct GramRing {
  uint64_t full[TST], conv[TST], mmad[TST], accd[2], tfree[2];
  int abort_flag;
  // role state (one thread each): next k-tile to load (pt) and to multiply (mt)
  int pt, mt;
  int nkt, i0, j0, gsh;
  long long kt0;
  uint32_t tmem, sm;
};

// One non-blocking step of the load role (producer) or of the MMA role: issue what the
// barriers allow, return.  Kept out of line so that only the two role threads pay for
// its registers.
__device__ __noinline__ void gram_poll(GramRing* R, const CUtensorMap* ma, const CUtensorMap* mb, bool producer) {
  if (producer) {
    int pt = R->pt;
    while (pt < R->nkt) {   // a stage is free once the MMAs of its previous tile are done
      const int s = pt % TST;
      if (pt >= TST && !ptx::mbar_test(&R->mmad[s], (uint32_t)((pt / TST) - 1) & 1u)) break;
      const uint32_t st = R->sm + (uint32_t)(s * TSTAGE);
      ptx::mbar_arrive_expect_tx(&R->full[s], 2 * TILE_A);
      const int g0 = (int)((R->kt0 + pt) * BK);
      tma2(st, ma, g0, R->i0, &R->full[s]);
      tma2(st + TILE_A, mb, g0, R->j0, &R->full[s]);
      ++pt;
    }
    R->pt = pt;
  } else {
    constexpr uint32_t IDESC = idesc_tf32(BM, GN);
    int mt = R->mt;
    while (mt < R->nkt) {
      const int s = mt % TST, c = mt >> R->gsh, b = c & 1;
      const int gm = (1 << R->gsh) - 1;
      if (!ptx::mbar_test(&R->conv[s], (uint32_t)(mt / TST) & 1u)) break;
      if ((mt & gm) == 0 && c >= 2 && !ptx::mbar_test(&R->tfree[b], (uint32_t)((c / 2) - 1) & 1u)) break;
      tc_after();
      const uint32_t h0 = R->sm + (uint32_t)(s * TSTAGE);
      const uint32_t l0 = R->sm + (uint32_t)((TST + mt % TLO) * TSTAGE);
      const uint32_t d = R->tmem + (uint32_t)(b * 2 * GN);
      mma_ktile<true>(d, d + GN, h0, l0, h0 + TILE_A, l0 + TILE_A, IDESC, (mt & gm) == 0);
      mma_commit(&R->mmad[s]);
      if ((mt & gm) == gm || mt == R->nkt - 1) mma_commit(&R->accd[b]);
      ++mt;
    }
    R->mt = mt;
  }
}

__global__ void __launch_bounds__(TTHREADS, 1)
k_gram_tma(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, long long nd, int nt,
           int nsplit, double* __restrict__ part, int* status, int gsh) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ GramRing R;
  __shared__ uint32_t tmem_base;
  const uint32_t raw = saddr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  int pr = blockIdx.x, ti = 0;
  while (pr >= nt - ti) { pr -= nt - ti; ++ti; }
  const int tj = ti + pr;
  const int sp = blockIdx.y;
  const long long nkt_all = (nd + BK - 1) / BK;
  const long long kt0 = nkt_all * sp / nsplit;
  const int nkt = (int)(nkt_all * (sp + 1) / nsplit - kt0);
  double* P = part + (size_t)(blockIdx.x * nsplit + sp) * (BM * GN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nkt <= 0) {
    for (int e = threadIdx.x; e < BM * GN; e += TTHREADS) P[e] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < TST; ++s) {
      mbar_init(&R.full[s], 1);
      mbar_init(&R.conv[s], NCTL);
      mbar_init(&R.mmad[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&R.accd[b], 1);
      mbar_init(&R.tfree[b], 16);
    }
    R.abort_flag = 0;
    R.pt = 0;
    R.mt = 0;
    R.nkt = nkt;
    R.gsh = gsh;
    R.i0 = ti * BM;
    R.j0 = tj * GN;
    R.kt0 = kt0;
    R.sm = saddr(sm);
    ptx::mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 4 * GN);   // two (D, Ds) pairs: 512 columns
  tc_before();
  __syncthreads();
  if (threadIdx.x == 0) R.tmem = tmem_base;
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  const int gm = (1 << gsh) - 1;
  const int nchunk = (nkt + gm) >> gsh;
  volatile int* abort_flag = &R.abort_flag;
  // warp 15 is the control warp: its lane 0 issues the loads and the MMAs, and the warp
  // drains its share of TMEM; warps 0..14 split the landed tiles and drain theirs
  const bool control = warp == NCTL;
  // bounded wait for a phase
  auto wait = [&](uint64_t* b, uint32_t parity) {
    const long long t0 = clock64();
    while (!ptx::mbar_test(b, parity)) {
      if (*abort_flag) return false;
      if (clock64() - t0 > (1LL << 32)) {
        *abort_flag = 1;
        return false;
      }
    }
    return true;
  };
  float ahi[32], alo[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) ahi[c] = alo[c] = 0.f;
  const int row = 32 * (warp & 3) + lane;          // TMEM lane = output row i
  const int col0 = (warp >> 2) * 32;                // 32 output columns j
  int drained = 0;
  auto drain_now = [&](int c) {
    const int b = c & 1;
    tc_after();
    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * 2 * GN + col0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {   // columns 16 h .. 16 h + 15: a_hi b_hi plus the small products
      float v[16], vs[16];
      tmem_ld16x2(ta + (uint32_t)(16 * h), ta + (uint32_t)(GN + 16 * h), v, vs);
#pragma unroll
      for (int q = 0; q < 16; ++q) two_sum(ahi[16 * h + q], alo[16 * h + q], v[q] + vs[q]);
    }
    tc_before();
    __syncwarp();
    if (lane == 0) arrive(&R.tfree[b]);
  };
  bool ok = true;
  if (control) {
    // steps of the two roles until every MMA is issued, draining each chunk as it
    // completes; bounded by the time without progress
    long long t0 = clock64();
    while (ok) {
      int progress = 0;
      if (lane == 0) {
        const int pt = R.pt, mt = R.mt;
        gram_poll(&R, &ma, &mb, true);
        gram_poll(&R, &ma, &mb, false);
        progress = (R.pt != pt) || (R.mt != mt);
      }
      progress = __shfl_sync(0xffffffffu, progress, 0);
      if (drained < nchunk) {
        const int b = drained & 1;
        const int ready = __shfl_sync(0xffffffffu, lane == 0 ? (int)ptx::mbar_test(&R.accd[b], (uint32_t)(drained / 2) & 1u) : 0, 0);
        if (ready) {
          drain_now(drained++);
          progress = 1;
        }
      }
      const int done = __shfl_sync(0xffffffffu, lane == 0 ? (int)(R.mt == nkt) : 0, 0);
      if (done && drained == nchunk) break;
      if (progress) t0 = clock64();
      if (*abort_flag) ok = false;
      else if (clock64() - t0 > (1LL << 32)) {
        *abort_flag = 1;
        ok = false;
      }
    }
  } else {
    for (int t = 0; t < nkt && ok; ++t) {
      const int s = t % TST;
      if (!wait(&R.full[s], (uint32_t)(t / TST) & 1u)) { ok = false; break; }
      // the low slot is free once the MMAs of k-tile t - TLO are done
      if (t >= TLO && !wait(&R.mmad[(t - TLO) % TST], (uint32_t)((t - TLO) / TST) & 1u)) { ok = false; break; }
      // split the 2048 16-byte chunks of the k-tile's A and B images: hi in place, lo to its slot
      uint8_t* hs = sm + s * TSTAGE;
      uint8_t* ls = sm + (TST + t % TLO) * TSTAGE;
#pragma unroll 1
      for (int f = (int)threadIdx.x; f < 2048; f += NCTL * 32) {
        const int off = (f < 1024 ? 0 : TILE_A) + 16 * (f & 1023);
        float4 x = *(const float4*)(hs + off), h, l;
        split4(x, h, l);
        *(float4*)(hs + off) = h;
        *(float4*)(ls + off) = l;
      }
      proxy_fence();
      __syncwarp();
      if (lane == 0) arrive(&R.conv[s]);
      if ((t & gm) == (gm + 1) / 2 && drained < (t >> gsh)) {
        ok = wait(&R.accd[drained & 1], (uint32_t)(drained / 2) & 1u);
        if (ok) drain_now(drained++);
      }
    }
    while (ok && drained < nchunk) {
      ok = wait(&R.accd[drained & 1], (uint32_t)(drained / 2) & 1u);
      if (ok) drain_now(drained++);
    }
  }
  if (ok) {
#pragma unroll
    for (int q = 0; q < 32; ++q) P[(size_t)(col0 + q) * BM + row] = (double)ahi[q] + (double)alo[q];
  }
  // wind down: the loads issued and the MMAs committed complete before TMEM is freed
  if (control && lane == 0) {
    const int pt = R.pt;
    for (int t = (pt > TST ? pt - TST : 0); t < pt; ++t) {
      const long long c0 = clock64();
      while (!ptx::mbar_test(&R.full[t % TST], (uint32_t)(t / TST) & 1u))
        if (clock64() - c0 > (1LL << 32)) break;
    }
    if (R.mt > 0) {
      const int mt = R.mt;
      const long long c0 = clock64();
      while (!ptx::mbar_test(&R.mmad[(mt - 1) % TST], (uint32_t)((mt - 1) / TST) & 1u))
        if (clock64() - c0 > (1LL << 32)) break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, STATUS_TIMEOUT);
  tc_after();
  if (warp == 0) tmem_free(tmem, 4 * GN);
}

// G[i + j ns] from the partials: fixed-order sum over splits; tile pairs below the
// diagonal are the transposes of those above (times sgn: 1 for a symmetric G, -1 for
// an antisymmetric one); diagonal tiles are (anti)symmetrised.
__global__ void k_gram_reduce(const double* __restrict__ part, int nt, int nsplit, int ns, double* __restrict__ G,
                              double sgn) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ns * ns) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  const int ti = i / BM, tj = j / GN, ii = i % BM, jj = j % GN;
  auto pidx = [&](int a, int b) { return a * nt - a * (a - 1) / 2 + (b - a); };
  const int p = ti <= tj ? pidx(ti, tj) : pidx(tj, ti);
  const double* P = part + (size_t)p * nsplit * (BM * GN);
  double a = 0.0, b = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    const double* Ps = P + (size_t)s * (BM * GN);
    if (ti <= tj) a += Ps[(size_t)jj * BM + ii];
    if (ti >= tj) b += Ps[(size_t)ii * BM + jj];
  }
  G[e] = ti < tj ? a : (ti > tj ? sgn * b : 0.5 * (a + sgn * b));
}

// JB = i B for complex B (nd x ns, ldb; JB leading dimension nd): (re, im) -> (-im, re)
__global__ void k_times_i(const float2* __restrict__ B, long long ldb, long long nd, int ns, float2* __restrict__ JB) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nd * ns) return;
  const long long g = e % nd, j = e / nd;
  const float2 v = B[g + j * ldb];
  JB[e] = make_float2(-v.y, v.x);
}

// G = Gre - i Gim (Gre = r(A)^T r(B), Gim = r(A)^T r(i B), both ns x ns)
__global__ void k_cgram_combine(const double* __restrict__ Gre, const double* __restrict__ Gim, long long nn,
                                double2* __restrict__ G) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nn) G[e] = make_double2(Gre[e], -Gim[e]);
}

// ------------------------------------------------------------------ rotation
// Shared-memory images of Yr: for column half nh (256 columns) and k-tile t,
// hi then lo, each 256 rows (columns n of Yr) x 32 values (rows k of Yr), swizzled.
// CPLX: Yr is complex (ns x ns, (re, im) pairs) and its real K = 2 ns rows are
// Re Yr over Im Yr.
template <bool CPLX>
__global__ void k_rot_pack(const double* __restrict__ Yr, int ns, int nk, int nkt, int nnh, float* __restrict__ bp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nnh * nkt * RN * BK) return;
  const int kk = (int)(e % BK), r = (int)((e / BK) % RN);
  const int t = (int)((e / (BK * RN)) % nkt), nh = (int)(e / ((long long)BK * RN * nkt));
  const int n = nh * RN + r, k = t * BK + kk;
  float x = 0.f;
  if (n < ns && k < nk) {
    if constexpr (CPLX) x = (float)(k < ns ? Yr[2 * (k + (size_t)n * ns)] : Yr[2 * ((k - ns) + (size_t)n * ns) + 1]);
    else x = (float)Yr[k + (size_t)n * ns];
  }
  float hi, lo;
  split(x, hi, lo);
  const size_t img = (size_t)(nh * nkt + t) * 2 * (RN * BK);
  const int off = r * BK + ((((kk >> 2) ^ (r & 7)) << 2) | (kk & 3));
  bp[img + off] = hi;
  bp[img + RN * BK + off] = lo;
}

// C[g + n ldc] = sum_k U[g + k ldu] Yr[k + n ns] for g in [128 blockIdx.y, +128),
// n in [256 blockIdx.x, +256), k < nk (= ns).  CPLX: U, C are the real views (2 nd
// rows) of complex columns and k runs over nk = 2 ns: column k >= ns of the operand
// is r(i U_{k - ns}), whose row g is -/+ row g ^ 1 of r(U_{k - ns}) (minus on the
// real parts, the even rows).
template <bool CPLX>
__global__ void __launch_bounds__(THREADS, 1)
k_rot_tc(const float* __restrict__ U, long long ldu, const float* __restrict__ bp, long long nd, int ns, int nk,
         int nkt_all, float* __restrict__ C, long long ldc, int* status, int upper) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar[RST];
  __shared__ uint32_t tmem_base;
  const uint32_t raw = saddr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int nh = blockIdx.x;
  const long long m0 = (long long)blockIdx.y * BM;
  // Yr upper triangular: columns of half nh take rows k < (nh + 1) RN only
  const int nkt = upper ? min(nkt_all, ((nh + 1) * RN + BK - 1) / BK) : nkt_all;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RST; ++s) mbar_init(&bar[s], 1);
    ptx::mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * RN);   // D (a_hi b_hi) and Ds (cross terms)
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t IDESC = idesc_tf32(BM, RN);
  // A: thread t loads grid row gl = t % 128 at 16 consecutive k (kh = t / 128 picks the half)
  const int gl = threadIdx.x & (BM - 1), kh = threadIdx.x >> 7;
  const long long g = m0 + gl;
  const bool gok = g < nd;
  auto load_a = [&](int t, float (&v)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = t * BK + kh * 16 + j;
      if constexpr (CPLX) {
        float x = 0.f;
        if (gok && k < nk) {
          if (k < ns) {
            x = __ldg(U + g + (long long)k * ldu);
          } else {
            x = __ldg(U + (g ^ 1) + (long long)(k - ns) * ldu);
            if (!(g & 1)) x = -x;
          }
        }
        v[j] = x;
      } else {
        v[j] = (gok && k < ns) ? __ldg(U + g + (long long)k * ldu) : 0.f;
      }
    }
  };
  auto load_b = [&](int t, int s) {   // the hi and lo images of Yr, 64 KB
    const float* src = bp + (size_t)(nh * nkt_all + t) * 2 * (RN * BK);
    const uint32_t dst = saddr(sm + s * RSTAGE + 2 * TILE_A);
#pragma unroll 4
    for (int q = 0; q < (2 * RN * BK * 4) / (16 * THREADS); ++q) {
      const int f = threadIdx.x + THREADS * q;
      cp_async16(dst + 16 * f, src + 4 * f);
    }
    cp_async_commit();
  };
  float ca[16], na[16];
  load_b(0, 0);
  load_a(0, ca);
  bool aborted = false;
  int last = -1;
  for (int t = 0; t < nkt; ++t) {
    const int s = t & 1, s1 = s ^ 1;
    bool ok = true;
    if (t + 1 < nkt) {
      if (t >= 1) ok = mbar_wait(&bar[s1], (uint32_t)((t - 1) >> 1) & 1u);   // MMAs of tile t - 1 done
      load_b(t + 1, s1);
      load_a(t + 1, na);
    }
    uint8_t* st = sm + s * RSTAGE;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {   // chunk kh*4 + c4 of row gl: k = kh*16 + 4*c4 .. +3
      float4 x = make_float4(ca[4 * c4], ca[4 * c4 + 1], ca[4 * c4 + 2], ca[4 * c4 + 3]), h, l;
      split4(x, h, l);
      const uint32_t off = swz(gl, kh * 4 + c4);
      *(float4*)(st + off) = h;
      *(float4*)(st + TILE_A + off) = l;
    }
    if (t + 1 < nkt) cp_async_wait<1>(); else cp_async_wait<0>();
    proxy_fence();
    if (__syncthreads_or(!ok)) { aborted = true; break; }
    if (threadIdx.x == 0) {
      tc_after();
      const uint32_t b0 = saddr(st);
      mma_ktile(tmem, tmem + RN, b0, b0 + TILE_A, b0 + 2 * TILE_A, b0 + 2 * TILE_A + RN * BK * 4, IDESC, t == 0);
      mma_commit(&bar[s]);
    }
    last = t;
#pragma unroll
    for (int j = 0; j < 16; ++j) ca[j] = na[j];
  }
  bool ok = true;
  if (last >= 0) ok = mbar_wait(&bar[last & 1], (uint32_t)(last >> 1) & 1u);
  if (!ok || aborted) {
    if (threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
  } else {
    tc_after();
    const int row = 32 * (warp & 3) + lane;
    const long long gr = m0 + row;
    const int c0 = (warp >> 2) * (RN / 2);
#pragma unroll
    for (int h = 0; h < RN / 64; ++h) {
      float v[32], vs[32];
      const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 32 * h);
      tmem_ld32(ta, v);
      tmem_ld32(ta + RN, vs);
      if (gr < nd) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int n = nh * RN + c0 + 32 * h + c;
          if (n < ns) C[gr + (long long)n * ldc] = v[c] + vs[c];
        }
      }
    }
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0) tmem_free(tmem, 2 * RN);
}

}  // namespace

// ------------------------------------------------------------------ host side
static int gram_nsplit(const sparc_ctx* ctx, int ns, long long nd) {
  const int nt = ceil_div(ns, BM);
  const int pairs = nt * (nt + 1) / 2;
  const long long nkt = (nd + BK - 1) / BK;
  int nsplit = std::max(1, ctx->nsm / pairs);
  return (int)std::max<long long>(1, std::min<long long>(nsplit, nkt));
}

size_t gram_scratch_bytes(const sparc_ctx* ctx, int ns, long long nd) {
  const int nt = ceil_div(ns, BM);
  return (size_t)(nt * (nt + 1) / 2) * gram_nsplit(ctx, ns, nd) * BM * GN * sizeof(double);
}

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
// Tensor map of a column-major nd x ns FP32 operand: boxes of 32 grid points x 128
// columns in the 128-byte swizzle (the K-major layout of the MMA's operand images);
// points past nd and columns past ns read as zero.
static bool map_operand(CUtensorMap* m, const float* X, long long ldx, long long nd, int ns) {
  const cuuint64_t dims[2] = {(cuuint64_t)nd, (cuuint64_t)ns};
  const cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t es[2] = {1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)X, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t gram(sparc_ctx* ctx, const float* A, long long lda, const float* B, long long ldb, long long nd, int ns,
                 double* G, void* scratch, cudaStream_t st, bool anti, bool fast) {
  const int gsh = fast ? GCH_FAST_LOG : GCH_ACC_LOG;
  const int nt = ceil_div(ns, BM);
  const int pairs = nt * (nt + 1) / 2;
  const int nsplit = gram_nsplit(ctx, ns, nd);
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && (nd % 4 == 0) && ((uintptr_t)A % 16 == 0) &&
                   ((uintptr_t)B % 16 == 0);
  cudaError_t e;
  CUtensorMap ma, mb;
  if (vec && encoder() != nullptr && map_operand(&ma, A, lda, nd, ns) && map_operand(&mb, B, ldb, nd, ns)) {
    e = cudaFuncSetAttribute(k_gram_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM);
    if (e != cudaSuccess) return e;
    k_gram_tma<<<dim3(pairs, nsplit), TTHREADS, TSMEM, st>>>(ma, mb, nd, nt, nsplit, (double*)scratch,
                                                              ctx->d_status, gsh);
  } else if (vec) {
    e = cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
    if (e != cudaSuccess) return e;
    k_gram_tc<true><<<dim3(pairs, nsplit), GTHREADS, GSMEM, st>>>(A, lda, B, ldb, nd, ns, nt, nsplit,
                                                                 (double*)scratch, ctx->d_status, gsh);
  } else {
    e = cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
    if (e != cudaSuccess) return e;
    k_gram_tc<false><<<dim3(pairs, nsplit), GTHREADS, GSMEM, st>>>(A, lda, B, ldb, nd, ns, nt, nsplit,
                                                                  (double*)scratch, ctx->d_status, gsh);
  }
  const long long nn = (long long)ns * ns;
  k_gram_reduce<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>((const double*)scratch, nt, nsplit, ns, G,
                                                             anti ? -1.0 : 1.0);
  ctx->launches += 2;
  return cudaGetLastError();
}

size_t cgram_scratch_bytes(const sparc_ctx* ctx, int ns, long long nd) {
  const size_t g = (gram_scratch_bytes(ctx, ns, 2 * nd) + 255) & ~(size_t)255;
  return g + 2 * (((size_t)ns * ns * sizeof(double) + 255) & ~(size_t)255);
}

cudaError_t cgram(sparc_ctx* ctx, const cf32* A, long long lda, const cf32* B, long long ldb, long long nd, int ns,
                  cf64* G, cf32* JB, void* scratch, cudaStream_t st, bool fast) {
  const size_t g = (gram_scratch_bytes(ctx, ns, 2 * nd) + 255) & ~(size_t)255;
  double* Gre = (double*)((char*)scratch + g);
  double* Gim = (double*)((char*)Gre + (((size_t)ns * ns * sizeof(double) + 255) & ~(size_t)255));
  const long long ne = nd * ns, nn = (long long)ns * ns;
  k_times_i<<<(unsigned)ceil_div(ne, 256), 256, 0, st>>>((const float2*)B, ldb, nd, ns, (float2*)JB);
  ++ctx->launches;
  cudaError_t e = gram(ctx, (const float*)A, 2 * lda, (const float*)B, 2 * ldb, 2 * nd, ns, Gre, scratch, st, false,
                       fast);
  if (e != cudaSuccess) return e;
  e = gram(ctx, (const float*)A, 2 * lda, (const float*)JB, 2 * nd, 2 * nd, ns, Gim, scratch, st, true, fast);
  if (e != cudaSuccess) return e;
  k_cgram_combine<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>(Gre, Gim, nn, (double2*)G);
  ++ctx->launches;
  return cudaGetLastError();
}

size_t rot_scratch_bytes(int ns, bool cplx) {
  const int nkt = ceil_div(cplx ? 2 * ns : ns, BK), nnh = ceil_div(ns, RN);
  return (size_t)nnh * nkt * 2 * RN * BK * sizeof(float);
}

cudaError_t rotate(sparc_ctx* ctx, const float* U, long long ldu, const double* Yr, long long nd, int ns, float* C,
                   long long ldc, void* scratch, cudaStream_t st, bool upper) {
  const int nkt = ceil_div(ns, BK), nnh = ceil_div(ns, RN);
  if ((nd + BM - 1) / BM > 65535) return cudaErrorInvalidValue;   // grid y limit
  const long long npack = (long long)nnh * nkt * RN * BK;
  k_rot_pack<false><<<(unsigned)ceil_div(npack, 256), 256, 0, st>>>(Yr, ns, ns, nkt, nnh, (float*)scratch);
  cudaError_t e = cudaFuncSetAttribute(k_rot_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RSMEM);
  if (e != cudaSuccess) return e;
  k_rot_tc<false><<<dim3(nnh, (unsigned)ceil_div(nd, BM)), THREADS, RSMEM, st>>>(
      U, ldu, (const float*)scratch, nd, ns, ns, nkt, C, ldc, ctx->d_status, upper ? 1 : 0);
  ctx->launches += 2;
  return cudaGetLastError();
}

cudaError_t crotate(sparc_ctx* ctx, const cf32* U, long long ldu, const cf64* Yr, long long nd, int ns, cf32* C,
                    long long ldc, void* scratch, cudaStream_t st) {
  const int nk = 2 * ns, nkt = ceil_div(nk, BK), nnh = ceil_div(ns, RN);
  const long long nr = 2 * nd;   // rows of the real views
  if ((nr + BM - 1) / BM > 65535) return cudaErrorInvalidValue;   // grid y limit
  const long long npack = (long long)nnh * nkt * RN * BK;
  k_rot_pack<true><<<(unsigned)ceil_div(npack, 256), 256, 0, st>>>((const double*)Yr, ns, nk, nkt, nnh,
                                                                   (float*)scratch);
  cudaError_t e = cudaFuncSetAttribute(k_rot_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RSMEM);
  if (e != cudaSuccess) return e;
  k_rot_tc<true><<<dim3(nnh, (unsigned)ceil_div(nr, BM)), THREADS, RSMEM, st>>>(
      (const float*)U, 2 * ldu, (const float*)scratch, nr, ns, nk, nkt, (float*)C, 2 * ldc, ctx->d_status, 0);
  ctx->launches += 2;
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace sparc

// ------------------------------------------------------------------ C ABI
using namespace sparc;

extern "C" sparc_status sparc_gram_f32(sparc_ctx* ctx, const float* A, int64_t lda, const float* B, int64_t ldb,
                                       int64_t nd, int ns, double* G, void* stream) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  if (!A || !B || !G || nd < 1 || ns < 1 || ns > 4096 || lda < nd || ldb < nd)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_gram_f32: need nd >= 1, 1 <= ns <= 4096, lda, ldb >= nd");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!ensure_ws(ctx, tc::gram_scratch_bytes(ctx, ns, nd)))
    return fail(ctx, SPARC_ERR_OOM, "sparc_gram_f32: workspace allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t t0 = timing_begin(ctx, st);
  SPARC_CUDA(ctx, tc::gram(ctx, A, lda, B, ldb, nd, ns, G, ctx->ws, st));
  timing_end(ctx, TK_GRAM, t0, st);
  return SPARC_OK;
}

extern "C" sparc_status sparc_rotate_f32(sparc_ctx* ctx, const float* U, int64_t ldu, const double* Yr, int64_t nd,
                                         int ns, float* C, int64_t ldc, void* stream) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  if (!U || !Yr || !C || nd < 1 || ns < 1 || ns > 4096 || ldu < nd || ldc < nd)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_rotate_f32: need nd >= 1, 1 <= ns <= 4096, ldu, ldc >= nd");
  const char* u0 = (const char*)U;
  const char* u1 = (const char*)(U + (size_t)ldu * (ns - 1) + nd);
  const char* c0 = (const char*)C;
  const char* c1 = (const char*)(C + (size_t)ldc * (ns - 1) + nd);
  if (u0 < c1 && c0 < u1) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_rotate_f32: C overlaps U");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!ensure_ws(ctx, tc::rot_scratch_bytes(ns)))
    return fail(ctx, SPARC_ERR_OOM, "sparc_rotate_f32: workspace allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t t0 = timing_begin(ctx, st);
  SPARC_CUDA(ctx, tc::rotate(ctx, U, ldu, Yr, nd, ns, C, ldc, ctx->ws, st));
  timing_end(ctx, TK_ROT, t0, st);
  return SPARC_OK;
}

extern "C" sparc_status sparc_gram_c64(sparc_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb,
                                       int64_t nd, int ns, void* G, void* stream) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  if (!A || !B || !G || nd < 1 || ns < 1 || ns > 4096 || lda < nd || ldb < nd)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_gram_c64: need nd >= 1, 1 <= ns <= 4096, lda, ldb >= nd");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t gb = align256(tc::cgram_scratch_bytes(ctx, ns, nd));
  if (!ensure_ws(ctx, gb + (size_t)nd * ns * sizeof(cf32)))
    return fail(ctx, SPARC_ERR_OOM, "sparc_gram_c64: workspace allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t t0 = timing_begin(ctx, st);
  SPARC_CUDA(ctx, tc::cgram(ctx, (const cf32*)A, lda, (const cf32*)B, ldb, nd, ns, (cf64*)G,
                            (cf32*)((char*)ctx->ws + gb), ctx->ws, st));
  timing_end(ctx, TK_GRAM, t0, st);
  return SPARC_OK;
}

extern "C" sparc_status sparc_rotate_c64(sparc_ctx* ctx, const void* U, int64_t ldu, const void* Yr, int64_t nd,
                                         int ns, void* C, int64_t ldc, void* stream) {
  if (!ctx) return SPARC_ERR_INVALID_ARG;
  if (!U || !Yr || !C || nd < 1 || ns < 1 || ns > 4096 || ldu < nd || ldc < nd)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_rotate_c64: need nd >= 1, 1 <= ns <= 4096, ldu, ldc >= nd");
  const char* u0 = (const char*)U;
  const char* u1 = (const char*)((const cf32*)U + (size_t)ldu * (ns - 1) + nd);
  const char* c0 = (const char*)C;
  const char* c1 = (const char*)((cf32*)C + (size_t)ldc * (ns - 1) + nd);
  if (u0 < c1 && c0 < u1) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_rotate_c64: C overlaps U");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!ensure_ws(ctx, tc::rot_scratch_bytes(ns, true)))
    return fail(ctx, SPARC_ERR_OOM, "sparc_rotate_c64: workspace allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t t0 = timing_begin(ctx, st);
  SPARC_CUDA(ctx, tc::crotate(ctx, (const cf32*)U, ldu, (const cf64*)Yr, nd, ns, (cf32*)C, ldc, ctx->ws, st));
  timing_end(ctx, TK_ROT, t0, st);
  return SPARC_OK;
}
