// One SCF iteration around the CheFSI step (Section 3.4 and Eq. EL; Section 5 names the
// solvers): the discrete pseudocharges and their self energy (Eqs. PseudochargeDiscrete,
// DiscreteEself), the Fermi level by Brent's method, the electron density, the Poisson
// equation by conjugate gradients, LDA exchange-correlation (Slater exchange,
// Perdew-Wang 1992 correlation), Anderson extrapolation of V_eff and the free energy
// (Eq. FreeEnergy:GroundState:DFT:discrete).  All grid arithmetic is FP64 and every
// reduction runs in a fixed order (per-block partial sums, then one block), so the
// iteration is bitwise deterministic.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rr.cuh"

namespace sparc {
namespace scf {

constexpr int TPB = 256;
constexpr int MAXHIST = 8;
constexpr int NPAIR = MAXHIST * (MAXHIST + 1) / 2 + MAXHIST;   // Anderson dot products
// slots of the scalar array
enum {
  S_MU = 0, S_EBAND, S_ENT, S_NEL, S_EXC, S_EEL, S_RES2, S_VOUT2, S_MEAN, S_ESELF,
  S_RHS2, S_RR0, S_RR1, S_DONE, S_ITERS, S_GAMMA = 16, S_RHOSUM = 24, S_COUNT = 32
};

struct Weights {
  double w[3][MAX_FD + 1];   // w_{p,s} of Eq. weightsLap (centre counted twice)
};

struct Atom {
  double R[3], Z, rc;
  int c[3], nb[3];           // nearest node (unwrapped) and cube half-width
};

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;   // valid in thread 0
}

// out[k] = sum_b part[b * stride + k] over nb blocks, fixed order (one thread per k)
__global__ void k_sum_parts(const double* __restrict__ part, int nb, int stride, int nk, double* out) {
  const int k = threadIdx.x;
  if (k >= nk) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(long long)b * stride + k];
  out[k] = s;
}

// ------------------------------------------------------------------ pseudocharges
__device__ __forceinline__ double vloc(double r, double Z, double rc) {
  // V_I(r) = -Z erf(r/rc)/r, and its limit at the nucleus
  return r < 1e-12 ? -2.0 * Z / (sqrt(M_PI) * rc) : -Z * erf(r / rc) / r;
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// b(g) = sum over atoms and periodic images whose cube holds g of -(1/4pi) lap_h V_I(g),
// and E_self partials 1/2 h1h2h3 b_I V_I (Eqs. PseudochargeDiscrete and DiscreteEself).
__global__ void __launch_bounds__(TPB) k_pseudocharge(int n1, int n2, int n3, double h1, double h2, double h3,
                                                      int no, Weights W, const Atom* __restrict__ atoms,
                                                      int natom, double* __restrict__ b, double* part) {
  __shared__ double sh[32];
  const long long nd = (long long)n1 * n2 * n3;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double bs = 0.0, es = 0.0;
  if (g < nd) {
    const int i = (int)(g % n1), j = (int)((g / n1) % n2), k = (int)(g / ((long long)n1 * n2));
    const int n[3] = {n1, n2, n3}, idx[3] = {i, j, k};
    const double h[3] = {h1, h2, h3};
    for (int I = 0; I < natom; ++I) {
      const Atom A = atoms[I];
      long long t0[3], t1[3];
      for (int s = 0; s < 3; ++s) {
        t0[s] = -floor_div((long long)idx[s] - A.c[s] + A.nb[s], n[s]);
        t1[s] = floor_div((long long)A.c[s] + A.nb[s] - idx[s], n[s]);
      }
      for (long long tz = t0[2]; tz <= t1[2]; ++tz)
        for (long long ty = t0[1]; ty <= t1[1]; ++ty)
          for (long long tx = t0[0]; tx <= t1[0]; ++tx) {
            const long long u[3] = {i + tx * n1, j + ty * n2, k + tz * n3};
            double x[3];
            for (int s = 0; s < 3; ++s) x[s] = -0.5 * n[s] * h[s] + (double)u[s] * h[s] - A.R[s];
            const double v0 = vloc(sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]), A.Z, A.rc);
            double lap = 0.0;
            for (int s = 0; s < 3; ++s) {
              double acc = 2.0 * W.w[s][0] * v0;
              for (int p = 1; p <= no; ++p) {
                double y[3] = {x[0], x[1], x[2]};
                y[s] = x[s] + p * h[s];
                const double vp = vloc(sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]), A.Z, A.rc);
                y[s] = x[s] - p * h[s];
                const double vm = vloc(sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]), A.Z, A.rc);
                acc += W.w[s][p] * (vp + vm);
              }
              lap += acc;
            }
            const double bI = -lap / (4.0 * M_PI);
            bs += bI;
            es += 0.5 * h1 * h2 * h3 * bI * v0;
          }
    }
    b[g] = bs;
  }
  const double t = block_sum(es, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ------------------------------------------------------------------ Fermi level (Brent)
__device__ __forceinline__ double fermi_occ(double lam, double mu, double kT) {
  const double x = (lam - mu) / kT;   // written so that exp never overflows
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// 2 sum_n w_n g_n(mu) - Ne (w: the k-point weight of each value, null: 1), summed by
// the block in a fixed order, result in every thread
__device__ double nel_minus(const double* lam, const double* wt, int ns, double mu, double kT, double Ne,
                            double* sh, double* bc) {
  double v = 0.0;
  for (int n = threadIdx.x; n < ns; n += blockDim.x) v += (wt ? wt[n] : 1.0) * fermi_occ(lam[n], mu, kT);
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) *bc = 2.0 * s - Ne;
  __syncthreads();
  const double r = *bc;
  __syncthreads();
  return r;
}

// lambda_f with 2 sum_n w_n g_n = Ne (Eq. EL; with k-points the Brillouin-zone sum
// weights each value by its k-point's weight w_n, null: 1), by Brent's method on
// [lam_min - 1, lam_max + 1]: inverse quadratic interpolation or secant steps when they
// stay inside the bracket and shrink fast enough, bisection otherwise.  Then the
// occupations, band energy, entropy term and electron count.
__global__ void __launch_bounds__(TPB) k_fermi(const double* __restrict__ lam, const double* __restrict__ wt,
                                               int ns, double Ne, double kT, double* __restrict__ occ,
                                               double* scal) {
  __shared__ double sh[32], bc;
  __shared__ double st[8];   // Brent state shared with the block: next abscissa, done flag
  double lo = lam[0], hi = lam[0];
  for (int n = 1; n < ns; ++n) { lo = fmin(lo, lam[n]); hi = fmax(hi, lam[n]); }
  double a = lo - 1.0, bb = hi + 1.0;
  double fa = nel_minus(lam, wt, ns, a, kT, Ne, sh, &bc);
  double fb = nel_minus(lam, wt, ns, bb, kT, Ne, sh, &bc);
  double c = a, fc = fa, d = bb - a, e = d;
  const double xtol = 1e-14, eps = 2.220446049250313e-16;
  for (int it = 0; it < 300; ++it) {
    // thread 0 decides the next point; every thread keeps the same state
    if (threadIdx.x == 0) {
      int done = 0;
      if ((fb > 0.0) == (fc > 0.0)) { c = a; fc = fa; d = bb - a; e = d; }
      if (fabs(fc) < fabs(fb)) { a = bb; bb = c; c = a; fa = fb; fb = fc; fc = fa; }
      const double tol1 = 2.0 * eps * fabs(bb) + 0.5 * xtol;
      const double xm = 0.5 * (c - bb);
      if (fabs(xm) <= tol1 || fb == 0.0) {
        done = 1;
      } else {
        if (fabs(e) >= tol1 && fabs(fa) > fabs(fb)) {
          const double s = fb / fa;
          double p, q;
          if (a == c) {   // secant
            p = 2.0 * xm * s;
            q = 1.0 - s;
          } else {        // inverse quadratic interpolation through a, b, c
            const double qq = fa / fc, r = fb / fc;
            p = s * (2.0 * xm * qq * (qq - r) - (bb - a) * (r - 1.0));
            q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
          }
          if (p > 0.0) q = -q;
          p = fabs(p);
          if (2.0 * p < fmin(3.0 * xm * q - fabs(tol1 * q), fabs(e * q))) { e = d; d = p / q; }
          else { d = xm; e = d; }
        } else {
          d = xm;
          e = d;
        }
        a = bb;
        fa = fb;
        bb += fabs(d) > tol1 ? d : (xm > 0.0 ? tol1 : -tol1);
      }
      st[0] = bb; st[1] = done; st[2] = a; st[3] = fa; st[4] = c; st[5] = fc; st[6] = d; st[7] = e;
    }
    __syncthreads();
    bb = st[0]; a = st[2]; fa = st[3]; c = st[4]; fc = st[5]; d = st[6]; e = st[7];
    const bool done = st[1] != 0.0;
    __syncthreads();
    if (done) break;
    fb = nel_minus(lam, wt, ns, bb, kT, Ne, sh, &bc);
  }
  const double mu = bb;
  double eb = 0.0, en = 0.0, ne = 0.0;
  for (int n = threadIdx.x; n < ns; n += blockDim.x) {
    const double g = fermi_occ(lam[n], mu, kT);
    const double w = wt ? wt[n] : 1.0;
    occ[n] = g;
    eb += w * g * lam[n];
    ne += w * g;
    if (g > 0.0 && g < 1.0) en += w * (g * log(g) + (1.0 - g) * log(1.0 - g));
  }
  const double seb = block_sum(eb, sh);
  const double sen = block_sum(en, sh);
  const double sne = block_sum(ne, sh);
  if (threadIdx.x == 0) {
    scal[S_MU] = mu;
    scal[S_EBAND] = 2.0 * seb;
    scal[S_ENT] = 2.0 * kT * sen;
    scal[S_NEL] = 2.0 * sne;
  }
}

// ------------------------------------------------------------------ density
// rho (+)= scale w sum_n g_n |U_n|^2: one k-point's share (accumulate after the first)
template <class T>
__global__ void __launch_bounds__(TPB) k_density(const T* __restrict__ U, long long ld, int ns, long long nd,
                                                 const double* __restrict__ occ, double scale, double w,
                                                 int accumulate, double* __restrict__ rho) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nd) return;
  double s = 0.0;
  for (int n = 0; n < ns; ++n) s += occ[n] * Tr<T>::abs2(U[g + (long long)n * ld]);
  const double v = scale * (w * s);
  rho[g] = accumulate ? rho[g] + v : v;
}

// ------------------------------------------------------------------ Poisson (CG)
// y = -(1/4pi) lap_h x (periodic, FD radius no); part[block] = sum x.y
__global__ void __launch_bounds__(TPB) k_lapA(const double* __restrict__ x, double* __restrict__ y, int n1,
                                              int n2, int n3, int no, Weights W, double* part,
                                              const double* scal) {
  __shared__ double sh[32];
  if (scal && scal[S_DONE] != 0.0) return;
  const long long nd = (long long)n1 * n2 * n3;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (g < nd) {
    const int i = (int)(g % n1), j = (int)((g / n1) % n2), k = (int)(g / ((long long)n1 * n2));
    const double xc = x[g];
    double lap = 2.0 * (W.w[0][0] + W.w[1][0] + W.w[2][0]) * xc;
    for (int p = 1; p <= no; ++p) {
      int ip = i + p; if (ip >= n1) ip -= n1;
      int im = i - p; if (im < 0) im += n1;
      int jp = j + p; if (jp >= n2) jp -= n2;
      int jm = j - p; if (jm < 0) jm += n2;
      int kp = k + p; if (kp >= n3) kp -= n3;
      int km = k - p; if (km < 0) km += n3;
      const long long row = ((long long)k * n2 + j) * n1;
      lap += W.w[0][p] * (x[row + ip] + x[row + im]);
      lap += W.w[1][p] * (x[((long long)k * n2 + jp) * n1 + i] + x[((long long)k * n2 + jm) * n1 + i]);
      lap += W.w[2][p] * (x[((long long)kp * n2 + j) * n1 + i] + x[((long long)km * n2 + j) * n1 + i]);
    }
    const double v = -lap / (4.0 * M_PI);
    y[g] = v;
    d = xc * v;
  }
  const double t = block_sum(d, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// every block sums the nb partials in the same order
__device__ __forceinline__ double sum_parts_all(const double* part, int nb, double* sh, double* bc) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
  // fixed order: per-thread strided sums, then the block sum in thread order
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) *bc = s;
  __syncthreads();
  const double r = *bc;
  __syncthreads();
  return r;
}

// alpha = rr / p.Ap; phi += alpha p; r -= alpha Ap; part_rr = sum r^2
__global__ void __launch_bounds__(TPB) k_cg_update(double* __restrict__ phi, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ Ap,
                                                   long long nd, const double* part_pap, int nb, int par,
                                                   double* scal, double* part_rr) {
  __shared__ double sh[32], bc;
  if (scal[S_DONE] != 0.0) return;
  const double pap = sum_parts_all(part_pap, nb, sh, &bc);
  const double alpha = scal[S_RR0 + par] / pap;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (g < nd) {
    phi[g] += alpha * p[g];
    const double rn = r[g] - alpha * Ap[g];
    r[g] = rn;
    s = rn * rn;
  }
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = t;
}

// rr' = sum r^2; beta = rr'/rr; p = r + beta p; convergence flag and iteration count
__global__ void __launch_bounds__(TPB) k_cg_dir(const double* __restrict__ r, double* __restrict__ p, long long nd,
                                                const double* part_rr, int nb, int par, double tol, double* scal) {
  __shared__ double sh[32], bc;
  if (scal[S_DONE] != 0.0) return;
  const double rr = sum_parts_all(part_rr, nb, sh, &bc);
  const double beta = rr / scal[S_RR0 + par];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nd) p[g] = r[g] + beta * p[g];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[S_RR0 + (par ^ 1)] = rr;
    scal[S_ITERS] += 1.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && sqrt(rr) <= tol * sqrt(scal[S_RHS2])) scal[S_DONE] = 1.0;
}

// r = rhs - mean - Ap (initial residual), p = r, part = r^2 and rhs^2 (two halves)
__global__ void __launch_bounds__(TPB) k_cg_init(const double* __restrict__ rho, const double* __restrict__ b,
                                                 const double* __restrict__ Ap, long long nd, const double* scal,
                                                 double* __restrict__ r, double* __restrict__ p, double* part) {
  __shared__ double sh[32];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0, q = 0.0;
  if (g < nd) {
    const double f = rho[g] + b[g] - scal[S_MEAN];
    const double rv = f - Ap[g];
    r[g] = rv;
    p[g] = rv;
    s = rv * rv;
    q = f * f;
  }
  const double t0 = block_sum(s, sh);
  const double t1 = block_sum(q, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = t0; part[gridDim.x + blockIdx.x] = t1; }
}

// part[block] = sum of (x + y) over the block
__global__ void __launch_bounds__(TPB) k_sum2(const double* __restrict__ x, const double* __restrict__ y, long long nd,
                                              double* part) {
  __shared__ double sh[32];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double v = g < nd ? x[g] + (y ? y[g] : 0.0) : 0.0;
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_shift(double* __restrict__ x, long long nd, const double* mean, double scale) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nd) x[g] -= *mean * scale;
}

__global__ void k_scale1(double* x, double s) { *x *= s; }

__global__ void k_neg(const double* __restrict__ x, double* __restrict__ y, long long nd) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nd) y[g] = -x[g];
}

// ------------------------------------------------------------------ starting density
// rho = max(-b + scale dy, 0) (the superposition of atomic densities -b plus a
// correction) and per-block partial sums of rho.
__global__ void k_guess(const double* __restrict__ b, const float* __restrict__ dy, double scale, long long nd,
                        double* __restrict__ rho, double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (g < nd) {
    r = -b[g] + (dy ? scale * (double)dy[g] : 0.0);
    r = r > 0.0 ? r : 0.0;
    rho[g] = r;
  }
  const double t = block_sum(r, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// rho *= N_e / (dv sum rho), V = phi + V_xc
__global__ void k_renorm_vin(double* __restrict__ rho, const double* __restrict__ scal, double Ne, double dv,
                             long long nd) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nd) rho[g] *= Ne / (dv * scal[S_RHOSUM]);
}
__global__ void k_add(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ z, long long nd) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nd) z[g] = x[g] + y[g];
}

// ------------------------------------------------------------------ LDA
// eps_xc, V_xc: Slater exchange and the Perdew-Wang 1992 correlation of the
// unpolarised gas (parameters A, alpha1, beta1..beta4).
__global__ void k_lda(const double* __restrict__ rho, long long nd, double* __restrict__ eps, double* __restrict__ v) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nd) return;
  const double r = rho[g];
  if (!(r > 1e-30)) { eps[g] = 0.0; v[g] = 0.0; return; }
  const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  const double ex = -0.75 * cbrt(3.0 / M_PI) * cbrt(r);
  const double rs = cbrt(3.0 / (4.0 * M_PI * r));
  const double srs = sqrt(rs);
  const double Q0 = -2.0 * A * (1.0 + a1 * rs);
  const double Q1 = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
  const double Q1p = A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs);
  const double L = log1p(1.0 / Q1);
  const double ec = Q0 * L;
  const double dec = -2.0 * A * a1 * L - Q0 * Q1p / (Q1 * Q1 + Q1);
  eps[g] = ex + ec;
  v[g] = (4.0 / 3.0) * ex + ec - rs / 3.0 * dec;
}

// V_out = phi + V_xc, and partials of the grid energy terms and residual norms:
// [0] sum (eps - vxc) rho, [1] sum 1/2 (b - rho) phi, [2] sum (vout - vin)^2, [3] sum vout^2
__global__ void __launch_bounds__(TPB) k_vout(const double* __restrict__ phi, const double* __restrict__ vxc,
                                              const double* __restrict__ eps, const double* __restrict__ rho,
                                              const double* __restrict__ b, const double* __restrict__ vin,
                                              long long nd, double* __restrict__ vout, double* __restrict__ fres,
                                              double* part) {
  __shared__ double sh[32];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  if (g < nd) {
    const double vo = phi[g] + vxc[g];
    vout[g] = vo;
    const double f = vo - vin[g];
    fres[g] = f;
    t[0] = (eps[g] - vxc[g]) * rho[g];
    t[1] = 0.5 * (b[g] - rho[g]) * phi[g];
    t[2] = f * f;
    t[3] = vo * vo;
  }
  for (int q = 0; q < 4; ++q) {
    const double s = block_sum(t[q], sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * 4 + q] = s;
  }
}

// ------------------------------------------------------------------ Anderson
// ring slot of iteration k
__device__ __forceinline__ int slot(int k, int nslot) { return ((k % nslot) + nslot) % nslot; }

// dots of the differences dF_a = F_{k-a} - F_{k-a-1} (a < mm) with each other (a <= b)
// and with F_k, one partial per block and pair
__global__ void __launch_bounds__(TPB) k_anderson_dots(const double* __restrict__ F, long long nd, int nslot, int k,
                                                       int mm, double* part) {
  __shared__ double sh[32];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double d[MAXHIST], fk = 0.0;
  for (int a = 0; a < MAXHIST; ++a) d[a] = 0.0;
  if (g < nd) {
    fk = F[(long long)slot(k, nslot) * nd + g];
    for (int a = 0; a < mm; ++a)
      d[a] = F[(long long)slot(k - a, nslot) * nd + g] - F[(long long)slot(k - a - 1, nslot) * nd + g];
  }
  int q = 0;
  for (int a = 0; a < mm; ++a)
    for (int b2 = a; b2 < mm; ++b2, ++q) {
      const double s = block_sum(d[a] * d[b2], sh);
      if (threadIdx.x == 0) part[(long long)blockIdx.x * NPAIR + q] = s;
    }
  for (int a = 0; a < mm; ++a, ++q) {
    const double s = block_sum(d[a] * fk, sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * NPAIR + q] = s;
  }
}

// gamma from the normal equations (dF^T dF + 1e-12 tr I) gamma = dF^T f_k (Cholesky, one thread)
__global__ void k_anderson_solve(const double* sums, int mm, double* scal) {
  if (threadIdx.x != 0 || mm == 0) return;
  double G[MAXHIST][MAXHIST], rhs[MAXHIST];
  int q = 0;
  for (int a = 0; a < mm; ++a)
    for (int b = a; b < mm; ++b, ++q) G[a][b] = G[b][a] = sums[q];
  for (int a = 0; a < mm; ++a, ++q) rhs[a] = sums[q];
  double tr = 0.0;
  for (int a = 0; a < mm; ++a) tr += G[a][a];
  for (int a = 0; a < mm; ++a) G[a][a] += 1e-12 * tr;
  for (int j = 0; j < mm; ++j) {   // G = L L^T in place (lower)
    double s = G[j][j];
    for (int k = 0; k < j; ++k) s -= G[j][k] * G[j][k];
    G[j][j] = sqrt(fmax(s, 1e-300));
    for (int i = j + 1; i < mm; ++i) {
      double t = G[i][j];
      for (int k = 0; k < j; ++k) t -= G[i][k] * G[j][k];
      G[i][j] = t / G[j][j];
    }
  }
  double y[MAXHIST];
  for (int i = 0; i < mm; ++i) {
    double t = rhs[i];
    for (int k = 0; k < i; ++k) t -= G[i][k] * y[k];
    y[i] = t / G[i][i];
  }
  for (int i = mm - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < mm; ++k) t -= G[k][i] * scal[S_GAMMA + k];
    scal[S_GAMMA + i] = t / G[i][i];
  }
}

// V_next = (x_k - sum_a gamma_a dX_a) + beta (f_k - sum_a gamma_a dF_a)
__global__ void k_anderson_next(const double* __restrict__ X, const double* __restrict__ F, long long nd, int nslot,
                                int k, int mm, double beta, const double* scal, double* __restrict__ vnext) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nd) return;
  double x = X[(long long)slot(k, nslot) * nd + g];
  double f = F[(long long)slot(k, nslot) * nd + g];
  for (int a = 0; a < mm; ++a) {
    const double ga = scal[S_GAMMA + a];
    const long long s0 = (long long)slot(k - a, nslot) * nd + g, s1 = (long long)slot(k - a - 1, nslot) * nd + g;
    x -= ga * (X[s0] - X[s1]);
    f -= ga * (F[s0] - F[s1]);
  }
  vnext[g] = x + beta * f;
}


// ------------------------------------------------------------------ forces (Section 3.6)
struct GWeights {
  double w[3][MAX_FD + 1];   // central first-derivative weights w~_{p,s} (gradient formula)
};

// lap_h V_I at the point y (relative to the atom), node spacing h
__device__ double lap_vloc(const double y[3], const double h[3], int no, const Weights& W, double Z, double rc) {
  double lap = 0.0;
  const double v0 = vloc(sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]), Z, rc);
  for (int s = 0; s < 3; ++s) {
    double acc = 2.0 * W.w[s][0] * v0;
    for (int p = 1; p <= no; ++p) {
      double a[3] = {y[0], y[1], y[2]};
      a[s] = y[s] + p * h[s];
      const double vp = vloc(sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]), Z, rc);
      a[s] = y[s] - p * h[s];
      const double vm = vloc(sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]), Z, rc);
      acc += W.w[s][p] * (vp + vm);
    }
    lap += acc;
  }
  return lap;
}

// Local force (Eq. LocalForce:Discrete): h1h2h3 sum over the atom's cube nodes of
// nabla_h b_I (phi - V_I), b_I = -(1/4pi) lap_h V_I evaluated at any node.
// Grid: (atom, blocks over the cube); part[(atom * gridDim.y + block) * 3 + s].
__global__ void __launch_bounds__(TPB) k_force_local(int n1, int n2, int n3, double h1, double h2, double h3, int no,
                                                     Weights W, GWeights G, const Atom* __restrict__ atoms,
                                                     const double* __restrict__ phi, double* part) {
  __shared__ double sh[32];
  const Atom A = atoms[blockIdx.x];
  const int m0 = 2 * A.nb[0] + 1, m1 = 2 * A.nb[1] + 1, m2 = 2 * A.nb[2] + 1;
  const long long ncube = (long long)m0 * m1 * m2;
  const long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x;
  const int n[3] = {n1, n2, n3};
  const double h[3] = {h1, h2, h3};
  double f[3] = {0.0, 0.0, 0.0};
  if (e < ncube) {
    const int u[3] = {A.c[0] - A.nb[0] + (int)(e % m0), A.c[1] - A.nb[1] + (int)((e / m0) % m1),
                      A.c[2] - A.nb[2] + (int)(e / ((long long)m0 * m1))};
    double x[3];
    int gi[3];
    for (int s = 0; s < 3; ++s) {
      x[s] = -0.5 * n[s] * h[s] + (double)u[s] * h[s] - A.R[s];
      gi[s] = (int)(((long long)u[s] % n[s] + n[s]) % n[s]);
    }
    const double pv = phi[((long long)gi[2] * n2 + gi[1]) * n1 + gi[0]] -
                      vloc(sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]), A.Z, A.rc);
    for (int s = 0; s < 3; ++s) {
      double gb = 0.0;
      for (int p = 1; p <= no; ++p) {
        double y[3] = {x[0], x[1], x[2]};
        y[s] = x[s] + p * h[s];
        const double lp = lap_vloc(y, h, no, W, A.Z, A.rc);
        y[s] = x[s] - p * h[s];
        const double lm = lap_vloc(y, h, no, W, A.Z, A.rc);
        gb += G.w[s][p] * (lp - lm);
      }
      f[s] = h1 * h2 * h3 * (-gb / (4.0 * M_PI)) * pv;
    }
  }
  for (int s = 0; s < 3; ++s) {
    const double t = block_sum(f[s], sh);
    if (threadIdx.x == 0) part[((long long)blockIdx.x * gridDim.y + blockIdx.y) * 3 + s] = t;
  }
}

// Nonlocal projections for the force: for projector p = blockIdx.x and orbital
// n = blockIdx.y, out[(p * ns + n) * 4 + {0, 1, 2, 3}] = sum over the box of chi U and of
// chi nabla_h U (Y and W without the h1h2h3 and normalisation factors).
template <class T>
__global__ void __launch_bounds__(TPB) k_force_proj(const T* __restrict__ U, long long ld, int n1, int n2, int n3, int no,
                                                    GWeights G, const long long* __restrict__ p_off,
                                                    const int* __restrict__ p_g, const double* __restrict__ p_val,
                                                    int ns, double* out) {
  __shared__ double sh[32];
  const int p = blockIdx.x, nn = blockIdx.y;
  const T* u = U + (long long)nn * ld;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long e = p_off[p] + threadIdx.x; e < p_off[p + 1]; e += blockDim.x) {
    const int g = p_g[e];
    const double c = p_val[e];
    const int i = g % n1, j = (g / n1) % n2, k = g / (n1 * n2);
    acc[0] += c * (double)u[g];
    double gr[3] = {0.0, 0.0, 0.0};
    for (int q = 1; q <= no; ++q) {
      int ip = i + q; if (ip >= n1) ip -= n1;
      int im = i - q; if (im < 0) im += n1;
      int jp = j + q; if (jp >= n2) jp -= n2;
      int jm = j - q; if (jm < 0) jm += n2;
      int kp = k + q; if (kp >= n3) kp -= n3;
      int km = k - q; if (km < 0) km += n3;
      const long long row = ((long long)k * n2 + j) * n1;
      gr[0] += G.w[0][q] * ((double)u[row + ip] - (double)u[row + im]);
      gr[1] += G.w[1][q] * ((double)u[((long long)k * n2 + jp) * n1 + i] - (double)u[((long long)k * n2 + jm) * n1 + i]);
      gr[2] += G.w[2][q] * ((double)u[((long long)kp * n2 + j) * n1 + i] - (double)u[((long long)km * n2 + j) * n1 + i]);
    }
    for (int s = 0; s < 3; ++s) acc[1 + s] += c * gr[s];
  }
  for (int q = 0; q < 4; ++q) {
    const double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) out[((long long)p * ns + nn) * 4 + q] = t;
  }
}

// The same projections for Bloch orbitals of one k-point (complex U, complex chi~ with the
// image phases of Eq. NonlocalPS:FD): out[(p * ns + n) * 8 + 2 q + {0, 1}] = (Re, Im) of
// sum conj(chi~) u (q = 0) and of sum conj(chi~) (nabla_h u)_s (q = 1 + s), where a
// neighbour across the upper face of axis s carries exp(+i k_s L_s) and across the lower
// face exp(-i k_s L_s) (the Bloch wrap of Section 3.1).
template <class T>
__global__ void __launch_bounds__(TPB) k_force_proj_c(const T* __restrict__ U, long long ld, int n1, int n2, int n3,
                                                      int no, GWeights G, const long long* __restrict__ p_off,
                                                      const int* __restrict__ p_g, const cf64* __restrict__ p_val,
                                                      double phr0, double phi0, double phr1, double phi1, double phr2,
                                                      double phi2, int ns, double* out) {
  __shared__ double sh[32];
  const int p = blockIdx.x, nn = blockIdx.y;
  const T* u = U + (long long)nn * ld;
  const double phr[3] = {phr0, phr1, phr2}, phi[3] = {phi0, phi1, phi2};
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  // u at node (i, j, k) times the phase of `t` face crossings along axis s (t in -1, 0, 1)
  auto val = [&](int i, int j, int k, int s, int t, double& re, double& im) {
    const T v = u[((long long)k * n2 + j) * n1 + i];
    const double vr = (double)v.x, vi = (double)v.y;
    if (t == 0) { re = vr; im = vi; return; }
    const double cr = phr[s], ci = t > 0 ? phi[s] : -phi[s];
    re = vr * cr - vi * ci;
    im = vr * ci + vi * cr;
  };
  for (long long e = p_off[p] + threadIdx.x; e < p_off[p + 1]; e += blockDim.x) {
    const int g = p_g[e];
    const cf64 c = p_val[e];
    const int i = g % n1, j = (g / n1) % n2, k = g / (n1 * n2);
    double ur, ui;
    val(i, j, k, 0, 0, ur, ui);
    double gr[3] = {0.0, 0.0, 0.0}, gi[3] = {0.0, 0.0, 0.0};
    for (int q = 1; q <= no; ++q) {
      double ar, ai, br, bi;
      {
        int ip = i + q, im = i - q, tp = 0, tm = 0;
        if (ip >= n1) { ip -= n1; tp = 1; }
        if (im < 0) { im += n1; tm = -1; }
        val(ip, j, k, 0, tp, ar, ai);
        val(im, j, k, 0, tm, br, bi);
        gr[0] += G.w[0][q] * (ar - br);
        gi[0] += G.w[0][q] * (ai - bi);
      }
      {
        int jp = j + q, jm = j - q, tp = 0, tm = 0;
        if (jp >= n2) { jp -= n2; tp = 1; }
        if (jm < 0) { jm += n2; tm = -1; }
        val(i, jp, k, 1, tp, ar, ai);
        val(i, jm, k, 1, tm, br, bi);
        gr[1] += G.w[1][q] * (ar - br);
        gi[1] += G.w[1][q] * (ai - bi);
      }
      {
        int kp = k + q, km = k - q, tp = 0, tm = 0;
        if (kp >= n3) { kp -= n3; tp = 1; }
        if (km < 0) { km += n3; tm = -1; }
        val(i, j, kp, 2, tp, ar, ai);
        val(i, j, km, 2, tm, br, bi);
        gr[2] += G.w[2][q] * (ar - br);
        gi[2] += G.w[2][q] * (ai - bi);
      }
    }
    // conj(c) * (x + i y) = (c.x x + c.y y) + i (c.x y - c.y x)
    acc[0] += c.x * ur + c.y * ui;
    acc[1] += c.x * ui - c.y * ur;
    for (int s2 = 0; s2 < 3; ++s2) {
      acc[2 + 2 * s2] += c.x * gr[s2] + c.y * gi[s2];
      acc[3 + 2 * s2] += c.x * gi[s2] - c.y * gr[s2];
    }
  }
  for (int q = 0; q < 8; ++q) {
    const double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) out[((long long)p * ns + nn) * 8 + q] = t;
  }
}

// fn[3 I + s] += -4 w h1h2h3 sum_{p of atom I} gamma_p sum_n g_n Re(conj(Y_pn) W_pns) for the
// projections of one k-point (Eq. NonlocForce:Discrete with the k-point weight w; fixed order).
__global__ void k_force_acc_k(const double* __restrict__ prj, const int* __restrict__ patom,
                              const double* __restrict__ gamma, int nproj, int ns, const double* __restrict__ occ,
                              double wdv, int natom, double* fn) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= natom) return;
  for (int s = 0; s < 3; ++s) {
    double acc = 0.0;
    for (int p = 0; p < nproj; ++p) {
      if (patom[p] != I) continue;
      double t = 0.0;
      for (int n = 0; n < ns; ++n) {
        const double* q = prj + ((long long)p * ns + n) * 8;
        t += occ[n] * (q[0] * q[2 + 2 * s] + q[1] * q[3 + 2 * s]);
      }
      acc += -4.0 * gamma[p] * wdv * t;
    }
    fn[3 * I + s] += acc;
  }
}

// f[I] = local partials (fixed order) into f[3 I + s]; fn copied into f[3 (natom + I) + s].
__global__ void k_force_fin(const double* __restrict__ loc, int nby, const double* __restrict__ fn, int natom,
                            double* f) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= natom) return;
  for (int s = 0; s < 3; ++s) {
    double fl = 0.0;
    for (int b = 0; b < nby; ++b) fl += loc[((long long)I * nby + b) * 3 + s];
    f[3 * I + s] = fl;
    f[3 * (natom + I) + s] = fn[3 * I + s];
  }
}

// f[atom] = local partials (fixed order) - 4 h1h2h3 sum_{p of atom} gamma_p sum_n g_n Y W
// (Eq. NonlocForce:Discrete; psi = U / sqrt(h1h2h3), so Y W = h1h2h3 (sum chi U)(sum chi grad U))
__global__ void k_force_sum(const double* __restrict__ loc, int nby, const double* __restrict__ prj,
                            const int* __restrict__ patom, const double* __restrict__ gamma, int nproj, int ns,
                            const double* __restrict__ occ, double dv, int natom, double* f) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= natom) return;
  for (int s = 0; s < 3; ++s) {
    double fl = 0.0;
    for (int b = 0; b < nby; ++b) fl += loc[((long long)I * nby + b) * 3 + s];
    double fn = 0.0;
    for (int p = 0; p < nproj; ++p) {
      if (patom[p] != I) continue;
      double t = 0.0;
      for (int n = 0; n < ns; ++n) t += occ[n] * prj[((long long)p * ns + n) * 4] * prj[((long long)p * ns + n) * 4 + 1 + s];
      fn += -4.0 * gamma[p] * dv * t;
    }
    f[3 * I + s] = fl;
    f[3 * (natom + I) + s] = fn;
  }
}
}  // namespace scf
}  // namespace sparc

// ------------------------------------------------------------------ SCF object
struct sparc_scf {
  sparc_ham* H = nullptr;
  int device = 0;                  // sparc_scf_destroy does not read H
  sparc::scf::Weights W{};
  std::vector<sparc::scf::Atom> atoms;
  double kT = 0.01, beta = 0.3, ptol = 1e-10, Ne = 0.0, e_self = 0.0;
  int hist = 7, nslot = 8, iter = 0, nblk = 0;
  int first_passes = 1;            // CheFSI passes of the first iteration
  sparc::scf::Atom* d_atoms = nullptr;
  double *d_b = nullptr, *d_rho = nullptr, *d_phi = nullptr, *d_eps = nullptr, *d_vxc = nullptr;
  double *d_vout = nullptr, *d_fres = nullptr, *d_vnext = nullptr;
  double *d_r = nullptr, *d_p = nullptr, *d_ap = nullptr;
  double *d_X = nullptr, *d_F = nullptr;
  double *d_part = nullptr, *d_sums = nullptr, *d_scal = nullptr, *d_occ = nullptr, *d_v0 = nullptr;
  void* d_Y = nullptr;
  size_t ybytes = 0;
  std::vector<sparc_ham*> Hk;      // one Hamiltonian per k-point (Hk[0] == H)
  std::vector<double> wk;          // k-point weights
  std::vector<std::vector<double>> lamk;   // Ritz values of the last step, per k
  double* d_wt = nullptr;          // weight of every Ritz value (nk > 1)
  int wt_n = 0;
  int nproj = 0;
  int* d_patom = nullptr;          // atom of each projector (forces); null if not given
  int last_ns = 0;                 // orbitals of the last iteration (occupations in d_occ)
};

namespace sparc {
namespace scf {

static void free_scf(sparc_scf* S) {
  void* ps[] = {S->d_atoms, S->d_b, S->d_rho, S->d_phi, S->d_eps, S->d_vxc, S->d_vout, S->d_fres,
                S->d_vnext, S->d_r, S->d_p, S->d_ap, S->d_X, S->d_F, S->d_part, S->d_sums,
                S->d_scal, S->d_occ, S->d_v0, S->d_Y, S->d_patom, S->d_wt};
  for (void* p : ps)
    if (p) cudaFree(p);
}

// V_xc of rho, V_out = phi + V_xc and the grid terms; then the Poisson solve before it.
static sparc_status poisson(sparc_scf* S, cudaStream_t st, int* iters) {
  sparc_ham* H = S->H;
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  const int nb = S->nblk;
  const int n1 = H->gd.n1, n2 = H->gd.n2, n3 = H->gd.n3, no = H->gd.no;
  // mean of rho + b (the truncation error of b), removed from the right-hand side
  k_sum2<<<nb, TPB, 0, st>>>(S->d_rho, S->d_b, nd, S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, nb, 1, 1, S->d_scal + S_MEAN);
  k_scale1<<<1, 1, 0, st>>>(S->d_scal + S_MEAN, 1.0 / (double)nd);
  // warm start from the previous phi: r = rhs - A phi, p = r
  k_lapA<<<nb, TPB, 0, st>>>(S->d_phi, S->d_ap, n1, n2, n3, no, S->W, S->d_part, nullptr);
  k_cg_init<<<nb, TPB, 0, st>>>(S->d_rho, S->d_b, S->d_ap, nd, S->d_scal, S->d_r, S->d_p, S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, nb, 1, 1, S->d_scal + S_RR0);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part + nb, nb, 1, 1, S->d_scal + S_RHS2);
  SPARC_CUDA(ctx, cudaMemsetAsync(S->d_scal + S_DONE, 0, 2 * sizeof(double), st));
  ctx->launches += 8;
  double* part2 = S->d_part + 2 * (size_t)nb;
  int it = 0;
  const int batch = 25, max_it = ctx->inject_cg_max > 0 ? ctx->inject_cg_max : 4000;
  double hs[2] = {0.0, 0.0};
  while (it < max_it) {
    for (int q = 0; q < batch; ++q, ++it) {
      const int par = it & 1;
      k_lapA<<<nb, TPB, 0, st>>>(S->d_p, S->d_ap, n1, n2, n3, no, S->W, S->d_part, S->d_scal);
      k_cg_update<<<nb, TPB, 0, st>>>(S->d_phi, S->d_r, S->d_p, S->d_ap, nd, S->d_part, nb, par, S->d_scal, part2);
      k_cg_dir<<<nb, TPB, 0, st>>>(S->d_r, S->d_p, nd, part2, nb, par, S->ptol, S->d_scal);
    }
    ctx->launches += 3 * batch;
    SPARC_CUDA(ctx, cudaMemcpyAsync(hs, S->d_scal + S_DONE, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    if (hs[0] != 0.0) break;
  }
  *iters = (int)hs[1];
  if (hs[0] == 0.0) return fail(ctx, SPARC_ERR_NO_CONVERGENCE, "Poisson CG did not reach its tolerance");
  // zero mean of phi
  k_sum2<<<nb, TPB, 0, st>>>(S->d_phi, nullptr, nd, S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, nb, 1, 1, S->d_scal + S_MEAN);
  k_shift<<<ceil_div(nd, TPB), TPB, 0, st>>>(S->d_phi, nd, S->d_scal + S_MEAN, 1.0 / (double)nd);
  ctx->launches += 3;
  return SPARC_OK;
}

}  // namespace scf
}  // namespace sparc

using namespace sparc;
using namespace sparc::scf;

extern "C" sparc_status sparc_scf_create_k(sparc_ham* const* Hs, int nk, const double* wk, const sparc_scf_desc* d,
                                           sparc_scf** out) {
  if (!Hs || nk < 1 || !Hs[0] || !wk || !d || !out) return SPARC_ERR_INVALID_ARG;
  *out = nullptr;
  sparc_ham* H = Hs[0];
  sparc_ctx* ctx = H->ctx;
  bool any_cplx = false;
  for (int k = 0; k < nk; ++k) {
    const sparc_ham* Hk = Hs[k];
    if (!Hk || Hk->ctx != ctx || !(wk[k] > 0.0) || !isfinite(wk[k]))
      return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_create_k: Hamiltonians on one context, weights > 0");
    for (int a = 0; a < 3; ++a)
      if (Hk->grid.n[a] != H->grid.n[a] || Hk->grid.h[a] != H->grid.h[a])
        return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_create_k: the k-points must share the grid");
    if (Hk->grid.fd_radius != H->grid.fd_radius || Hk->nproj != H->nproj)
      return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_create_k: the k-points must share stencil and projectors");
    any_cplx = any_cplx || Hk->gd.cplx;
  }
  if (d->natom < 1 || !d->R || !d->Z || !d->rc || !d->v0 || !(d->kT > 0.0) || !(d->mix_beta > 0.0) ||
      d->mix_history < 0 || d->mix_history > MAXHIST || !(d->poisson_tol > 0.0) || d->first_passes < 0 ||
      d->first_passes > 64)
    return fail(ctx, SPARC_ERR_INVALID_ARG,
                "sparc_scf_create: need natom >= 1, R, Z, rc, v0, kT > 0, mix_beta > 0, 0 <= mix_history <= 8, "
                "poisson_tol > 0, 0 <= first_passes <= 64");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  sparc_scf* S = new sparc_scf();
  S->H = H;
  S->Hk.assign(Hs, Hs + nk);
  S->wk.assign(wk, wk + nk);
  S->lamk.assign(nk, std::vector<double>());
  S->device = ctx->device;
  S->kT = d->kT;
  S->beta = d->mix_beta;
  S->hist = d->mix_history;
  S->nslot = d->mix_history + 1;
  S->ptol = d->poisson_tol;
  S->first_passes = std::max(1, d->first_passes);
  const long long nd = H->gd.nd;
  S->nblk = ceil_div(nd, TPB);
  for (int s = 0; s < 3; ++s)
    for (int p = 0; p <= MAX_FD; ++p) S->W.w[s][p] = p <= H->gd.no ? -2.0 * H->gd.coef[s][p] : 0.0;
  const int n[3] = {H->grid.n[0], H->grid.n[1], H->grid.n[2]};
  for (int I = 0; I < d->natom; ++I) {
    Atom A;
    A.Z = d->Z[I];
    A.rc = d->rc[I];
    if (!(A.Z > 0.0) || !(A.rc > 0.0)) {
      delete S;
      return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_create: Z and rc must be positive");
    }
    for (int s = 0; s < 3; ++s) {
      A.R[s] = d->R[3 * I + s];
      const double hs = H->grid.h[s];
      A.nb[s] = (int)ceil(6.0 * A.rc / hs);   // charge error below 1e-8 (Eq. PseudochargeRadiusChoice)
      A.c[s] = (int)nearbyint((A.R[s] + 0.5 * n[s] * hs) / hs);   // nearest node, ties to even
    }
    S->atoms.push_back(A);
    S->Ne += A.Z;
  }
  const size_t vb = (size_t)nd * sizeof(double);
  bool ok = cudaMalloc(&S->d_atoms, S->atoms.size() * sizeof(Atom)) == cudaSuccess;
  double** vecs[] = {&S->d_b, &S->d_rho, &S->d_phi, &S->d_eps, &S->d_vxc, &S->d_vout, &S->d_fres, &S->d_vnext,
                     &S->d_r, &S->d_p, &S->d_ap};
  for (double** v : vecs) ok = ok && cudaMalloc(v, vb) == cudaSuccess;
  ok = ok && cudaMalloc(&S->d_X, vb * S->nslot) == cudaSuccess && cudaMalloc(&S->d_F, vb * S->nslot) == cudaSuccess;
  ok = ok && cudaMalloc(&S->d_part, (size_t)S->nblk * std::max(NPAIR, 4) * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&S->d_sums, NPAIR * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&S->d_scal, S_COUNT * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&S->d_occ, 4096 * sizeof(double)) == cudaSuccess;
  const size_t v0b = vb * (any_cplx ? 2 : 1);
  ok = ok && cudaMalloc(&S->d_v0, v0b) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_scf(S);
    delete S;
    return fail(ctx, SPARC_ERR_OOM, "sparc_scf_create: device allocation failed");
  }
  // from here on, every failure return frees S; success releases it to the caller
  struct Owner {
    sparc_scf* s;
    ~Owner() { if (s) { free_scf(s); delete s; } }
  } owner{S};
  cudaStream_t st = 0;
  SPARC_CUDA(ctx, cudaMemcpy(S->d_atoms, S->atoms.data(), S->atoms.size() * sizeof(Atom), cudaMemcpyHostToDevice));
  SPARC_CUDA(ctx, cudaMemcpy(S->d_v0, d->v0, v0b, cudaMemcpyHostToDevice));
  S->nproj = H->nproj;
  if (d->proj_atom && H->nproj > 0) {
    for (int p = 0; p < H->nproj; ++p)
      if (d->proj_atom[p] < 0 || d->proj_atom[p] >= d->natom)
        return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_create: proj_atom out of range");
    SPARC_CUDA(ctx, cudaMalloc(&S->d_patom, H->nproj * sizeof(int)));
    SPARC_CUDA(ctx, cudaMemcpy(S->d_patom, d->proj_atom, H->nproj * sizeof(int), cudaMemcpyHostToDevice));
  }
  SPARC_CUDA(ctx, cudaMemset(S->d_phi, 0, vb));
  SPARC_CUDA(ctx, cudaMemset(S->d_scal, 0, S_COUNT * sizeof(double)));
  // pseudocharges and self energy
  k_pseudocharge<<<S->nblk, TPB, 0, st>>>(n[0], n[1], n[2], H->grid.h[0], H->grid.h[1], H->grid.h[2], H->gd.no,
                                          S->W, S->d_atoms, (int)S->atoms.size(), S->d_b, S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, S->nblk, 1, 1, S->d_scal + S_ESELF);
  // starting potential from a superposition of atomic densities: rho0 = -b (Gaussian
  // atoms, neutral with the pseudocharges, so phi0 = 0), V_in = V_xc(rho0)
  k_neg<<<S->nblk, TPB, 0, st>>>(S->d_b, S->d_rho, nd);
  k_lda<<<S->nblk, TPB, 0, st>>>(S->d_rho, nd, S->d_eps, S->d_vxc);
  ctx->launches += 4;
  SPARC_LAUNCH(ctx, "scf setup");
  sparc_status rc = SPARC_OK;
  for (int k = 0; k < nk && rc == SPARC_OK; ++k) rc = sparc_ham_set_veff(Hs[k], S->d_vxc, 1, st);
  if (rc != SPARC_OK) return rc;
  SPARC_CUDA(ctx, cudaMemcpy(&S->e_self, S->d_scal + S_ESELF, sizeof(double), cudaMemcpyDeviceToHost));
  owner.s = nullptr;
  *out = S;
  return SPARC_OK;
}

extern "C" sparc_status sparc_scf_create(sparc_ham* H, const sparc_scf_desc* d, sparc_scf** out) {
  const double one = 1.0;
  return sparc_scf_create_k(&H, 1, &one, d, out);
}

extern "C" void sparc_scf_destroy(sparc_scf* S) {
  if (!S) return;
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  free_scf(S);
  delete S;
}

extern "C" sparc_status sparc_scf_read(const sparc_scf* S, int which, double* dst, void* stream) {
  if (!S || !dst) return SPARC_ERR_INVALID_ARG;
  const double* src = nullptr;
  switch (which) {
    case 0: src = S->d_b; break;
    case 1: src = S->d_rho; break;
    case 2: src = S->d_phi; break;
    case 3: src = S->d_vxc; break;
    case 4: src = S->d_vout; break;
    case 5: src = S->H->d_veff; break;
    default: return fail(S->H->ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_read: which must be 0..5");
  }
  SPARC_CUDA(S->H->ctx, cudaMemcpyAsync(dst, src, (size_t)S->H->gd.nd * sizeof(double), cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
  return SPARC_OK;
}

extern "C" sparc_status sparc_scf_set_density(sparc_scf* S, const float* dy, double scale, void* stream) {
  if (!S) return SPARC_ERR_INVALID_ARG;
  sparc_ham* H = S->H;
  sparc_ctx* ctx = H->ctx;
  if (S->iter != 0) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_set_density: only before the first step");
  if (!isfinite(scale)) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_set_density: scale must be finite");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const long long nd = H->gd.nd;
  const int nb = S->nblk;
  const double dv = H->grid.h[0] * H->grid.h[1] * H->grid.h[2];
  k_guess<<<nb, TPB, 0, st>>>(S->d_b, dy, scale, nd, S->d_rho, S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, nb, 1, 1, S->d_scal + S_RHOSUM);
  k_renorm_vin<<<nb, TPB, 0, st>>>(S->d_rho, S->d_scal, S->Ne, dv, nd);
  ctx->launches += 3;
  SPARC_LAUNCH(ctx, "starting density");
  int piters = 0;
  sparc_status rc = poisson(S, st, &piters);
  if (rc != SPARC_OK) return rc;
  k_lda<<<nb, TPB, 0, st>>>(S->d_rho, nd, S->d_eps, S->d_vxc);
  k_add<<<nb, TPB, 0, st>>>(S->d_phi, S->d_vxc, S->d_vnext, nd);
  ctx->launches += 2;
  SPARC_LAUNCH(ctx, "starting potential");
  for (sparc_ham* Hk : S->Hk) {
    rc = sparc_ham_set_veff(Hk, S->d_vnext, 1, stream);
    if (rc != SPARC_OK) return rc;
  }
  return SPARC_OK;
}

extern "C" sparc_status sparc_scf_step(sparc_scf* S, sparc_dtype dtype, int m, void* U, int ns, int64_t ld,
                                       double* eig, sparc_scf_info* info, void* stream) {
  if (!S || !U || !eig || !info) return SPARC_ERR_INVALID_ARG;
  sparc_ham* H = S->H;
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  const int nk = (int)S->Hk.size();
  if (m < 1 || ns < 1 || ns > 4096 || ld < nd || (long long)nk * ns > 4096)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_step: need m >= 1, 1 <= nk ns <= 4096, ld >= Nd");
  if (2.0 * ns < S->Ne) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_step: 2 ns must hold the electrons");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = dtype == SPARC_F64 ? 8 : dtype == SPARC_F32 ? 4 : dtype == SPARC_C128 ? 16 : 8;
  const size_t kbytes = (size_t)ld * ns * es;   // one k-point's orbitals
  const size_t ybytes = kbytes * nk;
  if (ybytes > S->ybytes) {
    if (S->d_Y) cudaFree(S->d_Y);
    S->d_Y = nullptr;
    S->ybytes = 0;
    if (cudaMalloc(&S->d_Y, ybytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SPARC_ERR_OOM, "sparc_scf_step: filter buffer allocation failed");
    }
    S->ybytes = ybytes;
  }
  if (nk > 1 && S->wt_n != nk * ns) {   // the weight of every Ritz value
    std::vector<double> wt((size_t)nk * ns);
    for (int k = 0; k < nk; ++k)
      for (int n = 0; n < ns; ++n) wt[(size_t)k * ns + n] = S->wk[k];
    if (S->d_wt) cudaFree(S->d_wt);
    S->d_wt = nullptr;
    S->wt_n = 0;
    SPARC_CUDA(ctx, cudaMalloc(&S->d_wt, wt.size() * sizeof(double)));
    SPARC_CUDA(ctx, cudaMemcpy(S->d_wt, wt.data(), wt.size() * sizeof(double), cudaMemcpyHostToDevice));
    S->wt_n = nk * ns;
  }
  // 1. filter bounds per k: Lanczos upper bound; cutoff and lower end from the previous
  //    Ritz values, or the Lanczos lower end and a Weyl estimate at the first iteration
  std::vector<double> a0l(nk), b(nk), a0(nk), a(nk);
  sparc_status rc = SPARC_OK;
  for (int k = 0; k < nk; ++k) {
    rc = sparc_lanczos_bounds(S->Hk[k], 10, S->d_v0, &a0l[k], &b[k], stream);
    if (rc != SPARC_OK) return rc;
  }
  // 2. CheFSI: scaled filter and Rayleigh-Ritz (FP64, or mixed for FP32 data); the
  //    first iteration repeats it at the fixed starting potential (Section 4).  With
  //    k-points one batched filter serves all of them.
  const int passes = (S->iter == 0) ? S->first_passes : 1;
  const int mode = (dtype == SPARC_F32 || dtype == SPARC_C64) ? SPARC_RR_MIXED : SPARC_RR_FP64;
  for (int pass = 0; pass < passes; ++pass) {
    for (int k = 0; k < nk; ++k) {
      const std::vector<double>& lp = S->lamk[k];
      if ((int)lp.size() == ns) {
        a0[k] = lp.front();
        a[k] = lp.back();
      } else {
        a0[k] = a0l[k];
        a[k] = a0[k] + (b[k] - a0[k]) * pow((double)ns / (double)nd, 2.0 / 3.0);
      }
      if (!(a[k] < b[k])) a[k] = 0.5 * (a0[k] + b[k]);
      if (!(a0[k] < a[k])) a0[k] = a[k] - 1e-3 * (b[k] - a[k]);
    }
    if (nk == 1) rc = sparc_cheb_filter(H, dtype, m, a[0], b[0], a0[0], U, S->d_Y, ns, ld, stream);
    else rc = sparc_cheb_filter_batch(S->Hk.data(), nk, dtype, m, a.data(), b.data(), a0.data(), U, S->d_Y, ns, ld,
                                      stream);
    if (rc != SPARC_OK) return rc;
    for (int k = 0; k < nk; ++k) {
      rc = sparc_rayleigh_ritz(S->Hk[k], dtype, (char*)S->d_Y + k * kbytes, ns, ld, eig + (size_t)k * ns, mode, stream);
      if (rc != SPARC_OK) return rc;
    }
    SPARC_CUDA(ctx, cudaMemcpyAsync(U, S->d_Y, ybytes, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < nk; ++k) {
      S->lamk[k].assign(ns, 0.0);
      SPARC_CUDA(ctx, cudaMemcpyAsync(S->lamk[k].data(), eig + (size_t)k * ns, ns * sizeof(double),
                                      cudaMemcpyDeviceToHost, st));
    }
    if (pass + 1 < passes) SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  }
  // 3. Fermi level and occupations over all k-points
  k_fermi<<<1, TPB, 0, st>>>(eig, nk > 1 ? S->d_wt : nullptr, nk * ns, S->Ne, S->kT, S->d_occ, S->d_scal);
  // 4. density rho = 2 sum_k w_k sum_n g_nk |u_nk|^2 / (h1h2h3)
  const double dv = H->grid.h[0] * H->grid.h[1] * H->grid.h[2];
  const int nb = S->nblk;
  for (int k = 0; k < nk; ++k) {
    const char* Uk = (const char*)U + k * kbytes;
    const double* occk = S->d_occ + (size_t)k * ns;
    const double w = nk > 1 ? S->wk[k] : 1.0;
    switch (dtype) {
      case SPARC_F64: k_density<double><<<nb, TPB, 0, st>>>((const double*)Uk, ld, ns, nd, occk, 2.0 / dv, w, k, S->d_rho); break;
      case SPARC_F32: k_density<float><<<nb, TPB, 0, st>>>((const float*)Uk, ld, ns, nd, occk, 2.0 / dv, w, k, S->d_rho); break;
      case SPARC_C128: k_density<cf64><<<nb, TPB, 0, st>>>((const cf64*)Uk, ld, ns, nd, occk, 2.0 / dv, w, k, S->d_rho); break;
      case SPARC_C64: k_density<cf32><<<nb, TPB, 0, st>>>((const cf32*)Uk, ld, ns, nd, occk, 2.0 / dv, w, k, S->d_rho); break;
    }
  }
  ctx->launches += 1 + nk;
  SPARC_LAUNCH(ctx, "fermi and density");
  // 5. Poisson: -(1/4pi) lap phi = rho + b
  int piters = 0;
  rc = poisson(S, st, &piters);
  if (rc != SPARC_OK) return rc;
  // 6. LDA, V_out = phi + V_xc, energy terms, residual
  k_lda<<<nb, TPB, 0, st>>>(S->d_rho, nd, S->d_eps, S->d_vxc);
  k_vout<<<nb, TPB, 0, st>>>(S->d_phi, S->d_vxc, S->d_eps, S->d_rho, S->d_b, H->d_veff, nd, S->d_vout, S->d_fres,
                             S->d_part);
  k_sum_parts<<<1, 32, 0, st>>>(S->d_part, nb, 4, 4, S->d_scal + S_EXC);
  // 7. Anderson extrapolation of V_eff over the last mix_history iterations
  const int k = S->iter;
  const int sl = k % S->nslot;
  SPARC_CUDA(ctx, cudaMemcpyAsync(S->d_X + (size_t)sl * nd, H->d_veff, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SPARC_CUDA(ctx, cudaMemcpyAsync(S->d_F + (size_t)sl * nd, S->d_fres, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int mm = std::min(k, S->hist);
  if (mm > 0) {
    k_anderson_dots<<<nb, TPB, 0, st>>>(S->d_F, nd, S->nslot, k, mm, S->d_part);
    const int np = mm * (mm + 1) / 2 + mm;
    k_sum_parts<<<1, 64, 0, st>>>(S->d_part, nb, NPAIR, np, S->d_sums);
    k_anderson_solve<<<1, 32, 0, st>>>(S->d_sums, mm, S->d_scal);
    ctx->launches += 3;
  }
  k_anderson_next<<<nb, TPB, 0, st>>>(S->d_X, S->d_F, nd, S->nslot, k, mm, S->beta, S->d_scal, S->d_vnext);
  ctx->launches += 4;
  SPARC_LAUNCH(ctx, "xc, energy and mixing");
  for (sparc_ham* Hk : S->Hk) {
    rc = sparc_ham_set_veff(Hk, S->d_vnext, 1, stream);
    if (rc != SPARC_OK) return rc;
  }
  double hs[S_COUNT];
  SPARC_CUDA(ctx, cudaMemcpyAsync(hs, S->d_scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  const double e_xc = dv * hs[S_EXC], e_el = dv * hs[S_EEL];
  info->e_band = hs[S_EBAND];
  info->e_xc = e_xc;
  info->e_el = e_el;
  info->e_self = S->e_self;
  info->e_entropy = hs[S_ENT];
  info->free_energy = hs[S_EBAND] + e_xc + e_el - S->e_self + hs[S_ENT];
  info->fermi = hs[S_MU];
  info->nelec = hs[S_NEL];
  info->vresid = sqrt(hs[S_RES2] / std::max(hs[S_VOUT2], 1e-300));
  info->poisson_iters = piters;
  S->last_ns = ns;
  info->a0 = a0[0];   // the filter bounds of the first k-point
  info->a = a[0];
  info->b = b[0];
  ++S->iter;
  return SPARC_OK;
}

extern "C" sparc_status sparc_scf_forces(sparc_scf* S, sparc_dtype dtype, const void* U, int ns, int64_t ld,
                                         double* f_host, void* stream) {
  if (!S || !U || !f_host) return SPARC_ERR_INVALID_ARG;
  sparc_ham* H = S->H;
  sparc_ctx* ctx = H->ctx;
  const long long nd = H->gd.nd;
  if (S->last_ns != ns || ns < 1 || ld < nd)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_forces: needs the orbitals of the last sparc_scf_step");
  const int nk = (int)S->Hk.size();
  const bool cplx = dtype == SPARC_C128 || dtype == SPARC_C64;
  if ((int)dtype < 0 || (int)dtype > 3) return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_forces: unknown dtype");
  if (!cplx && (nk != 1 || H->gd.cplx))
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_forces: real orbitals need one k-point at Gamma");
  if (H->nproj > 0 && !S->d_patom)
    return fail(ctx, SPARC_ERR_INVALID_ARG, "sparc_scf_forces: sparc_scf_desc.proj_atom was not given");
  SPARC_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int natom = (int)S->atoms.size();
  GWeights G{};
  for (int s2 = 0; s2 < 3; ++s2) {
    const int no = H->gd.no;
    double fo = 1.0;
    for (int q = 2; q <= no; ++q) fo *= q;
    for (int p = 0; p <= MAX_FD; ++p) {
      if (p == 0 || p > no) { G.w[s2][p] = 0.0; continue; }
      double den = 1.0;
      for (int q = 2; q <= no - p; ++q) den *= q;
      for (int q = 2; q <= no + p; ++q) den *= q;
      G.w[s2][p] = ((p % 2) ? 1.0 : -1.0) * fo * fo / (H->grid.h[s2] * p * den);
    }
  }
  int maxcube = 1;
  for (const Atom& A : S->atoms) maxcube = std::max(maxcube, (2 * A.nb[0] + 1) * (2 * A.nb[1] + 1) * (2 * A.nb[2] + 1));
  const int nby = ceil_div(maxcube, TPB);
  // per-call buffers, freed on every return path
  struct DevDoubles {
    double* p = nullptr;
    ~DevDoubles() { if (p) cudaFree(p); }
  } loc, prj, fo;
  const int np = H->nproj;
  SPARC_CUDA(ctx, cudaMalloc(&loc.p, (size_t)natom * nby * 3 * sizeof(double)));
  SPARC_CUDA(ctx, cudaMalloc(&prj.p, (size_t)std::max(np, 1) * ns * (cplx ? 8 : 4) * sizeof(double)));
  SPARC_CUDA(ctx, cudaMalloc(&fo.p, (size_t)natom * (cplx ? 9 : 6) * sizeof(double)));
  double* const d_loc = loc.p;
  double* const d_prj = prj.p;
  double* const d_f = fo.p;
  k_force_local<<<dim3(natom, nby), TPB, 0, st>>>(H->gd.n1, H->gd.n2, H->gd.n3, H->grid.h[0], H->grid.h[1],
                                                   H->grid.h[2], H->gd.no, S->W, G, S->d_atoms, S->d_phi, d_loc);
  ++ctx->launches;
  const double dvk = H->grid.h[0] * H->grid.h[1] * H->grid.h[2];
  if (cplx) {
    // Bloch orbitals: the nonlocal force summed over the k-points with their weights
    double* d_fn = d_f + 6 * (size_t)natom;
    SPARC_CUDA(ctx, cudaMemsetAsync(d_fn, 0, 3 * (size_t)natom * sizeof(double), st));
    const size_t es = dtype == SPARC_C128 ? 16 : 8;
    for (int k = 0; k < nk && np > 0; ++k) {
      sparc_ham* Hk = S->Hk[k];
      sparc_status rc = ensure_vals(Hk, SPARC_C128);
      if (rc != SPARC_OK) return rc;
      const void* Uk = (const char*)U + (size_t)k * ld * ns * es;
      const cf64* pv = (const cf64*)Hk->d_p_val[SPARC_C128];
      const double* ph_r = Hk->gd.ph_re;
      const double* ph_i = Hk->gd.ph_im;
      if (dtype == SPARC_C128)
        k_force_proj_c<cf64><<<dim3(np, ns), TPB, 0, st>>>((const cf64*)Uk, ld, H->gd.n1, H->gd.n2, H->gd.n3, H->gd.no,
                                                            G, Hk->d_p_off, Hk->d_p_g, pv, ph_r[0], ph_i[0], ph_r[1],
                                                            ph_i[1], ph_r[2], ph_i[2], ns, d_prj);
      else
        k_force_proj_c<cf32><<<dim3(np, ns), TPB, 0, st>>>((const cf32*)Uk, ld, H->gd.n1, H->gd.n2, H->gd.n3, H->gd.no,
                                                            G, Hk->d_p_off, Hk->d_p_g, pv, ph_r[0], ph_i[0], ph_r[1],
                                                            ph_i[1], ph_r[2], ph_i[2], ns, d_prj);
      const double w = nk > 1 ? S->wk[k] : 1.0;
      k_force_acc_k<<<ceil_div(natom, 64), 64, 0, st>>>(d_prj, S->d_patom, H->d_gamma, np, ns, S->d_occ + (size_t)k * ns,
                                                        w * dvk, natom, d_fn);
      ctx->launches += 2;
    }
    k_force_fin<<<ceil_div(natom, 64), 64, 0, st>>>(d_loc, nby, d_fn, natom, d_f);
    ++ctx->launches;
    SPARC_LAUNCH(ctx, "forces");
    std::vector<double> hf((size_t)natom * 6);
    SPARC_CUDA(ctx, cudaMemcpyAsync(hf.data(), d_f, hf.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPARC_CUDA(ctx, cudaStreamSynchronize(st));
    for (int i = 0; i < 3 * natom; ++i) {
      f_host[i] = hf[i] + hf[3 * natom + i];
      f_host[3 * natom + i] = hf[i];
      f_host[6 * natom + i] = hf[3 * natom + i];
    }
    return SPARC_OK;
  }
  if (np > 0) {
    sparc_status rc = ensure_vals(H, SPARC_F64);
    if (rc != SPARC_OK) return rc;
    if (dtype == SPARC_F64)
      k_force_proj<double><<<dim3(np, ns), TPB, 0, st>>>((const double*)U, ld, H->gd.n1, H->gd.n2, H->gd.n3, H->gd.no,
                                                          G, H->d_p_off, H->d_p_g, (const double*)H->d_p_val[SPARC_F64],
                                                          ns, d_prj);
    else
      k_force_proj<float><<<dim3(np, ns), TPB, 0, st>>>((const float*)U, ld, H->gd.n1, H->gd.n2, H->gd.n3, H->gd.no,
                                                         G, H->d_p_off, H->d_p_g, (const double*)H->d_p_val[SPARC_F64],
                                                         ns, d_prj);
    ++ctx->launches;
  }
  const double dv = H->grid.h[0] * H->grid.h[1] * H->grid.h[2];
  k_force_sum<<<ceil_div(natom, 64), 64, 0, st>>>(d_loc, nby, d_prj, S->d_patom, H->d_gamma, np, ns, S->d_occ, dv,
                                                   natom, d_f);
  ++ctx->launches;
  SPARC_LAUNCH(ctx, "forces");
  std::vector<double> hf((size_t)natom * 6);
  SPARC_CUDA(ctx, cudaMemcpyAsync(hf.data(), d_f, hf.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPARC_CUDA(ctx, cudaStreamSynchronize(st));
  for (int i = 0; i < 3 * natom; ++i) {
    f_host[i] = hf[i] + hf[3 * natom + i];           // total
    f_host[3 * natom + i] = hf[i];                   // local part
    f_host[6 * natom + i] = hf[3 * natom + i];       // nonlocal part
  }
  return SPARC_OK;
}
