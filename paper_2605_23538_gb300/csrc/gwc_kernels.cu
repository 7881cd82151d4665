// gwc_kernels.cu -- CUDA kernels of the dark-siren likelihood (sm_103a).
//
//   k_prologue   several CTAs per Lambda (a 16-CTA cluster for small batches, three
//                CTAs otherwise), FP64: domain check, the d_L(z) inversion table
//                (Eq. 1), mass-model normalisations and smoothing-window tables, the
//                redshift-prior normalisation, and the constants each sample needs.
//   k_fused      the hot loop, persistent: a CTA stages a chunk of samples (or
//                injections) in shared memory once and its warps sweep them for a tile
//                of Lambda points, each warp accumulating the per-(chunk, Lambda)
//                logsumexp partial (max, sum w, sum w^2 and, with the gradient, 13 or 16
//                weighted statistics) of Eqs. 5-7 online in registers.
//   k_kde        the paper's KDE form of the event term (Eqs. 5-7 with a finite kernel).
//   k_plain_*    the single-Lambda baseline: per-sample weights written to memory and
//                reduced in separate passes.
//   k_merge      one CTA per Lambda, FP64: merges the partials of each event in a fixed
//                order into ln L_i and N_eff,i, the injection partials into ln xi, and
//                forms the total of Eq. 3 and its gradient.  Deterministic.
#include "gwc_internal.cuh"
#include "gwc_kernels.h"

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <mutex>
#include <type_traits>

#include <cooperative_groups.h>

namespace gwc {

__constant__ double c_glx[NGL];   // Gauss-Legendre nodes on [-1, 1] (the smoothing window)
__constant__ double c_glw[NGL];   // and weights
__constant__ double c_gzx[NGL_Z];  // the same for the z quadrature
__constant__ double c_gzw[NGL_Z];

// n-point Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on the Legendre
// polynomial from the three-term recurrence, started at the usual cosine estimate.
static void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// One upload per device for the life of the process (the values never change), shared by
// gwc_create and the context-free entry point.
struct ProArgs;
template <bool CL> __global__ void k_prologue(ProArgs A);

cudaError_t ensure_prologue_ready() {
  constexpr int MAX_DEV = 64;
  static std::mutex mu;
  static bool done[MAX_DEV] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (done[dev]) return cudaSuccess;
  double x[NGL], w[NGL], xz[NGL_Z], wz[NGL_Z];
  gauss_legendre(NGL, x, w);
  gauss_legendre(NGL_Z, xz, wz);
  e = cudaMemcpyToSymbol(c_glx, x, sizeof(double) * NGL);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_glw, w, sizeof(double) * NGL);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gzx, xz, sizeof(double) * NGL_Z);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gzw, wz, sizeof(double) * NGL_Z);
  // the small-batch shape is a cluster of 16 CTAs, beyond the portable size of 8
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prologue<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// ------------------------------------------------------------------ FP64 helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sums of V values (fixed order); every thread gets the totals
template <int V>
__device__ void block_sum(double (&v)[V], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < V; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
    for (int i = 0; i < V; ++i) red[i * 32 + w] = v[i];
  __syncthreads();
  if (threadIdx.x < V) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[threadIdx.x * 32 + k];
    red[threadIdx.x * 32] = s;
  }
  __syncthreads();
  for (int i = 0; i < V; ++i) v[i] = red[i * 32];
  __syncthreads();
}

// inclusive scan of V values over the block (fixed order)
template <int V>
__device__ void block_scan(double (&v)[V], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < V; ++i) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, v[i], o);
      if (lane >= o) v[i] += y;
    }
  }
  if (lane == 31)
    for (int i = 0; i < V; ++i) red[i * 32 + w] = v[i];
  __syncthreads();
  for (int i = 0; i < V; ++i) {
    double off = 0.0;
    for (int k = 0; k < w; ++k) off += red[i * 32 + k];
    v[i] += off;
  }
  __syncthreads();
  (void)nw;
}

__device__ __forceinline__ double softplus_d(double a) {
  return a > 0.0 ? a + log1p(exp(-a)) : log1p(exp(a));
}
__device__ __forceinline__ double sigmoid_d(double a) {
  return a >= 0.0 ? 1.0 / (1.0 + exp(-a)) : exp(a) / (1.0 + exp(a));
}

// S(m), 1 - S(m) and dS/d(delta_m) inside the smoothing window (0 < mp < dm), from
// r1 = 1/mp and r2 = 1/(mp - dm), which the callers reuse: on this GPU an FP64 division
// is a long sequence of FP64 instructions, each costing a whole warp-instruction
__device__ __forceinline__ void smooth_d(double mp, double dm, double r1, double r2, double& S,
                                         double& oneS, double& dSddm) {
  const double f = dm * (r1 + r2);
  const double e = exp(-fabs(f));
  const double q = 1.0 / (1.0 + e);
  S = f > 0.0 ? e * q : q;
  oneS = f > 0.0 ? q : e * q;
  dSddm = -S * oneS * (r1 + mp * (r2 * r2));
}

__device__ bool lambda_ok(const double* L, bool mp) {
  for (int i = 0; i < n_params(mp); ++i)
    if (!isfinite(L[i])) return false;
  const bool base = L[P_H0] > 0.0 && L[P_OM] >= 0.0 && L[P_OM] <= 1.0 && L[P_MMIN] > 0.0 &&
                    L[P_MMAX] > L[P_MMIN] && L[P_DM] >= 0.0 && L[P_MMIN] + L[P_DM] < L[P_MMAX] &&
                    L[P_SIG] > 0.0 && L[P_LAM] >= 0.0 && L[P_LAM] <= 1.0 && L[P_ZP] > -1.0;
  return base && (!mp || (L[P_SIG2] > 0.0 && L[P_LAM1] >= 0.0 && L[P_LAM1] <= 1.0));
}

// ln Z_G = ln of the mass of N(mu, sig) inside [mmin, mmax] (erfc forms without
// cancellation on either side) and d ln Z_G / d(mu, sig, mmin, mmax) into out[0..4]
// Called by a whole warp: its lanes evaluate the two erfc and the two exp side by side
// (the same instructions on arguments chosen by the lane), so the warp runs one erfc
// and one exp where a single thread would run two of each; lane 0 writes out.
__device__ void gauss_mass(double mu, double sig, double mmin, double mmax, double* out) {
  const int l = threadIdx.x & 31;
  const double is = 1.0 / sig;
  const double A_ = (mmin - mu) * is, B_ = (mmax - mu) * is, r2 = 0.70710678118654752440;
  // erfc arguments: A > 0: erfc(A) - erfc(B); B < 0: erfc(-B) - erfc(-A); else both tails
  const double x0 = A_ > 0.0 ? A_ : (B_ < 0.0 ? -B_ : B_);
  const double x1 = A_ > 0.0 ? B_ : -A_;
  const double ef = erfc((l == 1 ? x1 : x0) * r2);
  const double E0 = __shfl_sync(0xffffffffu, ef, 0), E1 = __shfl_sync(0xffffffffu, ef, 1);
  const double ZG = (A_ > 0.0 || B_ < 0.0) ? 0.5 * (E0 - E1) : 1.0 - 0.5 * (E0 + E1);
  const double ph = 0.39894228040143267794 * exp(-0.5 * (l == 1 ? B_ * B_ : A_ * A_));
  const double phA = __shfl_sync(0xffffffffu, ph, 0), phB = __shfl_sync(0xffffffffu, ph, 1);
  const double lz = log(ZG);
  const double iz = 1.0 / (sig * ZG);
  if (l == 0) {
    out[0] = lz;
    out[1] = (phA - phB) * iz;                // d ln Z_G / d mu
    out[2] = (A_ * phA - B_ * phB) * iz;      // d ln Z_G / d sigma
    out[3] = -phA * iz;                       // d ln Z_G / d m_min
    out[4] = phB * iz;                        // d ln Z_G / d m_max
  }
}

// ---------------------------------------------------------------------- prologue
constexpr int PRO_THREADS = 256;
constexpr int ZPANELS = 256;   // panels of the z quadrature (one per thread)

// (1) I(z) and J(z) = dI/dOm on the ZPANELS + 1 panel edges of [0, zmax] (an NGL_Z-point
// Gauss-Legendre rule per panel, one panel per thread, then a block scan), and D(z),
// D'(z) = I + (1+z)/E there.
__device__ void z_panels(double om, double zmax, double* sI, double* sJ, double* sD, double* sDp,
                         double* red) {
  const int tid = threadIdx.x;
  const double hz = zmax / ZPANELS;
  double v[2] = {0.0, 0.0};
  const double za = tid * hz;
  for (int q = 0; q < NGL_Z; ++q) {
    const double zq = za + 0.5 * hz * (1.0 + c_gzx[q]);
    const double u3m1 = zq * (3.0 + zq * (3.0 + zq));   // (1+z)^3 - 1
    const double iE = rsqrt(om * u3m1 + 1.0);            // 1/E
    v[0] += c_gzw[q] * iE;
    v[1] += c_gzw[q] * (-0.5 * u3m1 * (iE * iE * iE));
  }
  v[0] *= 0.5 * hz;
  v[1] *= 0.5 * hz;
  block_scan<2>(v, red);
  sI[tid + 1] = v[0];
  sJ[tid + 1] = v[1];
  if (tid == 0) { sI[0] = 0.0; sJ[0] = 0.0; }
  __syncthreads();
  for (int p = tid; p <= ZPANELS; p += PRO_THREADS) {
    const double zp_ = p * hz, u = 1.0 + zp_;
    sD[p] = u * sI[p];
    sDp[p] = sI[p] + u * rsqrt(om * (zp_ * (3.0 + zp_ * (3.0 + zp_))) + 1.0);
  }
  __syncthreads();
}

// The prologue's CTAs per Lambda point and their roles, in two shapes.  CL (small
// batches, whose few CTAs would leave most SMs idle): a thread-block cluster of 16 CTAs
// (the non-portable size), so that the FP64 work, which this GPU runs at 1/75 of its FP32
// rate, is spread over 16 SMs -- ranks 0..3 build a quarter of the d_L -> z inversion
// table each (each after step (1)), ranks 4 and 5 half of the redshift normalisation
// N'_z each (rank 4 adds them after the first barrier and writes it), ranks 6..15 each
// integrate a share of the smoothing window's panels.  After a cluster barrier every
// window rank gathers the panel integrals from their owners' shared memory and scans
// them; ranks 7..15 split the window tables' nodes while rank 6 gathers the window sums
// and writes the constants (xmax it reads from rank 0's shared memory), and a second
// barrier keeps every CTA's shared memory alive until all have read it.  Every CTA
// passes both barriers, except that all of them return at once for a Lambda outside the
// domain.  Not CL (large batches, where every SM has work anyway): three CTAs, no
// redundant work -- rank 0 the whole inversion table, rank 1 N'_z, rank 2 step (1), the
// whole window, the tables and the constants.
template <bool CL> struct ProShape {
  static constexpr int CTAS = CL ? 16 : 3;  // a cluster of 16 (the non-portable size) per point
  static constexpr int INV = CL ? 4 : 1;    // ranks [0, INV) build the inversion table
  static constexpr int NZR = INV;           // ranks [NZR, NZR + NNZ) sum N'_z; NZR writes it
  static constexpr int NNZ = CL ? 2 : 1;
  static constexpr int WIN0 = NZR + NNZ;    // ranks [WIN0, CTAS) integrate the window; WIN0 gathers
  static constexpr int NWIN = CTAS - WIN0;
};
constexpr int PRO_CLUSTER_MAX_K = 32;      // batches up to this size use the cluster shape

template <bool CL>
__global__ void __launch_bounds__(PRO_THREADS) k_prologue(ProArgs A) {
  namespace cg = cooperative_groups;
  using Sh = ProShape<CL>;
  extern __shared__ double sdyn[];               // 4 * nx doubles: P_n, D_n, then J_n, J'_n
  __shared__ double sI[ZPANELS + 1], sJ[ZPANELS + 1], sD[ZPANELS + 1], sDp[ZPANELS + 1];
  __shared__ double red[32 * 16];
  __shared__ double sc[32];                      // scalar broadcast
  __shared__ double s_wv[16];                    // a window CTA's share of the window sums
  __shared__ double s_pan[4][NW_WIN];            // and its panels' C-family integrals

  const int k = blockIdx.x, tid = threadIdx.x, rank = blockIdx.y;
  // the barrier across a Lambda point's CTAs (the cluster); without CL the roles exchange
  // nothing and only the CTA's own barrier is needed
  auto pro_sync = [&]() {
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
  };
  // a rank's shared memory (without CL only the CTA's own is ever asked for)
  auto peer = [&](double* p, int r) -> const double* {
    if constexpr (CL) return cg::this_cluster().map_shared_rank(p, r);
    else return p;
  };
  if (k == 0 && rank == 0 && tid == 0 && A.counter) *A.counter = 0;
  if (A.order && rank == 0 && tid < 32) {
    // this point's rank in the batch ordered by H0 (ties and NaN by index): the fused
    // kernel takes points in that order, so the warps of a CTA work on points whose
    // distance-redshift relations, and hence LOS cells, are alike
    const int np = n_params(A.mp != 0);
    const double hk = A.lam[(size_t)k * np + P_H0];
    const double kk = hk == hk ? hk : INFINITY;
    int r = 0;
    for (int j = tid; j < (int)gridDim.x; j += 32) {
      const double hj0 = A.lam[(size_t)j * np + P_H0];
      const double hj = hj0 == hj0 ? hj0 : INFINITY;
      r += (hj < kk || (hj == kk && j < k)) ? 1 : 0;
    }
    r = __reduce_add_sync(0xffffffffu, r);
    if (tid == 0) A.order[r] = k;
  }
  const bool mp = A.mp != 0;
  const double* L = A.lam + (size_t)k * n_params(mp);
  LamF* lf = A.lf + k;
  LamD* ld = A.ld + k;
  float* tb = A.tables + (size_t)k * A.tstride;
  const int nx = A.nx, nz = A.nz;
  const double zmax = A.zmax;

  if (!lambda_ok(L, mp)) {   // the same for every rank: the whole cluster returns
    if (tid == 0 && rank == Sh::WIN0) {
      LamF f;
      memset(&f, 0, sizeof(f));
      f.xmax = -1.f;
      *lf = f;
      ld->c = 0.0;
      ld->cz = 0.0;
      for (int i = 0; i < NP_MAX; ++i) ld->dc[i] = 0.0;
      ld->mp = mp ? 1 : 0;
      ld->lam1_sigma = 0;
      for (int i = 0; i < 3; ++i) ld->dcz[i] = 0.0;
      ld->flag = 1;
      ld->lam_sigma = 0;
    }
    return;
  }
  const double H0 = L[P_H0], om = L[P_OM], alpha = L[P_ALPHA], beta = L[P_BETA];
  const double mmin = L[P_MMIN], mmax = L[P_MMAX], dm = L[P_DM], mu = L[P_MU], sig = L[P_SIG];
  const double lam = L[P_LAM], gam = L[P_GAM], kap = L[P_KAP], zp = L[P_ZP];
  const double gpk = gam + kap, lp = log1p(zp);
  // multi-peak: the high peak and the low peak's share (lam1 = 1 leaves one Gaussian)
  const double mu2 = mp ? L[P_MU2] : 0.0, sig2 = mp ? L[P_SIG2] : 1.0, lam1 = mp ? L[P_LAM1] : 1.0;

  if (rank >= Sh::NZR && rank < Sh::NZR + Sh::NNZ) {
    // ---- (5) redshift normalisation N'_z = sum_j c_j dz pbar_j psi'(z_j) / (1 + z_j),
    //          psi' = (1+z)^gamma / (1 + ((1+z)/(1+zp))^(gamma+kappa)); the N'_z ranks
    //          split the grid, rank NZR adds their sums in rank order and writes N'_z
    const double dzg = zmax / (nz - 1);
    const int zr = rank - Sh::NZR;
    const int j0 = zr * nz / Sh::NNZ, j1 = (zr + 1) * nz / Sh::NNZ;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = j0 + tid; j < j1; j += PRO_THREADS) {
      const double zj = j * dzg, l = log1p(zj);
      const double r = gpk * (l - lp);
      const double term = ((j == 0 || j == nz - 1) ? 0.5 : 1.0) * dzg * A.pbar64[j] *
                          exp(gam * l - softplus_d(r) - l);
      const double s = sigmoid_d(r);
      v[0] += term;
      v[1] += term * (l - s * (l - lp));
      v[2] += term * (-s * (l - lp));
      v[3] += term * (s * gpk / (1.0 + zp));
    }
    block_sum<4>(v, red);
    if (tid < 4) s_wv[tid] = v[tid];
    auto write_nz = [&](const double* t) {
      ld->cz = -log(t[0]);
      ld->dcz[0] = -t[1] / t[0];
      ld->dcz[1] = -t[2] / t[0];
      ld->dcz[2] = -t[3] / t[0];
    };
    if constexpr (CL) {
      pro_sync();
      if (rank == Sh::NZR && tid == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < Sh::NNZ; ++r)
          for (int i = 0; i < 4; ++i) t[i] += peer(s_wv, Sh::NZR + r)[i];
        write_nz(t);
      }
      pro_sync();
    } else if (tid == 0) {
      write_nz(v);
    }
    return;
  }
  const double pscale = (double)(nz - 1) / zmax;   // LOS grid units per unit z

  if (rank < Sh::INV) {
  z_panels(om, zmax, sI, sJ, sD, sDp, red);
  const double hz = zmax / ZPANELS;
  const double xmax = sD[ZPANELS];
  const double dx = xmax / (nx - 1);

  // ---- (2) inversion table on the uniform x grid: each of the INV ranks owns nodes
  //          [own0, own1) and also evaluates node own1 (when there is one), the right
  //          neighbour that its last Hermite segment needs, leaving that node's table
  //          entries to the next rank
  const int own0 = rank * nx / Sh::INV, own1 = (rank + 1) * nx / Sh::INV;
  const int eval1 = own1 < nx ? own1 + 1 : nx;
  float4* aux = reinterpret_cast<float4*>(tb + 4 * nx);
  for (int n = own0 + tid; n < eval1; n += PRO_THREADS) {
    const double xn = (n == nx - 1) ? xmax : n * dx;
    double z = 0.0, Dp = 1.0, Jz = 0.0, jd = 0.0;
    if (n > 0) {
      int lo = 0, hi = ZPANELS - 1;   // largest p with sD[p] <= xn
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sD[mid] <= xn) lo = mid; else hi = mid - 1;
      }
      const int p = lo;
      const double z0 = p * hz;
      // start: invert the cubic Hermite interpolant of D on the panel (D and D' at its
      // edges; ~1e-11 from the root), three Newton steps on that cubic in s = (z-z0)/hz
      const double D0 = sD[p], D1 = sD[p + 1], d0 = sDp[p] * hz, d1 = sDp[p + 1] * hz;
      const double c2 = 3.0 * (D1 - D0) - 2.0 * d0 - d1, c3 = 2.0 * (D0 - D1) + d0 + d1;
      double sp = (xn - D0) / (D1 - D0);
      for (int it = 0; it < 3; ++it) {
        const double f = D0 + sp * (d0 + sp * (c2 + sp * c3)) - xn;
        const double fd = d0 + sp * (2.0 * c2 + 3.0 * sp * c3);
        sp = fmin(fmax(sp - f / fd, 0.0), 1.0);
      }
      z = z0 + sp * hz;
      // one Newton step on the exact D: I, J and E from one Gauss-Legendre pass; D' and
      // J are kept from that pass (the step moves z by ~1e-11)
      const double h = z - z0;
      double acc = 0.0, accj = 0.0;
      for (int q = 0; q < NGL_Z; ++q) {
        const double zq = z0 + 0.5 * h * (1.0 + c_gzx[q]);
        const double u3m1 = zq * (3.0 + zq * (3.0 + zq)), iE = rsqrt(om * u3m1 + 1.0);
        acc += c_gzw[q] * iE;
        accj += c_gzw[q] * (-0.5 * u3m1 * iE * iE * iE);
      }
      const double Iz = sI[p] + 0.5 * h * acc;
      Jz = sJ[p] + 0.5 * h * accj;
      const double u = 1.0 + z;
      const double u3m1 = z * (3.0 + z * (3.0 + z)), iE = rsqrt(om * u3m1 + 1.0);
      Dp = Iz + u * iE;
      z = fmin(fmax(z - (u * Iz - xn) / Dp, z0), z0 + hz);
      jd = -0.5 * u3m1 * iE * iE * iE;
    }
    sdyn[2 * n] = z * pscale;                // P_n
    sdyn[2 * n + 1] = pscale / Dp * dx;      // dP/dx * dx
    sdyn[2 * nx + n] = Jz;                   // J and dJ/dx * dx at the node
    sdyn[3 * nx + n] = jd / Dp * dx;
  }
  __syncthreads();
  float4* pos = reinterpret_cast<float4*>(tb);
  for (int n = own0 + tid; n < own1; n += PRO_THREADS) {
    const double P0 = sdyn[2 * n], D0 = sdyn[2 * n + 1];
    double c2 = 0.0, c3 = 0.0;
    if (n < nx - 1) {
      const double P1 = sdyn[2 * n + 2], D1 = sdyn[2 * n + 3];
      c2 = 3.0 * (P1 - P0) - 2.0 * D0 - D1;
      c3 = 2.0 * (P0 - P1) + D0 + D1;
    }
    const float hi = (float)P0;
    pos[n] = make_float4(hi, (float)(P0 - (double)hi), (float)D0, (float)c2);
    // J on the segment: the quadratic through J_n and J_{n+1} whose curvature is the mean
    // of the two nodes' slopes' difference, J = J_n + t (d - c) + t^2 c (error O(dx^3))
    const double J0 = sdyn[2 * nx + n];
    double dJ = 0.0, cJ = 0.0;
    if (n < nx - 1) {
      dJ = sdyn[2 * nx + n + 1] - J0;
      cJ = 0.5 * (sdyn[3 * nx + n + 1] - sdyn[3 * nx + n]);
    }
    aux[n] = make_float4((float)c3, (float)J0, (float)(dJ - cJ), (float)cJ);
  }
  if constexpr (CL) { pro_sync(); pro_sync(); }   // rank WIN0 reads xmax from rank 0 in between
  return;
  }   // the inversion ranks

  // ---- the window ranks; without CL the single window rank also needs step (1) for xmax
  if constexpr (!CL) z_panels(om, zmax, sI, sJ, sD, sDp, red);

  // ---- (3) mass-model normalisations (Z_P by warp 0, Z_G by warp 1, Z_G2 by warp 2,
  //          ln(sig sqrt(2 pi)) of the two peaks on threads 96 and 128, so the serial
  //          chains run in different warps), broadcast through shared memory.  Within a
  //          warp the lanes evaluate a chain's logarithms, expm1s, divisions and
  //          exponentials of one level side by side (the same instructions on arguments
  //          chosen by the lane): each level costs the warp one such evaluation
  if (tid < 32) {
    // Z_P = int_{mmin}^{mmax} m^-alpha dm = e^{t a} (b - a) phi1(t (b - a)), t = 1 - alpha
    const int l = tid;
    const unsigned full = 0xffffffffu;
    const double t = 1.0 - alpha;
    const double la = log(l == 1 ? mmax : mmin);                       // a (lane 0), b (lane 1)
    const double a = __shfl_sync(full, la, 0), b = __shfl_sync(full, la, 1);
    const double Lr = b - a, y = t * Lr;
    const bool small = fabs(y) < 1e-5;
    const double em = expm1(l == 1 ? -y : y);                          // expm1(y), expm1(-y)
    const double emp = __shfl_sync(full, em, 0), emm = __shfl_sync(full, em, 1);
    const double dv = 1.0 / (l == 1 ? (small ? 1.0 : -emm) : (small ? 1.0 : y));   // 1/y, -1/expm1(-y)
    const double iy = __shfl_sync(full, dv, 0), iq = __shfl_sync(full, dv, 1);
    const double phi1 = small ? 1.0 + y * (0.5 + y * (1.0 / 6.0)) : emp * iy;
    const double gy = small ? 0.5 + y * (1.0 / 12.0) : iq - iy;
    const double lg = log(l == 1 ? phi1 : Lr);                         // ln Lr, ln phi1
    const double lnZP = t * a + __shfl_sync(full, lg, 0) + __shfl_sync(full, lg, 1);
    const double ex = exp(-alpha * (l == 1 ? b : a) - lnZP);
    if (l == 0) {
      sc[0] = lnZP;
      sc[1] = -(a + Lr * gy);                        // d ln Z_P / d alpha
      sc[2] = -ex;                                   // d ln Z_P / d m_min
    } else if (l == 1) {
      sc[3] = ex;                                    // d ln Z_P / d m_max
    }
  } else if (tid < 64) {
    gauss_mass(mu, sig, mmin, mmax, sc + 4);         // Z_G = Phi(B) - Phi(A)
  } else if (tid < 96) {
    if (mp) gauss_mass(mu2, sig2, mmin, mmax, sc + 9);
  } else if (tid == 96) {
    sc[14] = log(sig) + 0.91893853320467274178;
  } else if (tid == 128) {
    sc[15] = log(sig2) + 0.91893853320467274178;
  }
  __syncthreads();
  const double lnZP = sc[0], dZPa = sc[1], dZPmin = sc[2], dZPmax = sc[3];
  const double lnZG = sc[4], dZGmu = sc[5], dZGsig = sc[6], dZGmin = sc[7], dZGmax = sc[8];
  const double lnZG2 = mp ? sc[9] : 0.0, dZG2mu = mp ? sc[10] : 0.0, dZG2sig = mp ? sc[11] : 0.0;
  const double dZG2min = mp ? sc[12] : 0.0, dZG2max = mp ? sc[13] : 0.0;
  const double lnsig2pi = sc[14];
  const double lnsig2pi2 = sc[15];

  // ---- (4) smoothing window [mmin, mmin + dm]: W = int h (1 - S), its derivatives,
  //          and the cumulative C-family integrals at the table nodes
  const double hw = dm / NW_WIN;
  //          (multi-peak: the Gaussian part is lam1 G + (1 - lam1) G2, and four more sums
  //          give the mu2, sig2, lam1 derivatives and the G2 part of the m_max one)
  //          The window ranks share the panels; a thread takes one Gauss-Legendre node at
  //          a time (eight consecutive threads one panel).
  const int wr = rank - Sh::WIN0;
  const int pa0 = wr * NW_WIN / Sh::NWIN, pa1 = (wr + 1) * NW_WIN / Sh::NWIN;   // this CTA's panels
  double wv[13] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const double isig = 1.0 / sig, isig2 = mp ? 1.0 / sig2 : 0.0;
  for (int base = 0; base < (pa1 - pa0) * NGL; base += PRO_THREADS) {   // uniform trip count
  const int pl = (base + tid) / NGL, q = tid % NGL;                        // panel (local), node
  double cum[4] = {0.0, 0.0, 0.0, 0.0};   // C, C_beta, J, K at this thread's node
  if (pa0 + pl < pa1 && dm > 0.0) {
    const double ma = mmin + (pa0 + pl) * hw;
    {
      const double m = ma + 0.5 * hw * (1.0 + c_glx[q]);
      const double mr = m - mmin, lm = log(m), im = 1.0 / m;
      double S, oneS, dSddm;
      smooth_d(mr, dm, 1.0 / mr, 1.0 / (mr - dm), S, oneS, dSddm);
      const double mb = exp(beta * lm);
      const double w = c_glw[q] * 0.5 * hw;
      cum[0] += w * mb * S;
      cum[1] += w * mb * lm * S;
      cum[2] += w * mb * im * S;
      cum[3] += w * mb * dSddm;
      const double P = exp(-alpha * lm - lnZP);
      const double zg = (m - mu) * isig;
      const double G1 = exp(-0.5 * zg * zg - lnsig2pi - lnZG);
      const double zg2 = (m - mu2) * isig2;
      const double G2 = mp ? exp(-0.5 * zg2 * zg2 - lnsig2pi2 - lnZG2) : 0.0;
      const double G = lam1 * G1, Gb = (1.0 - lam1) * G2;   // the two peaks' shares
      const double h = (1.0 - lam) * P + lam * (G + Gb);
      wv[0] += w * h * oneS;
      wv[1] += w * (1.0 - lam) * P * (-lm - dZPa) * oneS;
      wv[2] += w * (G + Gb - P) * oneS;
      wv[3] += w * lam * G * (zg * isig - dZGmu) * oneS;
      wv[4] += w * lam * G * ((zg * zg - 1.0) * isig - dZGsig) * oneS;
      wv[5] += w * P * oneS;
      wv[6] += w * G * oneS;
      wv[7] += w * ((1.0 - lam) * P * (-alpha * im - dZPmin) + lam * G * (-zg * isig - dZGmin) +
                    lam * Gb * (-zg2 * isig2 - dZG2min)) * oneS;
      wv[8] += w * (-h * dSddm);
      if (mp) {
        wv[9] += w * lam * Gb * (zg2 * isig2 - dZG2mu) * oneS;
        wv[10] += w * lam * Gb * ((zg2 * zg2 - 1.0) * isig2 - dZG2sig) * oneS;
        wv[11] += w * lam * (G1 - G2) * oneS;
        wv[12] += w * Gb * oneS;
      }
    }
  }
  // each panel's integrals: the sum over its NGL node threads (a fixed xor tree)
  for (int i = 0; i < 4; ++i)
    for (int o = 1; o < NGL; o <<= 1) cum[i] += __shfl_xor_sync(0xffffffffu, cum[i], o);
  if (q == 0 && pa0 + pl < pa1)
    for (int i = 0; i < 4; ++i) s_pan[i][pl] = cum[i];
  }
  block_sum<13>(wv, red);
  if (tid < 13) s_wv[tid] = wv[tid];
  pro_sync();
  // ---- every window rank gathers each panel's integrals from the CTA that owns it (one
  //      panel a thread) and scans them inclusively: thread p holds the cumulative
  //      integrals at node p + 1.  The window tables' nodes are then split over the
  //      window ranks; rank WIN0 also gathers the window sums and writes the constants.
  double cum[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid < NW_WIN) {
    int r = 0;
    while ((r + 1) * NW_WIN / Sh::NWIN <= tid) ++r;
    const double* o = peer(&s_pan[0][0], Sh::WIN0 + r);
    const int loc = tid - r * NW_WIN / Sh::NWIN;
    for (int i = 0; i < 4; ++i) cum[i] = o[i * NW_WIN + loc];
  }
  // the scan over the NW_WIN panels in the warps that hold them (the others would add
  // zeros, and an FP64 warp-instruction costs the same with no useful lane); the same
  // order of additions as block_scan, so the same sums
  static_assert(NW_WIN % 32 == 0 && NW_WIN <= PRO_THREADS, "panel scan layout");
  {
    const int lane = tid & 31, w = tid >> 5;
    if (tid < NW_WIN) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double y = __shfl_up_sync(0xffffffffu, cum[i], o);
          if (lane >= o) cum[i] += y;
        }
      }
      if (lane == 31)
        for (int i = 0; i < 4; ++i) red[i * 32 + w] = cum[i];
    }
    __syncthreads();
    if (tid < NW_WIN) {
      for (int i = 0; i < 4; ++i) {
        double off = 0.0;
        for (int k = 0; k < w; ++k) off += red[i * 32 + k];
        cum[i] += off;
      }
    }
    __syncthreads();
  }

  // window tables at nodes m_k = mmin + k hw: with R_X = X / (m^beta S(m)),
  //   Q_C = R_C dm / m'^2, Q_beta = R_beta / R_C, Q_J = R_J / R_C, Q_K = R_K dm / m'
  // and their m-derivatives (times hw).  Node 0 takes the m' -> 0 limits (1, ln mmin,
  // 1/mmin, -1) with secant slopes: weights there carry S(m1) < e^-127.
  float4* wval = reinterpret_cast<float4*>(tb + 8 * nx);
  float4* wslp = wval + (NW_WIN + 1);
  __shared__ double scum[4][NW_WIN + 1];
  __shared__ double sq[4][NW_WIN + 1];
  if (tid < NW_WIN)
    for (int i = 0; i < 4; ++i) scum[i][tid + 1] = cum[i];
  if (tid == 0)
    for (int i = 0; i < 4; ++i) scum[i][0] = 0.0;
  __syncthreads();
  // this rank's nodes [nd0, nd1) of the NW_WIN + 1.  With several window ranks, rank WIN0
  // takes none (it writes the constants meanwhile) and the others split them; the rank
  // with node 0 also evaluates node 1, whose value the secant slope at node 0 needs
  const int tw = Sh::NWIN > 1 ? Sh::NWIN - 1 : 1, tr = Sh::NWIN > 1 ? wr - 1 : 0;
  const int nd0 = tr >= 0 ? tr * (NW_WIN + 1) / tw : 0, nd1 = tr >= 0 ? (tr + 1) * (NW_WIN + 1) / tw : 0;
  const int node = nd0 + tid;
  const bool mine = node < nd1, eval = mine || (node == 1 && nd0 == 0 && nd1 > 0);
  double qv[4] = {1.0, 0.0, 0.0, -1.0}, qd[4] = {0.0, 0.0, 0.0, 0.0};
  if (eval) {   // the m' -> 0 limits (every node's values without a window)
    qv[1] = log(mmin);
    qv[2] = 1.0 / mmin;
  }
  if (eval && node > 0 && dm > 0.0) {
    // with r1 = 1/m', r2 = 1/(m' - dm), im = 1/m, 1/g and 1/R_C: five divisions where the
    // expressions written out would take about twenty (each a long FP64 sequence here)
    const double mr = node * hw, m = mmin + mr, lm = log(m), im = 1.0 / m, r1 = 1.0 / mr;
    double S = 1.0, oneS = 0.0, dSddm = 0.0, dlnS = 0.0, dSS = 0.0;
    if (node < NW_WIN) {
      const double r2 = 1.0 / (mr - dm);
      smooth_d(mr, dm, r1, r2, S, oneS, dSddm);
      dlnS = oneS * dm * (r1 * r1 + r2 * r2);
      dSS = -oneS * (r1 + mr * (r2 * r2));   // (dS/d delta_m) / S
    }
    const double ig = 1.0 / (exp(beta * lm) * S);
    const double gl = beta * im + dlnS;     // g'/g
    const double Rc = scum[0][node] * ig, Rb = scum[1][node] * ig;
    const double Rj = scum[2][node] * ig, Rk = scum[3][node] * ig;
    const double iRc = 1.0 / Rc;
    const double dRc = 1.0 - Rc * gl, dRb = lm - Rb * gl, dRj = im - Rj * gl, dRk = dSS - Rk * gl;
    qv[0] = Rc * dm * (r1 * r1);
    qv[1] = Rb * iRc;
    qv[2] = Rj * iRc;
    qv[3] = Rk * dm * r1;
    qd[0] = dm * (dRc * (r1 * r1) - 2.0 * Rc * (r1 * r1 * r1));
    qd[1] = (dRb - qv[1] * dRc) * iRc;
    qd[2] = (dRj - qv[2] * dRc) * iRc;
    qd[3] = dm * (dRk * r1 - Rk * (r1 * r1));
  }
  if (eval)
    for (int i = 0; i < 4; ++i) sq[i][node] = qv[i];
  __syncthreads();
  if (mine && node == 0 && dm > 0.0)
    for (int i = 0; i < 4; ++i) qd[i] = (sq[i][1] - sq[i][0]) / hw;
  if (mine) {
    wval[node] = make_float4((float)qv[0], (float)qv[1], (float)qv[2], (float)qv[3]);
    wslp[node] = make_float4((float)(qd[0] * hw), (float)(qd[1] * hw), (float)(qd[2] * hw), (float)(qd[3] * hw));
  }

  if (rank == Sh::WIN0) {
  // ---- rank WIN0: the window sums gathered in rank order, one component a lane
  __shared__ double s_wsum[13];
  __shared__ double s_tv[32];
  if (tid < 13) {
    double v = 0.0;
    for (int r = 0; r < Sh::NWIN; ++r) v += peer(s_wv, Sh::WIN0 + r)[tid];
    s_wsum[tid] = v;
  }
  const double xmax = *peer(&sD[ZPANELS], 0);   // D(z_max): rank 0's with CL, else this CTA's
  __syncthreads();
  for (int i = 0; i < 13; ++i) wv[i] = s_wsum[i];
  // Z_m1 = 1 - W with W = wv[0]; d ln Z_m1 / d theta = -dW/d theta / Z_m1
  const double dWa = wv[1], dWl = wv[2], dWmu = wv[3], dWsig = wv[4];
  const double dWmax = -(1.0 - lam) * dZPmax * wv[5] - lam * dZGmax * wv[6] - lam * dZG2max * wv[12];
  const double dWmin = wv[7], dWdm = wv[8];
  const double dWmu2 = wv[9], dWsig2 = wv[10], dWl1 = wv[11];

  // ---- (6) constants.  Their logarithms, exponentials and divisions are long FP64
  //      sequences; the lanes of a warp evaluate one kind of them side by side (the same
  //      expressions, one per lane, all lanes running the same instructions on arguments
  //      chosen by the lane), the logarithms in warp 0, log1p in warp 1, the divisions in
  //      warp 2 and mw^(1+beta) in warp 3, so that the four run on the SM's four
  //      schedulers at once, before thread 0 assembles the fields into s_tv[]:
  //        [0..5]   log of lam lam1, lam, mw, lam1, 1 - W, H0/c       [6, 7] log1p(-lam), log1p(-lam1)
  //        [8]      exp(eps log mw)
  //        [9..24]  1/sig, 1/sig2, 1/eps, N_w/dm, 1/dm, 1/H0, 1/(1+zp), 1/lam, 1/(1-lam),
  //                 1/(1-W), 1/lam1, 1/(1-lam1), gpk/(1+zp), (H0/c)/dx, zmax/(nz-1), 1/mw
  const double mw = mmin + dm, eps = 1.0 + beta;
  const double h0c = H0 * (1.0 / C_KMS);   // H0/c (within an ulp of the quotient)
  if (tid < 128) {
    const int l = tid & 31, wq = tid >> 5;
    const double W0 = wv[0];
    if (wq == 0) {
      const double la = l == 0 ? lam * lam1 : l == 1 ? lam : l == 2 ? mw : l == 3 ? lam1 : l == 4 ? 1.0 - W0
                      : l == 5 ? h0c : 1.0;
      const double vlog = log(la);
      if (l < 6) s_tv[l] = vlog;
    } else if (wq == 1) {
      const double vlog1p = log1p(l == 0 ? -lam : l == 1 ? -lam1 : 0.0);
      if (l < 2) s_tv[6 + l] = vlog1p;
    } else if (wq == 2) {
      // lane 22: (H0/c)/dx = (H0/c)(nx - 1)/xmax
      const double num = l == 12 ? (double)NW_WIN : l == 21 ? gpk : l == 22 ? h0c * (double)(nx - 1)
                       : l == 23 ? zmax : 1.0;
      const double den = l == 9 ? sig : l == 10 ? sig2 : l == 11 ? eps : l == 12 ? dm : l == 13 ? dm
                       : l == 14 ? H0 : l == 15 ? 1.0 + zp : l == 16 ? lam : l == 17 ? 1.0 - lam
                       : l == 18 ? 1.0 - W0 : l == 19 ? lam1 : l == 20 ? 1.0 - lam1 : l == 21 ? 1.0 + zp
                       : l == 22 ? xmax : l == 23 ? (double)(nz - 1) : l == 24 ? mw : 1.0;
      const double vdiv = num / den;
      if (l >= 9 && l < 25) s_tv[l] = vdiv;
    } else {
      const double vexp = exp(eps * log(mw));
      if (l == 0) s_tv[8] = vexp;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const double Cw = dm > 0.0 ? scum[0][NW_WIN] : 0.0;
    const double Cwb = dm > 0.0 ? scum[1][NW_WIN] : 0.0;
    const double Jw = dm > 0.0 ? scum[2][NW_WIN] : 0.0;
    const double Kw = dm > 0.0 ? scum[3][NW_WIN] : 0.0;
    const double LOG2E = 1.44269504088896340736;
    LamF f;
    memset(&f, 0, sizeof(f));
    f.H0c = (float)h0c;
    f.H0c_lo = (float)(h0c - (double)f.H0c);
    const double sxa = s_tv[22];
    f.sxa = (float)sxa;
    f.sxa_lo = (float)(sxa - (double)f.sxa);
    f.xmax = (float)xmax;
    f.live = 1.f;
    f.zstep = (float)s_tv[23];
    f.zstep_lo = (float)(s_tv[23] - (double)f.zstep);
    f.inv_zstep = (float)pscale;
    f.om = (float)om;
    f.lp2 = (float)(lp * LOG2E);
    f.gam = (float)gam;
    f.gam_m3 = (float)(gam - 3.0);
    f.gpk = (float)gpk;
    f.gpk_lo = (float)(gpk - (double)f.gpk);
    f.alpha = (float)alpha;
    f.beta = (float)beta;
    f.eps_b = (float)eps;
    f.alpha_lo = (float)(alpha - (double)f.alpha);
    f.beta_lo = (float)(beta - (double)f.beta);
    f.eps_b_lo = (float)(eps - (double)f.eps_b);
    f.mmin = (float)mmin;
    f.mmax = (float)mmax;
    f.dm = (float)dm;
    f.dm_l2 = (float)(dm * LOG2E);
    f.mw = (float)mw;
    f.mu = (float)mu;
    f.inv_sig = (float)s_tv[9];
    // the two components' log2 normalisations, less an anchor R (log2 units) that c
    // carries in FP64: only their difference is rounded to FP32, so the rounding no
    // longer shifts every sample's weight by the same amount
    // (multi-peak: the low peak carries lam lam1, the high one lam (1 - lam1))
    const double la2d = lam < 1.0 ? (s_tv[6] - lnZP) * LOG2E : -INFINITY;
    const double lb2d = lam > 0.0 && lam1 > 0.0 ? (s_tv[0] - lnsig2pi - lnZG) * LOG2E : -INFINITY;
    const double lc2d = mp && lam > 0.0 && lam1 < 1.0 ? (s_tv[1] + s_tv[7] - lnsig2pi2 - lnZG2) * LOG2E
                                                     : -INFINITY;
    const double R = lam < 1.0 ? la2d : (lb2d > -INFINITY ? lb2d : lc2d);
    f.la2 = lam < 1.0 ? (float)(la2d - R) : -INFINITY;
    f.lb2 = lb2d > -INFINITY ? (float)(lb2d - R) : -INFINITY;
    f.lc2 = lc2d > -INFINITY ? (float)(lc2d - R) : -INFINITY;
    f.mu2 = (float)mu2;
    f.inv_sig2 = (float)s_tv[10];
    const bool small = fabs(eps) < 1e-3;
    const double mw1b = s_tv[8];
    f.beta_small = small ? 1.f : 0.f;
    f.inv_eps_b = small ? 0.f : (float)s_tv[11];
    f.C0 = small ? 0.f : (float)(Cw - mw1b * s_tv[11]);
    f.Cw = (float)Cw;
    f.mw1b = (float)mw1b;
    f.lmw = (float)s_tv[2];
    f.inv_wh = dm > 0.0 ? (float)s_tv[12] : 0.f;
    f.inv_dm = dm > 0.0 ? (float)s_tv[13] : 0.f;
    f.invH0 = (float)s_tv[14];
    f.inv1zp = (float)s_tv[15];
    f.lam_edge = (lam > 0.0 && lam < 1.0) ? 0.f : 1.f;
    f.lam = (float)lam;
    f.lam_sig = lam >= 1.0 ? 1.f : (lam <= 0.0 ? -1.f : 0.f);
    // multi-peak bounds: lam1 at 0 or 1 (with lam > 0) takes the other peak's weight lam G2
    // (lam1 = 1) or lam G (lam1 = 0); at lam = 0 the mixture of the two peaks without lam
    const bool e1 = mp && lam > 0.0 && !(lam1 > 0.0 && lam1 < 1.0);
    f.lam1_edge = e1 ? 1.f : 0.f;
    f.o2_hi = lam1 >= 1.0 ? 1.f : 0.f;
    f.o2_l2 = !e1 ? 0.f
                  : (float)((s_tv[1] - (lam1 >= 1.0 ? lnsig2pi2 + lnZG2 : lnsig2pi + lnZG)) * LOG2E - R);
    f.lb1_2 = mp && lam1 > 0.0 ? (float)((s_tv[3] - lnsig2pi - lnZG) * LOG2E - R) : -INFINITY;
    f.lc1_2 = mp && lam1 < 1.0 ? (float)((s_tv[7] - lnsig2pi2 - lnZG2) * LOG2E - R) : -INFINITY;
    f.dZPa = (float)dZPa;
    f.dZPmin = (float)dZPmin;
    f.dZPmax = (float)dZPmax;
    f.dZGmu = (float)dZGmu;
    f.dZGsig = (float)dZGsig;
    f.dZGmin = (float)dZGmin;
    f.dZGmax = (float)dZGmax;
    f.Cwb = (float)Cwb;
    f.Cmin = (float)(beta * Jw - mw1b * s_tv[24]);
    f.Kw = (float)Kw;
    f.la0_2 = (float)(-lnZP * LOG2E - R);
    f.lb0_2 = (float)((-lnsig2pi - lnZG) * LOG2E - R);
    f.inv_lam = lam > 0.0 ? (float)s_tv[16] : 0.f;
    f.inv_1ml = lam < 1.0 ? (float)s_tv[17] : 0.f;
    *lf = f;
    // c = -ln Z_m1 + ln(H0 / c) + R ln 2 (the anchor taken out of la2, lb2); -ln N'_z
    // and its derivatives are in cz, dcz
    ld->c = -s_tv[4] + s_tv[5] + R * 0.69314718055994530942;
    double dc[NP_MAX];
    for (int i = 0; i < NP_MAX; ++i) dc[i] = 0.0;
    const double iZ = s_tv[18];   // -d ln Z_m1 = dW / Z_m1
    dc[P_H0] = s_tv[14];
    dc[P_ALPHA] = dWa * iZ;
    dc[P_MMIN] = dWmin * iZ;
    dc[P_MMAX] = dWmax * iZ;
    dc[P_DM] = dWdm * iZ;
    dc[P_MU] = dWmu * iZ;
    dc[P_SIG] = dWsig * iZ;
    dc[P_LAM] = dWl * iZ;
    if (mp) {
      dc[P_MU2] = dWmu2 * iZ;
      dc[P_SIG2] = dWsig2 * iZ;
      dc[P_LAM1] = dWl1 * iZ;
    }
    for (int i = 0; i < NP_MAX; ++i) ld->dc[i] = dc[i];
    ld->flag = 0;
    ld->lam_sigma = lam >= 1.0 ? 1 : (lam <= 0.0 ? -1 : 0);
    ld->mp = mp ? 1 : 0;
    ld->lam1_sigma = e1 ? (lam1 >= 1.0 ? 1 : -1) : 0;
    ld->dZG2min = dZG2min;
    ld->dZG2max = dZG2max;
    ld->dZG2mu = dZG2mu;
    ld->dZG2sig = dZG2sig;
    ld->inv_sig2 = s_tv[10];
    ld->inv_lam1 = lam1 > 0.0 ? s_tv[19] : 0.0;
    ld->inv_1ml1 = lam1 < 1.0 ? s_tv[20] : 0.0;
    ld->invH0 = s_tv[14];
    ld->dZPa = dZPa;
    ld->dZPmin = dZPmin;
    ld->dZPmax = dZPmax;
    ld->dZGmin = dZGmin;
    ld->dZGmax = dZGmax;
    ld->dZGmu = dZGmu;
    ld->dZGsig = dZGsig;
    ld->inv_sig = s_tv[9];
    ld->inv_lam = lam > 0.0 ? s_tv[16] : 0.0;
    ld->inv_1ml = lam < 1.0 ? s_tv[17] : 0.0;
    ld->gpk_inv1zp = s_tv[21];
  }
  }   // rank WIN0
  if constexpr (CL) pro_sync();   // the window CTAs' shared memory stays until rank WIN0 has read it
}

// ---------------------------------------------------------------- fused kernel
// A CTA owns one work item (a chunk of one event's samples, or of injections) and a
// tile of Lambda points.  Its 8 warps form 8/G groups of G warps; a group sweeps one
// Lambda at a time, each of its warps over 1/G of the staged samples, so the CTA's L1
// working set is 8/G Lambda points' tables plus the chunk's few LOS rows, and each
// lane amortises its per-Lambda work over chunk / (32 G) samples.  Every warp leaves
// its (max, sums) for each of its Lambda points in shared memory; after the tile the
// G entries of each Lambda are combined in warp order into one partial per
// (item, Lambda).
// Occupancy: three CTAs per SM (<= 80 registers per thread) for both kernels.  The
// gradient kernel fits there because each warp's Lambda index is formed by a warp
// reduction (a value the compiler knows to be the same in every lane), so the point's
// constants are loaded once per warp and kept out of the per-thread registers; with the
// index as a plain per-thread value the same bound spilled ~400 bytes per thread.
constexpr int MINB_VALUE = 3, MINB_GRAD = 3;

// One (item, Lambda-slab) unit: stage the item's samples, sweep them for the slab's
// Lambda points, combine the warp groups' sums into the unit's partials.
template <bool GRAD, bool KAHAN, typename RowT, bool MP>
__device__ __forceinline__ void fused_unit(const FusedArgs& A, int unit, float* sm, int* s_next) {
  constexpr int NS = n_params(MP);   // gradient statistics of the mass model
  using Sink = AccSink<GRAD, KAHAN, NS>;
  const int CH = A.chunk;
  // staged samples: {m1, m2, d_L, -log2 pi}, {log2 m1, log2 m2, pixel, 0} (two loads a
  // sample); the value kernel's partials need only (m, s1, s2)
  constexpr int PS = GRAD ? PSTRIDE : 4;
  float4* s_a = reinterpret_cast<float4*>(sm);
  float4* s_b = s_a + CH;
  float* s_part = reinterpret_cast<float*>(s_b + CH);   // [slab][G][PS]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = A.group, ngroups = WARPS / G;
  const int gidx = warp / G, wg = warp - gidx * G;
  const int ipos = unit / A.n_slabs, slab = unit - ipos * A.n_slabs;
  const int item = A.sched[ipos];
  const Item it = A.items[item];
  const bool inj = it.kind == 1;

  const float4* src = inj ? A.inj : A.smp;
  for (int i = tid; i < it.count; i += THREADS) {
    const float4 v = __ldg(src + it.begin + i);
    s_a[i] = make_float4(v.x, v.y, v.z, -to_log2(v.w));
    s_b[i] = make_float4(log2f(v.x), log2f(v.y), __int_as_float(inj ? 0 : __ldg(A.pix + it.begin + i)), 0.f);
  }
  if (tid == 0) *s_next = 0;
  __syncthreads();

  const int k0 = slab * A.slab;
  const int nk = min(A.slab, A.K - k0);
  const int nx = A.nx, nz = A.nz;
  const int a = (int)((long long)it.count * wg / G);
  const int b = (int)((long long)it.count * (wg + 1) / G);
  // With one warp per group each warp takes the next Lambda point of the tile from a
  // counter (the work per point varies, e.g. with how many samples fall outside the mass
  // support); a point's sums are still formed by one warp in one order, so the result
  // does not depend on which warp took it.  Groups of several warps take every
  // ngroups-th point.
  auto next_k = [&](int prev) {
    if (G != 1) return prev + ngroups;
    int v = 0;
    if (lane == 0) v = atomicAdd(s_next, 1);
    return __shfl_sync(0xffffffffu, v, 0);
  };
  for (int kk = (G == 1) ? next_k(0) : gidx; kk < nk; kk = next_k(kk)) {
    // the same k in every lane of the warp, formed so that the compiler can tell
    const int k = __reduce_max_sync(0xffffffffu, A.order ? A.order[k0 + kk] : k0 + kk);
    const LamF L = A.lf[k];
    Acc<GRAD, KAHAN, NS> acc;
    if (L.live != 0.f) {
      const float* tb = A.tables + (size_t)k * A.tstride;
      const float4* pos = reinterpret_cast<const float4*>(tb);
      const float4* aux = reinterpret_cast<const float4*>(tb + 4 * nx);
      const float4* wv = reinterpret_cast<const float4*>(tb + 8 * nx);
      const float4* ws = wv + (NW_WIN + 1);
      // every lane of the warp runs the same number of iterations (the per-sample
      // arithmetic votes over the warp); lanes past the end repeat the run's last sample
      // with valid = false.  Rare points (a mixture weight on a bound, |1+beta| < 1e-3) take
      // their own instance of the loop.
      auto sweep = [&](auto rare_tag) {
        constexpr bool RARE = decltype(rare_tag)::value;
        for (int base = a; base < b; base += 32) {
          const int i = min(base + lane, b - 1);
          SampleIn s;
          const float4 va = s_a[i];
          const float4 vb = s_b[i];
          s.m1 = va.x; s.m2 = va.y; s.dl = va.z; s.npe2 = va.w;
          s.lm1 = vb.x; s.lm2 = vb.y;
          s.valid = base + lane < b;
          float lw;
          Sink sink(acc);
          if (inj)
            sample_lnw<GRAD, float, Sink, true, MP, RARE>(L, s, A.pbar32, nz, pos, aux, nx, wv, ws, lw, sink);
          else
            sample_lnw<GRAD, RowT, Sink, true, MP, RARE>(L, s, reinterpret_cast<const RowT*>(A.los) +
                                                           (size_t)__float_as_int(vb.z) * nz, nz, pos, aux, nx, wv, ws,
                                                           lw, sink);
        }
      };
      if ((GRAD && (L.lam_edge != 0.f || (MP && L.lam1_edge != 0.f))) || L.beta_small != 0.f)
        sweep(std::true_type{});
      else
        sweep(std::false_type{});
      if (KAHAN) { acc.s1 -= acc.c1; acc.s2 -= acc.c2; }
    }
    // butterfly reduction across the warp (every lane ends with the same sums)
    using AccT = Acc<GRAD, KAHAN, NS>;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float om_ = __shfl_xor_sync(0xffffffffu, acc.m, o);
      const float o1 = __shfl_xor_sync(0xffffffffu, acc.s1, o);
      const float o2 = __shfl_xor_sync(0xffffffffu, acc.s2, o);
      float2 og[AccT::NG2];
      float omO[AccT::NO], osO[AccT::NO];
      if (GRAD) {
#pragma unroll
        for (int q = 0; q < AccT::NG2; ++q)
          og[q] = make_float2(__shfl_xor_sync(0xffffffffu, acc.g2[q].x, o),
                              __shfl_xor_sync(0xffffffffu, acc.g2[q].y, o));
#pragma unroll
        for (int q = 0; q < AccT::NO; ++q) {
          omO[q] = __shfl_xor_sync(0xffffffffu, acc.mO[q], o);
          osO[q] = __shfl_xor_sync(0xffffffffu, acc.sO[q], o);
        }
      }
      acc.merge(om_, o1, o2, og, omO, osO);
    }
    if (G == 1) {
      // one warp per point: the warp's sums are the partial; written straight to global
      // memory with the reference rounded up to an integer (the FP64 merge then rescales
      // by exact powers of two), no shared-memory combine
      float* out = A.partials + ((size_t)k * A.stride + A.slot0 + item) * PSTRIDE;
      const float M = ceilf(acc.m);
      const float sc = M > -INFINITY ? ex2(acc.m - M) : 0.f;
      if (lane == 0) {
        out[0] = M;
        out[1] = acc.s1 * sc;
        out[2] = acc.s2 * (sc * sc);
      }
      if (GRAD && lane < NS) {
        float gv = 0.f;
#pragma unroll
        for (int q = 0; q < NS; ++q) gv = (lane == q) ? acc.g(q) : gv;
        out[3 + lane] = gv * sc;
      }
      if (GRAD && lane < 2) {   // the other-component pairs
        const float mo = lane == 0 ? acc.mO[0] : (AccT::NO > 1 ? acc.mO[AccT::NO - 1] : -INFINITY);
        const float so = lane == 0 ? acc.sO[0] : (AccT::NO > 1 ? acc.sO[AccT::NO - 1] : 0.f);
        const float MO = ceilf(mo);
        out[lane == 0 ? PART_MO : PART_MO2] = MO;
        out[lane == 0 ? PART_SO : PART_SO2] = MO > -INFINITY ? so * ex2(mo - MO) : 0.f;
      }
      continue;
    }
    float* slot = s_part + ((size_t)kk * G + wg) * PS;
    if (lane == 0) {
      slot[0] = acc.m;
      slot[1] = acc.s1;
      slot[2] = acc.s2;
      if (GRAD) {
        slot[PART_MO] = acc.mO[0];
        slot[PART_SO] = acc.sO[0];
        slot[PART_MO2] = AccT::NO > 1 ? acc.mO[AccT::NO - 1] : -INFINITY;
        slot[PART_SO2] = AccT::NO > 1 ? acc.sO[AccT::NO - 1] : 0.f;
      }
    }
    if (GRAD && lane < NS) {
      float gv = 0.f;
#pragma unroll
      for (int q = 0; q < NS; ++q) gv = (lane == q) ? acc.g(q) : gv;
      slot[3 + lane] = gv;
    }
  }
  if (G == 1) return;   // the caller's barrier precedes the next unit's staging
  __syncthreads();
  // combine the G warps' sums of each Lambda in warp order: lane q owns component q.
  // The partial's reference is the warps' largest rounded up to an integer (the FP64
  // merge then rescales by exact powers of two).
  for (int kk = warp; kk < nk; kk += WARPS) {
    const float* sl = s_part + (size_t)kk * G * PS;
    float M = -INFINITY;
    for (int w = 0; w < G; ++w) M = fmaxf(M, sl[w * PS]);
    M = ceilf(M);
    const int kq = A.order ? A.order[k0 + kk] : k0 + kk;
    float* out = A.partials + ((size_t)kq * A.stride + A.slot0 + item) * PSTRIDE;
    const int ncomp = GRAD ? 2 + NS : 2;   // s1, s2 (and g)
    if (lane < ncomp) {
      float acc = 0.f;
      if (M > -INFINITY) {
        for (int w = 0; w < G; ++w) {
          const float mw = sl[w * PS];
          if (mw > -INFINITY) acc = fmaf(sl[w * PS + 1 + lane], lane == 1 ? ex2(2.f * (mw - M)) : ex2(mw - M), acc);
        }
      }
      out[1 + lane] = acc;
    }
    if (lane == 0) out[0] = M;
    if (GRAD && (lane == ncomp || lane == ncomp + 1)) {   // the lanes past the sums: one other pair each
      const int pm = lane == ncomp ? PART_MO : PART_MO2;
      float MO = -INFINITY;
      for (int w = 0; w < G; ++w) MO = fmaxf(MO, sl[w * PS + pm]);
      MO = ceilf(MO);
      float so = 0.f;
      if (MO > -INFINITY) {
        for (int w = 0; w < G; ++w) {
          const float mo = sl[w * PS + pm];
          if (mo > -INFINITY) so = fmaf(sl[w * PS + pm + 1], ex2(mo - MO), so);
        }
      }
      out[pm] = MO;
      out[pm + 1] = so;
    }
  }
}

template <bool GRAD, bool KAHAN, typename RowT, bool MP>
__global__ void __launch_bounds__(THREADS, GRAD ? MINB_GRAD : MINB_VALUE) k_fused(const __grid_constant__ FusedArgs A) {
  extern __shared__ __align__(16) float sm[];
  // persistent: each CTA takes (item, Lambda-slab) units from the counter until none
  // is left; the counter is zeroed by the prologue of the same call
  __shared__ int s_unit, s_next;
  const int n_units = A.n_sched * A.n_slabs;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(A.counter, 1);
    __syncthreads();
    const int unit = s_unit;
    if (unit >= n_units) break;
    fused_unit<GRAD, KAHAN, RowT, MP>(A, unit, sm, &s_next);
    __syncthreads();   // every warp is done with the staged samples (and the combine with s_part)
  }
}

// ------------------------------------------------------------------ KDE form
// The paper's own event term (Eqs. 5-7): for each (event, pixel) group, a Gaussian KDE
// in z of the group's samples weighted by w' (the weight without its LOS factor) on a
// uniform grid of G points over [0, z_max], times the pixel's LOS prior at the grid
// points, trapezoid rule.  One warp per (group, Lambda); the 8 warps of a CTA take 8
// Lambda points of one group, so the group's samples are read from L1 after the first.
// Pass 1: z and w' of every sample -> the pixel's N_eff and the moments (and, for the
// Silverman and biweight rules, order statistics: within a group the samples are sorted
// by d_L, so by z, and the samples with a z form a contiguous index range).  Pass 2:
// each sample adds w' times its kernel's trapezoid sum over the grid points within 6 h
// (the kernel's mass beyond is 2e-9).
namespace {

struct KdeSink {
  float z = -INFINITY;
  __device__ __forceinline__ bool any(bool p) { return p; }
  __device__ __forceinline__ bool weight(float, bool) { return false; }
  __device__ __forceinline__ void grad2(int, float, float) {}
  __device__ __forceinline__ void other(int, float, float) {}
  __device__ __forceinline__ void position(float zz, int, bool ok) {
    if (ok) z = zz;
  }
  __device__ __forceinline__ void reached(int, bool) {}
  __device__ __forceinline__ void windows(bool, bool, bool) {}
};

struct KdeCtx {
  bool mp;            // multi-peak mass model
  const LamF& L;
  const float4* pos;
  const float4* aux;
  const float4* wv;
  const float4* ws;
  int nx, nz;
  const float2* lm;   // the group's log2 masses
};

// z and log2 w' of a sample (z = -inf when d_L has no z; lw = -inf when w' = 0)
__device__ __forceinline__ void kde_sample(const KdeCtx& C, const float4 v, const float2 lm, float& z,
                                           float& lw) {
  SampleIn s;
  s.m1 = v.x; s.m2 = v.y; s.dl = v.z; s.npe2 = -to_log2(v.w);
  s.lm1 = lm.x; s.lm2 = lm.y;
  KdeSink sk;
  float l = -INFINITY;
  const float* none = nullptr;
  const bool ok = C.mp ? sample_lnw<false, float, KdeSink, false, true>(C.L, s, none, C.nz, C.pos, C.aux, C.nx,
                                                                        C.wv, C.ws, l, sk)
                       : sample_lnw<false, float, KdeSink, false, false>(C.L, s, none, C.nz, C.pos, C.aux, C.nx,
                                                                         C.wv, C.ws, l, sk);
  z = sk.z;
  lw = ok ? l : -INFINITY;
}

__device__ __forceinline__ float kde_z(const KdeCtx& C, const float4* smp, int64_t i) {
  float z, lw;
  kde_sample(C, __ldg(smp + i), C.lm[i], z, lw);
  return z;
}

// quantile q of the n z values starting at index v0 (sorted): linear between order statistics
__device__ float kde_quantile(const KdeCtx& C, const float4* smp, int64_t v0, int n, float q) {
  const float pos = q * (float)(n - 1);
  const int i = min((int)floorf(pos), n - 1);
  const float z0 = kde_z(C, smp, v0 + i);
  if (i + 1 >= n) return z0;
  return fmaf(pos - (float)i, kde_z(C, smp, v0 + i + 1) - z0, z0);
}

// k-th smallest (0-based) of |z_i - Q| over the n sorted values from v0, where the first
// `nl` values are <= Q (their deviations fall with i) and the rest are > Q (rise with i)
__device__ float kde_kth_dev(const KdeCtx& C, const float4* smp, int64_t v0, int n, int nl, float Q, int k) {
  // A[a] = Q - z[nl - 1 - a] (a < nl, ascending), B[b] = z[nl + b] - Q (b < n - nl, ascending)
  const int na = nl, nb = n - nl;
  int lo = max(0, k + 1 - nb), hi = min(k + 1, na);   // number taken from A
  for (int it = 0; it < 40 && lo < hi; ++it) {
    const int ta = (lo + hi) >> 1, tb = k + 1 - ta;
    // need A[ta-1] <= B[tb] and B[tb-1] <= A[ta]
    const float a_next = ta < na ? Q - kde_z(C, smp, v0 + nl - 1 - ta) : INFINITY;
    const float b_prev = tb > 0 ? kde_z(C, smp, v0 + nl + tb - 1) - Q : -INFINITY;
    if (b_prev > a_next) lo = ta + 1; else hi = ta;
  }
  const int ta = lo, tb = k + 1 - ta;
  const float a_last = ta > 0 ? Q - kde_z(C, smp, v0 + nl - ta) : -INFINITY;
  const float b_last = tb > 0 ? kde_z(C, smp, v0 + nl + tb - 1) - Q : -INFINITY;
  return fmaxf(a_last, b_last);
}

}  // namespace

__global__ void __launch_bounds__(THREADS) k_kde(KdeArgs A) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the Lambda index by a warp reduction: the compiler then knows it is the same in
  // every lane and keeps the point's constants out of the per-thread registers
  const int g = blockIdx.x, k = __reduce_max_sync(0xffffffffu, blockIdx.y * WARPS + warp);
  if (k >= A.K) return;
  const KdeGroup grp = A.groups[g];
  float* out = A.partials + ((size_t)k * A.stride + g) * PSTRIDE;
  const LamF L = A.lf[k];
  if (L.live == 0.f) {
    if (lane == 0) { out[0] = -INFINITY; out[1] = 0.f; out[2] = 0.f; }
    return;
  }
  const float* tb = A.tables + (size_t)k * A.tstride;
  const float4* pos = reinterpret_cast<const float4*>(tb);
  const float4* aux = reinterpret_cast<const float4*>(tb + 4 * A.nx);
  const float4* wv = reinterpret_cast<const float4*>(tb + 8 * A.nx);
  const KdeCtx C{A.mp != 0, L, pos, aux, wv, wv + (NW_WIN + 1), A.nx, A.nz, A.lm + grp.begin};
  const float4* smp = A.smp + grp.begin;
  const int n = grp.count;
  if (A.census && lane == 0) atomicAdd(A.census + 0, (unsigned long long)n);

  // ---- pass 1: weights (max, sum, sum of squares), Welford moments of z, valid range
  float m = -INFINITY, s1 = 0.f, s2 = 0.f;
  // Welford per lane and Chan's pairwise merge across lanes, all in FP32: this GPU's
  // FP64 pipe runs at 1/64 of the FP32 rate, and a few FP64 divisions per warp kept it
  // half busy for the whole kernel
  float fn = 0.f, fmean = 0.f, fM2 = 0.f;
  int vmin = INT_MAX, vmax = -1;
  for (int i = lane; i < n; i += 32) {
    float z, lw;
    kde_sample(C, __ldg(smp + i), C.lm[i], z, lw);
    if (z > -INFINITY) {
      vmin = min(vmin, i);
      vmax = max(vmax, i);
      fn += 1.f;
      const float d = z - fmean;
      fmean = fmaf(d, 1.f / fn, fmean);
      fM2 = fmaf(d, z - fmean, fM2);
    }
    if (lw > -INFINITY) {
      if (lw > m) {
        const float sc = ex2(m - lw);
        s1 = fmaf(s1, sc, 1.f);
        s2 = fmaf(s2, sc * sc, 1.f);
        m = lw;
      } else {
        const float t = ex2(lw - m);
        s1 += t;
        s2 = fmaf(t, t, s2);
      }
    }
  }
  float wn = fn, wmean = fmean, wM2 = fM2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float om = __shfl_xor_sync(0xffffffffu, m, o);
    const float o1 = __shfl_xor_sync(0xffffffffu, s1, o);
    const float o2 = __shfl_xor_sync(0xffffffffu, s2, o);
    const float M = fmaxf(m, om);
    if (M > -INFINITY) {
      const float ra = ex2(m - M), rb = ex2(om - M);
      s1 = s1 * ra + o1 * rb;
      s2 = s2 * ra * ra + o2 * rb * rb;
      m = M;
    }
    const float bn = __shfl_xor_sync(0xffffffffu, wn, o);
    const float bmean = __shfl_xor_sync(0xffffffffu, wmean, o);
    const float bM2 = __shfl_xor_sync(0xffffffffu, wM2, o);
    const float nn = wn + bn;   // exact: counts stay below 2^24
    if (nn > 0.f) {   // Chan et al.'s pairwise update of (n, mean, M2)
      const float d = bmean - wmean, r = bn / nn;
      wM2 = wM2 + bM2 + (d * d) * (wn * r);
      wmean = fmaf(d, r, wmean);
      wn = nn;
    }
    vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  // the two partners of a butterfly round differently; every lane takes lane 0's M2
  wM2 = __shfl_sync(0xffffffffu, wM2, 0);
  const int nv = (int)wn;
  bool keep = m > -INFINITY && nv >= 2 && s1 * s1 >= A.neff_min * s2;

  // ---- bandwidth (every lane computes the same value; the order statistics by lane 0)
  float h = 0.f;
  if (keep) {
    const float shrink = exp2f(-0.2f * log2f((float)nv));
    const float sigma = sqrtf(wM2 / (wn - 1.f));
    if (A.rule == 0) {
      h = 1.06f * sigma * shrink;
    } else {
      float hv = 0.f;
      if (lane == 0) {
        if (A.rule == 1) {
          const float iqr = kde_quantile(C, smp, vmin, nv, 0.75f) - kde_quantile(C, smp, vmin, nv, 0.25f);
          hv = 0.9f * fminf(sigma, iqr / 1.34f) * shrink;
        } else {
          const float Q = kde_quantile(C, smp, vmin, nv, 0.5f);
          // values <= Q: binary search on the sorted z
          int lo = 0, hi = nv;
          for (int it = 0; it < 40 && lo < hi; ++it) {
            const int mid = (lo + hi) >> 1;
            if (kde_z(C, smp, vmin + mid) <= Q) lo = mid + 1; else hi = mid;
          }
          const float pos = 0.5f * (float)(nv - 1);
          const int i0 = (int)floorf(pos);
          const float d0 = kde_kth_dev(C, smp, vmin, nv, lo, Q, i0);
          const float d1 = i0 + 1 < nv ? kde_kth_dev(C, smp, vmin, nv, lo, Q, i0 + 1) : d0;
          const float mad = fmaf(pos - (float)i0, d1 - d0, d0);
          hv = mad > 0.f ? Q : NAN;   // Q passed on; the sums below need every lane
          h = mad;
        }
      }
      if (A.rule == 1) {
        h = __shfl_sync(0xffffffffu, hv, 0);
      } else {
        const float Q = __shfl_sync(0xffffffffu, hv, 0);
        const float mad = __shfl_sync(0xffffffffu, h, 0);
        h = 0.f;
        if (mad > 0.f) {
          const float inv9 = 1.f / (9.f * mad);
          float num = 0.f, den = 0.f;
          for (int i = vmin + lane; i <= vmax; i += 32) {
            const float dz = kde_z(C, smp, i) - Q;
            const float u = dz * inv9;
            if (fabsf(u) < 1.f) {
              const float u2 = u * u, a = 1.f - u2, a2 = a * a;
              num = fmaf((dz * dz) * a2, a2, num);
              den = fmaf(a, fmaf(-5.f, u2, 1.f), den);
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
          }
          if (den != 0.f && num > 0.f) h = 1.06f * sqrtf((float)nv * num / (den * den)) * shrink;
        }
      }
    }
    keep = h > 0.f;
  }
  if (!keep) {
    if (lane == 0) { out[0] = -INFINITY; out[1] = 0.f; out[2] = 0.f; }
    return;
  }
  unsigned n_w = 0, n_terms = 0;   // census counts of this lane (measurement only)

  // ---- pass 2: sum_k w'_k sum_g c_g p_LOS(z_g) K_h(z_g - z_k), scaled by 2^-m; each
  //      kernel over the grid points within 6 h (its mass beyond is 2e-9), taken in
  //      aligned blocks of 4.  On a uniform grid the Gaussian's values follow a product
  //      recurrence: with e_j = 2^(c d_j^2), d_j = z_j - z, c = -log2(e) / (2 h^2),
  //      e_(j+1) = e_j r_j, r_j = 2^(c (2 d_j dz + dz^2)), r_(j+1) = r_j q, q = 2^(2 c dz^2);
  //      each block starts from its own e_0 and r_0 (two ex2), so the rounding drift stays
  //      within ~10 ulp.  For h >= dz a block's e_0 >= 2^-72 and r <= 2^14 (no underflow or
  //      overflow inside a block); narrower kernels take every value from ex2.
  const int GS = kde_row(A.G);
  const float* pg = A.pgrid + (size_t)grp.pix * GS;
  const float dzg = A.dzg, inv_dzg = 1.f / dzg, reach = 6.f * h;
  const float cexp = -0.5f * LOG2EF / (h * h);
  const bool recur = dzg <= h;
  const float lq = 2.f * cexp * dzg * dzg;        // log2 q
  float acc = 0.f;
  for (int i = lane; i < n; i += 32) {
    float z, lw;
    kde_sample(C, __ldg(smp + i), C.lm[i], z, lw);
    if (!(lw > -INFINITY)) continue;
    const int g0 = max(0, (int)ceilf((z - reach) * inv_dzg));
    const int g1 = min(A.G - 1, (int)floorf((z + reach) * inv_dzg));
    float T = 0.f;
    int lo = g0, hi = g1;                         // the grid points summed
    if (recur && g0 <= g1) {
      lo = g0 & ~(KDE_BLOCK - 1);
      hi = min(g1 | (KDE_BLOCK - 1), GS - 1);     // padding beyond the grid holds zeros
      const float ql = ex2(lq);
      for (int b = lo; b <= hi; b += KDE_BLOCK) {
        const float d0 = fmaf((float)b, dzg, -z);
        float e = ex2((cexp * d0) * d0);
        float r = ex2(cexp * fmaf(2.f * d0, dzg, dzg * dzg));
        static_assert(KDE_BLOCK == 4, "one float4 of grid values a block");
        const float4 pa = __ldg(reinterpret_cast<const float4*>(pg + b));
        const float pv[KDE_BLOCK] = {pa.x, pa.y, pa.z, pa.w};
#pragma unroll
        for (int j = 0; j < KDE_BLOCK; ++j) {
          T = fmaf(pv[j], e, T);
          e *= r;
          r *= ql;
        }
      }
      hi = min(hi, A.G - 1);
    } else {
      float gf = (float)g0;
      for (int gg = g0; gg <= g1; ++gg, gf += 1.f) {
        const float d = fmaf(gf, dzg, -z);
        T = fmaf(__ldg(pg + gg), ex2((cexp * d) * d), T);
      }
    }
    if (A.census) {
      ++n_w;
      n_terms += (unsigned)max(hi - lo + 1, 0);
    }
    // trapezoid: the two end points of the grid weigh half (when summed)
    if (lo == 0 && hi >= 0) T = fmaf(-0.5f * __ldg(pg), ex2((cexp * z) * z), T);
    if (hi == A.G - 1 && lo <= hi) {
      const float d = fmaf((float)(A.G - 1), dzg, -z);
      T = fmaf(-0.5f * __ldg(pg + A.G - 1), ex2((cexp * d) * d), T);
    }
    acc = fmaf(ex2(lw - m), T, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (A.census) {
    const unsigned a = __reduce_add_sync(0xffffffffu, n_w), b = __reduce_add_sync(0xffffffffu, n_terms);
    if (lane == 0) {
      atomicAdd(A.census + 1, 1ull);
      atomicAdd(A.census + 2, (unsigned long long)a);
      atomicAdd(A.census + 3, (unsigned long long)b);
    }
  }
  if (lane == 0) {
    // the reference rounded up to an integer for the merge, the sum scaled to it
    const float mi = ceilf(m);
    const float S = acc * dzg / (h * 2.50662827463100050242f) * ex2(m - mi);   // h sqrt(2 pi)
    out[0] = S > 0.f ? mi : -INFINITY;
    out[1] = S;
    out[2] = S * S;
  }
}

__global__ void k_los_grid(const float* __restrict__ los, int n_pix, int nz, double zmax, int G,
                           float* __restrict__ out) {
  const int GS = kde_row(G);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_pix * GS) return;
  const int p = (int)(t / GS), gq = (int)(t - (long long)p * GS);
  if (gq >= G) {   // padding of the row to whole blocks
    out[t] = 0.f;
    return;
  }
  const double zg = gq * (zmax / (G - 1));
  const double sc = (double)(nz - 1) / zmax;
  int j = (int)floor(zg * sc);
  if (j > nz - 2) j = nz - 2;
  if (j < 0) j = 0;
  const double tt = zg * sc - (double)j;
  const float* row = los + (size_t)p * nz;
  const double a = row[j], b = row[j + 1];
  out[t] = (float)(a + tt * (b - a));
}

__global__ void k_log2_masses(const float4* __restrict__ smp, long long n, float2* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = __ldg(smp + i);
  out[i] = make_float2(log2f(v.x), log2f(v.y));
}

cudaError_t launch_log2_masses(const float4* smp, long long n, float2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_log2_masses<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(smp, n, out);
  return cudaGetLastError();
}

cudaError_t launch_kde(const KdeArgs& a, cudaStream_t s) {
  if (a.n_groups <= 0 || a.K <= 0) return cudaSuccess;
  const dim3 grid((unsigned)a.n_groups, (unsigned)((a.K + WARPS - 1) / WARPS));
  k_kde<<<grid, THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_los_grid(const float* los, int n_pix, int nz, double zmax, int G, float* out,
                            cudaStream_t s) {
  const long long n = (long long)n_pix * kde_row(G);
  k_los_grid<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(los, n_pix, nz, zmax, G, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ plain path
// pass 1 (value) and pass 3 (gradient): one thread per sample, one Lambda, tables and
// samples straight from global memory.  Pass 1 writes ln w; pass 3 writes
// e^(ln w - m_item) d ln w / d Lambda for the item's max m from pass 2.
template <bool GRAD, typename RowT>
__global__ void __launch_bounds__(256) k_plain_sample(PlainArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n_total) return;
  const LamF L = A.lf[A.k];
  const bool inj = i >= A.n_samples;
  float4 v = inj ? __ldg(A.inj + (i - A.n_samples)) : __ldg(A.smp + i);
  SampleIn s;
  s.m1 = v.x; s.m2 = v.y; s.dl = v.z; s.npe2 = -to_log2(v.w);
  s.lm1 = log2f(v.x); s.lm2 = log2f(v.y);
  const float* tb = A.tables + (size_t)A.k * A.tstride;
  const int nx = A.nx;
  const float4* pos = reinterpret_cast<const float4*>(tb);
  const float4* aux = reinterpret_cast<const float4*>(tb + 4 * nx);
  const float4* wv = reinterpret_cast<const float4*>(tb + 8 * nx);
  const float4* ws = wv + (NW_WIN + 1);
  // the gradient pass knows its item's final maximum from the value pass
  const float m = GRAD ? A.partials[((size_t)A.k * A.n_items + A.sample_item[i]) * PSTRIDE] : -INFINITY;
  float lw = -INFINITY;
  TermSink ts;
  bool ok = false;
  if (L.live != 0.f) {
    if (inj)
      ok = sample_lnw<GRAD>(L, s, A.pbar32, A.nz, pos, aux, nx, wv, ws, lw, ts);
    else
      ok = sample_lnw<GRAD>(L, s, reinterpret_cast<const RowT*>(A.los) + (size_t)__ldg(A.pix + i) * A.nz,
                            A.nz, pos, aux, nx, wv, ws, lw, ts);
  }
  if (!GRAD) {
    A.lw[i] = ok ? lw : -INFINITY;
  } else {
    const float t = ok ? ex2(lw - m) : 0.f;
    for (int q = 0; q < NP; ++q) A.tg[(size_t)q * A.n_total + i] = ok ? t * ts.g[q] : 0.f;
    if (ok && ts.edge[0])   // sigma (t - t O/mix): may overflow for extreme samples
      A.tg[(size_t)S_LX * A.n_total + i] = ts.g[S_LX] * (t - ex2(lw - m + ts.lo[0]));
  }
}

// pass 2 / pass 4: one CTA per item reduces its range of the per-sample arrays
template <bool GRAD>
__global__ void __launch_bounds__(256) k_plain_reduce(PlainArgs A) {
  __shared__ float red[3][8];
  __shared__ float redg[NP][8];
  const int item = blockIdx.x;
  const Item it = A.items[item];
  const long long base = it.kind == 1 ? A.n_samples + it.begin : it.begin;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float* out = A.partials + ((size_t)A.k * A.n_items + item) * PSTRIDE;
  if (!GRAD) {
    float m = -INFINITY;
    for (int i = tid; i < it.count; i += 256) m = fmaxf(m, A.lw[base + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[0][w] = m;
    __syncthreads();
    m = red[0][0];
    for (int q = 1; q < 8; ++q) m = fmaxf(m, red[0][q]);
    m = ceilf(m);   // an integer reference for the merge (and the gradient pass)
    float s1 = 0.f, s2 = 0.f;
    if (m > -INFINITY)
      for (int i = tid; i < it.count; i += 256) {
        const float t = ex2(A.lw[base + i] - m);
        s1 += t;
        s2 += t * t;
      }
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    __syncthreads();
    if (lane == 0) { red[1][w] = s1; red[2][w] = s2; }
    __syncthreads();
    if (tid == 0) {
      float a = 0.f, b = 0.f;
      for (int q = 0; q < 8; ++q) { a += red[1][q]; b += red[2][q]; }
      out[0] = m;
      out[1] = a;
      out[2] = b;
      out[PART_MO] = -INFINITY;   // the plain path folds the lambda-edge term into its g
      out[PART_SO] = 0.f;
      out[PART_MO2] = -INFINITY;
      out[PART_SO2] = 0.f;
    }
  } else {
    float gs[NP];
    for (int q = 0; q < NP; ++q) gs[q] = 0.f;
    for (int i = tid; i < it.count; i += 256)
      for (int q = 0; q < NP; ++q) gs[q] += A.tg[(size_t)q * A.n_total + base + i];
    for (int q = 0; q < NP; ++q) {
      for (int o = 16; o > 0; o >>= 1) gs[q] += __shfl_xor_sync(0xffffffffu, gs[q], o);
      if (lane == 0) redg[q][w] = gs[q];
    }
    __syncthreads();
    if (tid < NP) {
      float a = 0.f;
      for (int q = 0; q < 8; ++q) a += redg[tid][q];
      out[3 + tid] = a;
    }
  }
}

// -------------------------------------------------------------------- merge
// Partial references arrive in log2 units and are integers (every producer rounds its
// reference up to one and scales its sums to it), so every rescale of the FP64 sums is
// an exact power of two: 2^k from the exponent field, without the FP64 exp2 sequence
// (GB300's FP64 pipe runs at 1/64 of the FP32 rate, and the merge of a small batch is
// a chain of such rescales).  Below the FP64 range the term is dropped (it is below
// 2^-1022 of the largest), above it the result is infinite.
__device__ __forceinline__ double pow2i(double k) {
  if (!(k >= -1022.0)) return 0.0;
  if (k > 1023.0) return INFINITY;
  return __longlong_as_double((long long)(1023 + (int)k) << 52);
}
constexpr double LN2D = 0.69314718055994530942;

// The CTA-wide sums of the merge.  Every thread holds NV values; the sum of each column
// over the CTA's threads is formed in shared memory in a fixed order (a transposed
// reduction): CB columns at a time, each thread first adds MB rows of one column, then
// the segment sums are added MB at a time until one is left.  GB300's FP64 pipe charges a
// warp-instruction the same whatever its active lanes, so this costs a few FP64
// instructions a column where a warp butterfly would spend five levels of every value
// in every warp and a serial pass over the warps.  nt (the CTA's threads) is a power of
// two from 32 to 256; the column sums land in res[NV].
constexpr int MERGE_CB = 8, MERGE_MB = 8;
template <int NV>
__device__ void merge_column_sums(const double (&v)[NV], double* buf, double* res) {
  const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
  for (int c0 = 0; c0 < NV; c0 += MERGE_CB) {
#pragma unroll
    for (int j = 0; j < MERGE_CB; ++j) buf[tid * MERGE_CB + j] = (c0 + j < NV) ? v[c0 + j] : 0.0;
    __syncthreads();
    int nseg = nt;   // rows still to be added, per column
    while (nseg > 1) {
      const int g = nseg < MERGE_MB ? nseg : MERGE_MB;
      const int out = nseg / g;
      double acc = 0.0;
      const int j = tid % MERGE_CB, s = tid / MERGE_CB;
      if (s < out) {
        acc = buf[(s * g) * MERGE_CB + j];
        for (int q = 1; q < g; ++q) acc += buf[(s * g + q) * MERGE_CB + j];
      }
      __syncthreads();
      if (s < out) buf[s * MERGE_CB + j] = acc;
      __syncthreads();
      nseg = out;
    }
    if (tid < MERGE_CB && c0 + tid < NV) res[c0 + tid] = buf[tid];
    __syncthreads();
  }
}

// CTA-wide maximum of an integer per thread, the same in every thread
__device__ int merge_imax(int x, int* s_i) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = __reduce_max_sync(0xffffffffu, x);
  if (lane == 0) s_i[w] = x;
  __syncthreads();
  int m = s_i[0];
  for (int q = 1; q < nw; ++q) m = max(m, s_i[q]);
  __syncthreads();
  return m;
}
// an integer-valued reference (or -inf) as an int, and back
__device__ __forceinline__ int ref_to_int(double m) { return m > -INFINITY ? (int)m : INT_MIN; }
__device__ __forceinline__ double int_to_ref(int m) { return m == INT_MIN ? -INFINITY : (double)m; }

template <bool GRAD, bool MP>
__global__ void __launch_bounds__(256, 1) k_merge(MergeArgs A) {
  constexpr int NPK = n_params(MP);   // gradient width of the mass model (a constant, so the
                                      // per-component arrays stay in registers)
  // per-thread columns: the events' sum of ln L_i, and with the gradient the events'
  // normalised statistics U (13/16), the events' other-component sums (2); the selection
  // sums S1, S2 (and G, 13/16) and its other-component sums (2), all rescaled to the
  // CTA's references
  constexpr int C_U = 1, C_OE = C_U + (GRAD ? NPK : 0), C_S1 = C_OE + (GRAD ? 2 : 0);
  constexpr int C_S2 = C_S1 + 1, C_G = C_S2 + 1, C_OS = C_G + (GRAD ? NPK : 0);
  constexpr int NV = C_OS + (GRAD ? 2 : 0);
  __shared__ double s_buf[256 * MERGE_CB];
  __shared__ double s_res[NV];
  __shared__ int s_i[8], s_ok[8], s_fail[8];
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nt = blockDim.x, nw = nt >> 5;   // sized to the work by launch_merge
  const LamD D = A.ld[k];
  const int ne = A.n_events;
  if (D.flag & 1) {
    for (int e = tid; e < ne; e += nt) {
      A.lnL_event[(size_t)k * ne + e] = -INFINITY;
      A.neff_event[(size_t)k * ne + e] = 0.0;
    }
    if (tid == 0) {
      A.ln_xi[k] = -INFINITY;
      A.neff_sel[k] = 0.0;
      if (A.lnL_total) A.lnL_total[k] = -INFINITY;
      if (A.sum_events) A.sum_events[k] = -INFINITY;
      A.flags[k] = 1;
      for (int i = 0; i < NPK; ++i) {
        if (GRAD && A.grad_total) A.grad_total[(size_t)k * NPK + i] = 0.0;
        if (GRAD && A.grad_events) A.grad_events[(size_t)k * NPK + i] = 0.0;
        if (GRAD && A.grad_ln_xi) A.grad_ln_xi[(size_t)k * NPK + i] = 0.0;
      }
    }
    return;
  }
  const int P = A.P;
  const float* pk = A.partials + (size_t)k * A.n_items * P * PSTRIDE;
  double v[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) v[c] = 0.0;

  // ---- events: thread-strided, each event merged in item order.  Its gradient
  // d ln L_i = stats_to_grad(st_i, S1_i) / S1_i + dc is linear in the statistics, so the
  // CTA sums st_i / S1_i (and the other-component sums / S1_i) and the tail applies
  // stats_to_grad once, with n_ok (the events with a weight) in place of S1
  double sumL = 0.0, cmp = 0.0;
  int fail = 0;   // bit 0: an event below the N_eff threshold; bit 1: an event with no weight
  int n_ok = 0;
  for (int e = tid; e < ne; e += nt) {
    const int s0 = A.ev_item0[e] * P, s1 = A.ev_item0[e + 1] * P;
    double M = -INFINITY;
    for (int s = s0; s < s1; ++s) M = fmax(M, (double)pk[(size_t)s * PSTRIDE]);
    double S1 = 0.0, S2 = 0.0, G[GRAD ? NP_MAX : 1], O[2] = {0.0, 0.0};
    if (GRAD)
      for (int i = 0; i < NPK; ++i) G[i] = 0.0;
    if (M > -INFINITY) {
      for (int s = s0; s < s1; ++s) {
        const float* p = pk + (size_t)s * PSTRIDE;
        if (!(p[0] > -INFINITY)) continue;
        const double r = pow2i((double)p[0] - M);
        S1 += (double)p[1] * r;
        S2 += (double)p[2] * r * r;
        if (GRAD)
          for (int i = 0; i < NPK; ++i) G[i] += (double)p[3 + i] * r;
      }
      if (GRAD && (D.lam_sigma != 0 || D.lam1_sigma != 0))   // other-component sums at the bounds
        for (int s = s0; s < s1; ++s) {
          const float* p = pk + (size_t)s * PSTRIDE;
          if (D.lam_sigma != 0 && p[PART_MO] > -INFINITY) O[0] += (double)p[PART_SO] * pow2i((double)p[PART_MO] - M);
          if (D.lam1_sigma != 0 && p[PART_MO2] > -INFINITY) O[1] += (double)p[PART_SO2] * pow2i((double)p[PART_MO2] - M);
        }
    }
    double lnL = -INFINITY, neff = 0.0;
    if (S1 > 0.0) {
      lnL = M * LN2D + log(S1) - A.ln_ev_n[e] + lamd_c(D);
      neff = S1 * S1 / S2;
      if constexpr (GRAD) {
        const double iS1 = 1.0 / S1;
#pragma unroll
        for (int i = 0; i < NPK; ++i) v[C_U + i] = fma(G[i], iS1, v[C_U + i]);
        v[C_OE] = fma(O[0], iS1, v[C_OE]);
        v[C_OE + 1] = fma(O[1], iS1, v[C_OE + 1]);
      }
    }
    A.lnL_event[(size_t)k * ne + e] = lnL;
    A.neff_event[(size_t)k * ne + e] = neff;
    if (!(neff >= A.neff_min_event)) fail |= 1;
    if (!(S1 > 0.0)) {
      fail |= 2;   // a zero-weight event makes the product of Eq. 3 vanish
      continue;
    }
    ++n_ok;
    // Neumaier-compensated sum in this thread's event order
    const double t = sumL + lnL;
    if (fabs(sumL) >= fabs(lnL)) cmp += (sumL - t) + lnL; else cmp += (lnL - t) + sumL;
    sumL = t;
  }
  v[0] = sumL + cmp;

  // ---- injections: online merge of the injection partials
  double sM = -INFINITY, sS1 = 0.0, sS2 = 0.0, sG[GRAD ? NP_MAX : 1];
  double oM[2] = {-INFINITY, -INFINITY}, oS[2] = {0.0, 0.0};   // other-component pairs at the bounds
  if (GRAD)
    for (int i = 0; i < NPK; ++i) sG[i] = 0.0;
  for (int s = A.inj_item0 * P + tid; s < A.n_items * P; s += nt) {
    const float* p = pk + (size_t)s * PSTRIDE;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int pm = q == 0 ? PART_MO : PART_MO2;
      if (GRAD && (q == 0 ? D.lam_sigma : D.lam1_sigma) != 0 && p[pm] > -INFINITY) {
        const double mo = p[pm];
        if (mo > oM[q]) { oS[q] = oS[q] * pow2i(oM[q] - mo) + (double)p[pm + 1]; oM[q] = mo; }
        else oS[q] += (double)p[pm + 1] * pow2i(mo - oM[q]);
      }
    }
    const double m = p[0];
    if (!(m > -INFINITY)) continue;
    if (m > sM) {
      const double r = pow2i(sM - m);
      sS1 *= r;
      sS2 *= r * r;
      if (GRAD)
        for (int i = 0; i < NPK; ++i) sG[i] *= r;
      sM = m;
    }
    const double r = pow2i(m - sM);
    sS1 += (double)p[1] * r;
    sS2 += (double)p[2] * r * r;
    if (GRAD)
      for (int i = 0; i < NPK; ++i) sG[i] += (double)p[3 + i] * r;
  }

  // ---- the CTA's references: every partial reference is an integer (or -inf), and so
  // are the threads' maxima, so the CTA-wide maxima are exact integer maxima; each thread
  // rescales its sums to them by exact powers of two, which leaves plain column sums
  const double M = int_to_ref(merge_imax(ref_to_int(sM), s_i));
  {
    const double r = (M > -INFINITY && sM > -INFINITY) ? pow2i(sM - M) : 0.0;
    v[C_S1] = sS1 * r;
    v[C_S2] = sS2 * r * r;
    if constexpr (GRAD)
#pragma unroll
      for (int i = 0; i < NPK; ++i) v[C_G + i] = sG[i] * r;
  }
  double MO[2] = {-INFINITY, -INFINITY};
  if constexpr (GRAD) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      MO[q] = int_to_ref(merge_imax(ref_to_int(oM[q]), s_i));
      v[C_OS + q] = (MO[q] > -INFINITY && oM[q] > -INFINITY) ? oS[q] * pow2i(oM[q] - MO[q]) : 0.0;
    }
  }
  {
    const int f = __reduce_or_sync(0xffffffffu, fail), c = __reduce_add_sync(0xffffffffu, n_ok);
    if (lane == 0) { s_fail[w] = f; s_ok[w] = c; }
  }
  merge_column_sums<NV>(v, s_buf, s_res);   // (its barriers also publish s_fail, s_ok)
  int fl = 0, nok = 0;
  for (int q = 0; q < nw; ++q) { fl |= s_fail[q]; nok += s_ok[q]; }

  // ---- the tail: ln xi, N_eff,sel, flags and the total; the gradient components one
  // lane each
  const double S1 = s_res[C_S1], S2 = s_res[C_S2];
  int flag = (fl & 1) ? 2 : 0;
  const bool dead = (fl & 2) != 0;
  double lnxi = -INFINITY, neffs = 0.0;
  if (S1 > 0.0) {
    lnxi = M * LN2D + log(S1) - A.ln_n_draw + lamd_c(D);
    neffs = S1 * S1 / S2;
  } else {
    flag |= 8;
  }
  if (A.neff_min_sel > 0.0 && !(neffs >= A.neff_min_sel)) flag |= 4;
  const double tot = s_res[0];
  if (tid == 0) {
    A.ln_xi[k] = lnxi;
    A.neff_sel[k] = neffs;
    A.flags[k] = flag;
    if (A.lnL_total) A.lnL_total[k] = (flag || dead) ? -INFINITY : tot - (double)ne * lnxi;
    if (A.sum_events) A.sum_events[k] = dead ? -INFINITY : tot;
  }
  if constexpr (GRAD) {
   if (w == 0) {
    // the events' gradient: stats_to_grad of the summed normalised statistics with n_ok
    // for S1, the other-component sums, and n_ok times the per-Lambda constant's
    // derivative; the selection's: stats_to_grad(G, S1) less its other-component sums,
    // over S1.  Every lane forms both (FP64 instructions cost the same for one lane as
    // for the warp) and lane i writes component i.
    double st[NP_MAX], ge[NP_MAX], gs[NP_MAX];
#pragma unroll
    for (int i = 0; i < NPK; ++i) st[i] = s_res[C_U + i];
    stats_to_grad(st, (double)nok, D, ge);
#pragma unroll
    for (int i = 0; i < NPK; ++i) st[i] = s_res[C_G + i];
    stats_to_grad(st, S1, D, gs);
    if (D.lam_sigma != 0) {
      ge[P_LAM] -= D.lam_sigma * s_res[C_OE];
      if (MO[0] > -INFINITY && M > -INFINITY) gs[P_LAM] -= D.lam_sigma * s_res[C_OS] * pow2i(MO[0] - M);
    }
    if (D.lam1_sigma != 0) {
      ge[P_LAM1] -= D.lam1_sigma * s_res[C_OE + 1];
      if (MO[1] > -INFINITY && M > -INFINITY) gs[P_LAM1] -= D.lam1_sigma * s_res[C_OS + 1] * pow2i(MO[1] - M);
    }
    const double iS = S1 > 0.0 ? 1.0 / S1 : 0.0;   // one division for all components
    double gev = 0.0, gsel = 0.0;
#pragma unroll
    for (int i = 0; i < NPK; ++i)
      if (lane == i) {
        gev = ge[i] + (double)nok * lamd_dc(D, i);
        gsel = gs[i] * iS + lamd_dc(D, i);
      }
    if (lane < NPK) {
      if (A.grad_total)
        A.grad_total[(size_t)k * NPK + lane] = (flag || dead) ? 0.0 : gev - (double)ne * gsel;
      if (A.grad_events) A.grad_events[(size_t)k * NPK + lane] = dead ? 0.0 : gev;
      if (A.grad_ln_xi) A.grad_ln_xi[(size_t)k * NPK + lane] = S1 > 0.0 ? gsel : 0.0;
    }
   }
  }
}

// --------------------------------------------------------- per-sample terms (tests)
template <typename RowT, bool MP>
__global__ void __launch_bounds__(256) k_sample_terms(TermsArgs A) {
  constexpr int NS = n_params(MP);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    A.c[0] = lamd_c(*A.ld);
    for (int q = 0; q < NS; ++q) A.c[1 + q] = lamd_dc(*A.ld, q);
  }
  if (i >= A.n_total) return;
  const LamF L = A.lf[0];
  const bool inj = i >= A.n_samples;
  const float4 v = inj ? __ldg(A.inj + (i - A.n_samples)) : __ldg(A.smp + i);
  SampleIn s;
  s.m1 = v.x; s.m2 = v.y; s.dl = v.z; s.npe2 = -to_log2(v.w);
  s.lm1 = log2f(v.x); s.lm2 = log2f(v.y);
  const float* tb = A.tables;
  const int nx = A.nx;
  const float4* pos = reinterpret_cast<const float4*>(tb);
  const float4* aux = reinterpret_cast<const float4*>(tb + 4 * nx);
  const float4* wv = reinterpret_cast<const float4*>(tb + 8 * nx);
  const float4* ws = wv + (NW_WIN + 1);
  float lw = -INFINITY;
  TermSink ts;
  bool ok = false;
  if (L.live != 0.f) {
    if (inj) {
      ok = sample_lnw<true, float, TermSink, true, MP>(L, s, A.pbar32, A.nz, pos, aux, nx, wv, ws, lw, ts);
    } else {
      const int px = __ldg(A.pix + i);
      if (px >= 0 && px < A.n_pix)   // a pixel outside the table reads nothing and gets w = 0
        ok = sample_lnw<true, RowT, TermSink, true, MP>(L, s, reinterpret_cast<const RowT*>(A.los) + (size_t)px * A.nz,
                                                        A.nz, pos, aux, nx, wv, ws, lw, ts);
    }
  }
  if (A.cell) A.cell[i] = ts.cell;
  A.lnw[i] = ok ? lw * LN2F : -INFINITY;
  if (A.dlnw) {
    double st[NP_MAX], G[NP_MAX];
    for (int q = 0; q < NS; ++q) st[q] = ok ? (double)ts.g[q] : 0.0;
    stats_to_grad(st, ok ? 1.0 : 0.0, *A.ld, G);
    // at a mixture bound: sigma (1 - O/mix) (may overflow), and for the multi-peak
    // model's lambda_low the other peak's share taken off
    if (ok && ts.edge[0]) G[P_LAM] *= 1.0 - exp2((double)ts.lo[0]);
    if (ok && ts.edge[1]) G[P_LAM1] -= A.ld->lam1_sigma * exp2((double)ts.lo[1]);
    for (int q = 0; q < NS; ++q) A.dlnw[(size_t)q * A.n_total + i] = ok ? (float)G[q] : 0.f;
  }
}

cudaError_t launch_sample_terms(const TermsArgs& a, bool bf16, cudaStream_t s) {
  const int grid = (int)std::max(1LL, (a.n_total + 255) / 256);
  if (a.mp) {
    if (bf16) k_sample_terms<__nv_bfloat16, true><<<grid, 256, 0, s>>>(a);
    else k_sample_terms<float, true><<<grid, 256, 0, s>>>(a);
  } else {
    if (bf16) k_sample_terms<__nv_bfloat16, false><<<grid, 256, 0, s>>>(a);
    else k_sample_terms<float, false><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ path census (measurement)
// The value arithmetic of the fused kernel, once per (sample, Lambda), counting which
// stages each evaluation reaches (see gwc_path_census in gwc.h for the slots).
struct CensusSink {
  unsigned c[GWC_CENSUS_SLOTS] = {0};
  __device__ __forceinline__ bool any(bool p) { return p; }
  __device__ __forceinline__ bool weight(float, bool live) {
    c[7] += live;
    w = live;
    return false;
  }
  __device__ __forceinline__ void grad2(int, float, float) {}
  __device__ __forceinline__ void other(int, float, float) {}
  __device__ __forceinline__ void position(float, int, bool ok) { c[1] += ok; }
  __device__ __forceinline__ void reached(int st, bool ok) { c[st] += ok; }
  __device__ __forceinline__ void windows(bool a, bool b, bool ok) {
    if (!ok) return;
    ++c[4];
    w1 = a;
    w2 = b;
    c[5] += a;
    c[6] += b;
  }
  bool w = false, w1 = false, w2 = false;
};

template <typename RowT, bool MP>
__global__ void __launch_bounds__(256) k_census(CensusArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  CensusSink cs;
  if (i < A.n_total) {
    const bool inj = i >= A.n_samples;
    const float4 v = inj ? __ldg(A.inj + (i - A.n_samples)) : __ldg(A.smp + i);
    SampleIn s;
    s.m1 = v.x; s.m2 = v.y; s.dl = v.z; s.npe2 = -to_log2(v.w);
    s.lm1 = log2f(v.x); s.lm2 = log2f(v.y);
    const RowT* row = inj ? nullptr : reinterpret_cast<const RowT*>(A.los) + (size_t)__ldg(A.pix + i) * A.nz;
    const int nx = A.nx;
    for (int k = 0; k < A.K; ++k) {
      const LamF L = A.lf[k];
      if (L.live == 0.f) continue;
      ++cs.c[0];
      const float* tb = A.tables + (size_t)k * A.tstride;
      const float4* pos = reinterpret_cast<const float4*>(tb);
      const float4* aux = reinterpret_cast<const float4*>(tb + 4 * nx);
      const float4* wv = reinterpret_cast<const float4*>(tb + 8 * nx);
      const float4* ws = wv + (NW_WIN + 1);
      float lw;
      cs.w = false;
      if (inj)
        sample_lnw<false, float, CensusSink, true, MP>(L, s, A.pbar32, A.nz, pos, aux, nx, wv, ws, lw, cs);
      else
        sample_lnw<false, RowT, CensusSink, true, MP>(L, s, row, A.nz, pos, aux, nx, wv, ws, lw, cs);
      if (cs.w) {
        cs.c[8] += cs.w1;
        cs.c[9] += cs.w2;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GWC_CENSUS_SLOTS; ++q) {
    const unsigned t = __reduce_add_sync(0xffffffffu, cs.c[q]);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(A.counts + q, (unsigned long long)t);
  }
}

cudaError_t launch_census(const CensusArgs& a, bool bf16, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * GWC_CENSUS_SLOTS, s);
  if (e != cudaSuccess || a.n_total <= 0) return e;
  const unsigned grid = (unsigned)((a.n_total + 255) / 256);
  if (a.mp) {
    if (bf16) k_census<__nv_bfloat16, true><<<grid, 256, 0, s>>>(a);
    else k_census<float, true><<<grid, 256, 0, s>>>(a);
  } else {
    if (bf16) k_census<__nv_bfloat16, false><<<grid, 256, 0, s>>>(a);
    else k_census<float, false><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ cell index (tests)
__global__ void k_los_cell(const float* z, long long n, int nz, double zmax, int* cell) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zv = (double)z[i];
  int j = -1;
  if (zv >= 0.0 && zv <= zmax) {
    const double s = (double)(nz - 1) / zmax;
    j = (int)floor(zv * s);
    j = min(max(j, 0), nz - 2);
  }
  cell[i] = j;
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_prologue(const ProArgs& a, int K, cudaStream_t s) {
  const size_t smem = sizeof(double) * 4 * (size_t)a.nx;
  const bool cl = K <= PRO_CLUSTER_MAX_K;
  if (smem > 48 * 1024) {
    cudaError_t e = cl ? cudaFuncSetAttribute(k_prologue<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k_prologue<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (!cl) {
    k_prologue<false><<<dim3(K, ProShape<false>::CTAS), PRO_THREADS, smem, s>>>(a);
    return cudaGetLastError();
  }
  // one cluster of ProShape<true>::CTAS CTAs per Lambda point (grid y = cluster y)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(K, ProShape<true>::CTAS, 1);
  cfg.blockDim = dim3(PRO_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = ProShape<true>::CTAS;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_prologue<true>, a);
}

template <bool G, bool KH, typename RT, bool MP>
static cudaError_t launch_fused_t(const FusedArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_fused<G, KH, RT, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem_max());
  if (e != cudaSuccess) return e;
  k_fused<G, KH, RT, MP><<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool G, bool KH, typename RT, bool MP>
static cudaError_t occupancy_t(size_t smem, int* out) {
  cudaError_t e = cudaFuncSetAttribute(k_fused<G, KH, RT, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem_max());
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_fused<G, KH, RT, MP>, THREADS, smem);
}

// the instance for (gradient, compensated sums, bf16 LOS rows, multi-peak)
template <template <bool, bool, typename, bool> class F, typename... Args>
static cudaError_t fused_dispatch(bool grad, bool kahan, bool bf16, bool mp, Args... args) {
#define GWC_FUSED_CASE(G_, K_, B_, M_)                                                           \
  if (grad == G_ && kahan == K_ && bf16 == B_ && mp == M_)                                      \
    return F<G_, K_, std::conditional_t<B_, __nv_bfloat16, float>, M_>::run(args...);
  GWC_FUSED_CASE(true, false, false, false) GWC_FUSED_CASE(true, true, false, false)
  GWC_FUSED_CASE(true, false, true, false) GWC_FUSED_CASE(true, true, true, false)
  GWC_FUSED_CASE(false, false, false, false) GWC_FUSED_CASE(false, true, false, false)
  GWC_FUSED_CASE(false, false, true, false) GWC_FUSED_CASE(false, true, true, false)
  GWC_FUSED_CASE(true, false, false, true) GWC_FUSED_CASE(true, true, false, true)
  GWC_FUSED_CASE(true, false, true, true) GWC_FUSED_CASE(true, true, true, true)
  GWC_FUSED_CASE(false, false, false, true) GWC_FUSED_CASE(false, true, false, true)
  GWC_FUSED_CASE(false, false, true, true) GWC_FUSED_CASE(false, true, true, true)
#undef GWC_FUSED_CASE
  return cudaErrorInvalidValue;
}
template <bool G, bool KH, typename RT, bool MP> struct FusedLaunch {
  static cudaError_t run(const FusedArgs& a, int grid, size_t smem, cudaStream_t s) {
    return launch_fused_t<G, KH, RT, MP>(a, grid, smem, s);
  }
};
template <bool G, bool KH, typename RT, bool MP> struct FusedOccupancy {
  static cudaError_t run(size_t smem, int* out) { return occupancy_t<G, KH, RT, MP>(smem, out); }
};

size_t fused_smem_bytes(int chunk, int slab, int group, bool grad) {
  // one warp per point writes its partials directly: no combine buffer
  const size_t part = group == 1 ? 0 : (size_t)slab * group * (grad ? PSTRIDE : 4) * sizeof(float);
  return (size_t)chunk * 8 * sizeof(float) + part;
}
size_t fused_smem_max() { return fused_smem_bytes(4096, MAX_SLAB_GROUP / 2, 2, true); }   // the largest shape

cudaError_t launch_fused(const FusedArgs& a, bool grad, bool kahan, bool bf16, int grid, cudaStream_t s) {
  const size_t smem = fused_smem_bytes(a.chunk, a.slab, a.group, grad);
  return fused_dispatch<FusedLaunch>(grad, kahan, bf16, a.mp != 0, a, grid, smem, s);
}

cudaError_t fused_blocks_per_sm(const FusedArgs& a, bool grad, bool kahan, bool bf16, int* out) {
  const size_t smem = fused_smem_bytes(a.chunk, a.slab, a.group, grad);
  return fused_dispatch<FusedOccupancy>(grad, kahan, bf16, a.mp != 0, smem, out);
}

// ------------------------------------------------------------ event-shard merge
__global__ void k_merge_parts(int R, int K, int P, const double* __restrict__ parts, double* lnL_total,
                              double* ln_xi, double* neff_sel, int32_t* flags, double* grad_total) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) merge_parts_point(R, K, P, parts, k, lnL_total, ln_xi, neff_sel, flags, grad_total);
}

cudaError_t launch_merge_parts(int R, int K, int P, const double* parts, double* lnL_total, double* ln_xi,
                               double* neff_sel, int32_t* flags, double* grad_total, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  k_merge_parts<<<(K + 127) / 128, 128, 0, s>>>(R, K, P, parts, lnL_total, ln_xi, neff_sel, flags, grad_total);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ HMC leapfrog
__global__ void __launch_bounds__(32) k_hmc(HmcArgs A) {
  const int k = blockIdx.x, i = threadIdx.x;
  const bool on = i < A.np;
  const size_t o = (size_t)k * A.np + (on ? i : 0);
  if (A.mode == 0) {
    if (on) A.q0[o] = A.q[o];
    if (i == 0) A.div[k] = 0;
    return;
  }
  const bool bad = A.flags[k] != 0 || !(A.lnL[k] > -INFINITY);
  int div = A.div[k] | (bad ? 1 : 0);
  const double eps = A.eps[k];
  const double im = on ? A.inv_mass[i] : 0.0;
  double p = on ? A.p[o] : 0.0;
  const double g = on ? A.grad[o] : 0.0;
  auto kinetic = [&](double pv) {
    double t = on ? 0.5 * im * pv * pv : 0.0;
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
  };
  if (A.mode == 1) {
    if (on) A.grad0[o] = g;
    const double ke = kinetic(p);
    if (i == 0) {
      A.lnL0[k] = A.lnL[k];
      A.H[(size_t)k * 2] = div ? INFINITY : -A.lnL[k] + ke;
    }
  }
  if (A.mode == 1 || A.mode == 2) {
    if (!div && on) {
      p += (A.mode == 1 ? 0.5 : 1.0) * eps * g;
      A.p[o] = p;
      A.q[o] += eps * im * p;
    }
    if (i == 0) A.div[k] = div;
    return;
  }
  // mode 3: close the trajectory and accept or reject
  if (!div && on) {
    p += 0.5 * eps * g;
    A.p[o] = p;
  }
  const double ke = kinetic(p);
  const double H1 = div ? INFINITY : -A.lnL[k] + ke;
  const double H0 = A.H[(size_t)k * 2];
  const bool acc = !div && H0 < INFINITY && A.log_u[k] < H0 - H1;
  if (on) {
    if (!acc) A.q[o] = A.q0[o];
    A.grad_out[o] = acc ? g : A.grad0[o];
  }
  if (i == 0) {
    A.H[(size_t)k * 2 + 1] = H1;
    A.accept[k] = acc ? 1 : 0;
    A.lnL_out[k] = acc ? A.lnL[k] : A.lnL0[k];
    A.div[k] = div;
  }
}

cudaError_t launch_hmc(const HmcArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_hmc<<<a.K, 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_plain_sample(const PlainArgs& a, bool grad, bool bf16, cudaStream_t s) {
  const int grid = (int)((a.n_total + 255) / 256);
  if (grad) {
    if (bf16) k_plain_sample<true, __nv_bfloat16><<<grid, 256, 0, s>>>(a);
    else k_plain_sample<true, float><<<grid, 256, 0, s>>>(a);
  } else {
    if (bf16) k_plain_sample<false, __nv_bfloat16><<<grid, 256, 0, s>>>(a);
    else k_plain_sample<false, float><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_reduce(const PlainArgs& a, bool grad, cudaStream_t s) {
  if (grad) k_plain_reduce<true><<<a.n_items, 256, 0, s>>>(a);
  else k_plain_reduce<false><<<a.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// One CTA per Lambda point, with one thread per event or injection partial up to 256: a
// small catalogue (an HMC chain's) then reduces over one or two warps, whose FP64
// butterflies (1/64 of the FP32 rate on this GPU) would otherwise run in all eight.
cudaError_t launch_merge(const MergeArgs& a, int K, bool grad, cudaStream_t s) {
  const long long work = std::max<long long>(a.n_events, (long long)(a.n_items - a.inj_item0) * a.P);
  int threads = 32;   // a power of two (the column sums' segments halve evenly)
  while (threads < 256 && threads < work) threads *= 2;
  if (a.mp) {
    if (grad) k_merge<true, true><<<K, threads, 0, s>>>(a);
    else k_merge<false, true><<<K, threads, 0, s>>>(a);
  } else {
    if (grad) k_merge<true, false><<<K, threads, 0, s>>>(a);
    else k_merge<false, false><<<K, threads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_los_cell(const float* z, long long n, int nz, double zmax, int* cell, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_los_cell<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, n, nz, zmax, cell);
  return cudaGetLastError();
}

}  // namespace gwc
