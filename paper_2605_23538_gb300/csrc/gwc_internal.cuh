// gwc_internal.cuh -- layouts shared by the library's kernels and the per-sample arithmetic.
//
// Each Lambda point gets, from the prologue kernel, a block of FP32 constants (LamF),
// a block of FP64 constants for the merge (LamD) and a few tables:
//   * the LOS-grid position P(x) = z(x) (n_z - 1) / z_max of the inverted distance
//     relation on a uniform x = d_L H0 / c grid, as cubic Hermite segments stored in a
//     split (hi + lo) form so the cell index and the in-cell fraction keep ~1e-7 of a cell;
//   * J(x) = d I / d Om at z(x) (gradient only), I(z) = int_0^z dz'/E;
//   * four smoothing-window tables over m in [m_min, m_min + delta_m] (the value path
//     uses the first).  With m' = m - m_min, g = m^beta S(m) and R_X = X(m) / g for the
//     integrals C = int m^beta S, C_beta = int m^beta ln m S, J = int m^(beta-1) S and
//     K = int m^beta dS/d delta_m from m_min, the tables hold the smooth, positive-definite
//     ratios Q_C = R_C delta_m / m'^2 (-> 1 at m_min), Q_beta = R_beta / R_C (-> ln m_min),
//     Q_J = R_J / R_C (-> 1/m_min) and Q_K = R_K delta_m / m' (-> -1), which a cubic Hermite
//     interpolates to FP32 precision right down to m_min.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gwc {

constexpr int NP = 13;               // hyperparameters of the power law + peak mass model
constexpr int NP_MP = 16;            // of the multi-peak model
constexpr int NP_MAX = 16;
__host__ __device__ constexpr int n_params(bool mp) { return mp ? NP_MP : NP; }
constexpr double C_KMS = 299792.458;
constexpr int WARPS = 8;             // warps per CTA of the sample kernels
constexpr int THREADS = WARPS * 32;
constexpr int NW_WIN = 128;          // panels of the smoothing-window tables
constexpr int PSTRIDE = 23;          // floats per partial sum: m, s1, s2, g[16], mO, sO, mO2, sO2
constexpr int PART_MO = 3 + NP_MAX, PART_SO = 4 + NP_MAX;     // where mO, sO sit
constexpr int PART_MO2 = 5 + NP_MAX, PART_SO2 = 6 + NP_MAX;   // the second pair (multi-peak)
constexpr int NGL = 8;               // Gauss-Legendre nodes per panel of the smoothing window (near
                                     // m_min its integrand m^beta S(m) changes by many e-folds a panel)
constexpr int NGL_Z = 4;             // and per panel of the z quadrature (1/E is smooth, the panels
                                     // narrow: 4 nodes are exact there to far below FP64 rounding)

// The multi-peak model appends the higher-mass Gaussian and the lower one's share of
// the Gaussian fraction; (mu_g, sigma_g, lambda_peak) are then the low peak's
// (mu_low, sigma_low) and lambda_g.
enum { P_H0, P_OM, P_ALPHA, P_BETA, P_MMIN, P_MMAX, P_DM, P_MU, P_SIG, P_LAM, P_GAM, P_KAP, P_ZP,
       P_MU2, P_SIG2, P_LAM1 };

// The sample kernels do not sum the 13 derivatives of ln w (16 for the multi-peak model)
// themselves but as many weighted statistics that they are linear in; the FP64 merge applies the Lambda-only coefficients
// (stats_to_grad).  For one sample of weight t (pa, pb: mixture responsibilities,
// zz = (m1s - mu)/sig, sr = sigmoid of the rate's turnover, lu2 = log2(1+z)):
//   S_H0   t Gz x / D'            (d/dH0 = S_H0 / H0)
//   S_OM   t d ln w / d Om
//   S_A1   t pa                   S_LX  t pb  (at lambda_peak = 0, 1: t times the
//                                             lambda-derivative before the other-component term)
//   S_AL   t pa log2 m1s          S_BE  t d ln w / d beta
//   S_MMIN t (smoothing and C(m1) parts of d/dm_min)   S_DM  t d ln w / d delta_m
//   S_MU   t pb zz                S_SIG t pb zz^2
//   S_LU   t lu2                  S_SRD t sr (lu2 - log2(1+z_p))      S_SR  t sr
// and for the multi-peak model (pb then being the low peak's responsibility, pb2 the
// high peak's, zz2 = (m1s - mu2)/sig2):
//   S_MU2  t pb2 zz2              S_SIG2 t pb2 zz2^2                  S_LX2 t pb2
enum { S_H0, S_OM, S_A1, S_LX, S_AL, S_BE, S_MMIN, S_DM, S_MU, S_SIG, S_LU, S_SRD, S_SR,
       S_MU2, S_SIG2, S_LX2 };

// FP32 constants of one Lambda point for the sample kernels (68 floats = 17 float4).
// Fields ending in 2 are in log2 units (the value path works in log2 so that the
// special-function unit's ex2/lg2 apply directly).
struct __align__(16) LamF {
  float H0c, H0c_lo, sxa, sxa_lo;        // H0/c as a hi + lo pair; H0/(c dx) (the table
                                         // coordinate per Mpc) as a hi + lo pair
  float xmax, live, zstep, inv_zstep;     // live = 0: skip this Lambda; z_max/(n_z-1) and inverse
  float om, lp2, gam, gam_m3;             // log2(1+z_p); gamma; gamma - 3
  float gpk, alpha, beta, eps_b;          // gamma+kappa; 1+beta
  float mmin, mmax, dm, mw;               // mw = m_min + delta_m
  float mu, inv_sig, la2, lb2;            // log2 of (1-lam)/Z_P and of lam/(sig sqrt(2 pi) Z_G),
                                          // less the anchor R carried in FP64 by c
  float C0, inv_eps_b, Cw, mw1b;          // C above the window = C0 + m1^(1+beta)/(1+beta);
                                          // C(mw) = int_{m_min}^{mw} m^beta S; mw^(1+beta)
  float lmw, inv_wh, inv_dm, beta_small;  // ln mw; N_w/delta_m; 1/delta_m; 1 if |1+beta| < 1e-3
  float invH0, inv1zp, lam_edge, lam;     // lam_edge = 1 when lambda_peak is 0 or 1
  float dZPa, dZPmin, dZPmax, dZGmu;      // d ln Z_P / d(alpha, m_min, m_max); d ln Z_G / d mu
  float dZGsig, dZGmin, dZGmax, Cwb;      // d ln Z_G / d(sig, m_min, m_max); int m^beta ln m S
  float Cmin, Kw, la0_2, lb0_2;           // dC/dm_min above the window; int m^beta dS/d delta_m;
                                          // log2 of 1/Z_P and of 1/(sig sqrt(2 pi) Z_G)
  float inv_lam, inv_1ml, dm_l2, zstep_lo;   // dm log2(e) formed in FP64; z_max/(n_z-1) - zstep
  float alpha_lo, beta_lo, eps_b_lo, gpk_lo;   // alpha, beta, 1+beta, gamma+kappa less their
                                               // float values (they multiply logs of up to ~8)
  float mu2, inv_sig2, lc2, lam_sig;      // multi-peak: the high peak, log2 of its weight
                                          // lam (1-lam1)/(sig2 sqrt(2 pi) Z_G2) less R;
                                          // lam_sig = +1 / -1 at lambda_peak = 1 / 0, else 0
  float lam1_edge, o2_hi, o2_l2, lb1_2;   // multi-peak, lam1 at 0 or 1 with lam > 0: the
                                          // other peak's log2 weight o2_l2 = log2(lam /
                                          // (sig sqrt(2 pi) Z_G)) less R of the high (o2_hi
                                          // = 1, lam1 = 1) or the low peak; at lam = 0 the
                                          // peaks' log2 weights without lam: lb1_2, lc1_2
  float lc1_2, pad1, pad2, pad3;
};
static_assert(sizeof(LamF) == 68 * 4, "LamF layout");

// FP64 constants of one Lambda point for the merge: ln w = (per-sample term) + c.
// lam_sigma = +1 at lambda_peak = 1, -1 at lambda_peak = 0, else 0 (see Acc); for the
// multi-peak model lam1_sigma the same for lambda_low (0 when lambda_peak = 0).
struct LamD {
  double c;
  double dc[NP_MAX];
  int32_t flag;
  int32_t lam_sigma;
  // coefficients of stats_to_grad
  double invH0, dZPa, dZPmin, dZPmax, dZGmin, dZGmax, dZGmu, dZGsig;
  double inv_sig, inv_lam, inv_1ml, gpk_inv1zp;
  // multi-peak (mp = 1): the high peak's d ln Z_G2 / d(m_min, m_max, mu2, sig2), 1/sig2,
  // 1/lam1, 1/(1 - lam1) (a reciprocal is 0 where its weight is 0)
  int32_t mp, lam1_sigma;
  double dZG2min, dZG2max, dZG2mu, dZG2sig, inv_sig2, inv_lam1, inv_1ml1;
  // -ln N'_z and its gamma, kappa, z_p derivatives, written by a prologue CTA of their own
  double cz, dcz[3];
};

// the per-Lambda constant of ln w and its gradient: the parts in c, dc and in cz, dcz
__host__ __device__ inline double lamd_c(const LamD& D) { return D.c + D.cz; }
__host__ __device__ inline double lamd_dc(const LamD& D, int i) {
  return D.dc[i] + (i == P_GAM ? D.dcz[0] : i == P_KAP ? D.dcz[1] : i == P_ZP ? D.dcz[2] : 0.0);
}

// The derivative sums G (before division by the weight sum S1; 13, or 16 for the
// multi-peak model) from the statistics.
template <typename T>
__host__ __device__ inline void stats_to_grad(const T* st, T S1, const LamD& D, T* G) {
  const T LN2 = (T)0.69314718055994530942;
  if (D.mp) {
    const T A1 = st[S_A1], B1 = st[S_LX], B2 = st[S_LX2];
    G[P_H0] = (T)D.invH0 * st[S_H0];
    G[P_OM] = st[S_OM];
    G[P_ALPHA] = -LN2 * st[S_AL] - (T)D.dZPa * A1;
    G[P_BETA] = st[S_BE];
    G[P_MMIN] = st[S_MMIN] - (T)D.dZPmin * A1 - (T)D.dZGmin * B1 - (T)D.dZG2min * B2;
    G[P_MMAX] = -(T)D.dZPmax * A1 - (T)D.dZGmax * B1 - (T)D.dZG2max * B2;
    G[P_DM] = st[S_DM];
    G[P_MU] = (T)D.inv_sig * st[S_MU] - (T)D.dZGmu * B1;
    G[P_SIG] = (T)D.inv_sig * (st[S_SIG] - B1) - (T)D.dZGsig * B1;
    G[P_MU2] = (T)D.inv_sig2 * st[S_MU2] - (T)D.dZG2mu * B2;
    G[P_SIG2] = (T)D.inv_sig2 * (st[S_SIG2] - B2) - (T)D.dZG2sig * B2;
    // d ln mix / d lam = (pb + pb2)/lam - pa/(1-lam); d / d lam1 = pb/lam1 - pb2/(1-lam1).
    // At a bound the term whose weight is 0 has 0 responsibility and a 0 reciprocal, and
    // what remains is the one-sided derivative less the other component's share, which
    // the caller subtracts (sigma times the other-component sum, see Acc): at lam = 1,
    // S1 - sum t P/mix; at lam = 0, sum t (lam1 G + (1-lam1) G2)/P - S1; at lam1 = 1,
    // sum t pb - sum t lam G2/mix; at lam1 = 0, sum t lam G/mix - sum t pb2
    G[P_LAM] = (T)D.inv_lam * (B1 + B2) - (T)D.inv_1ml * A1;
    G[P_LAM1] = (T)D.inv_lam1 * B1 - (T)D.inv_1ml1 * B2;
    G[P_GAM] = LN2 * (st[S_LU] - st[S_SRD]);
    G[P_KAP] = -LN2 * st[S_SRD];
    G[P_ZP] = (T)D.gpk_inv1zp * st[S_SR];
    return;
  }
  T A1 = st[S_A1], B1 = st[S_LX];
  if (D.lam_sigma != 0) {          // one component only: pa, pb are 0 or 1
    A1 = D.lam_sigma < 0 ? S1 : (T)0;
    B1 = D.lam_sigma > 0 ? S1 : (T)0;
    G[P_LAM] = st[S_LX];
  } else {
    G[P_LAM] = (T)D.inv_lam * B1 - (T)D.inv_1ml * A1;
  }
  G[P_H0] = (T)D.invH0 * st[S_H0];
  G[P_OM] = st[S_OM];
  G[P_ALPHA] = -LN2 * st[S_AL] - (T)D.dZPa * A1;
  G[P_BETA] = st[S_BE];
  G[P_MMIN] = st[S_MMIN] - (T)D.dZPmin * A1 - (T)D.dZGmin * B1;
  G[P_MMAX] = -(T)D.dZPmax * A1 - (T)D.dZGmax * B1;
  G[P_DM] = st[S_DM];
  G[P_MU] = (T)D.inv_sig * st[S_MU] - (T)D.dZGmu * B1;
  G[P_SIG] = (T)D.inv_sig * (st[S_SIG] - B1) - (T)D.dZGsig * B1;
  G[P_GAM] = LN2 * (st[S_LU] - st[S_SRD]);
  G[P_KAP] = -LN2 * st[S_SRD];
  G[P_ZP] = (T)D.gpk_inv1zp * st[S_SR];
}

// Per-Lambda table block (floats):
//   [0, 4 NX)          float4 pos[NX]  {hi, lo, D, c2}: P(x_n) = hi + lo; cubic in t on
//                      segment n: P = P_n + t (D + t (c2 + t c3)), t in [0, 1)
//   [4 NX, 8 NX)       float4 aux[NX]  {c3, J_n, d - c, c}: J = J_n + t (d - c) + t^2 c on
//                      segment n, d = J_{n+1} - J_n, c half the difference of the nodes'
//                      slopes dJ/dx dx
//   [8 NX, 8 NX + 4 (NW_WIN + 1))   float4 wval[NW_WIN + 1] {Q_C, Q_beta, Q_J, Q_K}
//   [.., + 4 (NW_WIN + 1))           float4 wslp[NW_WIN + 1] the same times dQ/dm * h
//                      (Hermite in m over [m_min, m_min + delta_m])
__host__ __device__ constexpr int table_floats(int nx) { return 8 * nx + 8 * (NW_WIN + 1); }

struct Item {          // one work item: a contiguous run of samples of one event, or of injections
  int64_t begin;
  int32_t count;
  int32_t kind;        // 0: event samples, 1: injections
};

// ---------------------------------------------------------------- device helpers
constexpr float LN2F = 0.69314718055994530942f;
constexpr float LOG2EF = 1.44269504088896340736f;
constexpr float HALF_LOG2EF = 0.72134752044448170368f;
// log2(e) as an unevaluated sum of two floats: x * log2(e) to about half an ulp, where the
// single float constant (relative error -1.3e-8) would shift every ln pi of magnitude ~20
// by the same ~3e-7, an error that grows with the number of events in the total
constexpr float LOG2E_LO = 1.9259629911e-08f;
__device__ __forceinline__ float to_log2(float x) { return fmaf(x, LOG2EF, x * LOG2E_LO); }

// the special-function unit's approximations (PTX ex2/lg2/rcp .approx): relative errors
// of a few 2^-23, which keeps every term of ln w at FP32 rounding level
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// lg2: the special-function unit's approximation, for log2(1+z).  lg2_acc: the accurate
// log2f, for the logarithm of the product of all ratio terms.  With the approximation in
// both places the weighted mean error of ln w over 1e6 injections was +2e-7 to +5e-7, a
// bias every sample shares and that reaches the total multiplied by the number of
// events; with log2f for the product, ln xi at 5e7 injections is within 5e-8 of the FP64
// value and the total at 10,000 events within 7.1e-4 (log2f in both places: 7.4e-4, and
// about 2% slower).  ex2.approx and rcp.approx showed no comparable bias.
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_acc(float x) { return log2f(x); }
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// derivative with respect to t (multiply by 1/h for d/dm)
__device__ __forceinline__ float hermite_dt(float2 a, float2 b, float t) {
  const float d = b.x - a.x;
  const float c2 = fmaf(3.f, d, -fmaf(2.f, a.y, b.y));
  const float c3 = fmaf(-2.f, d, a.y + b.y);
  return fmaf(t, fmaf(3.f * t, c3, 2.f * c2), a.y);
}

// cubic Hermite basis at t: f = h00 f0 + h10 f0'h + h01 f1 + h11 f1'h
struct HermiteBasis {
  float h00, h10, h01, h11;
  __device__ __forceinline__ explicit HermiteBasis(float t) {
    const float t2 = t * t, tm = t - 1.f;
    h01 = t2 * fmaf(-2.f, t, 3.f);
    h00 = 1.f - h01;
    h10 = t * tm * tm;
    h11 = t2 * tm;
  }
  __device__ __forceinline__ float operator()(float f0, float d0, float f1, float d1) const {
    return fmaf(h00, f0, fmaf(h10, d0, fmaf(h01, f1, h11 * d1)));
  }
};

struct SampleIn {
  float m1, m2, dl, npe2, lm1, lm2;  // detector-frame masses, distance, -log2 pi (the PE
                                     // prior or draw density), log2 m1, log2 m2
  bool valid = true;                 // false: a lane past the end of its run (its fields
                                     // hold another sample of the run; it adds nothing)
};

__device__ __forceinline__ float ld_row(const float* __restrict__ r, int j) { return __ldg(r + j); }
__device__ __forceinline__ float ld_row(const __nv_bfloat16* __restrict__ r, int j) {
  return __bfloat162float(r[j]);
}

// floor(v) for |v| < 2^22 without a float-to-int conversion (those share the
// special-function unit's quarter-rate pipe): v + 1.5*2^23 lies in [2^23, 2^24), where
// the floats are exactly the integers, so the exact sum rounded down is floor(v) +
// 1.5*2^23.  floor_biased returns that sum; biased_int its integer, biased_float its value
// (both exact).  Outside |v| < 2^22 (and for NaN) the integer is meaningless but finite;
// every caller clamps it to a table.
constexpr float FLOOR_BIAS = 12582912.f;          // 1.5 * 2^23
constexpr unsigned FLOOR_BIAS_BITS = 0x4B400000u;
__device__ __forceinline__ float floor_biased(float v) { return __fadd_rd(v, FLOOR_BIAS); }
__device__ __forceinline__ int biased_int(float f) { return (int)((unsigned)__float_as_int(f) - FLOOR_BIAS_BITS); }
__device__ __forceinline__ float biased_float(float f) { return f - FLOOR_BIAS; }

// lw2 = log2 of w without the per-Lambda constant c (ln w = lw2 ln 2 + c) and, for GRAD,
// g = d ln w / d Lambda (natural units, without dc).
//   ln w = ln p_LOS(z) + (gamma - 3) ln u - softplus(r) + ln p_mix(m1) + beta ln m2 + ln S(m2)
//          - ln C(m1) - ln D'(z) - ln pi,   u = 1 + z, r = (gamma + kappa) ln(u / (1 + z_p))
// with every log1p term folded into one logarithm of a product.  row: the sample's LOS
// row (or the pixel-averaged row for injections); pos/aux/wval/wslp: this Lambda's tables.
// When L.lam_edge is set (lambda_peak = 1 or 0) the mixture is one component and the
// lambda derivative is sigma (1 - O/mix), where O is the other component's density
// (P at lambda = 1, G at lambda = 0) and sigma = +1 / -1.  O/mix can exceed the float
// range for samples far from the present component, so statistic S_LX holds sigma and
// lam_lb holds log2(O/mix); the accumulator keeps sum w O/mix as its own (max, sum) pair
// and the FP64 merge subtracts it.  Returns false where w = 0.
//
// Control flow.  The sample's cuts (d_L outside the distance table, m2 > m1, source
// masses outside [m_min, m_max], a zero LOS prior, m2 on the lower mass edge, w = 0) clear
// a per-lane flag `live` instead of returning, and the function returns early only where
// sink.any(live) is false: for the warp-wide sinks that is a vote over the warp (one
// uniform branch, no divergent exits), for per-thread sinks the thread's own flag.  A lane
// that is not live keeps computing on its own, possibly meaningless, values; every table
// index is clamped, the smoothing-window branches are taken only by live lanes, its weight
// is zero and the sink adds none of its derivatives.
//
// The gradient is not returned per sample: `sink` receives the sample's weight t
// relative to the running reference (after any rescaling) through sink.weight(lw2, live)
// and then each derivative through sink.grad(i, value), so the 13 terms are folded into
// their accumulators as soon as they exist (fewer live registers).  Samples whose lw2
// falls more than 48 below the reference skip the derivative work: their weight is below
// 2^-48 of the sum's largest.
constexpr float GRAD_SKIP = 48.f;
// how far above an accumulator's reference a sample may lie before the reference is raised
constexpr float RESCALE_HEADROOM = 32.f;

// WITH_LOS = false leaves out the LOS factor (the weight w' of the KDE form, whose LOS
// prior enters through the grid integral instead).  Every sample whose d_L maps into
// [0, z_max] reports its z and the LOS cell j it interpolates in through
// sink.position(z, j, ok), whatever its weight; sink.reached(2, ok) and sink.reached(3, ok)
// mark the mass-order and mass-support cuts passed, and sink.windows(win1, win2, ok) the
// whole value about to be formed, with the smoothing-window branches taken (a path census
// uses them).  MP selects the multi-peak mass model (a second Gaussian in the
// primary-mass mixture).  RARE = false leaves out the code of two rare kinds of Lambda
// point: a mixture weight on a bound (the other-component sums and sigma in S_LX) and
// |1 + beta| < 1e-3 (the series form of C(m1)); a caller may pass it only for points with
// L.lam_edge = 0, L.lam1_edge = 0 (multi-peak model) and L.beta_small = 0.
template <bool GRAD, typename RowT, typename Sink, bool WITH_LOS = true, bool MP = false, bool RARE = true>
__device__ __forceinline__ bool sample_lnw(const LamF& L, const SampleIn& s,
                                           const RowT* __restrict__ row, int nz,
                                           const float4* __restrict__ pos,
                                           const float4* __restrict__ aux, int nx,
                                           const float4* __restrict__ wval,
                                           const float4* __restrict__ wslp, float& lw2,
                                           Sink& sink) {
  // x = d_L H0 / c, and the table coordinate d_L H0 / (c dx) carried with its rounding
  // error (an exact product by FMA and the constant's own low part), so the LOS-grid
  // position keeps ~1e-7 of a cell
  const float x = s.dl * L.H0c;
  bool live = s.valid && x > 0.f && !(x > L.xmax);
  if (!sink.any(live)) return false;
  const float sx = s.dl * L.sxa;
  const float sx_lo = fmaf(s.dl, L.sxa, -sx) + s.dl * L.sxa_lo;

  // --- d_L -> z: position on the LOS grid from the Hermite table (split precision)
  const int n = min(max(biased_int(floor_biased(sx)), 0), nx - 2);   // floor(sx), in the table
  const float t = (sx - (float)n) + sx_lo;
  const float4 nd = __ldg(pos + n);
  const float4 ax = __ldg(aux + n);
  const float frac = nd.y + t * (nd.z + t * (nd.w + t * ax.x));
  const float fj = floor_biased(nd.x + frac);
  int j = biased_int(fj);
  float tl = (nd.x - biased_float(fj)) + frac;
  // The rounded sum hi + lo can land on the other side of a node when the position lies
  // within half an ulp of it (1.2e-4 cells near the end of a 2048-node grid); the
  // in-cell fraction tl is accurate to ~1e-7, so the cell follows its sign.
  const int dj = tl < 0.f ? -1 : (tl >= 1.f ? 1 : 0);
  j += dj;
  tl -= (float)dj;
  {  // the last cell extends to the end of the grid, the first to its start
    const int jc = min(max(j, 0), nz - 2);
    tl += (float)(j - jc);
    j = jc;
  }
  const float jt = (float)j + tl;
  const float z = fmaf(jt, L.zstep, jt * L.zstep_lo);   // the step in two floats
  sink.position(z, j, live);
  live = live && !(s.m2 > s.m1);
  sink.reached(2, live);
  const float u = 1.f + z;
  const float ru = rcp(u);

  // --- source-frame masses (the support cuts first: warps with no sample inside skip the rest)
  const float m1s = s.m1 * ru, m2s = s.m2 * ru;
  live = live && !(m1s > L.mmax || m2s < L.mmin);
  sink.reached(3, live);
  if (!sink.any(live)) return false;
  const float lu2 = lg2(u);
  const float lm1s2 = s.lm1 - lu2, lm2s2 = s.lm2 - lu2;

  // --- LOS prior of the sample's pixel, linear in z (convex form: no cancellation)
  float p0 = 1.f, p1 = 1.f, plos = 1.f;
  if (WITH_LOS) {
    p0 = ld_row(row, j);
    p1 = ld_row(row, j + 1);
    plos = fmaf(tl, p1, (1.f - tl) * p0);
    live = live && plos > 0.f;
  }

  // p(m1): (1-lam) m^-alpha / Z_P + lam N(m; mu, sig) / Z_G as max + log2(1 + e^-|a-b|);
  // multi-peak: the three components' log2 weights a2, b2, c2 as max + log2 of the sum of
  // their powers relative to it (mixf in [1, 3])
  const float a2 = fmaf(-L.alpha, lm1s2, fmaf(-L.alpha_lo, lm1s2, L.la2));
  const float zz = (m1s - L.mu) * L.inv_sig;
  const float b2 = fmaf(-HALF_LOG2EF * zz, zz, L.lb2);
  float mx, eab = 0.f, mixf, zz2 = 0.f, ea = 0.f, eb = 0.f, ec = 0.f;
  if (!MP) {
    mx = fmaxf(a2, b2);
    eab = ex2(fminf(a2, b2) - mx);
    mixf = 1.f + eab;
  } else {
    zz2 = (m1s - L.mu2) * L.inv_sig2;
    const float c2 = fmaf(-HALF_LOG2EF * zz2, zz2, L.lc2);
    mx = fmaxf(fmaxf(a2, b2), c2);
    ea = ex2(a2 - mx);
    eb = ex2(b2 - mx);
    ec = ex2(c2 - mx);
    mixf = ea + eb + ec;
  }
  float lin = mx;     // log2 terms outside the product
  float den;          // denominators of the product

  // smoothing of m2: ln S = -softplus(f), f = dm/m' + dm/(m' - dm)
  const bool win2 = live && m2s < L.mw;
  float mp2 = 0.f, i1 = 0.f, i2 = 0.f, f2 = 0.f, ef2 = 0.f;
  if (win2) {
    mp2 = m2s - L.mmin;
    live = mp2 > 0.f;              // S(m_min) = 0
    i1 = rcp(mp2);
    i2 = rcp(mp2 - L.dm);
    f2 = L.dm_l2 * (i1 + i2);
    ef2 = ex2(-fabsf(f2));
    lin -= fmaxf(f2, 0.f);
  }

  // normaliser of p(m2 | m1): in the window C(m1) = m1^beta S(m1) Q_C m'^2 / dm, whose
  // S(m1) cancels against p(m1); above it C = C0 + m1^(1+beta) / (1+beta)
  const bool win1 = live && m1s < L.mw;
  float Cx, mp1 = 0.f, Qc = 0.f, A = 0.f, dlm = 0.f, wt = 0.f;
  int wk = 0;
  if (win1) {
    mp1 = m1s - L.mmin;
    const float ws = mp1 * L.inv_wh;
    const float fw = floor_biased(ws);
    wk = min(biased_int(fw), NW_WIN - 1);
    wt = ws - (float)wk;
    const HermiteBasis hb(wt);
    const float4 v0 = __ldg(wval + wk), v1 = __ldg(wval + wk + 1);
    const float4 d0 = __ldg(wslp + wk), d1 = __ldg(wslp + wk + 1);
    Qc = hb(v0.x, d0.x, v1.x, d1.x);
    Cx = Qc * (mp1 * mp1) * L.inv_dm;
    const float dl21 = lm2s2 - lm1s2;
    lin = fmaf(L.beta, dl21, fmaf(L.beta_lo, dl21, lin));
  } else {
    if (!(RARE && L.beta_small != 0.f)) {
      A = ex2(fmaf(L.eps_b, lm1s2, L.eps_b_lo * lm1s2));   // m1s^(1+beta)
      Cx = fmaf(A, L.inv_eps_b, L.C0);
    } else {                                          // |1+beta| < 1e-3: series in y
      dlm = fmaf(lm1s2, LN2F, -L.lmw);
      const float y = L.eps_b * dlm;
      const float phi1 = fmaf(y, fmaf(y, fmaf(y, 1.f / 24.f, 1.f / 6.f), 0.5f), 1.f);
      A = L.mw1b * fmaf(y, phi1, 1.f);
      Cx = fmaf(L.mw1b * dlm, phi1, L.Cw);
    }
    lin = fmaf(L.beta, lm2s2, fmaf(L.beta_lo, lm2s2, lin));
  }
  den = win2 ? Cx * (1.f + ef2) : Cx;

  // rate psi(z)/(1+z) and the (1+z)^-2 mass Jacobian: (gam - 3) log2 u - softplus(r)/ln 2
  const float dlp = lu2 - L.lp2;
  const float r2 = fmaf(L.gpk, dlp, L.gpk_lo * dlp);
  const float er = ex2(-fabsf(r2));
  lin -= fmaxf(r2, 0.f);

  // d d_L / dz = (c/H0) D'(z), D' = I(z) + u/E with I(z) = x/u on the root
  const float u3m1 = z * fmaf(z, z + 3.f, 3.f);        // (1+z)^3 - 1 without cancellation
  const float rE = rsqrtf(fmaf(L.om, u3m1, 1.f));
  const float Dp = fmaf(x, ru, u * rE);
  den *= Dp * (1.f + er);

  sink.windows(win1, win2, live);
  lw2 = fmaf(L.gam_m3, lu2, lin) + lg2_acc(plos * mixf * rcp(den));
  lw2 += s.npe2;
  live = live && lw2 > -INFINITY;
  const bool has_grad = sink.weight(lw2, live);
  // at a mixture bound every live sample adds to the other-component sum, whatever its
  // weight (its weight under the absent component can be large)
  const bool edge = RARE && (L.lam_edge != 0.f || (MP && L.lam1_edge != 0.f));

  if (GRAD && sink.any(has_grad || (edge && live))) {
    // other-component sums at the mixture's bounds (the same branch for every lane of a
    // Lambda point): log2 of O/mix for the component whose weight is 0
    if (RARE && L.lam_edge != 0.f) {
      float lo;
      if (!MP) {
        lo = L.lam >= 1.f ? fmaf(-L.alpha, lm1s2, L.la0_2) - b2             // mix = G: P/G
                          : fmaf(-HALF_LOG2EF * zz, zz, L.lb0_2) - a2;      // mix = P: G/P
      } else if (L.lam >= 1.f) {                                            // P/mix
        lo = fmaf(-L.alpha, lm1s2, L.la0_2) - (mx + lg2(mixf));
      } else {                                          // mix = P: (lam1 G + (1-lam1) G2)/P
        const float q1 = fmaf(-HALF_LOG2EF * zz, zz, L.lb1_2);
        const float q2 = fmaf(-HALF_LOG2EF * zz2, zz2, L.lc1_2);
        const float qm = fmaxf(q1, q2);
        lo = qm + lg2(ex2(q1 - qm) + ex2(q2 - qm)) - (mx + lg2(mixf));
      }
      sink.other(0, lw2, lo);
    }
    if (RARE && MP && L.lam1_edge != 0.f) {             // lam G2/mix (lam1 = 1) or lam G/mix
      const float zo = L.o2_hi != 0.f ? zz2 : zz;
      sink.other(1, lw2, fmaf(-HALF_LOG2EF * zo, zo, L.o2_l2) - (mx + lg2(mixf)));
    }
    const float lm1s = lm1s2 * LN2F, lm2s = lm2s2 * LN2F;
    float pa, pb, pb2 = 0.f;                           // mixture responsibilities
    if (!MP) {
      const float inv1e = rcp(mixf);
      pa = a2 >= b2 ? inv1e : eab * inv1e;
      pb = 1.f - pa;
    } else {
      const float inv = rcp(mixf);
      pa = ea * inv;
      pb = eb * inv;
      pb2 = ec * inv;
    }
    const float invr = rcp(1.f + er);
    const float sr = r2 >= 0.f ? invr : er * invr;     // sigmoid(r)
    const float invDp = rcp(Dp);
    const float rE3 = rE * rE * rE;

    // smoothing derivatives of m2 (and of m1 in the window)
    float dS2_dm = 0.f, dS2_ddm = 0.f;
    if (win2) {
      const float inv = rcp(1.f + ef2);
      const float sf2 = f2 >= 0.f ? inv : ef2 * inv;
      dS2_dm = sf2 * L.dm * fmaf(i1, i1, i2 * i2);      // d ln S / dm = -d ln S / d m_min
      dS2_ddm = -sf2 * fmaf(mp2 * i2, i2, i1);
    }
    float dS1_dmin = 0.f, dS1_ddm = 0.f, dlnC_db, dlnC_dmin, dlnC_ddm, Gc;
    if (win1) {
      const float j1 = rcp(mp1), j2 = rcp(mp1 - L.dm);
      const float f1 = L.dm_l2 * (j1 + j2);
      const float ef1 = ex2(-fabsf(f1));
      const float inv = rcp(1.f + ef1);
      const float sf1 = f1 >= 0.f ? inv : ef1 * inv;
      dS1_dmin = -sf1 * L.dm * fmaf(j1, j1, j2 * j2);
      dS1_ddm = -sf1 * fmaf(mp1 * j2, j2, j1);
      // the four window tables share one Hermite basis (reloads hit L1)
      const HermiteBasis hb(wt);
      const float4 v0 = __ldg(wval + wk), v1 = __ldg(wval + wk + 1);
      const float4 d0 = __ldg(wslp + wk), d1 = __ldg(wslp + wk + 1);
      const float Qb = hb(v0.y, d0.y, v1.y, d1.y);
      const float Qj = hb(v0.z, d0.z, v1.z, d1.z);
      const float Qk = hb(v0.w, d0.w, v1.w, d1.w);
      const float2 qa = make_float2(v0.x, d0.x), qb = make_float2(v1.x, d1.x);
      const float iQ = rcp(Qc);
      dlnC_db = Qb;                                      // R_beta / R_C
      dlnC_dmin = fmaf(L.beta, Qj, -rcp(Cx));            // (-1 + beta R_J) / R_C
      dlnC_ddm = Qk * iQ * j1;                           // R_K / R_C
      // -ln R_C(m1s) through m1s = m1/u:  m1s (Q_C'/Q_C + 2/m') / u
      Gc = m1s * fmaf(hermite_dt(qa, qb, wt) * L.inv_wh, iQ, 2.f * j1);
    } else {
      const float iC = rcp(Cx);
      float dC_db;
      if (!(RARE && L.beta_small != 0.f)) {
        // dC/dbeta = C_beta(mw) + (A ln m1s - mw^(1+beta) ln mw - (C - C(mw))) / (1+beta)
        dC_db = fmaf(fmaf(A, lm1s, -fmaf(L.mw1b, L.lmw, Cx - L.Cw)), L.inv_eps_b, L.Cwb);
      } else {
        const float y = L.eps_b * dlm;
        const float phi1 = fmaf(y, fmaf(y, fmaf(y, 1.f / 24.f, 1.f / 6.f), 0.5f), 1.f);
        const float phi1p = fmaf(y, fmaf(y, 0.125f, 1.f / 3.f), 0.5f);
        dC_db = fmaf(L.mw1b * dlm, fmaf(L.lmw, phi1, dlm * phi1p), L.Cwb);
      }
      dlnC_db = dC_db * iC;
      dlnC_dmin = L.Cmin * iC;
      dlnC_ddm = L.Kw * iC;
      Gc = fmaf(A, iC, -L.beta);   // -ln C(m1s) and beta ln m2s through u (times 1/u below)
    }
    // total z-derivative of ln w at fixed detector-frame data
    float Gz = (p1 - p0) * L.inv_zstep * rcp(plos);
    const float gpeak = MP ? fmaf(pb * zz, L.inv_sig, pb2 * zz2 * L.inv_sig2) * m1s : pb * zz * m1s * L.inv_sig;
    const float inner = L.gam - 3.f - L.gpk * sr + fmaf(pa, L.alpha, gpeak) - m2s * dS2_dm + Gc;
    Gz = fmaf(inner, ru, Gz);
    const float D2 = fmaf(-1.5f * L.om * (u3m1 + 1.f), rE3, 2.f * rE);
    Gz = fmaf(-D2, invDp, Gz);

    // z depends on H0 and Om through x and the inverted distance relation; J = dI/dOm at
    // z(x), a quadratic on the table segment.  The statistics go to the sink in pairs
    // (packed FP32 pairs in the accumulator).
    const float J = fmaf(t, fmaf(t, ax.w, ax.z), ax.y);
    sink.grad2(S_H0, Gz * x * invDp, fmaf(Gz, -u * J * invDp, -fmaf(-0.5f * u * u3m1, rE3, J) * invDp));
    // S_LX: pb, or sigma at lambda_peak = 1 / 0 for the single-peak model (the merge takes
    // the lambda derivative from it and the other-component sum)
    sink.grad2(S_A1, pa, (RARE && !MP && L.lam_edge != 0.f) ? L.lam_sig : pb);
    sink.grad2(S_AL, pa * lm1s2, lm2s - dlnC_db);
    sink.grad2(S_MMIN, dS1_dmin - dS2_dm - dlnC_dmin, dS1_ddm + dS2_ddm - dlnC_ddm);
    const float pbz = pb * zz;
    sink.grad2(S_MU, pbz, pbz * zz);
    sink.grad2(S_LU, lu2, sr * dlp);
    const float pbz2 = pb2 * zz2;                      // 0 for the single-peak model
    sink.grad2(S_SR, sr, pbz2);                        // S_SR, S_MU2
    if (MP) sink.grad2(S_SIG2, pbz2 * zz2, pb2);       // S_SIG2, S_LX2

  }
  return live;
}

// Sink that folds a sample into the online (reference, sums) accumulator of its lane;
// any() votes over the warp, so every lane of the warp must call sample_lnw together
template <bool GRAD, bool KAHAN, int NS = NP> struct Acc;
template <bool GRAD, bool KAHAN, int NS = NP>
struct AccSink {
  Acc<GRAD, KAHAN, NS>& a;
  float t = 0.f;
  bool hg = false;    // this lane's derivatives are summed
  bool lv = false;    // this lane's sample has a weight
  __device__ __forceinline__ explicit AccSink(Acc<GRAD, KAHAN, NS>& acc) : a(acc) {}
  __device__ __forceinline__ bool any(bool p) { return __any_sync(0xffffffffu, p); }
  __device__ __forceinline__ bool weight(float lw, bool live) {
    // the rescale is rare: one warp-uniform branch, each lane's own part selected inside
    const bool up = live && lw > a.m + RESCALE_HEADROOM;
    if (__any_sync(0xffffffffu, up)) a.rescale(lw, up);
    t = a.add(lw, live);
    lv = live;
    hg = GRAD && live && !(lw < a.m - GRAD_SKIP);
    return hg;
  }
  // statistics i and i + 1 (i even) as one packed FP32 pair
  __device__ __forceinline__ void grad2(int i, float v0, float v1) {
    if (hg) a.g2[i >> 1] = __ffma2_rn(make_float2(t, t), make_float2(v0, v1), a.g2[i >> 1]);
  }
  __device__ __forceinline__ void position(float, int, bool) {}
  __device__ __forceinline__ void reached(int, bool) {}
  __device__ __forceinline__ void windows(bool, bool, bool) {}
  __device__ __forceinline__ void other(int q, float lw, float lo) {
    if (lv) a.add_other(q, lw + lo);
  }
};

// Sink that keeps one sample's value and derivatives (per-sample outputs; one thread each)
struct TermSink {
  float g[NP_MAX];
  float lo[2] = {0.f, 0.f};     // log2 of O/mix at the mixture's bounds (see sample_lnw)
  bool edge[2] = {false, false};
  int cell = -1;      // the LOS cell the sample interpolates in (-1: d_L outside [0, z_max])
  __device__ __forceinline__ bool any(bool p) { return p; }
  __device__ __forceinline__ bool weight(float, bool live) { return live; }
  __device__ __forceinline__ void grad2(int i, float v0, float v1) {
    g[i] = v0;
    g[i + 1] = v1;
  }
  __device__ __forceinline__ void position(float, int j, bool ok) { cell = ok ? j : -1; }
  __device__ __forceinline__ void reached(int, bool) {}
  __device__ __forceinline__ void windows(bool, bool, bool) {}
  __device__ __forceinline__ void other(int q, float, float l) {
    lo[q] = l;
    edge[q] = true;
  }
};

// Online accumulator of one lane, l in log2 units: a reference m and the sums
// s1 = sum 2^(l-m), s2 = sum 2^(2(l-m)), g = sum 2^(l-m) dl (as packed pairs g2), plus
// (mO, sO) = (max, sum 2^(l + lo - mO)) of the other-component weights at a mixture bound
// (one pair, two for the multi-peak model's lambda_peak and lambda_low; zero otherwise).
// NS statistics (13, or 16 multi-peak).  The reference is the value of some summed sample
// and is raised (rescaling the sums) only when a sample exceeds it by more than
// RESCALE_HEADROOM, so every term is at most 2^32 and s2 at most 2^64 a term (float holds
// 2^127); s1 >= 1 once a sample is in.  Partials and merges only use m as a common
// reference, never as the maximum.
template <bool GRAD, bool KAHAN, int NS>
struct Acc {
  static constexpr int NG2 = GRAD ? (NS + 1) / 2 : 1;   // packed statistic pairs
  static constexpr int NO = NS > NP ? 2 : 1;            // other-component pairs
  float m = -INFINITY, s1 = 0.f, s2 = 0.f, c1 = 0.f, c2 = 0.f;
  float mO[NO], sO[NO];
  float2 g2[NG2];
  __device__ __forceinline__ Acc() {
#pragma unroll
    for (int i = 0; i < NG2; ++i) g2[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NO; ++q) { mO[q] = -INFINITY; sO[q] = 0.f; }
  }
  __device__ __forceinline__ float g(int i) const { return (i & 1) ? g2[i >> 1].y : g2[i >> 1].x; }
  // raise the reference to lw where up is set (the sums rescaled; 0 on the first sample)
  __device__ __forceinline__ void rescale(float lw, bool up) {
    const float sc = up ? ex2(m - lw) : 1.f;
    s1 *= sc;
    s2 *= sc * sc;
    c1 *= sc;
    c2 *= sc * sc;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < NG2; ++i) g2[i] = __fmul2_rn(g2[i], make_float2(sc, sc));
    }
    m = up ? lw : m;
  }
  // add a sample of log2 weight lw (when live) to the value sums, once the reference
  // admits it (lw <= m + RESCALE_HEADROOM); returns its weight 2^(lw - m), 0 when not live
  __device__ __forceinline__ float add(float lw, bool live) {
    const float tt = live ? ex2(lw - m) : 0.f;
    if (KAHAN) {
      float y1 = tt - c1, t1 = s1 + y1;
      c1 = (t1 - s1) - y1;
      s1 = t1;
      float y2 = tt * tt - c2, t2 = s2 + y2;
      c2 = (t2 - s2) - y2;
      s2 = t2;
    } else {
      s1 += tt;
      s2 = fmaf(tt, tt, s2);
    }
    return tt;
  }
  // the other component's weight 2^l at a mixture bound, into pair q
  __device__ __forceinline__ void add_other(int q, float l) {
    if (l > mO[q]) {
      sO[q] = fmaf(sO[q], ex2(mO[q] - l), 1.f);
      mO[q] = l;
    } else {
      sO[q] += ex2(l - mO[q]);
    }
  }
  // merge another lane's sums (fixed shuffle tree keeps the result deterministic)
  __device__ __forceinline__ void merge(float om, float os1, float os2, const float2* og2,
                                        const float* omO, const float* osO) {
    const float M = fmaxf(m, om);
    if (M > -INFINITY) {
      const float sa = ex2(m - M), sb = ex2(om - M);
      s1 = s1 * sa + os1 * sb;
      s2 = s2 * sa * sa + os2 * sb * sb;
      if (GRAD) {
#pragma unroll
        for (int i = 0; i < NG2; ++i)
          g2[i] = __ffma2_rn(g2[i], make_float2(sa, sa), __fmul2_rn(og2[i], make_float2(sb, sb)));
      }
      m = M;
    }
    if (GRAD) {
#pragma unroll
      for (int q = 0; q < NO; ++q) {
        const float MO = fmaxf(mO[q], omO[q]);
        if (MO > -INFINITY) {
          sO[q] = sO[q] * ex2(mO[q] - MO) + osO[q] * ex2(omO[q] - MO);
          mO[q] = MO;
        }
      }
    }
  }
};

}  // namespace gwc
