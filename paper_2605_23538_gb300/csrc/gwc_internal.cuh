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

constexpr int NP = 13;
constexpr double C_KMS = 299792.458;
constexpr int WARPS = 8;             // warps per CTA of the sample kernels
constexpr int THREADS = WARPS * 32;
constexpr int NW_WIN = 128;          // panels of the smoothing-window tables
constexpr int PSTRIDE = 16;          // floats per partial sum: m, s1, s2, g[13]
constexpr int NGL = 8;               // Gauss-Legendre nodes per panel in the prologue

enum { P_H0, P_OM, P_ALPHA, P_BETA, P_MMIN, P_MMAX, P_DM, P_MU, P_SIG, P_LAM, P_GAM, P_KAP, P_ZP };

// FP32 constants of one Lambda point for the sample kernels (48 floats = 12 float4).
struct __align__(16) LamF {
  float H0c, xmax, inv_dx, live;       // x = dL * H0/c; table spacing; 0 = skip this Lambda
  float H0c_lo, inv_dx_lo, inv_dm, lam_edge;   // low parts of H0/c and (nx-1)/xmax; 1/delta_m;
                                               // 1 when lambda_peak is 0 or 1 (see Acc)
  float om, zstep, inv_zstep, lp;      // Om; z_max/(n_z-1); its inverse; ln(1+z_p)
  float alpha, beta, mmin, mmax;
  float dm, mw, mu, inv_sig;           // mw = m_min + delta_m
  float la, lb, Cw, mw1b;              // ln(1-lam) - ln Z_P; ln lam - ln(sig sqrt(2 pi)) - ln Z_G;
                                       // C(mw) = int_{m_min}^{mw} m^beta S; mw^(1+beta)
  float eps_b, inv_eps_b, lmw, gam;    // 1+beta; 1/(1+beta) (0 when |1+beta| < 1e-30); ln mw
  float gpk, inv_wh, invH0, inv1zp;    // gamma+kappa; N_w/delta_m; 1/H0; 1/(1+z_p)
  float dZPa, dZPmin, dZPmax, dZGmu;   // d ln Z_P / d(alpha, m_min, m_max); d ln Z_G / d mu
  float dZGsig, dZGmin, dZGmax, Cwb;   // d ln Z_G / d(sig, m_min, m_max); int m^beta ln m S
  float Jw, Kw, la0, lb0;              // int m^(beta-1) S; int m^beta dS/d delta_m; la, lb without ln(1-lam), ln lam
  float lam, inv_lam, inv_1ml, pad;    // lambda_peak, 1/lambda, 1/(1-lambda)
};
static_assert(sizeof(LamF) == 48 * 4, "LamF layout");

// FP64 constants of one Lambda point for the merge: ln w = (per-sample term) + c.
struct LamD {
  double c;
  double dc[NP];
  int32_t flag;
  int32_t pad;
};

// Per-Lambda table block (floats):
//   [0, 4 NX)          float4 pos[NX]  {hi, lo, D, c2}: P(x_n) = hi + lo; cubic in t on
//                      segment n: P = P_n + t (D + t (c2 + t c3)), t in [0, 1)
//   [4 NX, 5 NX)       float c3[NX]
//   [5 NX, 7 NX)       float2 jtab[NX] {J, dJ/dx * dx} (Hermite)
//   [7 NX, 7 NX + 8 (NW_WIN + 1))  float2 win[4][NW_WIN + 1] {Q, dQ/dm * h}: Q_C, Q_beta,
//                      Q_J, Q_K (Hermite in m over [m_min, m_min + delta_m])
__host__ __device__ inline int table_floats(int nx) { return 7 * nx + 8 * (NW_WIN + 1); }

struct Item {          // one work item: a contiguous run of samples of one event, or of injections
  int64_t begin;
  int32_t count;
  int32_t kind;        // 0: event samples, 1: injections
};

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float hermite_val(float2 a, float2 b, float t) {
  // a = {f0, f0' h}, b = {f1, f1' h}
  const float t2 = t * t, t3 = t2 * t;
  const float h00 = 2.f * t3 - 3.f * t2 + 1.f, h10 = t3 - 2.f * t2 + t;
  const float h01 = -2.f * t3 + 3.f * t2, h11 = t3 - t2;
  return h00 * a.x + h10 * a.y + h01 * b.x + h11 * b.y;
}
// derivative with respect to t (multiply by 1/h for d/dm)
__device__ __forceinline__ float hermite_dt(float2 a, float2 b, float t) {
  const float t2 = t * t;
  const float d00 = 6.f * t2 - 6.f * t, d10 = 3.f * t2 - 4.f * t + 1.f;
  const float d01 = -6.f * t2 + 6.f * t, d11 = 3.f * t2 - 2.f * t;
  return d00 * a.x + d10 * a.y + d01 * b.x + d11 * b.y;
}

struct SampleIn {
  float m1, m2, dl, lpe, lm1, lm2;   // detector-frame masses, distance, ln pi, ln m1, ln m2
};

// Smoothing window: for m' = m - m_min in (0, delta_m), f = dm/m' + dm/(m' - dm),
// ln S = -softplus(f).  Returns ln S and (GRAD) sf = sigmoid(f) = 1 - S, mp.
__device__ __forceinline__ float ln_smooth(float m, float mmin, float dm, float& sf, float& mp) {
  mp = m - mmin;
  const float f = dm / mp + dm / (mp - dm);
  const float e = expf(-fabsf(f));
  const float inv = __frcp_rn(1.f + e);
  sf = f >= 0.f ? inv : e * inv;
  return -(fmaxf(f, 0.f) + log1pf(e));
}

__device__ __forceinline__ float ld_row(const float* __restrict__ r, int j) { return __ldg(r + j); }
__device__ __forceinline__ float ld_row(const __nv_bfloat16* __restrict__ r, int j) {
  return __bfloat162float(r[j]);
}

// ln w (without the per-Lambda constant c) and, for GRAD, d ln w / d Lambda.
// row: the sample's LOS row (or the pixel-averaged row for injections).
// pos/pc3/jtab/win: this Lambda's tables (global memory, read through L1).
// When L.lam_edge is set (lambda_peak = 0 or 1) the lambda derivative
// e^(ln G - mix) - e^(ln P - mix) can exceed the float range for samples far from one
// mixture component, although its product with the sample's weight does not; g[P_LAM]
// then holds ln P - mix and lam_lb holds ln G - mix, and the accumulator forms the
// weighted difference in the exponent (lam_edge_term).
// Returns false where w = 0.
template <bool GRAD, typename RowT>
__device__ __forceinline__ bool sample_lnw(const LamF& L, const SampleIn& s,
                                           const RowT* __restrict__ row, int nz,
                                           const float4* __restrict__ pos,
                                           const float* __restrict__ pc3, int nx,
                                           const float2* __restrict__ jtab,
                                           const float2* __restrict__ win, float& lw, float* g,
                                           float& lam_lb) {
  // x = d_L H0 / c and the table coordinate x / dx carried with their rounding errors
  // (exact products by FMA), so the LOS-grid position keeps ~1e-7 of a cell
  const float x = s.dl * L.H0c;
  if (!(x > 0.f) || x > L.xmax) return false;
  if (s.m2 > s.m1) return false;
  const float x_lo = fmaf(s.dl, L.H0c, -x) + s.dl * L.H0c_lo;
  const float sx = x * L.inv_dx;
  const float sx_lo = fmaf(x, L.inv_dx, -sx) + fmaf(x, L.inv_dx_lo, x_lo * L.inv_dx);

  // --- d_L -> z: position on the LOS grid from the Hermite table (split precision)
  const int n = min((int)sx, nx - 2);
  const float t = (sx - (float)n) + sx_lo;
  const float4 nd = __ldg(pos + n);
  const float frac = nd.y + t * (nd.z + t * (nd.w + t * __ldg(pc3 + n)));
  int j = (int)floorf(nd.x + frac);
  float tl = (nd.x - (float)j) + frac;
  if (j > nz - 2) { tl += (float)(j - (nz - 2)); j = nz - 2; }
  if (j < 0) { tl += (float)j; j = 0; }
  const float z = ((float)j + tl) * L.zstep;
  const float u = 1.f + z;
  const float ru = __frcp_rn(u);
  const float lu = logf(u);

  // --- LOS prior of the sample's pixel, linear in z
  const float p0 = ld_row(row, j), p1 = ld_row(row, j + 1);
  const float dp = p1 - p0;
  const float plos = fmaf(tl, p1, (1.f - tl) * p0);   // convex form: no cancellation in tails
  if (!(plos > 0.f)) return false;

  // --- source-frame masses
  const float m1s = s.m1 * ru, m2s = s.m2 * ru;
  if (m1s > L.mmax || m2s < L.mmin) return false;
  const float lm1s = s.lm1 - lu, lm2s = s.lm2 - lu;

  // p(m1): log of (1-lam) m^-alpha/Z_P + lam N(m; mu, sig)/Z_G
  const float a = L.la - L.alpha * lm1s;
  const float zz = (m1s - L.mu) * L.inv_sig;
  const float b = fmaf(-0.5f * zz, zz, L.lb);
  const float mx = fmaxf(a, b), mn = fminf(a, b);
  const float eab = expf(mn - mx);

  // p(m2 | m1) = m2^beta S(m2) / C(m1)
  float lnS2 = 0.f, sf2 = 0.f, mp2 = 0.f;
  const bool win2 = m2s < L.mw;
  if (win2) {
    lnS2 = ln_smooth(m2s, L.mmin, L.dm, sf2, mp2);
    if (!(mp2 > 0.f)) return false;
  }
  const bool win1 = m1s < L.mw;
  float Cx, Cprod, lmass;   // the normaliser (C, or R_C in the window), its share of the
                            // one-log product below, and the remaining log-mass terms
  float y = 0.f, Q = 0.f, A = 0.f, dlm = 0.f;
  float2 wa = make_float2(0.f, 0.f), wb = wa;
  float wt = 0.f;
  int wk = 0;
  float mp1 = 0.f, Qc = 0.f;
  if (win1) {
    // in the window C(m1) = m1^beta S(m1) R_C(m1) with R_C = Q_C m'^2 / delta_m;
    // S(m1) cancels against p(m1)
    mp1 = m1s - L.mmin;
    const float ws = mp1 * L.inv_wh;
    wk = min((int)ws, NW_WIN - 1);
    wt = ws - (float)wk;
    wa = __ldg(win + wk);
    wb = __ldg(win + wk + 1);
    Qc = hermite_val(wa, wb, wt);
    Cx = Qc * (mp1 * mp1) * L.inv_dm;   // R_C >= ~1e-14 (m' >= one float ulp of m_min)
    Cprod = 1.f;                         // R_C can be small near m_min: keep its log separate
    lmass = L.beta * (lm2s - lm1s) - logf(Cx);
  } else {
    // above it C(m1) = C(mw) + mw^(1+beta) (exp((1+beta)(ln m1 - ln mw)) - 1) / (1+beta)
    dlm = lm1s - L.lmw;
    y = L.eps_b * dlm;
    Q = fabsf(y) < 1e-3f ? dlm * fmaf(y, fmaf(y, 1.f / 6.f, 0.5f), 1.f) : expm1f(y) * L.inv_eps_b;
    Cx = fmaf(L.mw1b, Q, L.Cw);
    Cprod = Cx;
    lmass = L.beta * lm2s;
  }

  // rate psi(z) / (1+z) and the (1+z)^-2 mass Jacobian: (gam - 3) ln u - softplus(r)
  const float r = L.gpk * (lu - L.lp);
  const float er = expf(-fabsf(r));

  // d d_L / dz = (c/H0) D'(z), D' = I(z) + u/E with I(z) = x/u on the root
  const float u3m1 = z * fmaf(z, z + 3.f, 3.f);   // (1+z)^3 - 1 without cancellation
  const float E2 = fmaf(L.om, u3m1, 1.f);
  const float rE = rsqrtf(E2);
  const float Dp = fmaf(x, ru, u * rE);

  // one logarithm for the product of the remaining factors
  const float prod = plos * (1.f + eab) / (Dp * Cprod * (1.f + er));
  lw = (L.gam - 3.f) * lu - fmaxf(r, 0.f) + mx + lnS2 + lmass + logf(prod) - s.lpe;
  if (!(lw > -INFINITY) || lw != lw) return false;

  if (GRAD) {
    const float inv1e = __frcp_rn(1.f + eab);
    const float pa = a >= b ? inv1e : eab * inv1e;   // mixture responsibilities
    const float pb = 1.f - pa;
    const float invr = __frcp_rn(1.f + er);
    const float sr = r >= 0.f ? invr : er * invr;   // sigmoid(r)
    const float invDp = __frcp_rn(Dp);
    const float rE3 = rE * rE * rE;

    // smoothing derivatives of m2 (and of m1 in the window)
    float dS2_dm = 0.f, dS2_dmin = 0.f, dS2_ddm = 0.f;
    if (win2) {
      const float i1 = __frcp_rn(mp2), i2 = __frcp_rn(mp2 - L.dm);
      const float q = L.dm * (i1 * i1 + i2 * i2);
      dS2_dm = sf2 * q;
      dS2_dmin = -sf2 * q;
      dS2_ddm = -sf2 * (i1 + mp2 * i2 * i2);
    }
    float dS1_dmin = 0.f, dS1_ddm = 0.f;
    float dlnC_db, dlnC_dmin, dlnC_ddm, Gc;
    if (win1) {
      float sf1, mp1;
      ln_smooth(m1s, L.mmin, L.dm, sf1, mp1);
      const float i1 = __frcp_rn(mp1), i2 = __frcp_rn(mp1 - L.dm);
      dS1_dmin = -sf1 * L.dm * (i1 * i1 + i2 * i2);
      dS1_ddm = -sf1 * (i1 + mp1 * i2 * i2);
      const float Qb = hermite_val(__ldg(win + (NW_WIN + 1) + wk), __ldg(win + (NW_WIN + 1) + wk + 1), wt);
      const float Qj = hermite_val(__ldg(win + 2 * (NW_WIN + 1) + wk), __ldg(win + 2 * (NW_WIN + 1) + wk + 1), wt);
      const float Qk = hermite_val(__ldg(win + 3 * (NW_WIN + 1) + wk), __ldg(win + 3 * (NW_WIN + 1) + wk + 1), wt);
      const float iQ = __frcp_rn(Qc), im = __frcp_rn(mp1);
      dlnC_db = Qb;                                     // R_beta / R_C
      dlnC_dmin = fmaf(L.beta, Qj, -__frcp_rn(Cx));     // (-1 + beta R_J) / R_C
      dlnC_ddm = Qk * iQ * im;                          // R_K / R_C
      // -ln R_C(m1s) through m1s = m1/u:  m1s (Q_C'/Q_C + 2/m') / u
      Gc = m1s * fmaf(hermite_dt(wa, wb, wt) * L.inv_wh, iQ, 2.f * im);
    } else {
      const float iC = __frcp_rn(Cx);
      A = L.mw1b * (Q * L.eps_b + 1.f);   // m1s^(1+beta)
      float phi2;
      if (fabsf(y) < 1e-2f) phi2 = fmaf(y, fmaf(y, 0.125f, 1.f / 3.f), 0.5f);
      else phi2 = (y * expf(y) - expm1f(y)) / (y * y);
      dlnC_db = (L.Cwb + L.mw1b * fmaf(L.lmw, Q, dlm * dlm * phi2)) * iC;
      dlnC_dmin = (L.beta * L.Jw - L.mw1b / L.mw) * iC;
      dlnC_ddm = L.Kw * iC;
      Gc = (A * iC - L.beta);   // -ln C(m1s) and beta ln m2s through u (times 1/u below)
    }
    // total z-derivative of ln w at fixed detector-frame data
    float Gz = dp * L.inv_zstep / plos;
    Gz += (L.gam - L.gpk * sr - 3.f) * ru;
    Gz += fmaf(pa, L.alpha, pb * zz * m1s * L.inv_sig) * ru;
    Gz -= m2s * dS2_dm * ru;
    Gz += Gc * ru;
    const float D2 = 2.f * rE - 1.5f * L.om * (u3m1 + 1.f) * rE3;
    Gz -= D2 * invDp;

    // z depends on H0 and Om through x and the inverted distance relation
    const float J = hermite_val(__ldg(jtab + n), __ldg(jtab + n + 1), t);
    g[P_H0] = Gz * x * L.invH0 * invDp;
    const float dz_dom = -u * J * invDp;
    const float dDp_dom = J - 0.5f * u * u3m1 * rE3;
    g[P_OM] = fmaf(Gz, dz_dom, -dDp_dom * invDp);
    g[P_ALPHA] = pa * (-lm1s - L.dZPa);
    g[P_BETA] = lm2s - dlnC_db;
    g[P_MMIN] = -pa * L.dZPmin - pb * L.dZGmin + dS1_dmin + dS2_dmin - dlnC_dmin;
    g[P_MMAX] = -pa * L.dZPmax - pb * L.dZGmax;
    g[P_DM] = dS1_ddm + dS2_ddm - dlnC_ddm;
    g[P_MU] = pb * (zz * L.inv_sig - L.dZGmu);
    g[P_SIG] = pb * (fmaf(zz, zz, -1.f) * L.inv_sig - L.dZGsig);
    if (L.lam_edge == 0.f) {
      g[P_LAM] = pb * L.inv_lam - pa * L.inv_1ml;
    } else {
      const float mix = mx + log1pf(eab);
      g[P_LAM] = L.la0 - L.alpha * lm1s - mix;         // ln P - mix
      lam_lb = fmaf(-0.5f * zz, zz, L.lb0) - mix;      // ln G - mix
    }
    const float dl = lu - L.lp;
    g[P_GAM] = lu - sr * dl;
    g[P_KAP] = -sr * dl;
    g[P_ZP] = sr * L.gpk * L.inv1zp;
  }
  return true;
}

// e^d (e^lb - e^la) without forming either exponential on its own
__device__ __forceinline__ float lam_edge_term(float d, float la, float lb) {
  return expf(d + lb) - expf(d + la);
}

// Online (max, sum e^(l-max), sum e^(2(l-max)), sum e^(l-max) dl) accumulator.
template <bool GRAD, bool KAHAN>
struct Acc {
  float m = -INFINITY, s1 = 0.f, s2 = 0.f, c1 = 0.f, c2 = 0.f;
  float g[GRAD ? NP : 1];
  __device__ __forceinline__ Acc() {
#pragma unroll
    for (int i = 0; i < (GRAD ? NP : 1); ++i) g[i] = 0.f;
  }
  __device__ __forceinline__ void add(float lw, const float* dg, bool lam_edge = false,
                                      float lam_lb = 0.f) {
    if (lw > m) {
      const float sc = expf(m - lw);   // 0 on the first sample
      s1 = fmaf(s1, sc, 1.f);
      s2 = fmaf(s2, sc * sc, 1.f);
      c1 *= sc;
      c2 *= sc * sc;
      if (GRAD) {
        const float dl = lam_edge ? lam_edge_term(0.f, dg[P_LAM], lam_lb) : dg[P_LAM];
#pragma unroll
        for (int i = 0; i < NP; ++i) g[i] = fmaf(g[i], sc, i == P_LAM ? dl : dg[i]);
      }
      m = lw;
    } else {
      const float tt = expf(lw - m);
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
      if (GRAD) {
        const float cl = lam_edge ? lam_edge_term(lw - m, dg[P_LAM], lam_lb) : tt * dg[P_LAM];
#pragma unroll
        for (int i = 0; i < NP; ++i) g[i] = i == P_LAM ? g[i] + cl : fmaf(tt, dg[i], g[i]);
      }
    }
  }
  // merge another lane's sums (fixed shuffle tree keeps the result deterministic)
  __device__ __forceinline__ void merge(float om, float os1, float os2, const float* og) {
    const float M = fmaxf(m, om);
    if (M == -INFINITY) return;
    const float sa = expf(m - M), sb = expf(om - M);
    s1 = s1 * sa + os1 * sb;
    s2 = s2 * sa * sa + os2 * sb * sb;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < NP; ++i) g[i] = g[i] * sa + og[i] * sb;
    }
    m = M;
  }
};

}  // namespace gwc
