// gwc_oracle.cpp -- FP64 CPU oracle for the dark-siren hierarchical log-likelihood.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, independent restatement of
// the method against which the CUDA library is checked.  Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark load it.  The library never
// calls it, and the two share no code, header, table or constant generator.
//
// What it computes, and the passage each step follows (Papadopoulos et al.,
// "Scalable Dark Siren Cosmology with gwcosmo"):
//   * Eq. 1: luminosity distance d_L(z) = (1+z) * int_0^z c dz'/H(z'),
//     H(z) = H0 sqrt(Om (1+z)^3 + OL), read as flat LCDM (OL = 1 - Om, no radiation).
//   * Eqs. 2-4: hierarchical likelihood; the selection function alpha(Lambda)
//     (called xi here) enters as xi^-Ndet; a scale-free rate prior removes p(Ndet|Lambda).
//   * Eq. hier_pixels (Sec. 2.1): each posterior sample carries its sky pixel; the
//     pixel's line-of-sight (LOS) redshift prior multiplies the population model;
//     detection does not depend on sky position, so the selection term uses the
//     pixel-averaged LOS prior.
//   * Eqs. 5-6: per-sample weights w = p_pop(z, theta'|Lambda) / pi_PE.  The Gaussian
//     kernel of Eq. 5 is taken in its zero-width limit, so each event term is the
//     Monte-Carlo mean of w over the event's samples.
//   * Eq. 7: effective sample size (sum w)^2 / sum w^2, applied per event.
//   * The KDE form of Eqs. 5-7 (per-pixel Gaussian KDE on a redshift grid, per-pixel
//     N_eff cut, bandwidth rules of the appendix) is evaluated by orc_loglik_kde.
// The mass models (power law + Gaussian peak, and the multi-peak model of the paper's
// simulated catalogue, App. A, Table 2, both with low-mass smoothing) and the
// Madau-Dickinson rate are named but not written out in the paper; the standard
// population-literature definitions are used (see the functions below).  A Lambda row of
// 13 entries selects the first mass model, one of 16 the second.
//
// Numerics are deliberately direct: every integral is an adaptive Gauss-Kronrod
// quadrature of its own definition, z(d_L) is a safeguarded Newton root of
// D(z) = x, and sums over samples are explicit logsumexp's in FP64.  Gradients are
// exact forward-mode derivatives of the same code (13-component dual numbers), with
// the root's derivative taken by one Newton step from the converged root (implicit
// function theorem).
//
// Parity status: every function here is pinned by tests of closed forms, invariants,
// unit normalisations and brute force (tests/test_oracle_*.py); none is "unpinned".

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NP = 13;                       // hyperparameters, power law + peak
constexpr int NP_MP = 16;                    // hyperparameters, multi-peak
constexpr int NP_MAX = 16;
constexpr double C_KMS = 299792.458;         // speed of light [km/s]
constexpr double NEG_INF = -std::numeric_limits<double>::infinity();
constexpr double LN_SQRT_2PI = 0.91893853320467274178032973640562;

// Lambda layout: [H0, Om, alpha, beta, m_min, m_max, delta_m, mu_g, sigma_g,
//                 lambda_peak, gamma, kappa, z_p]
// and for the multi-peak mass model three more, the second (higher-mass) Gaussian and
// the share of the Gaussian fraction in the first (lower-mass) one:
//                 [..., mu_high, sigma_high, lambda_low]
// (mu_g, sigma_g, lambda_peak are then mu_low, sigma_low and lambda_g of Table 2).
enum { P_H0, P_OM, P_ALPHA, P_BETA, P_MMIN, P_MMAX, P_DM, P_MU, P_SIG, P_LAM, P_GAM, P_KAP, P_ZP,
       P_MU2, P_SIG2, P_LAM1 };
enum { MODEL_PLP = 0, MODEL_MP = 1 };
inline int n_params(int model) { return model == MODEL_MP ? NP_MP : NP; }
inline int model_of(int n_par) { return n_par == NP ? MODEL_PLP : n_par == NP_MP ? MODEL_MP : -1; }

// ---------------------------------------------------------------- dual numbers
// value and N first derivatives (N = 13 or 16: one per hyperparameter of the model)
template <int N> struct DualT {
  double v;
  double d[N];
  DualT() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  DualT(double c) : v(c) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT: implicit on purpose
};
using Dual = DualT<NP>;
using DualM = DualT<NP_MP>;

inline double val(double x) { return x; }
template <int N> double val(const DualT<N>& x) { return x.v; }

template <int N> DualT<N> operator+(const DualT<N>& a, const DualT<N>& b) {
  DualT<N> r; r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> DualT<N> operator-(const DualT<N>& a, const DualT<N>& b) {
  DualT<N> r; r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> DualT<N> operator-(const DualT<N>& a) {
  DualT<N> r; r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> DualT<N> operator*(const DualT<N>& a, const DualT<N>& b) {
  DualT<N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> DualT<N> operator/(const DualT<N>& a, const DualT<N>& b) {
  DualT<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> DualT<N> operator+(const DualT<N>& a, double b) { DualT<N> r = a; r.v += b; return r; }
template <int N> DualT<N> operator+(double a, const DualT<N>& b) { DualT<N> r = b; r.v += a; return r; }
template <int N> DualT<N> operator-(const DualT<N>& a, double b) { DualT<N> r = a; r.v -= b; return r; }
template <int N> DualT<N> operator-(double a, const DualT<N>& b) { DualT<N> r = -b; r.v += a; return r; }
template <int N> DualT<N> operator*(const DualT<N>& a, double b) {
  DualT<N> r; r.v = a.v * b;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> DualT<N> operator*(double a, const DualT<N>& b) { return b * a; }
template <int N> DualT<N> operator/(const DualT<N>& a, double b) { return a * (1.0 / b); }
template <int N> DualT<N> operator/(double a, const DualT<N>& b) { return DualT<N>(a) / b; }

// f(a) with f(a.v) = fv and f'(a.v) = dfv
template <int N> DualT<N> chain(const DualT<N>& a, double fv, double dfv) {
  DualT<N> r; r.v = fv;
  for (int i = 0; i < N; ++i) r.d[i] = dfv * a.d[i];
  return r;
}

inline double fexp(double x) { return std::exp(x); }
inline double flog(double x) { return std::log(x); }
inline double flog1p(double x) { return std::log1p(x); }
inline double fsqrt(double x) { return std::sqrt(x); }
inline double ferf(double x) { return std::erf(x); }
template <int N> DualT<N> fexp(const DualT<N>& a) { const double e = std::exp(a.v); return chain(a, e, e); }
template <int N> DualT<N> flog(const DualT<N>& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
template <int N> DualT<N> flog1p(const DualT<N>& a) { return chain(a, std::log1p(a.v), 1.0 / (1.0 + a.v)); }
template <int N> DualT<N> fsqrt(const DualT<N>& a) {
  const double s = std::sqrt(a.v);
  return chain(a, s, 0.5 / s);
}
template <int N> DualT<N> ferf(const DualT<N>& a) {
  return chain(a, std::erf(a.v), 1.12837916709551257389615890312154 * std::exp(-a.v * a.v));
}
// ln(1 + e^a), stable for either sign of a
template <class T> T softplus(const T& a) {
  if (val(a) > 0.0) return a + flog1p(fexp(-a));
  return flog1p(fexp(a));
}

// component access used by the quadrature's convergence test
inline int ncomp(double) { return 1; }
template <int N> int ncomp(const DualT<N>&) { return N + 1; }
inline double comp(double x, int) { return x; }
template <int N> double comp(const DualT<N>& x, int i) { return i == 0 ? x.v : x.d[i - 1]; }
inline double cabs_comp(double x, int) { return std::fabs(x); }
template <int N> double cabs_comp(const DualT<N>& x, int i) { return std::fabs(comp(x, i)); }

// the variable for hyperparameter i: its value, with unit derivative in slot i
inline void seed(double& v, double x, int) { v = x; }
template <int N> void seed(DualT<N>& v, double x, int i) {
  v = DualT<N>(x);
  if (i < N) v.d[i] = 1.0;
}

// ------------------------------------------------------ adaptive Gauss-Kronrod
// Kronrod's 15-point extension of the 7-point Gauss-Legendre rule on [-1, 1]
// (abscissae in decreasing order; the Gauss nodes are the odd-indexed ones and 0).
const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
const double WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

constexpr int NC_MAX = NP_MAX + 1;

template <class T, class F>
void gk15(const F& f, const T& a, const T& b, T& K, T& G, double* kabs) {
  const T c = (a + b) * 0.5;
  const T h = (b - a) * 0.5;
  const T fc = f(c);
  K = fc * WGK[7];
  G = fc * WG[3];
  const int nc = ncomp(K);
  for (int i = 0; i < nc; ++i) kabs[i] = WGK[7] * cabs_comp(fc, i);
  for (int j = 0; j < 7; ++j) {
    const T dx = h * XGK[j];
    const T f1 = f(c - dx);
    const T f2 = f(c + dx);
    K = K + (f1 + f2) * WGK[j];
    if (j % 2 == 1) G = G + (f1 + f2) * WG[j / 2];
    for (int i = 0; i < nc; ++i) kabs[i] += WGK[j] * (cabs_comp(f1, i) + cabs_comp(f2, i));
  }
  K = K * h;
  G = G * h;
  const double hv = std::fabs(val(h));
  for (int i = 0; i < nc; ++i) kabs[i] *= hv;
}

// Convergence of one component: |K - G| within the relative tolerance, within its share
// of the absolute tolerance, or at the noise level of the local integral of |f| below
// which splitting cannot improve the estimate (50 ulp for values; 1e-13 for derivative
// components, whose integrands carry chain-rule rounding).  Every call also has a
// budget of splits, so the recursion always ends.
template <class T, class F>
T adapt_rec(const F& f, const T& a, const T& b, double rtol, const double* atol_density, int depth,
            int& budget) {
  T K, G;
  double kabs[NC_MAX];
  gk15(f, a, b, K, G, kabs);
  const double w = std::fabs(val(b) - val(a));
  bool ok = true;
  for (int i = 0; i < ncomp(K) && ok; ++i) {
    const double err = std::fabs(comp(K, i) - comp(G, i));
    const double floor_ = (i == 0 ? 50.0 * DBL_EPSILON : 1e-13) * kabs[i];
    const double rt = i == 0 ? rtol : std::max(rtol, 1e-11);
    ok = err <= rt * std::fabs(comp(K, i)) + atol_density[i] * w + floor_;
  }
  if (ok || depth >= 30 || budget <= 0) return K;
  --budget;
  const T m = (a + b) * 0.5;
  return adapt_rec(f, a, m, rtol, atol_density, depth + 1, budget) +
         adapt_rec(f, m, b, rtol, atol_density, depth + 1, budget);
}

// int_a^b f, to relative tolerance rtol of the integral of |f| (per component).
template <class T, class F>
T integrate(const F& f, const T& a, const T& b, double rtol) {
  if (!(val(b) > val(a))) return (b - a) * f(a);  // zero-width: keeps the Leibniz term
  T K, G;
  double kabs[NC_MAX], atol_density[NC_MAX];
  gk15(f, a, b, K, G, kabs);
  const double w = val(b) - val(a);
  for (int i = 0; i < ncomp(K); ++i) atol_density[i] = 1e-2 * rtol * kabs[i] / w;
  int budget = 20000;
  return adapt_rec(f, a, b, rtol, atol_density, 0, budget);
}

// ------------------------------------------------------------------ cosmology
// E(z) = H(z)/H0 for flat LCDM (Eq. 1 with OL = 1 - Om), written as
// E^2 = 1 + Om ((1+z)^3 - 1) = 1 + Om z (3 + 3z + z^2), which avoids the cancellation
// in (1+z)^3 - 1 at small z (it matters for d/dOm)
template <class T> T E_of(const T& z, const T& om) {
  return fsqrt(1.0 + om * (z * (3.0 + z * (3.0 + z))));
}
// I(z) = int_0^z dz'/E(z'); D(z) = (1+z) I(z) = d_L H0 / c
template <class T> T I_of(const T& z, const T& om) {
  auto f = [&om](const T& zp) { return 1.0 / E_of(zp, om); };
  return integrate(f, T(0.0), z, 1e-14);
}
template <class T> T D_of(const T& z, const T& om) { return (1.0 + z) * I_of(z, om); }
template <class T> T Dprime_of(const T& z, const T& om) {
  return I_of(z, om) + (1.0 + z) / E_of(z, om);
}

// root of D(z) = x on [0, zmax] by Newton's method kept inside a bisection bracket.
// For 0 <= Om <= 1 and z >= 0, E >= 1, so D(z) <= z (1+z): the Om = 0 inverse is a
// lower bound and a safe start.
double z_root(double x, double om, double zmax) {
  double lo = 0.0, hi = zmax;
  double z = 0.5 * (std::sqrt(1.0 + 4.0 * x) - 1.0);
  z = std::min(std::max(z, lo), hi);
  for (int it = 0; it < 200; ++it) {
    const double I = I_of(z, om);
    const double F = (1.0 + z) * I - x;
    if (F > 0.0) hi = z; else lo = z;
    const double Dp = I + (1.0 + z) / E_of(z, om);
    double zn = z - F / Dp;
    if (!(zn >= lo && zn <= hi)) zn = 0.5 * (lo + hi);
    const bool done = std::fabs(zn - z) <= 1e-15 * (1.0 + z);
    z = zn;
    if (done) break;
  }
  return z;
}

// z(x; Om) with derivatives: one Newton step from the converged root z0.
template <class T> T z_of_x(const T& x, const T& om, double z0) {
  const T z(z0);
  const T I = I_of(z, om);
  const T u = 1.0 + z;
  const T F = u * I - x;
  const T Dp = I + u / E_of(z, om);
  return z - F / Dp;
}

// ----------------------------------------------------------------- population
template <class T> struct Pop {
  int model = MODEL_PLP;
  T H0, om, alpha, beta, mmin, mmax, dm, mu, sig, lam, gam, kap, zp;
  T mu2, sig2, lam1;   // multi-peak only: the second Gaussian, the first one's share
  T lnZP;    // ln int_{mmin}^{mmax} m^-alpha dm
  T lnZG;    // ln of the Gaussian's mass inside [mmin, mmax]
  T lnZG2;   // the same for the second Gaussian (multi-peak)
  T lnZm1;   // ln int p_unnormalised(m1) dm1
  T lnNz;    // ln of the redshift-prior normalisation over the pixel-averaged LOS prior
  double xmax;  // D(z_max; Om)
};

// ln S(m): low-mass smoothing.  S = 0 below m_min, 1 above m_min + dm, and
// 1/(1 + exp(dm/m' + dm/(m' - dm))) with m' = m - m_min in between (S = 0 at m' = 0).
// Returns false where S = 0.
template <class T> bool ln_S(const T& m, const T& mmin, const T& dm, T& out) {
  if (val(m) < val(mmin)) return false;
  if (val(m) >= val(mmin) + val(dm)) { out = T(0.0); return true; }
  const T mp = m - mmin;
  if (!(val(mp) > 0.0)) return false;
  const T f = dm / mp + dm / (mp - dm);
  out = -softplus(f);
  return true;
}

// N(m; mu, sig) / Z, Z its mass inside [mmin, mmax] (a Gaussian truncated to the range)
template <class T> T gauss_trunc(const T& m, const T& mu, const T& sig, const T& lnZ) {
  const T zg = (m - mu) / sig;
  return fexp(-0.5 * zg * zg - flog(sig) - LN_SQRT_2PI - lnZ);
}

// unnormalised primary-mass density before smoothing:
//   power law + peak:  (1-lam) m^-alpha/Z_P + lam G(m; mu, sig)
//   multi-peak:        (1-lam) m^-alpha/Z_P + lam [lam1 G(m; mu, sig) + (1-lam1) G(m; mu2, sig2)]
// with G truncated Gaussians; the multi-peak model is the power law with two peaks of the
// population literature (Abbott et al. 2021, ApJL 913 L7), mixed and smoothed like the
// single peak.  At lam1 = 1 it is the power law + peak model with the first Gaussian.
template <class T> T m1_mixture(const T& m, const Pop<T>& P) {
  const T pl = fexp(-P.alpha * flog(m) - P.lnZP);
  const T ga = gauss_trunc(m, P.mu, P.sig, P.lnZG);
  if (P.model != MODEL_MP) return (1.0 - P.lam) * pl + P.lam * ga;
  const T ga2 = gauss_trunc(m, P.mu2, P.sig2, P.lnZG2);
  return (1.0 - P.lam) * pl + P.lam * (P.lam1 * ga + (1.0 - P.lam1) * ga2);
}

template <class T> T m1_unnormalised(const T& m, const Pop<T>& P) {
  T ls;
  if (!ln_S(m, P.mmin, P.dm, ls)) return T(0.0) * m;
  return m1_mixture(m, P) * fexp(ls);
}

// C(m1) = int_{mmin}^{m1} m^beta S(m) dm, the normaliser of p(m2 | m1)
template <class T> T C_of(const T& m1, const Pop<T>& P) {
  auto fw = [&P](const T& m) {
    T ls;
    if (!ln_S(m, P.mmin, P.dm, ls)) return T(0.0) * m;
    return fexp(P.beta * flog(m) + ls);
  };
  auto fa = [&P](const T& m) { return fexp(P.beta * flog(m)); };
  const T mw = P.mmin + P.dm;
  if (val(m1) <= val(mw)) return integrate(fw, P.mmin, m1, 1e-13);
  return integrate(fw, P.mmin, mw, 1e-13) + integrate(fa, mw, m1, 1e-13);
}

template <class T> bool ln_p_m1(const T& m1, const Pop<T>& P, T& out) {
  if (val(m1) > val(P.mmax)) return false;
  T ls;
  if (!ln_S(m1, P.mmin, P.dm, ls)) return false;
  const T mix = m1_mixture(m1, P);
  if (!(val(mix) > 0.0)) return false;
  out = flog(mix) + ls - P.lnZm1;
  return true;
}

template <class T> bool ln_p_m2(const T& m2, const T& m1, const Pop<T>& P, T& out) {
  if (val(m2) > val(m1)) return false;
  T ls;
  if (!ln_S(m2, P.mmin, P.dm, ls)) return false;
  const T C = C_of(m1, P);
  if (!(val(C) > 0.0)) return false;
  out = P.beta * flog(m2) + ls - flog(C);
  return true;
}

// Madau-Dickinson shape, psi(0) = 1:
//   psi(z) = [1 + (1+zp)^-(g+k)] (1+z)^g / [1 + ((1+z)/(1+zp))^(g+k)]
template <class T> T ln_psi(const T& z, const Pop<T>& P) {
  const T gk = P.gam + P.kap;
  const T lu = flog(1.0 + z);
  const T lp = flog(1.0 + P.zp);
  return softplus(-gk * lp) + P.gam * lu - softplus(gk * (lu - lp));
}

// N_z = trapezoid over the LOS grid of pbar(z_j) psi(z_j) / (1 + z_j)
template <class T> T Nz_of(const std::vector<double>& pbar, double zmax, const Pop<T>& P) {
  const int nz = (int)pbar.size();
  const double dz = zmax / (double)(nz - 1);
  T acc(0.0);
  for (int j = 0; j < nz; ++j) {
    const double zj = (double)j * dz;
    const double cj = (j == 0 || j == nz - 1) ? 0.5 : 1.0;
    acc = acc + (cj * pbar[j] * dz) * fexp(ln_psi(T(zj), P)) / (1.0 + zj);
  }
  return acc;
}

template <class T> void set_norms(Pop<T>& P, const std::vector<double>& pbar, double zmax) {
  auto fpl = [&P](const T& m) { return fexp(-P.alpha * flog(m)); };
  P.lnZP = flog(integrate(fpl, P.mmin, P.mmax, 1e-14));
  const double r2 = 0.70710678118654752440084436210485;
  P.lnZG = flog(0.5 * (ferf((P.mmax - P.mu) / P.sig * r2) - ferf((P.mmin - P.mu) / P.sig * r2)));
  if (P.model == MODEL_MP)
    P.lnZG2 = flog(0.5 * (ferf((P.mmax - P.mu2) / P.sig2 * r2) - ferf((P.mmin - P.mu2) / P.sig2 * r2)));
  // Z_m1 over [mmin, mmin+dm] and [mmin+dm, mmax]; the upper piece is split around the
  // peak (fixed split points do not change the integral, only help the adaptivity)
  auto fm = [&P](const T& m) { return m1_unnormalised(m, P); };
  const T mw = P.mmin + P.dm;
  T Z = integrate(fm, P.mmin, mw, 1e-14);
  std::vector<double> cuts;
  for (double k : {-5.0, 0.0, 5.0}) {
    const double c = val(P.mu) + k * val(P.sig);
    if (c > val(mw) && c < val(P.mmax)) cuts.push_back(c);
    if (P.model == MODEL_MP) {
      const double c2 = val(P.mu2) + k * val(P.sig2);
      if (c2 > val(mw) && c2 < val(P.mmax)) cuts.push_back(c2);
    }
  }
  std::sort(cuts.begin(), cuts.end());
  T lo = mw;
  for (double c : cuts) { Z = Z + integrate(fm, lo, T(c), 1e-14); lo = T(c); }
  Z = Z + integrate(fm, lo, P.mmax, 1e-14);
  P.lnZm1 = flog(Z);
  P.lnNz = flog(Nz_of(pbar, zmax, P));
  P.xmax = D_of(zmax, val(P.om));
}

bool lambda_in_domain(const double* L, int model = MODEL_PLP) {
  for (int i = 0; i < n_params(model); ++i) if (!std::isfinite(L[i])) return false;
  const bool base = L[P_H0] > 0.0 && L[P_OM] >= 0.0 && L[P_OM] <= 1.0 && L[P_MMIN] > 0.0 &&
                    L[P_MMAX] > L[P_MMIN] && L[P_DM] >= 0.0 && L[P_MMIN] + L[P_DM] < L[P_MMAX] &&
                    L[P_SIG] > 0.0 && L[P_LAM] >= 0.0 && L[P_LAM] <= 1.0 && L[P_ZP] > -1.0;
  if (model != MODEL_MP) return base;
  return base && L[P_SIG2] > 0.0 && L[P_LAM1] >= 0.0 && L[P_LAM1] <= 1.0;
}

// The population at Lambda; with T a dual number, hyperparameter i carries the unit
// derivative in slot i (all n_params(model) of them, so T must be wide enough)
template <class T>
Pop<T> make_pop(const double* L, int model, const std::vector<double>& pbar, double zmax) {
  T v[NP_MAX];
  for (int i = 0; i < n_params(model); ++i) seed(v[i], L[i], i);
  Pop<T> P;
  P.model = model;
  P.H0 = v[0]; P.om = v[1]; P.alpha = v[2]; P.beta = v[3]; P.mmin = v[4]; P.mmax = v[5];
  P.dm = v[6]; P.mu = v[7]; P.sig = v[8]; P.lam = v[9]; P.gam = v[10]; P.kap = v[11]; P.zp = v[12];
  if (model == MODEL_MP) { P.mu2 = v[P_MU2]; P.sig2 = v[P_SIG2]; P.lam1 = v[P_LAM1]; }
  set_norms(P, pbar, zmax);
  return P;
}

// ---------------------------------------------------------------------- LOS
// The grid cell of z on z_j = j * zmax / (nz - 1): the exact floor of z (nz - 1) / zmax,
// clamped to [0, nz - 2] (z = zmax lies in the last cell); -1 outside [0, zmax].
int los_cell_of(double zv, int nz, double zmax) {
  if (zv < 0.0 || zv > zmax) return -1;
  const double s = (double)(nz - 1) / zmax;
  int j = (int)std::floor(zv * s);
  if (j > nz - 2) j = nz - 2;
  if (j < 0) j = 0;
  return j;
}

// linear interpolation of a row tabulated at z_j = j * zmax / (nz - 1); zero outside
// [0, zmax], in the cell los_cell_of gives.
template <class T> bool los_interp(const double* row, int nz, double zmax, const T& z, T& p) {
  const double zv = val(z);
  const int j = los_cell_of(zv, nz, zmax);
  if (j < 0) return false;
  const double s = (double)(nz - 1) / zmax;
  const T t = z * s - (double)j;
  p = row[j] + t * (row[j + 1] - row[j]);
  return val(p) > 0.0;
}

// Size of the jump of d ln p_LOS / dz at a grid node within `kappa` cells of z (0 if
// none): the LOS prior is piecewise linear, so at a node the derivative has two valid
// one-sided values.  Tests use it to accept either side (see grad_kink below).
double los_kink(const double* row, int nz, double zmax, double zv, double p, double kappa) {
  const double s = (double)(nz - 1) / zmax;
  const double pos = zv * s;
  const int k = (int)std::floor(pos + 0.5);
  if (std::fabs(pos - k) > kappa || k <= 0 || k >= nz - 1 || !(p > 0.0)) return 0.0;
  const double left = row[k] - row[k - 1], right = row[k + 1] - row[k];
  return std::fabs(right - left) * s / p;
}

// ----------------------------------------------------------------- one sample
// ln w for one detector-frame sample (m1d, m2d, dL) with PE prior ln pi:
//   ln w = ln p_LOS(z) + ln psi(z) - ln(1+z) - ln N_z            (redshift prior, Eq. hier_pixels)
//        + ln p(m1s) + ln p(m2s | m1s)                           (source-frame masses)
//        - 2 ln(1+z) - ln(d d_L/dz)                              (Jacobian to detector frame)
//        - ln pi_PE                                              (Eq. 6)
// with z solving D(z) = d_L H0 / c and m_s = m_d / (1+z).  Returns false where w = 0.
inline void kink_parts(const double&, double, double*) {}
template <int N> void kink_parts(const DualT<N>& z, double jump, double* kink) {
  for (int i = 0; i < N; ++i) kink[i] = jump * std::fabs(z.d[i]);
}

// row == NULL leaves out the LOS factor (the weight w' of the KDE form, Eq. 6); *z_out
// (when given) receives z whenever d_L maps into [0, zmax], whatever the weight.
template <class T>
bool ln_w(const Pop<T>& P, const double* row, int nz, double zmax, double m1d, double m2d,
          double dl, double lnpi, T& out, double* kink = nullptr, double* z_out = nullptr) {
  if (z_out) *z_out = NEG_INF;
  if (!(dl > 0.0)) return false;
  const T x = dl * P.H0 / C_KMS;
  if (val(x) > P.xmax) return false;
  const double z0 = z_root(val(x), val(P.om), zmax);
  const T z = z_of_x(x, P.om, z0);
  if (z_out) *z_out = val(z);
  T plos = T(1.0);
  if (row && !los_interp(row, nz, zmax, z, plos)) return false;
  const T u = 1.0 + z;
  const T m1s = m1d / u;
  const T m2s = m2d / u;
  T lp1, lp2;
  if (!ln_p_m1(m1s, P, lp1)) return false;
  if (!ln_p_m2(m2s, m1s, P, lp2)) return false;
  const T ddl_dz = (C_KMS / P.H0) * Dprime_of(z, P.om);
  const T lu = flog(u);
  out = ln_psi(z, P) - lu - P.lnNz + lp1 + lp2 - 2.0 * lu - flog(ddl_dz) - lnpi;
  if (row) out = out + flog(plos);
  if (kink && row) kink_parts(z, los_kink(row, nz, zmax, val(z), val(plos), 2e-5), kink);
  return true;
}

// ------------------------------------------------------------ sums of weights
// (max, sum e^(l - max), sum e^(2(l - max)), sum e^(l - max) dl/dLambda) over a set
template <class T> struct Sums {
  double m = NEG_INF, s1 = 0.0, s2 = 0.0;
  double g[NP_MAX] = {0};      // sum e^(l - m) dl/dLambda
  double gabs[NP_MAX] = {0};   // sum e^(l - m) |dl/dLambda| (a magnitude scale for tests)
  double gkink[NP_MAX] = {0};  // sum e^(l - m) (one-sided derivative ambiguity at LOS nodes)
  long n_pos = 0;
};

inline void grad_parts(const double&, double*, double*, double) {}
template <int N> void grad_parts(const DualT<N>& l, double* g, double* gabs, double t) {
  for (int i = 0; i < N; ++i) {
    g[i] += t * l.d[i];
    gabs[i] += t * std::fabs(l.d[i]);
  }
}

// kinks: np values per entry of ls (or none)
template <class T> Sums<T> sums_of(const std::vector<T>& ls, const std::vector<double>& kinks, int np) {
  Sums<T> S;
  for (const T& l : ls) S.m = std::max(S.m, val(l));
  for (size_t q = 0; q < ls.size(); ++q) {
    const T& l = ls[q];
    const double t = std::exp(val(l) - S.m);
    S.s1 += t;
    S.s2 += t * t;
    grad_parts(l, S.g, S.gabs, t);
    if (!kinks.empty())
      for (int i = 0; i < np; ++i) S.gkink[i] += t * kinks[q * np + i];
    ++S.n_pos;
  }
  return S;
}

template <class T> Sums<T> merge(const std::vector<Sums<T>>& parts) {
  Sums<T> S;
  for (const auto& p : parts) S.m = std::max(S.m, p.m);
  if (S.m == NEG_INF) return S;
  for (const auto& p : parts) {
    if (p.n_pos == 0) continue;
    const double r = std::exp(p.m - S.m);
    S.s1 += p.s1 * r;
    S.s2 += p.s2 * r * r;
    for (int i = 0; i < NP_MAX; ++i) {
      S.g[i] += p.g[i] * r;
      S.gabs[i] += p.gabs[i] * r;
      S.gkink[i] += p.gkink[i] * r;
    }
    S.n_pos += p.n_pos;
  }
  return S;
}

struct Inputs {
  int32_t n_events;
  int32_t pad0;
  const int64_t* offsets;
  const float* m1;
  const float* m2;
  const float* dl;
  const float* lnpe;
  const int32_t* pix;
  int32_t n_pix;
  int32_t n_z;
  double z_max;
  const float* los;
  int64_t n_inj;
  double n_draw;
  const float* im1;
  const float* im2;
  const float* idl;
  const float* ilnpd;
};

std::vector<double> pixel_mean(const Inputs& in) {
  std::vector<double> pbar((size_t)in.n_z, 0.0);
  for (int p = 0; p < in.n_pix; ++p)
    for (int j = 0; j < in.n_z; ++j) pbar[(size_t)j] += (double)in.los[(size_t)p * in.n_z + j];
  for (double& v : pbar) v /= (double)in.n_pix;
  return pbar;
}

bool inputs_valid(const Inputs& in) {
  if (in.n_events < 0 || in.n_pix < 1 || in.n_z < 2 || !(in.z_max > 0.0)) return false;
  if (in.n_inj < 1 || !(in.n_draw >= (double)in.n_inj)) return false;
  if (in.offsets[0] != 0) return false;
  for (int e = 0; e < in.n_events; ++e)
    if (in.offsets[e + 1] <= in.offsets[e]) return false;
  const int64_t ns = in.offsets[in.n_events];
  for (int64_t k = 0; k < ns; ++k)
    if (in.pix[k] < 0 || in.pix[k] >= in.n_pix) return false;
  return true;
}

template <class T>
void eval_lambda(const Inputs& in, const std::vector<double>& pbar, const double* L, int model,
                 double neff_min_event, double neff_min_sel, double* lnL_event, double* neff_event,
                 double* ln_xi, double* neff_sel, double* lnL_total, int32_t* flag, double* grad,
                 double* gscale, double* gkink) {
  const int ne = in.n_events;
  const double zmax = in.z_max;
  const int nz = in.n_z;
  const int np = n_params(model);
  *flag = 0;
  if (grad) for (int i = 0; i < np; ++i) grad[i] = 0.0;
  if (gscale) for (int i = 0; i < np; ++i) gscale[i] = 0.0;
  if (gkink) for (int i = 0; i < np; ++i) gkink[i] = 0.0;
  if (!lambda_in_domain(L, model)) {
    *flag = 1;
    for (int e = 0; e < ne; ++e) { lnL_event[e] = NEG_INF; neff_event[e] = 0.0; }
    *ln_xi = NEG_INF; *neff_sel = 0.0; *lnL_total = NEG_INF;
    return;
  }
  const Pop<T> P = make_pop<T>(L, model, pbar, zmax);

  // ---- numerator: one event at a time
  std::vector<double> ev_grad((size_t)ne * np, 0.0), ev_gabs((size_t)ne * np, 0.0),
      ev_gkink((size_t)ne * np, 0.0);
  const bool want_kink = gkink != nullptr;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < ne; ++e) {
    std::vector<T> ls;
    std::vector<double> kinks;
    std::vector<double> row((size_t)nz);
    int cur_pix = -1;
    double kk[NP_MAX];
    for (int64_t k = in.offsets[e]; k < in.offsets[e + 1]; ++k) {
      if (in.pix[k] != cur_pix) {
        cur_pix = in.pix[k];
        for (int j = 0; j < nz; ++j) row[(size_t)j] = (double)in.los[(size_t)cur_pix * nz + j];
      }
      T l;
      if (ln_w(P, row.data(), nz, zmax, in.m1[k], in.m2[k], in.dl[k], in.lnpe[k], l,
               want_kink ? kk : nullptr)) {
        ls.push_back(l);
        if (want_kink) kinks.insert(kinks.end(), kk, kk + np);
      }
    }
    const Sums<T> S = sums_of(ls, kinks, np);
    const double n_i = (double)(in.offsets[e + 1] - in.offsets[e]);
    if (S.n_pos == 0) {
      lnL_event[e] = NEG_INF;
      neff_event[e] = 0.0;
    } else {
      lnL_event[e] = S.m + std::log(S.s1) - std::log(n_i);
      neff_event[e] = S.s1 * S.s1 / S.s2;
      for (int i = 0; i < np; ++i) {
        ev_grad[(size_t)e * np + i] = S.g[i] / S.s1;
        ev_gabs[(size_t)e * np + i] = S.gabs[i] / S.s1;
        ev_gkink[(size_t)e * np + i] = S.gkink[i] / S.s1;
      }
    }
  }

  // ---- selection: injections against the pixel-averaged LOS prior, in chunks small
  // enough that every thread gets several (the chunk size changes only the order of
  // the FP64 sums)
#ifdef _OPENMP
  const int64_t nthreads = omp_get_max_threads();
#else
  const int64_t nthreads = 1;
#endif
  const int64_t chunk = std::min<int64_t>(65536, std::max<int64_t>(1024, in.n_inj / (4 * nthreads) + 1));
  const int64_t nchunk = (in.n_inj + chunk - 1) / chunk;
  std::vector<Sums<T>> parts((size_t)nchunk);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nchunk; ++c) {
    std::vector<T> ls;
    std::vector<double> kinks;
    double kk[NP_MAX];
    const int64_t a = c * chunk, b = std::min(in.n_inj, a + chunk);
    for (int64_t k = a; k < b; ++k) {
      T l;
      if (ln_w(P, pbar.data(), nz, zmax, in.im1[k], in.im2[k], in.idl[k], in.ilnpd[k], l,
               want_kink ? kk : nullptr)) {
        ls.push_back(l);
        if (want_kink) kinks.insert(kinks.end(), kk, kk + np);
      }
    }
    parts[(size_t)c] = sums_of(ls, kinks, np);
  }
  const Sums<T> Ssel = merge(parts);
  double sel_grad[NP_MAX] = {0}, sel_gabs[NP_MAX] = {0}, sel_gkink[NP_MAX] = {0};
  if (Ssel.n_pos == 0) {
    *ln_xi = NEG_INF;
    *neff_sel = 0.0;
  } else {
    *ln_xi = Ssel.m + std::log(Ssel.s1) - std::log(in.n_draw);
    *neff_sel = Ssel.s1 * Ssel.s1 / Ssel.s2;
    for (int i = 0; i < np; ++i) {
      sel_grad[i] = Ssel.g[i] / Ssel.s1;
      sel_gabs[i] = Ssel.gabs[i] / Ssel.s1;
      sel_gkink[i] = Ssel.gkink[i] / Ssel.s1;
    }
  }

  // ---- total = sum_i ln L_i - N_det ln xi (Neumaier-compensated sum in event order)
  bool neff_fail = false, dead = false;
  double sum = 0.0, comp_ = 0.0;
  for (int e = 0; e < ne; ++e) {
    if (!(neff_event[e] >= neff_min_event)) neff_fail = true;
    if (lnL_event[e] == NEG_INF) { dead = true; continue; }   // the product of Eq. 3 vanishes
    const double v = lnL_event[e];
    const double t = sum + v;
    if (std::fabs(sum) >= std::fabs(v)) comp_ += (sum - t) + v; else comp_ += (v - t) + sum;
    sum = t;
  }
  // flags: bit 1 some event below the N_eff threshold, bit 2 selection below its
  // threshold (only when one is set), bit 3 every injection weight is zero.  Any
  // flag makes the total -inf.
  if (neff_fail) *flag |= 2;
  if (neff_min_sel > 0.0 && !(*neff_sel >= neff_min_sel)) *flag |= 4;
  if (Ssel.n_pos == 0) *flag |= 8;
  if (*flag || dead) {
    *lnL_total = NEG_INF;
    return;
  }
  *lnL_total = (sum + comp_) - (double)ne * (*ln_xi);
  if (grad) {
    for (int i = 0; i < np; ++i) {
      double g = 0.0;
      for (int e = 0; e < ne; ++e) g += ev_grad[(size_t)e * np + i];
      grad[i] = g - (double)ne * sel_grad[i];
    }
  }
  if (gscale) {
    for (int i = 0; i < np; ++i) {
      double a = 0.0;
      for (int e = 0; e < ne; ++e) a += ev_gabs[(size_t)e * np + i];
      gscale[i] = a + (double)ne * sel_gabs[i];
    }
  }
  if (gkink) {
    for (int i = 0; i < np; ++i) {
      double a = 0.0;
      for (int e = 0; e < ne; ++e) a += ev_gkink[(size_t)e * np + i];
      gkink[i] = a + (double)ne * sel_gkink[i];
    }
  }
}

// ------------------------------------------------------------ KDE numerator
// The paper's own per-event term (Eqs. 5-7): in each sky pixel j of event i, a Gaussian
// KDE in z of the pixel's samples weighted by w' = p_pop(z, theta'|Lambda) / pi_PE (the
// weight of Eq. 6, i.e. the Monte-Carlo weight without its LOS factor), evaluated on a
// uniform grid of n_grid points over [0, zmax], multiplied by the pixel's LOS prior and
// integrated by the trapezoid rule:
//     L_ij = sum_g c_g p_LOS(z_g | j) sum_k w'_k K_h(z_g - z_k),   K_h = N(0, h^2) density
//     L_i  = (1 / N_i) sum_{j kept} L_ij
// A pixel is kept when its N_eff = (sum w')^2 / sum w'^2 (Eq. 7) reaches the threshold
// and its bandwidth is positive.  With a LOS prior linear in z and every sample more
// than a few h inside the grid, L_i equals the Monte-Carlo term exactly; that is the
// kernel's zero-width limit for any h.
enum { BW_SCOTT = 0, BW_SILVERMAN = 1, BW_BIWEIGHT = 2 };

// quantile of sorted values, linear between order statistics at position q (n - 1)
double quantile_sorted(const std::vector<double>& s, double q) {
  const double pos = q * (double)(s.size() - 1);
  const size_t i = (size_t)std::floor(pos);
  if (i + 1 >= s.size()) return s.back();
  return s[i] + (pos - (double)i) * (s[i + 1] - s[i]);
}

// Bandwidth of one pixel's z samples (unweighted), by the rules of the paper's appendix:
//   Scott      1.06 sigma n^-1/5 (sigma: sample standard deviation, n - 1 in the divisor)
//   Silverman  0.9 min(sigma, IQR / 1.34) n^-1/5
//   biweight   1.06 s_bi n^-1/5 with s_bi^2 the biweight midvariance (the expression the
//              appendix prints, about the median Q with u = (z - Q) / (9 MAD))
// 0 when it is undefined (n < 2, or a zero scale).
double bandwidth(std::vector<double> z, int rule) {
  const size_t n = z.size();
  if (n < 2) return 0.0;
  const double nf = (double)n, shrink = std::pow(nf, -0.2);
  double mean = 0.0;
  for (double v : z) mean += v;
  mean /= nf;
  double ss = 0.0;
  for (double v : z) ss += (v - mean) * (v - mean);
  const double sigma = std::sqrt(ss / (nf - 1.0));
  if (rule == BW_SCOTT) return 1.06 * sigma * shrink;
  std::sort(z.begin(), z.end());
  if (rule == BW_SILVERMAN) {
    const double iqr = quantile_sorted(z, 0.75) - quantile_sorted(z, 0.25);
    return 0.9 * std::min(sigma, iqr / 1.34) * shrink;
  }
  const double Q = quantile_sorted(z, 0.5);
  std::vector<double> dev(n);
  for (size_t i = 0; i < n; ++i) dev[i] = std::fabs(z[i] - Q);
  std::sort(dev.begin(), dev.end());
  const double mad = quantile_sorted(dev, 0.5);
  if (!(mad > 0.0)) return 0.0;
  double num = 0.0, den = 0.0;
  for (double v : z) {
    const double u = (v - Q) / (9.0 * mad);
    if (std::fabs(u) < 1.0) {
      const double a = 1.0 - u * u;
      num += (v - Q) * (v - Q) * a * a * a * a;
      den += a * (1.0 - 5.0 * u * u);
    }
  }
  if (!(den != 0.0) || !(num > 0.0)) return 0.0;
  return 1.06 * std::sqrt(nf * num / (den * den)) * shrink;
}

// ln L_i and the effective number of kept pixels (sum_j L_ij)^2 / sum_j L_ij^2 of one event
void kde_event(const Inputs& in, const Pop<double>& P, int e, int rule, int n_grid,
               double neff_min_pixel, double* lnL, double* neff) {
  const int nz = in.n_z;
  const double zmax = in.z_max;
  const double dzg = zmax / (n_grid - 1);
  std::vector<int> pixels;
  for (int64_t k = in.offsets[e]; k < in.offsets[e + 1]; ++k)
    if (std::find(pixels.begin(), pixels.end(), in.pix[k]) == pixels.end()) pixels.push_back(in.pix[k]);
  std::vector<double> lnLj;   // ln L_ij of the kept pixels
  for (int pj : pixels) {
    std::vector<double> zs, zw, lw;   // valid z of the pixel; z and ln w' of positive weights
    for (int64_t k = in.offsets[e]; k < in.offsets[e + 1]; ++k) {
      if (in.pix[k] != pj) continue;
      double l, z;
      const bool pos = ln_w(P, nullptr, nz, zmax, in.m1[k], in.m2[k], in.dl[k], in.lnpe[k], l,
                            nullptr, &z);
      if (z == NEG_INF) continue;   // d_L outside the distance range
      zs.push_back(z);
      if (pos) { zw.push_back(z); lw.push_back(l); }
    }
    if (lw.empty()) continue;
    double m = NEG_INF;
    for (double v : lw) m = std::max(m, v);
    double s1 = 0.0, s2 = 0.0;
    for (double v : lw) { const double t = std::exp(v - m); s1 += t; s2 += t * t; }
    if (!(s1 * s1 / s2 >= neff_min_pixel)) continue;
    const double h = bandwidth(zs, rule);
    if (!(h > 0.0)) continue;
    std::vector<double> row((size_t)nz);
    for (int j = 0; j < nz; ++j) row[(size_t)j] = (double)in.los[(size_t)pj * nz + j];
    // the grid sum of Eq. 5 times the LOS prior, in the paper's order: the KDE at each
    // grid point, then the trapezoid over the grid
    const double norm = 1.0 / (h * std::sqrt(2.0 * M_PI));
    double Lj = 0.0;
    for (int g = 0; g < n_grid; ++g) {
      const double zg = g * dzg;
      double p;
      if (!los_interp(row.data(), nz, zmax, zg, p)) continue;
      double f = 0.0;
      for (size_t k = 0; k < zw.size(); ++k) {
        const double u = (zg - zw[k]) / h;
        f += std::exp(lw[k] - m - 0.5 * u * u) * norm;
      }
      Lj += ((g == 0 || g == n_grid - 1) ? 0.5 : 1.0) * dzg * p * f;
    }
    if (Lj > 0.0) lnLj.push_back(m + std::log(Lj));
  }
  const double n_i = (double)(in.offsets[e + 1] - in.offsets[e]);
  if (lnLj.empty()) { *lnL = NEG_INF; *neff = 0.0; return; }
  double M = NEG_INF;
  for (double v : lnLj) M = std::max(M, v);
  double a = 0.0, b = 0.0;
  for (double v : lnLj) { const double t = std::exp(v - M); a += t; b += t * t; }
  *lnL = M + std::log(a) - std::log(n_i);
  *neff = a * a / b;
}

void eval_lambda_kde(const Inputs& in, const std::vector<double>& pbar, const double* L, int model,
                     int rule, int n_grid, double neff_min_pixel, double neff_min_sel,
                     double* lnL_event, double* neff_event, double* ln_xi, double* neff_sel,
                     double* lnL_total, int32_t* flag) {
  const int ne = in.n_events;
  // the selection term is the Monte-Carlo one; the event terms are replaced below
  eval_lambda<double>(in, pbar, L, model, 0.0, neff_min_sel, lnL_event, neff_event, ln_xi, neff_sel,
                      lnL_total, flag, nullptr, nullptr, nullptr);
  if (*flag & 1) return;
  const Pop<double> P = make_pop<double>(L, model, pbar, in.z_max);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < ne; ++e)
    kde_event(in, P, e, rule, n_grid, neff_min_pixel, lnL_event + e, neff_event + e);
  bool dead = false;
  double sum = 0.0, comp_ = 0.0;
  for (int e = 0; e < ne; ++e) {
    if (lnL_event[e] == NEG_INF) { dead = true; continue; }
    const double v = lnL_event[e];
    const double t = sum + v;
    if (std::fabs(sum) >= std::fabs(v)) comp_ += (sum - t) + v; else comp_ += (v - t) + sum;
    sum = t;
  }
  *flag &= ~2;   // the per-pixel cut replaces the per-event one
  *lnL_total = (*flag || dead) ? NEG_INF : (sum + comp_) - (double)ne * (*ln_xi);
}

std::vector<double> row_to_double(const float* row, int nz) {
  std::vector<double> r((size_t)nz);
  for (int j = 0; j < nz; ++j) r[(size_t)j] = (double)row[j];
  return r;
}

// ln w of n samples with gradient slots of type D (Dual or DualM): out_grad[n][np] and,
// when non-NULL, out_kink[n][np]; row_of(k, row) fills sample k's LOS row
template <class D, class RowOf>
void ln_w_grad(const double* L, int model, const std::vector<double>& norm_row, double zmax,
               int64_t n, const float* m1, const float* m2, const float* dl, const float* lnpi,
               int nz, const RowOf& row_of, double* out, double* out_grad, double* out_kink) {
  const int np = n_params(model);
  const Pop<D> P = make_pop<D>(L, model, norm_row, zmax);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n; ++k) {
    std::vector<double> row((size_t)nz);
    row_of(k, row);
    D l;
    double kk[NP_MAX] = {0};
    const bool ok = ln_w(P, row.data(), nz, zmax, m1[k], m2[k], dl[k], lnpi[k], l, kk);
    out[k] = ok ? l.v : NEG_INF;
    for (int i = 0; i < np; ++i) {
      out_grad[(size_t)k * np + i] = ok ? l.d[i] : 0.0;
      if (out_kink) out_kink[(size_t)k * np + i] = ok ? kk[i] : 0.0;
    }
  }
}

template <class RowOf>
int ln_w_any(const double* L, int32_t n_par, const std::vector<double>& norm_row, double zmax,
             int64_t n, const float* m1, const float* m2, const float* dl, const float* lnpi, int nz,
             const RowOf& row_of, double* out, double* out_grad, double* out_kink) {
  const int model = model_of(n_par);
  if (model < 0 || !lambda_in_domain(L, model)) return -1;
  if (!out_grad) {
    const Pop<double> P = make_pop<double>(L, model, norm_row, zmax);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
      std::vector<double> row((size_t)nz);
      row_of(k, row);
      double l;
      out[k] = ln_w(P, row.data(), nz, zmax, m1[k], m2[k], dl[k], lnpi[k], l) ? l : NEG_INF;
    }
  } else if (model == MODEL_MP) {
    ln_w_grad<DualM>(L, model, norm_row, zmax, n, m1, m2, dl, lnpi, nz, row_of, out, out_grad, out_kink);
  } else {
    ln_w_grad<Dual>(L, model, norm_row, zmax, n, m1, m2, dl, lnpi, nz, row_of, out, out_grad, out_kink);
  }
  return 0;
}

}  // namespace

// ============================================================== C entry points
extern "C" {

// Full likelihood for K Lambda points lam[K][n_par]; n_par = 13 selects the power law +
// peak mass model, 16 the multi-peak model.  Arrays are host memory; outputs are
// lnL_event[K][n_events], neff_event[K][n_events], ln_xi[K], neff_sel[K],
// lnL_total[K], flags[K] and, if grad_total != NULL, grad_total[K][n_par]
// (want_grad != 0 selects the dual-number pass).  grad_scale[K][n_par] (may be NULL)
// receives sum_i sum_k p_ik |d ln w_ik| + N_det sum_m q_m |d ln w_m|, the size of the
// terms whose difference is the gradient.  grad_kink[K][n_par] (may be NULL) receives the
// same weighted sum of the one-sided-derivative ambiguity of samples lying within 2e-5
// LOS cells of a grid node (where either one-sided derivative is correct).  Returns 0,
// or -1 on invalid inputs.
int orc_loglik(const Inputs* in, int32_t K, const double* lam, int32_t n_par, int32_t want_grad,
               double neff_min_event, double neff_min_sel, int32_t n_threads, double* lnL_event,
               double* neff_event, double* ln_xi, double* neff_sel, double* lnL_total,
               int32_t* flags, double* grad_total, double* grad_scale, double* grad_kink) {
  const int model = model_of(n_par);
  if (!in || K < 0 || model < 0 || !inputs_valid(*in)) return -1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  const std::vector<double> pbar = pixel_mean(*in);
  const int ne = in->n_events;
  for (int k = 0; k < K; ++k) {
    double* g = (want_grad && grad_total) ? grad_total + (size_t)k * n_par : nullptr;
    double* gs = (want_grad && grad_scale) ? grad_scale + (size_t)k * n_par : nullptr;
    double* gk = (want_grad && grad_kink) ? grad_kink + (size_t)k * n_par : nullptr;
    const double* Lk = lam + (size_t)k * n_par;
    double* le = lnL_event + (size_t)k * ne;
    double* nf = neff_event + (size_t)k * ne;
    if (want_grad && model == MODEL_MP)
      eval_lambda<DualM>(*in, pbar, Lk, model, neff_min_event, neff_min_sel, le, nf, ln_xi + k,
                         neff_sel + k, lnL_total + k, flags + k, g, gs, gk);
    else if (want_grad)
      eval_lambda<Dual>(*in, pbar, Lk, model, neff_min_event, neff_min_sel, le, nf, ln_xi + k,
                        neff_sel + k, lnL_total + k, flags + k, g, gs, gk);
    else
      eval_lambda<double>(*in, pbar, Lk, model, neff_min_event, neff_min_sel, le, nf, ln_xi + k,
                          neff_sel + k, lnL_total + k, flags + k, nullptr, nullptr, nullptr);
  }
  return 0;
}

// The KDE form of the likelihood (Eqs. 5-7; see kde_event): bw_rule 0 Scott, 1
// Silverman, 2 biweight; n_grid KDE grid points on [0, zmax]; pixels below
// neff_min_pixel are dropped.  neff_event receives the effective number of kept pixels.
// Flags as orc_loglik, without bit 1 (there is no per-event N_eff cut).
int orc_loglik_kde(const Inputs* in, int32_t K, const double* lam, int32_t n_par, int32_t bw_rule,
                   int32_t n_grid, double neff_min_pixel, double neff_min_sel, int32_t n_threads,
                   double* lnL_event, double* neff_event, double* ln_xi, double* neff_sel,
                   double* lnL_total, int32_t* flags) {
  const int model = model_of(n_par);
  if (!in || K < 0 || model < 0 || !inputs_valid(*in) || n_grid < 2 || bw_rule < 0 || bw_rule > 2)
    return -1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  const std::vector<double> pbar = pixel_mean(*in);
  const int ne = in->n_events;
  for (int k = 0; k < K; ++k)
    eval_lambda_kde(*in, pbar, lam + (size_t)k * n_par, model, bw_rule, n_grid, neff_min_pixel, neff_min_sel,
                    lnL_event + (size_t)k * ne, neff_event + (size_t)k * ne, ln_xi + k,
                    neff_sel + k, lnL_total + k, flags + k);
  return 0;
}

// bandwidth of n values by rule bw_rule (as above)
double orc_bandwidth(const double* z, int64_t n, int32_t bw_rule) {
  return bandwidth(std::vector<double>(z, z + n), bw_rule);
}

// hyperparameters of mass model 0 (power law + peak) or 1 (multi-peak)
int orc_num_params(int32_t model) { return model == MODEL_MP ? NP_MP : model == MODEL_PLP ? NP : -1; }

// --- pieces, exposed for the pin tests ---------------------------------------
double orc_E(double z, double om) { return E_of(z, om); }
double orc_I(double z, double om) { return I_of(z, om); }
double orc_D(double z, double om) { return D_of(z, om); }
double orc_Dprime(double z, double om) { return Dprime_of(z, om); }
double orc_z_of_x(double x, double om, double zmax) { return z_of_x(x, om, z_root(x, om, zmax)); }

double orc_S(double m, double mmin, double dm) {
  double ls;
  return ln_S(m, mmin, dm, ls) ? std::exp(ls) : 0.0;
}

// The pieces below take Lambda as L[n_par] (13: power law + peak, 16: multi-peak) and
// return NaN for any other n_par.
static Pop<double> pop_from(const double* L, int model) {
  std::vector<double> pbar(2, 1.0);  // N_z is not needed by the mass and rate pieces
  return make_pop<double>(L, model, pbar, 1.0);
}
constexpr double NaN_ = std::numeric_limits<double>::quiet_NaN();

double orc_ln_p_m1(double m1, const double* L, int32_t n_par) {
  if (model_of(n_par) < 0) return NaN_;
  const Pop<double> P = pop_from(L, model_of(n_par));
  double o;
  return ln_p_m1(m1, P, o) ? o : NEG_INF;
}
double orc_ln_p_m2(double m2, double m1, const double* L, int32_t n_par) {
  if (model_of(n_par) < 0) return NaN_;
  const Pop<double> P = pop_from(L, model_of(n_par));
  double o;
  return ln_p_m2(m2, m1, P, o) ? o : NEG_INF;
}
double orc_C(double m1, const double* L, int32_t n_par) {
  return model_of(n_par) < 0 ? NaN_ : C_of(m1, pop_from(L, model_of(n_par)));
}
double orc_ln_Zm1(const double* L, int32_t n_par) {
  return model_of(n_par) < 0 ? NaN_ : pop_from(L, model_of(n_par)).lnZm1;
}
double orc_ln_psi(double z, const double* L, int32_t n_par) {
  return model_of(n_par) < 0 ? NaN_ : ln_psi(z, pop_from(L, model_of(n_par)));
}

double orc_ln_Nz(const double* L, int32_t n_par, const double* pbar, int32_t nz, double zmax) {
  if (model_of(n_par) < 0) return NaN_;
  std::vector<double> pb(pbar, pbar + nz);
  return flog(Nz_of(pb, zmax, pop_from(L, model_of(n_par))));
}

// The LOS grid cell of z, as used by los_interp above and as the CUDA library documents
// it: floor(z * ((nz - 1) / zmax)) in double precision, clamped to [0, nz - 2]; -1 for
// z outside [0, zmax].
int32_t orc_los_cell(float zf, int32_t nz, double zmax) { return los_cell_of((double)zf, nz, zmax); }

// For n samples of distance dl (Mpc) at Lambda L: the LOS grid cell that ln_w
// interpolates in (los_cell_of of the sample's exact redshift; -1 where d_L does not map
// into [0, zmax], i.e. d_L <= 0 or x > D(zmax)) and, in pos (may be NULL), the exact grid
// position z (nz - 1) / zmax (NaN where the cell is -1).
int orc_sample_cells(const double* L, int32_t n_par, int64_t n, const float* dl, int32_t nz,
                     double zmax, int32_t* cell, double* pos) {
  const int model = model_of(n_par);
  if (model < 0 || !lambda_in_domain(L, model)) return 1;
  const double H0 = L[P_H0], om = L[P_OM];
  const double xmax = D_of(zmax, om);
  const double s = (double)(nz - 1) / zmax;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t k = 0; k < n; ++k) {
    const double d = (double)dl[k];
    cell[k] = -1;
    if (pos) pos[k] = NaN_;
    if (!(d > 0.0)) continue;
    const double x = d * H0 / C_KMS;
    if (x > xmax) continue;
    const double z = z_of_x(x, om, z_root(x, om, zmax));
    cell[k] = los_cell_of(z, nz, zmax);
    if (pos && cell[k] >= 0) pos[k] = z * s;
  }
  return 0;
}

// ln w for n samples against one LOS row that also defines N_z (as the pixel average
// does for injections).  out_grad[n][n_par] is filled when non-NULL.  Samples with
// w = 0 get -inf (and a zero gradient).
int orc_ln_w_row(const double* L, int32_t n_par, int64_t n, const float* m1, const float* m2,
                 const float* dl, const float* lnpi, const float* row_f32, int32_t nz, double zmax,
                 double* out, double* out_grad) {
  const std::vector<double> row = row_to_double(row_f32, nz);
  auto row_of = [&row](int64_t, std::vector<double>& r) { r = row; };
  return ln_w_any(L, n_par, row, zmax, n, m1, m2, dl, lnpi, nz, row_of, out, out_grad, nullptr);
}

// ln w of n samples as the likelihood uses them: event samples (pix != NULL) against their
// pixel's LOS row, injections (pix == NULL) against the pixel mean; N_z from the pixel
// mean in both cases.  -inf where w = 0; out_grad[n][n_par] when non-NULL, and
// out_kink[n][n_par] (with out_grad) the one-sided-derivative ambiguity of samples near a
// LOS grid node.
int orc_ln_w_samples(const double* L, int32_t n_par, int64_t n, const float* m1, const float* m2,
                     const float* dl, const float* lnpi, const int32_t* pix, const float* los,
                     int32_t n_pix, int32_t nz, double zmax, double* out, double* out_grad,
                     double* out_kink) {
  std::vector<double> pbar((size_t)nz, 0.0);
  for (int p = 0; p < n_pix; ++p)
    for (int j = 0; j < nz; ++j) pbar[(size_t)j] += (double)los[(size_t)p * nz + j];
  for (double& v : pbar) v /= (double)n_pix;
  auto row_of = [&](int64_t k, std::vector<double>& row) {
    if (!pix) { row = pbar; return; }
    for (int j = 0; j < nz; ++j) row[(size_t)j] = (double)los[(size_t)pix[k] * nz + j];
  };
  return ln_w_any(L, n_par, pbar, zmax, n, m1, m2, dl, lnpi, nz, row_of, out, out_grad, out_kink);
}

// single application of the 15-point Kronrod (which = 0) or 7-point Gauss
// (which = 1) rule to x^k on [-1, 1]; used to pin the quadrature constants.
double orc_rule_poly(int32_t k, int32_t which) {
  auto f = [k](const double& x) { return std::pow(x, (double)k); };
  double K, G, kabs[NC_MAX];
  gk15(f, -1.0, 1.0, K, G, kabs);
  return which == 0 ? K : G;
}

}  // extern "C"
