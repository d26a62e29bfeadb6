// Host-side kernel tables: prolate window and polynomial forms of the residual
// Stokes kernels.  See tables.h for the stored functions.
//
// The prolate psi_0^c (Sec. 2.4) is computed in the orthonormal Legendre basis:
// the prolate differential operator -((1-x^2)psi')' + c^2 x^2 psi has matrix
// diag(k(k+1)) + c^2 X^2 there, X the Jacobi matrix of multiplication by x with
// off-diagonal a_k = k / sqrt(4k^2 - 1).  Restricted to even k it is symmetric
// tridiagonal; psi_0^c belongs to its smallest eigenvalue, found here by
// Sturm-sequence bisection followed by inverse iteration.
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace dmk {

namespace {

// ---- Table 2: 3c/pi for the prolate split at eps = 1e-3, 1e-6, 1e-9, 1e-12
const double kLogEps[4] = {-12.0, -9.0, -6.0, -3.0};
const double kStokeslet3c[4] = {31.0, 25.0, 17.0, 10.0};
const double kStresslet3c[4] = {32.0, 25.0, 17.0, 9.0};

double interp_table(const double* vals, double le) {
  for (int i = 0; i < 3; ++i) {
    if (le >= kLogEps[i] - 1e-9 && le <= kLogEps[i + 1] + 1e-9) {
      double t = (le - kLogEps[i]) / (kLogEps[i + 1] - kLogEps[i]);
      return vals[i] + t * (vals[i + 1] - vals[i]);
    }
  }
  return -1.0;
}

double legendre_antideriv_at0(int k) {
  // A_k(x) = (P_{k+1}(x) - P_{k-1}(x))/(2k+1) at x = 0 for k >= 1
  // P_n(0) = 0 for odd n, (-1)^{n/2} (n-1)!!/n!! for even n.
  auto p0 = [](int n) {
    if (n % 2) return 0.0;
    double v = 1.0;
    for (int j = 1; j <= n / 2; ++j) v *= -(2.0 * j - 1.0) / (2.0 * j);
    return v;
  };
  return (p0(k + 1) - p0(k - 1)) / (2.0 * k + 1.0);
}

}  // namespace

double bandlimit_for_eps(double eps, int kernels) {
  if (!(eps > 0.0)) return -1.0;
  double le = std::log10(eps);
  if (le < -12.0 - 1e-9 || le > -3.0 + 1e-9) return -1.0;
  double v = 0.0;
  if (kernels & 1) v = std::max(v, std::ceil(interp_table(kStokeslet3c, le) - 1e-9));
  if (kernels & 2) v = std::max(v, std::ceil(interp_table(kStresslet3c, le) - 1e-9));
  return v * M_PI / 3.0;
}

int leaf_capacity_for_eps(double eps, int dim) {
  const double n3[4] = {3000.0, 2000.0, 1200.0, 600.0};
  const double n2[4] = {480.0, 360.0, 240.0, 120.0};
  double le = std::log10(eps);
  le = std::min(-3.0, std::max(-12.0, le));
  double v = interp_table(dim == 3 ? n3 : n2, le);
  return static_cast<int>(std::lround(v));
}

// ---------------------------------------------------------------- prolate
int prolate_series(double c, ProlateSeries* out) {
  int nt = static_cast<int>(c) + 48;            // even terms k = 0, 2, ..., 2nt-2
  if (2 * nt > 256) return 1;
  std::vector<double> a(2 * nt + 3, 0.0);       // a_k = k / sqrt(4k^2-1), a_0 = 0
  for (int k = 1; k < static_cast<int>(a.size()); ++k)
    a[k] = k / std::sqrt(4.0 * k * k - 1.0);
  std::vector<double> d(nt), e(nt, 0.0);        // diagonal, super-diagonal
  for (int i = 0; i < nt; ++i) {
    int k = 2 * i;
    d[i] = k * (k + 1.0) + c * c * (a[k] * a[k] + a[k + 1] * a[k + 1]);
    if (i + 1 < nt) e[i] = c * c * a[k + 1] * a[k + 2];
  }
  // Sturm count: number of eigenvalues < x
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < nt; ++i) {
      double qq = (q == 0.0) ? 1e-300 : q;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < nt; ++i) {
    double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < nt ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= 1) hi = mid; else lo = mid;
  }
  double lam = 0.5 * (lo + hi);
  // inverse iteration with a shift just below lam (T - sigma I is then
  // positive definite; plain LDL^T elimination is stable)
  double sigma = lam - 1e-9 * std::max(1.0, std::fabs(lam));
  std::vector<double> v(nt, 1.0), piv(nt), lo_f(nt), y(nt);
  piv[0] = d[0] - sigma;
  for (int i = 1; i < nt; ++i) {
    lo_f[i] = e[i - 1] / piv[i - 1];
    piv[i] = d[i] - sigma - lo_f[i] * e[i - 1];
  }
  for (int it = 0; it < 4; ++it) {
    y[0] = v[0];
    for (int i = 1; i < nt; ++i) y[i] = v[i] - lo_f[i] * y[i - 1];
    v[nt - 1] = y[nt - 1] / piv[nt - 1];
    for (int i = nt - 2; i >= 0; --i) v[i] = (y[i] - e[i] * v[i + 1]) / piv[i];
    double nrm = 0.0;
    for (int i = 0; i < nt; ++i) nrm += v[i] * v[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < nt; ++i) v[i] /= nrm;
  }
  // standard-basis coefficients of psi, then phi = psi / int psi (int psi = 2 c_0)
  std::memset(out->coef, 0, sizeof(out->coef));
  out->n = 2 * nt;
  for (int i = 0; i < nt; ++i) out->coef[2 * i] = v[i] * std::sqrt(2 * i + 0.5);
  double psi0 = 0.0;   // psi(0) = sum c_k P_k(0)
  {
    double p = 1.0;
    for (int i = 0; i < nt; ++i) {
      psi0 += out->coef[2 * i] * p;
      p *= -(2.0 * i + 1.0) / (2.0 * i + 2.0);
    }
  }
  double scale = 1.0 / (2.0 * out->coef[0]);
  if (psi0 < 0) scale = -scale;                    // sign convention psi(0) > 0
  if (out->coef[0] * scale < 0) return 2;
  for (int k = 0; k < out->n; ++k) out->coef[k] *= scale;
  out->chi = lam;
  return 0;
}

static void legendre_all(int n, double x, double* P, double* dP) {
  P[0] = 1.0;
  if (n > 1) P[1] = x;
  for (int k = 1; k + 1 < n; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
  if (dP) {
    dP[0] = 0.0;
    if (n > 1) dP[1] = 1.0;
    for (int k = 1; k + 1 < n; ++k) dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
}

double series_phi(const ProlateSeries& s, double x) {
  if (std::fabs(x) > 1.0) return 0.0;
  double P[258];
  legendre_all(s.n, x, P, nullptr);
  double v = 0.0;
  for (int k = s.n - 1; k >= 0; --k) v += s.coef[k] * P[k];
  return v;
}

double series_dphi(const ProlateSeries& s, double x) {
  if (std::fabs(x) > 1.0) return 0.0;
  double P[258], dP[258];
  legendre_all(s.n, x, P, dP);
  double v = 0.0;
  for (int k = s.n - 1; k >= 0; --k) v += s.coef[k] * dP[k];
  return v;
}

double series_int0(const ProlateSeries& s, double x) {
  double xc = std::max(-1.0, std::min(1.0, x));
  double P[260];
  legendre_all(s.n + 1, xc, P, nullptr);
  double v = s.coef[0] * xc;   // int_0^x P_0
  for (int k = s.n - 1; k >= 1; --k)
    v += s.coef[k] * ((P[k + 1] - P[k - 1]) / (2.0 * k + 1.0) - legendre_antideriv_at0(k));
  return v;
}

// ------------------------------------------------------- polynomial fits
namespace {

constexpr int kFitN = 64;

// Chebyshev coefficients of f sampled at t_j = cos(pi (j + 1/2) / n)
void cheb_coeffs(const double* fv, int n, double* cf) {
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    // angle pi k (2j+1) / (2n), reduced exactly modulo 2 pi in integers first
    for (int j = 0; j < n; ++j) s += fv[j] * std::cos(M_PI * ((k * (2 * j + 1)) % (4 * n)) / (2.0 * n));
    cf[k] = (k == 0 ? 1.0 : 2.0) * s / n;
  }
}

// monomial coefficients (in t) of sum_{k<m} cf_k T_k(t)
void cheb_to_mono(const double* cf, int m, double* mono) {
  std::vector<double> Tkm1(m + 1, 0.0), Tk(m + 1, 0.0), Tkp1(m + 1, 0.0);
  std::fill(mono, mono + m, 0.0);
  Tkm1[0] = 1.0;                 // T_0
  if (m > 0) mono[0] += cf[0];
  if (m > 1) {
    Tk[1] = 1.0;                 // T_1
    mono[1] += cf[1];
  }
  for (int k = 1; k + 1 < m; ++k) {
    std::fill(Tkp1.begin(), Tkp1.end(), 0.0);
    for (int j = 0; j < m; ++j) {
      if (j + 1 <= m) Tkp1[j + 1] += 2.0 * Tk[j];
      Tkp1[j] -= Tkm1[j];
    }
    for (int j = 0; j < m; ++j) mono[j] += cf[k + 1] * Tkp1[j];
    Tkm1 = Tk;
    Tk = Tkp1;
  }
}

int truncate_len(const double* cf, int n, double tol_abs) {
  int last = 0;
  for (int k = 0; k < n; ++k)
    if (std::fabs(cf[k]) > tol_abs) last = k;
  return last + 1;
}

void fit(const double* fv, double fp32_tol, int* n64, double* p64, int* n32, float* p32) {
  double cf[kFitN];
  cheb_coeffs(fv, kFitN, cf);
  double mx = 0.0;
  for (int j = 0; j < kFitN; ++j) mx = std::max(mx, std::fabs(fv[j]));
  mx = std::max(mx, 1e-300);
  // coefficients below ~4e-16 max|f| are rounding noise of the interpolation
  int m64 = std::min(kMaxTerms, truncate_len(cf, kFitN, 1e-15 * mx));
  int m32 = std::min(kMaxTerms, truncate_len(cf, kFitN, fp32_tol * mx));
  double mono[kMaxTerms];
  cheb_to_mono(cf, m64, mono);
  *n64 = m64;
  for (int j = 0; j < m64; ++j) p64[j] = mono[j];
  cheb_to_mono(cf, m32, mono);
  *n32 = m32;
  for (int j = 0; j < m32; ++j) p32[j] = static_cast<float>(mono[j]);
}

// d/ds of a polynomial in t = 2s - 1: 2 * d/dt
void deriv_s(const double* p, int n, double* dp, int* dn) {
  *dn = std::max(1, n - 1);
  dp[0] = 0.0;
  for (int j = 1; j < n; ++j) dp[j - 1] = 2.0 * j * p[j];
}

}  // namespace

// ------------------------------------------------------------- 2D (App. B)
namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the
// three-term recurrence, initial guesses cos(pi (i + 3/4) / (n + 1/2)))
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

const double kR2 = 1.0 + std::sqrt(2.0);   // truncation radius R = 1 + sqrt(d), Sec. 2.3

// Bessel-combination series below z = 2.  With j0_m the z^{2m} coefficient
// of J0 and j1_m the z^{2m+1} coefficient of J1:
//   d : J0 - J1/z                             = sum (j0_m - j1_m) z^{2m}
//   o : (2 J1 - z J0)/z^3                     = sum (2 j1_m - j0_m) z^{2m-2}
//   td: (4 J1 - 2 z J0 - z^2 J1)/z^3          = sum (4 j1_m - 2 j0_m - j1_{m-1}) z^{2m-2}
//   to: ((8/3) J1 - (4/3) z J0 - z^2 J1/3)/z^5 = sum ((8/3) j1_m - (4/3) j0_m - j1_{m-1}/3) z^{2m-4}
// (the terms with negative powers vanish identically).
double combo_series(int kind, double z) {
  double z2 = z * z;
  double sum = 0.0, j0m = 1.0, j1m = 0.5, j1prev = 0.0, zp = 1.0;   // m = 0
  for (int m = 0; m < 40; ++m) {
    double coef = 0.0;
    int pw = 0;
    switch (kind) {
      case 0: coef = j0m - j1m; pw = 2 * m; break;
      case 1: coef = 2.0 * j1m - j0m; pw = 2 * m - 2; break;
      case 2: coef = 4.0 * j1m - 2.0 * j0m - j1prev; pw = 2 * m - 2; break;
      default: coef = (8.0 / 3.0) * j1m - (4.0 / 3.0) * j0m - j1prev / 3.0; pw = 2 * m - 4; break;
    }
    if (pw >= 0) {
      sum += coef * zp;
      zp *= z2;
    }
    j1prev = j1m;
    j0m *= -1.0 / (4.0 * (m + 1.0) * (m + 1.0));
    j1m *= -1.0 / (4.0 * (m + 1.0) * (m + 2.0));
  }
  return sum;
}

double combo(int kind, double z) {
  if (z < 2.0) return combo_series(kind, z);
  const double J0 = std::cyl_bessel_j(0.0, z), J1 = std::cyl_bessel_j(1.0, z);
  switch (kind) {
    case 0: return J0 - J1 / z;
    case 1: return (2.0 * J1 - z * J0) / (z * z * z);
    case 2: return (4.0 * J1 - 2.0 * z * J0 - z * z * J1) / (z * z * z);
    default: return ((8.0 / 3.0) * J1 - (4.0 / 3.0) * z * J0 - z * z * J1 / 3.0) / (z * z * z * z * z);
  }
}

// B-hat^R(k) = (1 - J0(Rk) - R k J1(Rk)/2) / k^4 (Eq. (Btrunc_hat), d = 2);
// series sum_{m>=2} (-1)^m (m - 1) (z/2)^{2m} / (m!)^2 below z = 1/2.
double bhat_trunc2(double k) {
  const double z = kR2 * k;
  double num;
  if (z < 0.5) {
    num = 0.0;
    double t = 1.0;    // (z/2)^{2m} / (m!)^2
    for (int m = 1; m < 30; ++m) {
      t *= (z * z / 4.0) / (double(m) * m);
      num += ((m % 2) ? -1.0 : 1.0) * (m - 1.0) * t;
    }
    if (k == 0.0) return std::pow(kR2, 4) / 64.0;
  } else {
    num = 1.0 - std::cyl_bessel_j(0.0, z) - 0.5 * z * std::cyl_bessel_j(1.0, z);
  }
  return num / (k * k * k * k);
}

}  // namespace

static int build_tables_2d(const ProlateSeries& ser, double c, double fp32_tol, KernelTables* out) {
  // gamma-hat(k) = phi-hat(k) - k phi-hat'(k)/2 on Gauss-Legendre nodes of [0, c]
  // (Eq. (gammaB_in_phi); phi-hat(k) = 2 int_0^1 phi(t) cos(kt) dt)
  std::vector<double> tx, tw, kx, kw;
  gauss_legendre(200, tx, tw);
  gauss_legendre(160, kx, kw);
  const int nt = 200, nk = 160;
  std::vector<double> tn(nt), phit(nt);
  for (int i = 0; i < nt; ++i) {
    tn[i] = 0.5 * (tx[i] + 1.0);
    phit[i] = series_phi(ser, tn[i]);
  }
  std::vector<double> kn(nk), weight(nk);
  for (int j = 0; j < nk; ++j) {
    const double k = 0.5 * c * (kx[j] + 1.0);
    double ph = 0.0, dph = 0.0;
    for (int i = 0; i < nt; ++i) {
      ph += tw[i] * phit[i] * std::cos(k * tn[i]);
      dph -= tw[i] * tn[i] * phit[i] * std::sin(k * tn[i]);
    }
    // 2 int_0^1 = int_{-1}^{1} with the half-interval Jacobian 1/2 folded in
    const double gam = ph - 0.5 * k * dph;
    kn[j] = k;
    weight[j] = 0.5 * c * kw[j] * bhat_trunc2(k) * gam;
  }
  // M-functions at unit scale: m = 4 int k^p G(k rho) B-hat^R gamma-hat dk (+ 2(1 - log R) for m_d)
  const int pw[4] = {3, 5, 5, 7};
  auto mfun = [&](int kind, double rho) {
    double s = 0.0;
    for (int j = 0; j < nk; ++j) s += std::pow(kn[j], pw[kind]) * combo(kind, kn[j] * rho) * weight[j];
    s *= 4.0;
    if (kind == 0) s += 2.0 * (1.0 - std::log(kR2));
    return s;
  };
  double fv[4][kFitN];
  for (int j = 0; j < kFitN; ++j) {
    const double t = std::cos(M_PI * (j + 0.5) / kFitN);
    const double rho = std::sqrt(0.5 * (t + 1.0));
    for (int kind = 0; kind < 4; ++kind) fv[kind][j] = mfun(kind, rho);
  }
  const int ids[4] = {P_GS, P_HS, P_PT, P_QT};
  for (int kind = 0; kind < 4; ++kind)
    fit(fv[kind], fp32_tol, &out->n64[ids[kind]], out->p64[ids[kind]], &out->n32[ids[kind]], out->p32[ids[kind]]);
  // lim_{r->0} Mdiag(r)/r = 2 int B-hat^R gamma-hat k^3 dk + 2(1 - log R) (Eqs. (msdiag0), (msdiag))
  double s = 0.0;
  for (int j = 0; j < nk; ++j) s += kn[j] * kn[j] * kn[j] * weight[j];
  out->self2d_m0 = 2.0 * s + 2.0 * (1.0 - std::log(kR2));
  return 0;
}

int build_tables(int dim, double c, double fp32_tol, KernelTables* out) {
  *out = KernelTables();
  out->dim = dim;
  out->c = c;
  ProlateSeries ser;
  if (prolate_series(c, &ser)) return 1;
  out->phi0 = series_phi(ser, 0.0);
  if (dim == 2) return build_tables_2d(ser, c, fp32_tol, out);
  if (dim != 3) return 3;

  double fg[kFitN], fh[kFitN], fp[kFitN], fq[kFitN];
  for (int j = 0; j < kFitN; ++j) {
    double t = std::cos(M_PI * (j + 0.5) / kFitN);
    double s = 0.5 * (t + 1.0);
    double rho = std::sqrt(s);
    double I = series_int0(ser, rho);
    double ph = series_phi(ser, rho);
    double dph = series_dphi(ser, rho);
    fg[j] = -2.0 * (I / rho + ph);
    fh[j] = -2.0 * (I / rho - ph);
    fp[j] = -2.0 * rho * dph;
    fq[j] = -2.0 * I / rho + 2.0 * ph - (2.0 / 3.0) * rho * dph;
  }
  fit(fg, fp32_tol, &out->n64[P_GS], out->p64[P_GS], &out->n32[P_GS], out->p32[P_GS]);
  fit(fh, fp32_tol, &out->n64[P_HS], out->p64[P_HS], &out->n32[P_HS], out->p32[P_HS]);
  fit(fp, fp32_tol, &out->n64[P_PT], out->p64[P_PT], &out->n32[P_PT], out->p32[P_PT]);
  fit(fq, fp32_tol, &out->n64[P_QT], out->p64[P_QT], &out->n32[P_QT], out->p32[P_QT]);
  for (int id : {P_GS, P_HS, P_PT, P_QT}) {
    int dn;
    double dp[kMaxTerms];
    deriv_s(out->p64[id], out->n64[id], dp, &dn);
    int did = (id == P_GS) ? P_DGS : (id == P_HS) ? P_DHS : (id == P_PT) ? P_DPT : P_DQT;
    out->n64[did] = dn;
    for (int j = 0; j < dn; ++j) out->p64[did][j] = dp[j];
    deriv_s(out->p64[id], out->n32[id] < out->n64[id] ? std::min(out->n64[id], out->n32[id] + 1)
                                                       : out->n64[id], dp, &dn);
    out->n32[did] = dn;
    for (int j = 0; j < dn; ++j) out->p32[did][j] = static_cast<float>(dp[j]);
  }
  return 0;
}

}  // namespace dmk
