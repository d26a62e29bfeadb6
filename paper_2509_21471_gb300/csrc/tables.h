// Host-side kernel tables for the residual Stokes kernels (built once per plan).
//
// The residual kernels of Sec. 5.2 (Eqs. (res_stokeslet), (Soffdiag),
// (res_stresslet), (T-offd)) depend on the window phi through Phi(rho),
// rho*phi(rho) and rho^2*phi'(rho).  Each is "1 + odd function of rho" or
// "odd function of rho", so dividing the odd part by rho leaves an even,
// smooth function of s = rho^2 on [0, 1] (the remark closing Sec. 5.2: the
// real-space functions are precomputed as polynomials).  We store them as
// polynomials in t = 2 s - 1 (monomial form, evaluated by Horner):
//
//   3D  gS(s) = (Sdiag(rho) - 1)/rho,  hS(s) = (Soffd(rho) - 1)/rho
//       pT(s) =  Tdiag(rho)/rho,       qT(s) = (Toffd(rho) - 1)/rho
//       dgS, dhS, dpT, dqT = d/ds of gS, hS, pT, qT      (gradient kernels)
//   so that, with nu the residual scale, r < nu:
//       S_R = (1/r + gS/nu) delta/(8 pi) + (1/r^3 + hS/(nu r^2)) x x/(8 pi)
//       T_R = pT/(8 pi nu r^2) (delta x + ...) - (3/4pi)(1/r^5 + qT/(nu r^4)) x x x
//
//   2D  (App. B numerics; stored the same way, see build_tables_2d).
#pragma once
#include <cstdint>

namespace dmk {

constexpr int kMaxTerms = 48;

enum PolyId { P_GS = 0, P_HS = 1, P_PT = 2, P_QT = 3, P_DGS = 4, P_DHS = 5, P_DPT = 6, P_DQT = 7, P_COUNT = 8 };

struct KernelTables {
  int dim = 3;
  double c = 0.0;          // PSWF bandlimit
  double phi0 = 0.0;       // phi(0)
  double self2d_m0 = 0.0;  // 2D: lim_{r->0} S_M,diag(r)/r at nu = 1 (App. B, Eq. (msdiag0))
  int n64[P_COUNT] = {0};
  double p64[P_COUNT][kMaxTerms] = {{0}};
  int n32[P_COUNT] = {0};
  float p32[P_COUNT][kMaxTerms] = {{0}};
};

// PSWF bandlimit c for tolerance eps (Table 2 rows, 3c/pi interpolated
// linearly in log10(eps) and rounded up).  kernels: bit 1 Stokeslet, bit 2 stresslet.
// Returns < 0 if eps is outside [1e-12, 1e-3].
double bandlimit_for_eps(double eps, int kernels);

// Paper's leaf capacity n_s for eps (Sec. 8): 3D 600/1200/2000/3000, 2D
// 120/240/360/480 at eps = 1e-3/1e-6/1e-9/1e-12, interpolated in log10(eps).
int leaf_capacity_for_eps(double eps, int dim);

// Builds all polynomial tables for dimension dim (2 or 3) and bandlimit c.
// fp32_tol: truncation tolerance of the FP32 tables (relative to max |f|).
// Returns 0 on success.
int build_tables(int dim, double c, double fp32_tol, KernelTables* out);

// Reference evaluation of the window (used by the tables and by tests of the
// table builder): phi, phi', int_0^x phi for the prolate window of bandlimit c.
struct ProlateSeries {
  int n = 0;                // number of Legendre coefficients (standard basis)
  double coef[256] = {0};   // phi = sum coef_k P_k on [-1, 1]
  double chi = 0.0;         // prolate characteristic value
};
int prolate_series(double c, ProlateSeries* out);
double series_phi(const ProlateSeries& s, double x);
double series_dphi(const ProlateSeries& s, double x);
double series_int0(const ProlateSeries& s, double x);   // int_0^x phi

}  // namespace dmk
