// Single-level PSWF Ewald sum for the periodic 3D Stokeslet (components = ALL
// of a periodic plan): the "fast Ewald version" of the paper's Sec. 8, faster
// than DMK for uniformly distributed points.
//
// Sec. 5.3, Eqs. (ewald_local), (ewald_far) with the one-level split at scale
// nu: u = u_local + u_far + u_self (+ u0, zero for the Stokeslet), where
//   u_local, u_self   the near pass on a uniform tree at level L (every pair
//                     scale nu_ts = nu = 2^-(L+1), the self term at nu);
//   u_far(x_t)        = sum_{k in 2 pi Z^3, k != 0} S-hat_M(k) rho-hat(k) e^{i k.x_t},
//   S-hat_M(k)        = (k^2 I - k k^T) gamma-hat(|k| nu) / |k|^4      (Eqs. (moll_stokeslet),
//                       (generalbiharkdefs), gamma-hat of Eq. (gammaB_in_phi)),
//   rho-hat(k)        = sum_s f_s e^{-i k.x_s}.
// The Fourier sum is cut at |k_i| <= 2 pi m_max, m_max = ceil(1.1 c / (2 pi nu)):
// beyond |k| nu ~ c the window's gamma-hat falls to the level of phi(1) ~ eps
// (the edge of the truncated window), and the dropped tail changes the total
// far below eps.
//
// rho-hat and the sum over k are evaluated by a non-uniform FFT (spread the
// forces onto a uniform grid of n_g^3 points with a compact kernel psi, FFT,
// divide by psi-hat, multiply, inverse FFT, divide by psi-hat, interpolate with
// psi).  psi is the "exponential of semicircle" kernel of Barnett, Magland and
// af Klinteberg (SIAM J. Sci. Comput. 41, 2019), psi(x) = exp(beta (sqrt(1 -
// (x/alpha)^2) - 1)) for |x| < alpha = w h / 2, with w = ceil(log10(1/eps)) + 1
// grid points per direction, beta = 2.30 w, and a grid of at least twice the
// kept modes per direction (upsampling 2).  With h the grid spacing,
//   rho-hat(k) ~ h^3 B-hat[m] / psi-hat(k),   u(x_t) ~ h^3 sum_g psi(x_t - x_g) u~[g],
//   u~ = inverse FFT of S-hat_M rho-hat / psi-hat,
// so the per-mode factor is gamma-hat / (|k|^4 psi-hat^2) h^6 (precomputed per
// plan), the 3x3 tensor applied per mode.  The FFTs are cuFFT (plain library
// transforms); spreading, the per-mode product and interpolation are kernels
// here, all in FP64.
#include <cufft.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace dmk {

namespace {

const char* cufft_msg(cufftResult r) {
  switch (r) {
    case CUFFT_ALLOC_FAILED: return "cuFFT allocation failed";
    case CUFFT_INVALID_VALUE: return "cuFFT invalid value";
    case CUFFT_EXEC_FAILED: return "cuFFT execution failed";
    case CUFFT_SETUP_FAILED: return "cuFFT setup failed";
    case CUFFT_INVALID_SIZE: return "cuFFT invalid size";
    default: return "cuFFT error";
  }
}
#define DMK_CUFFT_TRY(expr)                                                                            \
  do {                                                                                                 \
    cufftResult _r = (expr);                                                                           \
    if (_r != CUFFT_SUCCESS)                                                                           \
      throw ::dmk::Error{_r == CUFFT_ALLOC_FAILED ? DMK_ERR_NOMEM : DMK_ERR_CUDA,                      \
                         std::string(#expr) + ": " + cufft_msg(_r)};                                   \
  } while (0)

// smallest even n >= lo whose prime factors are 2, 3, 5, 7
int fft_size(int lo) {
  for (int n = std::max(lo, 8);; ++n) {
    if (n & 1) continue;
    int m = n;
    for (int p : {2, 3, 5, 7})
      while (m % p == 0) m /= p;
    if (m == 1) return n;
  }
}

}  // namespace

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

namespace {

// ---------------------------------------------------------------- kernels
// ES kernel weights of one coordinate: the w grid points g0 .. g0 + w - 1
// nearest x (periodic), values psi((g h - x)), g0 = ceil(x / h - w / 2)
__device__ __forceinline__ int es_weights(double x, int ng, int w, double beta, double* wt) {
  const double t = x * ng - 0.5 * w;
  const int g0 = static_cast<int>(ceil(t));
  const double inv_half = 2.0 / w;
  for (int j = 0; j < w; ++j) {
    const double z = (g0 + j - x * ng) * inv_half;   // (g h - x) / alpha
    const double s = 1.0 - z * z;
    wt[j] = s > 0.0 ? exp(beta * (sqrt(s) - 1.0)) : 0.0;
  }
  return g0;
}

constexpr int kMaxW = 16;

// one thread per source (sorted order): its force spread onto the 3 grids
__global__ void k_ewald_spread(int64_t N, const double* __restrict__ wpos, const int32_t* __restrict__ perm,
                               const double* __restrict__ f, int ng, int w, double beta, double* __restrict__ grid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double wx[kMaxW], wy[kMaxW], wz[kMaxW];
  const int gx = es_weights(wpos[i], ng, w, beta, wx);
  const int gy = es_weights(wpos[N + i], ng, w, beta, wy);
  const int gz = es_weights(wpos[2 * N + i], ng, w, beta, wz);
  const int64_t o = perm[i];
  const double f0 = f[o * 3], f1 = f[o * 3 + 1], f2 = f[o * 3 + 2];
  const int64_t plane = static_cast<int64_t>(ng) * ng * ng;
  for (int a = 0; a < w; ++a) {
    const int ix = ((gx + a) % ng + ng) % ng;
    for (int b = 0; b < w; ++b) {
      const int iy = ((gy + b) % ng + ng) % ng;
      const double wab = wx[a] * wy[b];
      const int64_t row = (static_cast<int64_t>(ix) * ng + iy) * ng;
      for (int c = 0; c < w; ++c) {
        const int iz = ((gz + c) % ng + ng) % ng;
        const double v = wab * wz[c];
        atomicAdd(grid + row + iz, v * f0);
        atomicAdd(grid + plane + row + iz, v * f1);
        atomicAdd(grid + 2 * plane + row + iz, v * f2);
      }
    }
  }
}

// per-mode factor gamma-hat(|k| nu) h^6 / (|k|^4 psi-hat(k)^2) on the
// half spectrum (m1, m2 in [0, ng), m3 in [0, ng/2]), zero outside the kept
// modes and at k = 0
__global__ void k_ewald_mult(int ng, int mmax, const double* __restrict__ gtab, const double* __restrict__ psihat,
                             double h6, double* __restrict__ mult) {
  const int nh = ng / 2 + 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(ng) * ng * nh) return;
  const int m3 = static_cast<int>(i % nh);
  const int m2u = static_cast<int>((i / nh) % ng), m1u = static_cast<int>(i / (static_cast<int64_t>(nh) * ng));
  const int m1 = m1u <= ng / 2 ? m1u : m1u - ng, m2 = m2u <= ng / 2 ? m2u : m2u - ng;
  double v = 0.0;
  if (abs(m1) <= mmax && abs(m2) <= mmax && m3 <= mmax) {
    const int q = m1 * m1 + m2 * m2 + m3 * m3;
    if (q > 0) {
      const double k2 = 4.0 * M_PI * M_PI * q;
      const double ps = psihat[abs(m1)] * psihat[abs(m2)] * psihat[m3];
      v = gtab[q] * h6 / (k2 * k2 * ps * ps);
    }
  }
  mult[i] = v;
}

// U = mult (k^2 F - k (k.F)) per mode, the 3 components in place
__global__ void k_ewald_apply(int ng, const double* __restrict__ mult, cufftDoubleComplex* __restrict__ spec) {
  const int nh = ng / 2 + 1;
  const int64_t M = static_cast<int64_t>(ng) * ng * nh;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double s = mult[i];
  if (s == 0.0) {
    for (int a = 0; a < 3; ++a) spec[a * M + i] = make_cuDoubleComplex(0.0, 0.0);
    return;
  }
  const int m3 = static_cast<int>(i % nh);
  const int m2u = static_cast<int>((i / nh) % ng), m1u = static_cast<int>(i / (static_cast<int64_t>(nh) * ng));
  const double k[3] = {2.0 * M_PI * (m1u <= ng / 2 ? m1u : m1u - ng), 2.0 * M_PI * (m2u <= ng / 2 ? m2u : m2u - ng),
                       2.0 * M_PI * m3};
  const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  cufftDoubleComplex F[3];
  for (int a = 0; a < 3; ++a) F[a] = spec[a * M + i];
  const double kfr = k[0] * F[0].x + k[1] * F[1].x + k[2] * F[2].x;
  const double kfi = k[0] * F[0].y + k[1] * F[1].y + k[2] * F[2].y;
  for (int a = 0; a < 3; ++a)
    spec[a * M + i] = make_cuDoubleComplex(s * (k2 * F[a].x - k[a] * kfr), s * (k2 * F[a].y - k[a] * kfi));
}

// one thread per target (sorted order): u[caller] += sum_g psi(x_t - x_g) u~[g]
__global__ void k_ewald_interp(int64_t N, const double* __restrict__ wpos, const int32_t* __restrict__ perm,
                               int ng, int w, double beta, const double* __restrict__ grid, double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double wx[kMaxW], wy[kMaxW], wz[kMaxW];
  const int gx = es_weights(wpos[i], ng, w, beta, wx);
  const int gy = es_weights(wpos[N + i], ng, w, beta, wy);
  const int gz = es_weights(wpos[2 * N + i], ng, w, beta, wz);
  const int64_t plane = static_cast<int64_t>(ng) * ng * ng;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int a = 0; a < w; ++a) {
    const int ix = ((gx + a) % ng + ng) % ng;
    for (int b = 0; b < w; ++b) {
      const int iy = ((gy + b) % ng + ng) % ng;
      const double wab = wx[a] * wy[b];
      const int64_t row = (static_cast<int64_t>(ix) * ng + iy) * ng;
      for (int c = 0; c < w; ++c) {
        const int iz = ((gz + c) % ng + ng) % ng;
        const double v = wab * wz[c];
        s0 = fma(v, grid[row + iz], s0);
        s1 = fma(v, grid[plane + row + iz], s1);
        s2 = fma(v, grid[2 * plane + row + iz], s2);
      }
    }
  }
  const int64_t o = perm[i];
  u[o * 3] += s0;
  u[o * 3 + 1] += s1;
  u[o * 3 + 2] += s2;
}

}  // namespace

struct EwaldState {
  int L = 0, ng = 0, w = 0, mmax = 0;
  double nu = 0.0, beta = 0.0;
  double* grid = nullptr;                 // real grids [3][ng^3]
  cufftDoubleComplex* spec = nullptr;     // half spectra [3][ng ng (ng/2+1)]
  double* mult = nullptr;                 // per-mode factor [ng ng (ng/2+1)]
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
};

// Uniform tree level for the Ewald split: the smallest L >= 1 with at most
// ns points per box (ns = the plan's leaf capacity, default 4000), at most 4.
// Each level down costs 8x the grid of the Fourier part and saves 8x the
// near pairs; on GB300 the grid (FFTs, spreading traffic) costs more than the
// near pairs down to a few thousand points per box.
int ewald_level(int64_t N, int ns) {
  if (ns <= 0) ns = 4000;
  int L = 1;
  while (L < 4 && static_cast<double>(N) / std::ldexp(1.0, 3 * L) > ns) ++L;
  return L;
}

void ewald_setup(Plan& p, int L) {
  auto* E = new EwaldState();
  p.ewald = E;
  const double eps = p.opts.eps, c = p.tables.c;
  E->L = L;
  E->nu = std::ldexp(1.0, -(L + 1));
  E->mmax = static_cast<int>(std::ceil(1.1 * c / (2.0 * M_PI * E->nu)));
  E->ng = fft_size(2 * (2 * E->mmax + 1));
  E->w = std::min(kMaxW, static_cast<int>(std::ceil(-std::log10(eps))) + 1);
  E->beta = 2.30 * E->w;
  const int ng = E->ng, w = E->w, mmax = E->mmax;
  const double h = 1.0 / ng, alpha = 0.5 * w * h;
  // psi-hat(k) = alpha int_{-1}^{1} exp(beta (sqrt(1 - z^2) - 1)) cos(k alpha z) dz,
  // z = sin(theta) (smooth integrand), Gauss-Legendre in theta, k = 2 pi m
  std::vector<double> gx, gw;
  gauss_legendre(256, gx, gw);
  std::vector<double> psihat(ng / 2 + 1);
  for (int m = 0; m <= ng / 2; ++m) {
    const double k = 2.0 * M_PI * m;
    double s = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
      const double th = 0.5 * M_PI * gx[i];
      s += gw[i] * std::exp(E->beta * (std::cos(th) - 1.0)) * std::cos(k * alpha * std::sin(th)) * std::cos(th);
    }
    psihat[m] = alpha * 0.5 * M_PI * s;
  }
  // gamma-hat(kappa) = phi-hat - kappa phi-hat' / 2 = 2 int_0^1 phi(t) (cos(kappa t) + kappa t sin(kappa t) / 2) dt
  // at kappa = 2 pi sqrt(q) nu for every integer q = |m|^2 of the kept modes
  ProlateSeries ser;
  if (prolate_series(c, &ser) != 0) throw Error{DMK_ERR_CUDA, "prolate series failed"};
  std::vector<double> tx, tw;
  gauss_legendre(200, tx, tw);
  std::vector<double> phit(tx.size());
  for (size_t i = 0; i < tx.size(); ++i) phit[i] = series_phi(ser, 0.5 * (tx[i] + 1.0));
  const int qmax = 3 * mmax * mmax;
  std::vector<double> gtab(qmax + 1);
  for (int q = 0; q <= qmax; ++q) {
    const double kap = 2.0 * M_PI * std::sqrt(static_cast<double>(q)) * E->nu;
    double s = 0.0;
    for (size_t i = 0; i < tx.size(); ++i) {
      const double t = 0.5 * (tx[i] + 1.0);
      s += tw[i] * phit[i] * (std::cos(kap * t) + 0.5 * kap * t * std::sin(kap * t));
    }
    gtab[q] = s;                                       // 2 int_0^1 = sum with weights w_i / 2 * 2
  }
  if (std::fabs(gtab[0] - 1.0) > 1e-12) throw Error{DMK_ERR_CUDA, "window normalisation check failed"};
  cudaStream_t s = p.stream;
  const int nh = ng / 2 + 1;
  const int64_t cells = static_cast<int64_t>(ng) * ng * ng, modes = static_cast<int64_t>(ng) * ng * nh;
  E->grid = p.arena.alloc<double>(3 * cells);
  E->spec = p.arena.alloc<cufftDoubleComplex>(3 * modes);
  E->mult = p.arena.alloc<double>(modes);
  double* d_g = p.arena.alloc<double>(gtab.size());
  double* d_ps = p.arena.alloc<double>(psihat.size());
  DMK_CUDA_TRY(cudaMemcpyAsync(d_g, gtab.data(), gtab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  DMK_CUDA_TRY(cudaMemcpyAsync(d_ps, psihat.data(), psihat.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  const double h6 = std::pow(h, 6);
  k_ewald_mult<<<grid_for(modes, 256), 256, 0, s>>>(ng, mmax, d_g, d_ps, h6, E->mult);
  ++p.launches;
  DMK_CUDA_TRY(cudaGetLastError());
  int n3[3] = {ng, ng, ng};
  DMK_CUFFT_TRY(cufftPlanMany(&E->fwd, 3, n3, nullptr, 1, static_cast<int>(cells), nullptr, 1,
                              static_cast<int>(modes), CUFFT_D2Z, 3));
  E->have_fwd = true;
  DMK_CUFFT_TRY(cufftPlanMany(&E->inv, 3, n3, nullptr, 1, static_cast<int>(modes), nullptr, 1,
                              static_cast<int>(cells), CUFFT_Z2D, 3));
  E->have_inv = true;
  // the host tables above must outlive their copies
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
}

void ewald_free(Plan& p) {
  EwaldState* E = p.ewald;
  if (!E) return;
  if (E->have_fwd) cufftDestroy(E->fwd);
  if (E->have_inv) cufftDestroy(E->inv);
  delete E;                                            // device arrays live in the plan's arena
  p.ewald = nullptr;
}

void ewald_far(const Plan& p, const double* d_f, double* d_u, cudaStream_t s) {
  const EwaldState* E = p.ewald;
  const DeviceTree& T = p.tree;
  const int64_t N = T.N;
  if (!E || N == 0) return;
  const int ng = E->ng, nh = ng / 2 + 1;
  const int64_t cells = static_cast<int64_t>(ng) * ng * ng, modes = static_cast<int64_t>(ng) * ng * nh;
  DMK_CUDA_TRY(cudaMemsetAsync(E->grid, 0, 3 * cells * sizeof(double), s));
  k_ewald_spread<<<grid_for(N, 128), 128, 0, s>>>(N, T.w, T.perm, d_f, ng, E->w, E->beta, E->grid);
  DMK_CUDA_TRY(cudaGetLastError());
  DMK_CUFFT_TRY(cufftSetStream(E->fwd, s));
  DMK_CUFFT_TRY(cufftExecD2Z(E->fwd, E->grid, E->spec));
  k_ewald_apply<<<grid_for(modes, 256), 256, 0, s>>>(ng, E->mult, E->spec);
  DMK_CUDA_TRY(cudaGetLastError());
  DMK_CUFFT_TRY(cufftSetStream(E->inv, s));
  DMK_CUFFT_TRY(cufftExecZ2D(E->inv, E->spec, E->grid));
  k_ewald_interp<<<grid_for(N, 128), 128, 0, s>>>(N, T.w, T.perm, ng, E->w, E->beta, E->grid, d_u);
  DMK_CUDA_TRY(cudaGetLastError());
  p.launches += 3;
}

void ewald_info(const Plan& p, int32_t info[4]) {
  const EwaldState* E = p.ewald;
  info[0] = E ? E->L : 0;
  info[1] = E ? E->ng : 0;
  info[2] = E ? E->mmax : 0;
  info[3] = E ? E->w : 0;
}

}  // namespace dmk
