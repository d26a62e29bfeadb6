// DMK far field in 3D (components = ALL): proxy charges, plane-wave colleague
// interactions, the root kernel and interpolation down the tree.
//
// Sec. 6.1 Steps 1(c), 2, 3 and Sec. 6.2, with the parameters of Sec. 7 / Table 2:
//   * every box B of the tree (centre c_B, side r_l = 2^-l) carries a p x p x p
//     grid z = c_B + (r_l / 2) xi, xi the Chebyshev points of the first kind;
//   * upward pass: leaf proxy charges q_j = sum_s L_j(xi_s) rho_s (L the tensor
//     Lagrange basis, rho = f for the Stokeslet, the symmetric part of g (x) n
//     for the stresslet); a parent takes its children's charges through the
//     same basis;
//   * level-l plane waves, k = h m, h = 2 pi / (3 r_l), |m_i| <= M = (N1 - 1)/2:
//         O_B(m)  = K-hat_D,l(hm) . sum_j q_j e^{-i h m.(z_j - c_B)}      (outgoing, contracted)
//         I_B(m)  = sum_{colleagues C = B + delta} e^{-2 pi i m.delta/3} O_C(m)
//         pot_B  += Re (h / 2pi)^3 sum_m e^{i h m.(z - c_B)} I_B(m)
//     with K-hat_D,l the difference of the mollified kernels at r_{l+1} and
//     r_l (Eqs. (moll_stokeslet), (moll_stresslet)); every level uses the same
//     matrices because h (z - c_B) = pi xi / 3, and the kernel contraction is
//     applied to the outgoing side (the remark after Step 4);
//   * root: the periodic Fourier series of K_M,0 (Sec. 6.2, N_per modes a side)
//     or the truncated kernel of Eq. (Bmollhat_trunc) by the trapezoidal rule
//     (free space), plus K_corr = sum f / (4 pi R) for the free-space Stokeslet;
//   * downward pass: parents interpolate their potential grids to their
//     children; leaves evaluate their grids at their targets.
//
// GPU layout.  The box hierarchy and every job list are built on the host when
// the plan is made.  The separable tensor-product transforms (child merges,
// interpolation, outgoing and incoming plane waves, the root) all run in one
// kernel, k_rot, which contracts the slowest axis of a [n_in][rest] tensor with
// a small matrix and writes the result as [rest][n_out] (the contracted axis
// moves last, so three stages return the original axis order).  Spectra keep
// m_0 >= 0 only (the potential is real).  Arithmetic is FP32 when the plan's
// pair terms are FP32 (MIXED at eps >= 2e-7), FP64 otherwise; the target
// velocities are accumulated in FP64.
#include "common.cuh"
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <memory>
#include <unordered_map>
#include <vector>

namespace dmk {

namespace {

constexpr int kMaxP = 64;          // proxy order and mode counts a side (Table 2 needs <= 63)
constexpr int kRotTile = 32;       // rest columns per k_rot block
constexpr int kRotThreads = 256;
constexpr double kRTrunc = 2.7320508075688772;   // R = 1 + sqrt(3), Eq. (Btrunc_hat)

struct BoxGeo {
  double x, y, z, w;   // centre and half side, in-cell coordinates
};

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

// one stage of a separable transform: Y[r][m] (=, +=, = Re, += Re) sum_j A[m][j] X[j][r]
// over the job's one or two inputs (the second with the second matrix), r < rest
struct RotJob {
  int64_t x0, x1;   // element offsets into the launch's X base (x1 < 0: none; x0 < 0: zero input)
  int64_t y;        // element offset into the Y base
  int32_t a0, a1;   // matrix of each input (0 or 1)
};

// shared-memory sub-arrays of k_rot start on 16-byte boundaries
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ inline void rot_smem_layout(size_t bytesA, size_t bytesX, size_t* offX, size_t* offY) {
  *offX = align16(bytesA);
  *offY = *offX + align16(bytesX);
}

// MODE 0: write, 1: accumulate (for YC == false with complex arithmetic: the real part)
template <typename R, bool XC, bool AC, bool YC, int MODE>
__global__ void __launch_bounds__(kRotThreads) k_rot(const RotJob* __restrict__ jobs, const void* __restrict__ Xb,
                                                     void* __restrict__ Yb, int64_t xoff, int64_t yoff,
                                                     const void* __restrict__ A0, const void* __restrict__ A1,
                                                     int two_mats, int n_in, int n_out, int rest) {
  using C = typename Cplx<R>::T;
  using TX = typename std::conditional<XC, C, R>::type;
  using TA = typename std::conditional<AC, C, R>::type;
  using TY = typename std::conditional<YC, C, R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const RotJob J = jobs[blockIdx.x];
  const int r0 = blockIdx.y * kRotTile;
  if (r0 >= rest) return;
  const int ninp = J.x1 >= 0 ? 2 : 1;
  const int nmat = two_mats ? 2 : 1;
  size_t offX, offY;
  rot_smem_layout(nmat * n_out * n_in * sizeof(TA), 2 * n_in * kRotTile * sizeof(TX), &offX, &offY);
  TA* sA = reinterpret_cast<TA*>(smem);                                        // [nmat][n_out][n_in]
  TX* sX = reinterpret_cast<TX*>(smem + offX);                                 // [2][n_in][kRotTile]
  TY* sY = reinterpret_cast<TY*>(smem + offY);                                 // [kRotTile][n_out]
  for (int i = threadIdx.x; i < nmat * n_out * n_in; i += blockDim.x) {
    const int which = i / (n_out * n_in), e = i - which * n_out * n_in;
    sA[i] = (which == 0 ? static_cast<const TA*>(A0) : static_cast<const TA*>(A1))[e];
  }
  const int ncol = min(kRotTile, rest - r0);
  for (int k = 0; k < ninp; ++k) {
    const int64_t xo = (k == 0 ? J.x0 : J.x1);
    const TX* X = static_cast<const TX*>(Xb) + xoff + xo;
    for (int i = threadIdx.x; i < n_in * kRotTile; i += blockDim.x) {
      const int j = i / kRotTile, c = i - j * kRotTile;
      TX v;
      if constexpr (XC) {
        v.x = R(0);
        v.y = R(0);
      } else {
        v = R(0);
      }
      if (xo >= 0 && c < ncol) v = X[static_cast<int64_t>(j) * rest + r0 + c];
      sX[k * n_in * kRotTile + i] = v;
    }
  }
  __syncthreads();
  const int c = threadIdx.x & (kRotTile - 1);
  for (int m = threadIdx.x / kRotTile; m < n_out; m += blockDim.x / kRotTile) {
    R ar = R(0), ai = R(0);
    for (int k = 0; k < ninp; ++k) {
      const int am = (k == 0 ? J.a0 : J.a1);
      const TA* Am = sA + (am * n_out + m) * n_in;
      const TX* Xk = sX + k * n_in * kRotTile + c;
      for (int j = 0; j < n_in; ++j) {
        const TA a = Am[j];
        const TX x = Xk[j * kRotTile];
        if constexpr (AC && XC) {
          ar = fma(a.x, x.x, ar);
          ar = fma(-a.y, x.y, ar);
          ai = fma(a.x, x.y, ai);
          ai = fma(a.y, x.x, ai);
        } else if constexpr (AC) {
          ar = fma(a.x, x, ar);
          ai = fma(a.y, x, ai);
        } else if constexpr (XC) {
          ar = fma(a, x.x, ar);
          ai = fma(a, x.y, ai);
        } else {
          ar = fma(a, x, ar);
        }
      }
    }
    TY out;
    if constexpr (YC) {
      out.x = ar;
      out.y = ai;
    } else {
      out = ar;
    }
    sY[c * n_out + m] = out;
  }
  __syncthreads();
  TY* Y = static_cast<TY*>(Yb) + yoff + J.y + static_cast<int64_t>(r0) * n_out;
  for (int i = threadIdx.x; i < ncol * n_out; i += blockDim.x) {
    if constexpr (MODE == 1) {
      if constexpr (YC) {
        TY o = Y[i];
        o.x += sY[i].x;
        o.y += sY[i].y;
        Y[i] = o;
      } else {
        Y[i] += sY[i];
      }
    } else {
      Y[i] = sY[i];
    }
  }
}

// Lagrange basis at the Chebyshev points of the first kind in barycentric form
// (weights (-1)^j sin((2j+1) pi / 2p)); exact at a node
template <typename R>
__device__ inline void lagrange_row(double t, int p, const double* nodes, const double* bw, R* out, int stride = 1) {
  double s = 0.0;
  int hit = -1;
  for (int j = 0; j < p; ++j) {
    const double d = t - nodes[j];
    if (d == 0.0) hit = j;
    else s += bw[j] / d;
  }
  for (int j = 0; j < p; ++j) {
    double v;
    if (hit >= 0) v = (j == hit) ? 1.0 : 0.0;
    else v = (bw[j] / (t - nodes[j])) / s;
    out[j * stride] = static_cast<R>(v);
  }
}

// leaf proxy charges: q[box][slot+k][a][b][c] = sum_s L_a(x_s) L_b(y_s) L_c(z_s) v_s,k
// for the three components of group grp0 + blockIdx.y (0: f; 1: rho_00, rho_11,
// rho_22; 2: rho_01, rho_02, rho_12 of the symmetric part of g (x) n)
constexpr int kAntChunk = 32;
constexpr int kAntC = 8;
template <typename R>
__global__ void __launch_bounds__(256) k_far_anterp(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                    const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                                                    const double* __restrict__ w, int64_t N, const int32_t* __restrict__ perm,
                                                    const BoxGeo* __restrict__ box_geo, const double* __restrict__ f,
                                                    const double* __restrict__ g, const double* __restrict__ nrm, int grp0,
                                                    int slot_f, int slot_t, int ncomp, R* __restrict__ q, int p,
                                                    const double* __restrict__ nodes, const double* __restrict__ bw) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sW = reinterpret_cast<R*>(smem);                          // [3][kAntChunk][p]
  R* sV = sW + 3 * kAntChunk * p;                              // [kAntChunk][3]
  __shared__ double s_nodes[kMaxP], s_bw[kMaxP];
  const int li = leaf_list[blockIdx.x];
  const int box = leaf_box[blockIdx.x];
  const int grp = grp0 + blockIdx.y;
  const int slot = grp == 0 ? slot_f : slot_t + 3 * (grp - 1);
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  const BoxGeo geo = box_geo[box];                            // centre x, y, z, half side
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const int nchunk = (p + kAntC - 1) / kAntC;
  const int ntask = p * p * nchunk;
  const int64_t p3 = static_cast<int64_t>(p) * p * p;
  R* qb = q + (static_cast<int64_t>(box) * ncomp + slot) * p3;
  __syncthreads();
  for (int t0 = 0; t0 < ntask; t0 += blockDim.x) {
    const int task = t0 + threadIdx.x;
    const bool on = task < ntask;
    const int a = on ? task / (p * nchunk) : 0;
    const int rem = on ? task - a * p * nchunk : 0;
    const int b = rem / nchunk;
    const int c0 = (rem - b * nchunk) * kAntC;
    R acc[kAntC][3];
#pragma unroll
    for (int cc = 0; cc < kAntC; ++cc) acc[cc][0] = acc[cc][1] = acc[cc][2] = R(0);
    for (int sc = 0; sc < ns; sc += kAntChunk) {
      const int nc = min(kAntChunk, ns - sc);
      __syncthreads();
      for (int i = threadIdx.x; i < 3 * kAntChunk; i += blockDim.x) {
        const int ax = i / kAntChunk, sl = i - ax * kAntChunk;
        R* dst = sW + (ax * kAntChunk + sl) * p;
        if (sl < nc) {
          const int64_t si = s0 + sc + sl;
          const double ctr = ax == 0 ? geo.x : (ax == 1 ? geo.y : geo.z);
          lagrange_row<R>((w[ax * N + si] - ctr) / geo.w, p, s_nodes, s_bw, dst);
        } else {
          for (int j = 0; j < p; ++j) dst[j] = R(0);
        }
      }
      for (int sl = threadIdx.x; sl < kAntChunk; sl += blockDim.x) {
        double v0 = 0, v1 = 0, v2 = 0;
        if (sl < nc) {
          const int64_t o = perm[s0 + sc + sl];
          if (grp == 0) {
            v0 = f[o * 3];
            v1 = f[o * 3 + 1];
            v2 = f[o * 3 + 2];
          } else {
            const double g0 = g[o * 3], g1 = g[o * 3 + 1], g2 = g[o * 3 + 2];
            const double n0 = nrm[o * 3], n1 = nrm[o * 3 + 1], n2 = nrm[o * 3 + 2];
            if (grp == 1) {
              v0 = g0 * n0;
              v1 = g1 * n1;
              v2 = g2 * n2;
            } else {
              v0 = 0.5 * (g0 * n1 + g1 * n0);
              v1 = 0.5 * (g0 * n2 + g2 * n0);
              v2 = 0.5 * (g1 * n2 + g2 * n1);
            }
          }
        }
        sV[sl * 3] = static_cast<R>(v0);
        sV[sl * 3 + 1] = static_cast<R>(v1);
        sV[sl * 3 + 2] = static_cast<R>(v2);
      }
      __syncthreads();
      if (on) {
        for (int sl = 0; sl < nc; ++sl) {
          const R wab = sW[sl * p + a] * sW[(kAntChunk + sl) * p + b];
          const R* wc = sW + (2 * kAntChunk + sl) * p;
          const R f0 = sV[sl * 3], f1 = sV[sl * 3 + 1], f2 = sV[sl * 3 + 2];
#pragma unroll
          for (int cc = 0; cc < kAntC; ++cc) {
            const int ci = c0 + cc;
            const R wv = ci < p ? wab * wc[ci] : R(0);
            acc[cc][0] = fma(wv, f0, acc[cc][0]);
            acc[cc][1] = fma(wv, f1, acc[cc][1]);
            acc[cc][2] = fma(wv, f2, acc[cc][2]);
          }
        }
      }
    }
    if (on) {
#pragma unroll
      for (int cc = 0; cc < kAntC; ++cc) {
        const int ci = c0 + cc;
        if (ci < p)
          for (int k = 0; k < 3; ++k) qb[k * p3 + (static_cast<int64_t>(a) * p + b) * p + ci] = acc[cc][k];
      }
    }
  }
}

// kernel contraction of one proxy-charge component's spectrum rh (m_0 >= 0 half,
// layout [nh][nm][nm]) into the outgoing expansion O[box][3][modes]:
//   Stokeslet component l:      O_j += sS t (q delta_jl - m_j m_l) rh
//   stresslet component (l, n): O_j += i sT t [q (2 (G m)_j + m_j tr G) - 2 m_j (m.G.m)] rh
// with q = |m|^2, t = tab[q], G the basis tensor of the component, sS = h and
// sT = h^2 at level l (h = 2 pi 2^l / 3) or the root's factors
template <typename R>
__global__ void k_far_contract(int njob, const int32_t* __restrict__ job_box, const int32_t* __restrict__ box_level,
                               const typename Cplx<R>::T* __restrict__ rh, int64_t rh_stride,
                               typename Cplx<R>::T* __restrict__ O, int comp, int first, const R* __restrict__ tab,
                               double sS0, double sT0, int level_scaled, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  const int64_t modes = static_cast<int64_t>(nh) * nm * nm;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= njob * modes) return;
  const int jb = static_cast<int>(idx / modes);
  const int64_t mi = idx - jb * modes;
  const int box = job_box[jb];
  const int i1 = static_cast<int>(mi / (nm * nm));
  const int i2 = static_cast<int>((mi / nm) % nm);
  const int i3 = static_cast<int>(mi % nm);
  const R m[3] = {R(i1), R(i2 - Mh), R(i3 - Mh)};
  const int qi = i1 * i1 + (i2 - Mh) * (i2 - Mh) + (i3 - Mh) * (i3 - Mh);
  double h = 1.0;
  if (level_scaled) h = 2.0 * M_PI / 3.0 * static_cast<double>(1 << box_level[box]);
  const R t = tab[qi];
  const R q = R(qi);
  const C x = rh[jb * rh_stride + mi];
  R cr[3], ci[3];                     // O_j += (cr_j + i ci_j) x
  if (comp < 3) {
    const R s = static_cast<R>(sS0 * h) * t;
    for (int j = 0; j < 3; ++j) {
      cr[j] = s * ((j == comp ? q : R(0)) - m[j] * m[comp]);
      ci[j] = R(0);
    }
  } else {
    const R s = static_cast<R>(sT0 * h * h) * t;
    const int c = comp - 3;
    for (int j = 0; j < 3; ++j) {
      R v;
      if (c < 3) {          // diagonal (c, c)
        v = q * (R(2) * (j == c ? m[c] : R(0)) + m[j]) - R(2) * m[j] * m[c] * m[c];
      } else {              // off-diagonal (l, n)
        const int l = c == 3 ? 0 : (c == 4 ? 0 : 1);
        const int n = c == 3 ? 1 : 2;
        v = R(2) * q * ((j == l ? m[n] : R(0)) + (j == n ? m[l] : R(0))) - R(4) * m[j] * m[l] * m[n];
      }
      cr[j] = R(0);
      ci[j] = s * v;
    }
  }
  C* Ob = O + static_cast<int64_t>(box) * 3 * modes + mi;
  for (int j = 0; j < 3; ++j) {
    C add;
    add.x = cr[j] * x.x - ci[j] * x.y;
    add.y = cr[j] * x.y + ci[j] * x.x;
    if (first) {
      Ob[j * modes] = add;
    } else {
      C o = Ob[j * modes];
      o.x += add.x;
      o.y += add.y;
      Ob[j * modes] = o;
    }
  }
}

// incoming expansions: I[tb][k][m] = sum over the 27 colleague slots of
// e^{-2 pi i m.delta / 3} O[colleague][k][m]  (slot s: delta_a = ((s / 3^a) % 3) - 1)
template <typename R>
__global__ void k_far_colleague(int ntb, const int32_t* __restrict__ coll, const typename Cplx<R>::T* __restrict__ O,
                                typename Cplx<R>::T* __restrict__ I, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  const int64_t modes = static_cast<int64_t>(nh) * nm * nm;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(ntb) * 3 * modes) return;
  const int tb = static_cast<int>(idx / (3 * modes));
  const int64_t rem = idx - static_cast<int64_t>(tb) * 3 * modes;
  const int k = static_cast<int>(rem / modes);
  const int64_t mi = rem - k * modes;
  const int m0 = static_cast<int>(mi / (nm * nm));
  const int m1 = static_cast<int>((mi / nm) % nm) - Mh;
  const int m2 = static_cast<int>(mi % nm) - Mh;
  const R c120 = R(-0.5), s120 = R(0.86602540378443864676);
  R sr = 0, si = 0;
  for (int s = 0; s < 27; ++s) {
    const int cb = coll[tb * 27 + s];
    if (cb < 0) continue;
    const int d0 = s % 3 - 1, d1 = (s / 3) % 3 - 1, d2 = s / 9 - 1;
    int e = (m0 * d0 + m1 * d1 + m2 * d2) % 3;
    if (e < 0) e += 3;
    const C o = O[(static_cast<int64_t>(cb) * 3 + k) * modes + mi];
    if (e == 0) {
      sr += o.x;
      si += o.y;
    } else {
      // e^{-2 pi i e / 3}: e = 1 -> (-1/2, -sqrt3/2), e = 2 -> (-1/2, +sqrt3/2)
      const R sn = e == 1 ? -s120 : s120;
      sr += c120 * o.x - sn * o.y;
      si += c120 * o.y + sn * o.x;
    }
  }
  C r;
  r.x = sr;
  r.y = si;
  I[idx] = r;
}

// free-space Stokeslet constant K_corr sum_s f_s = (1 / 4 pi R) sum_j q_root,j
// (the Lagrange basis sums to one) added to the root potential grid
template <typename R>
__global__ void k_far_corr(const R* __restrict__ q_root, int slot_f, R* __restrict__ pot_root, int64_t p3) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < p3; i += blockDim.x) s += static_cast<double>(q_root[(slot_f + k) * p3 + i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const R add = static_cast<R>(red[0] / (4.0 * M_PI * kRTrunc));
  for (int64_t i = threadIdx.x; i < p3; i += blockDim.x) pot_root[k * p3 + i] += add;
}

// leaf evaluation: u[caller][k] += sum_abc L_a(x) L_b(y) L_c(z) pot[box][k][a][b][c]
// (one thread per target; the leaf's grid is read slab by slab through shared memory)
constexpr int kEvThreads = 128;
template <typename R>
__global__ void __launch_bounds__(kEvThreads) k_far_eval(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                         const int32_t* __restrict__ t_start, const int32_t* __restrict__ t_count,
                                                         const double* __restrict__ tw,
                                                         int64_t NT, const int32_t* __restrict__ tperm,
                                                         const BoxGeo* __restrict__ box_geo, const R* __restrict__ pot, int p,
                                                         const double* __restrict__ nodes, const double* __restrict__ bw,
                                                         double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sL = reinterpret_cast<R*>(smem);                    // [3][p][kEvThreads]
  R* sP = sL + 3 * p * kEvThreads;                       // [3][p][p] slab of the grid
  __shared__ double s_nodes[kMaxP], s_bw[kMaxP];
  const int li = leaf_list[blockIdx.x];
  const int box = leaf_box[blockIdx.x];
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  const BoxGeo geo = box_geo[box];
  const int t0 = t_start[li], nt = t_count ? t_count[li] : t_start[li + 1] - t0;
  const int64_t p2 = static_cast<int64_t>(p) * p, p3 = p2 * p;
  const R* P = pot + static_cast<int64_t>(box) * 3 * p3;
  __syncthreads();
  for (int base = 0; base < nt; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const bool on = t < nt;
    if (on) {
      for (int ax = 0; ax < 3; ++ax) {
        const double ctr = ax == 0 ? geo.x : (ax == 1 ? geo.y : geo.z);
        lagrange_row<R>((tw[ax * NT + t0 + t] - ctr) / geo.w, p, s_nodes, s_bw, sL + ax * p * kEvThreads + threadIdx.x,
                        kEvThreads);
      }
    }
    R acc0 = 0, acc1 = 0, acc2 = 0;
    for (int a = 0; a < p; ++a) {
      __syncthreads();
      for (int i = threadIdx.x; i < 3 * p2; i += blockDim.x) {
        const int k = static_cast<int>(i / p2);
        const int64_t e = i - k * p2;
        sP[i] = P[k * p3 + a * p2 + e];
      }
      __syncthreads();
      if (on) {
        const R la = sL[(0 * p + a) * kEvThreads + threadIdx.x];
        for (int b = 0; b < p; ++b) {
          const R lab = la * sL[(1 * p + b) * kEvThreads + threadIdx.x];
          const R* row = sP + b * p;
          R r0 = 0, r1 = 0, r2 = 0;
          for (int c = 0; c < p; ++c) {
            const R lc = sL[(2 * p + c) * kEvThreads + threadIdx.x];
            r0 = fma(lc, row[c], r0);
            r1 = fma(lc, row[p2 + c], r1);
            r2 = fma(lc, row[2 * p2 + c], r2);
          }
          acc0 = fma(lab, r0, acc0);
          acc1 = fma(lab, r1, acc1);
          acc2 = fma(lab, r2, acc2);
        }
      }
    }
    if (on) {
      const int64_t o = tperm[t0 + t];
      u[o * 3] += static_cast<double>(acc0);
      u[o * 3 + 1] += static_cast<double>(acc1);
      u[o * 3 + 2] += static_cast<double>(acc2);
    }
  }
}

// ------------------------------------------------------------------ host side
// gamma-hat(kappa) = 2 int_0^1 phi(t) (cos(kappa t) + kappa t sin(kappa t) / 2) dt
// (Eq. (gammaB_in_phi)), Gauss-Legendre on [0, 1]
struct GammaHat {
  std::vector<double> t, wphi;
  explicit GammaHat(double c) {
    ProlateSeries ser;
    if (prolate_series(c, &ser) != 0) throw Error{DMK_ERR_CUDA, "prolate series failed"};
    std::vector<double> x, w;
    gauss_legendre(256, x, w);
    t.resize(x.size());
    wphi.resize(x.size());
    for (size_t i = 0; i < x.size(); ++i) {
      t[i] = 0.5 * (x[i] + 1.0);
      wphi[i] = w[i] * series_phi(ser, t[i]);       // 2 * (1/2) w_i phi(t_i)
    }
  }
  double operator()(double kap) const {
    double s = 0.0;
    for (size_t i = 0; i < t.size(); ++i) s += wphi[i] * (std::cos(kap * t[i]) + 0.5 * kap * t[i] * std::sin(kap * t[i]));
    return s;
  }
};

// B-hat^R(k) in 3D, Eq. (Btrunc_hat); Taylor series of the bracket near k = 0
double b_trunc_hat(double k) {
  const double x = k * kRTrunc;
  if (x > 1e-2) return (1.0 + 0.5 * std::cos(x) - 1.5 * std::sin(x) / x) / (k * k * k * k);
  const double R4 = kRTrunc * kRTrunc * kRTrunc * kRTrunc;
  return R4 * (1.0 / 120.0 - x * x / 2520.0 + x * x * x * x / 120960.0);
}

// Table 2 columns and the rules that reproduce them: N1 = 2 (3c/pi) - 1, N_per = 2 floor(c / 2pi) + 1;
// p interpolated linearly in log10 eps between the rows and rounded up
int table2_p(double eps, int kernels) {
  static const double e_rows[4] = {-12, -9, -6, -3};
  static const double p_s[4] = {44, 33, 23, 12}, p_t[4] = {44, 33, 22, 11};
  const double e = std::log10(eps);
  auto interp = [&](const double* v) {
    for (int i = 0; i < 3; ++i)
      if (e >= e_rows[i] - 1e-9 && e <= e_rows[i + 1] + 1e-9) {
        const double tt = (e - e_rows[i]) / (e_rows[i + 1] - e_rows[i]);
        return static_cast<int>(std::ceil(v[i] + tt * (v[i + 1] - v[i]) - 1e-9));
      }
    return static_cast<int>(v[0]);
  };
  int p = 0;
  if (kernels & DMK_KERNEL_STOKESLET) p = std::max(p, interp(p_s));
  if (kernels & DMK_KERNEL_STRESSLET) p = std::max(p, interp(p_t));
  return p;
}

struct RotLaunch {
  RotJob* jobs = nullptr;   // device
  int n = 0;
};

template <typename T>
T* upload(Plan& p, const std::vector<T>& v) {
  T* d = p.arena.alloc<T>(std::max<size_t>(v.size(), 1));
  if (!v.empty()) DMK_CUDA_TRY(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p.stream));
  return d;
}

}  // namespace

struct FarState {
  int fp32 = 1;
  int p = 0, M = 0, nh = 0, nm = 0;           // level modes: m_0 in [0, M], m_1, m_2 in [-M, M]
  int rK = 0, rnh = 0, rnm = 0;               // root modes
  int ncomp = 0, slot_f = -1, slot_t = -1;
  int nbox = 0, maxlev = 0, nsrc_box = 0, ntrg_box = 0;
  int nsrc_leaf = 0, ntrg_leaf = 0;
  int64_t p3 = 0, modes = 0, rmodes = 0, scr_stride = 0;   // scratch stride in complex elements
  double sT_root = 1.0;
  // device arrays
  BoxGeo* box_geo = nullptr;
  int32_t* box_level = nullptr;
  double* nodes = nullptr;
  double* bw = nullptr;
  int32_t* src_leaf = nullptr;       // [nsrc_leaf] leaf index, then box id at + nsrc_leaf
  int32_t* trg_leaf = nullptr;
  int32_t* src_box_list = nullptr;   // boxes with sources (outgoing jobs order)
  int32_t* coll = nullptr;           // [ntrg_box][27]
  int32_t* root_box = nullptr;       // {0}
  void* mats = nullptr;              // matrix bank
  size_t m_T0 = 0, m_T1 = 0, m_T0t = 0, m_T1t = 0, m_Eh = 0, m_E = 0, m_Fh = 0, m_F = 0;
  size_t m_REh = 0, m_RE = 0, m_RFh = 0, m_RF = 0, m_tab = 0, m_rtab = 0;
  // big buffers (stream-ordered allocations)
  void* q = nullptr;                 // [nbox][ncomp][p^3] R
  void* pot = nullptr;               // [nbox][3][p^3] R
  void* O = nullptr;                 // [nbox][3][modes] C
  void* I = nullptr;                 // [ntrg_box][3][modes] C
  void* s1 = nullptr;                // scratch [max jobs][scr_stride] C
  void* s2 = nullptr;
  void* rO = nullptr;                // root outgoing [3][rmodes] C
  // job lists
  std::vector<RotLaunch> merge[3];   // per level (index = parent level), 3 stages
  std::vector<int> merge_level;
  std::vector<RotLaunch> interp[3];
  std::vector<int> interp_level;
  RotLaunch out1, out2, out3, ev1, ev2, ev3, r1, r2, r3, rv1, rv2, rv3;
  size_t bytes = 0;
};

namespace {

size_t elem_r(const FarState& F) { return F.fp32 ? sizeof(float) : sizeof(double); }

template <typename R>
void launch_rot_t(const FarState& F, const RotLaunch& L, const void* X, void* Y, int64_t xoff, int64_t yoff,
                  size_t matA0, size_t matA1, bool two_mats, int n_in, int n_out, int rest, int xc, int ac, int yc,
                  int mode, cudaStream_t s) {
  if (L.n == 0) return;
  using C = typename Cplx<R>::T;
  const size_t sa = ac ? sizeof(C) : sizeof(R), sx = xc ? sizeof(C) : sizeof(R), sy = yc ? sizeof(C) : sizeof(R);
  size_t offX, offY;
  rot_smem_layout((two_mats ? 2 : 1) * n_out * n_in * sa, 2 * n_in * kRotTile * sx, &offX, &offY);
  const size_t shm = offY + kRotTile * n_out * sy;
  const dim3 grid(L.n, (rest + kRotTile - 1) / kRotTile);
  const char* base = static_cast<const char*>(F.mats);
  const void* A0 = base + matA0;
  const void* A1 = base + matA1;
  const int tm = two_mats ? 1 : 0;
#define DMK_ROT(XC_, AC_, YC_, MODE_)                                                                         \
  do {                                                                                                        \
    auto kern = k_rot<R, XC_, AC_, YC_, MODE_>;                                                               \
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm))); \
    kern<<<grid, kRotThreads, shm, s>>>(L.jobs, X, Y, xoff, yoff, A0, A1, tm, n_in, n_out, rest);            \
  } while (0)
  if (!xc && !ac && !yc && mode == 0) DMK_ROT(false, false, false, 0);
  else if (!xc && !ac && !yc && mode == 1) DMK_ROT(false, false, false, 1);
  else if (!xc && ac && yc && mode == 0) DMK_ROT(false, true, true, 0);
  else if (xc && ac && yc && mode == 0) DMK_ROT(true, true, true, 0);
  else if (xc && ac && !yc && mode == 0) DMK_ROT(true, true, false, 0);
  else if (xc && ac && !yc && mode == 1) DMK_ROT(true, true, false, 1);
  else throw Error{DMK_ERR_CUDA, "unsupported transform stage"};
#undef DMK_ROT
  DMK_CUDA_TRY(cudaGetLastError());
}

void launch_rot(const Plan& p, const RotLaunch& L, const void* X, void* Y, int64_t xoff, int64_t yoff, size_t A0,
                size_t A1, bool two, int n_in, int n_out, int rest, int xc, int ac, int yc, int mode, cudaStream_t s) {
  const FarState& F = *p.far;
  if (L.n == 0) return;
  if (F.fp32) launch_rot_t<float>(F, L, X, Y, xoff, yoff, A0, A1, two, n_in, n_out, rest, xc, ac, yc, mode, s);
  else launch_rot_t<double>(F, L, X, Y, xoff, yoff, A0, A1, two, n_in, n_out, rest, xc, ac, yc, mode, s);
  ++p.launches;
}

RotLaunch make_launch(Plan& p, const std::vector<RotJob>& jobs) {
  RotLaunch L;
  L.n = static_cast<int>(jobs.size());
  if (L.n) L.jobs = upload(p, jobs);
  return L;
}

}  // namespace

void far_setup(Plan& p) {
  const DeviceTree& T = p.tree;
  const dmk_stokes_opts_t& o = p.opts;
  cudaStream_t s = p.stream;
  auto Fp = std::make_unique<FarState>();
  FarState& F = *Fp;
  F.fp32 = fp32_pair_terms(o) ? 1 : 0;
  const double c = p.tables.c;
  const int tcp = static_cast<int>(std::lround(3.0 * c / M_PI));
  F.p = table2_p(o.eps, o.kernels);
  if (o.bandlimit > 0) F.p = std::max(F.p, static_cast<int>(std::ceil(1.3 * tcp)));
  F.M = tcp - 1;                                   // N1 = 2 (3c/pi) - 1 modes a side
  F.nh = F.M + 1;
  F.nm = 2 * F.M + 1;
  if (F.p > kMaxP || F.nm > kMaxP) throw Error{DMK_ERR_UNSUPPORTED, "far-field order beyond the compiled maximum"};
  F.p3 = static_cast<int64_t>(F.p) * F.p * F.p;
  F.modes = static_cast<int64_t>(F.nh) * F.nm * F.nm;
  const bool wS = o.kernels & DMK_KERNEL_STOKESLET, wT = o.kernels & DMK_KERNEL_STRESSLET;
  F.slot_f = wS ? 0 : -1;
  F.slot_t = wT ? (wS ? 3 : 0) : -1;
  F.ncomp = (wS ? 3 : 0) + (wT ? 6 : 0);
  const double h0 = 2.0 * M_PI / (2.0 + 2.0 * std::sqrt(3.0));
  if (o.periodic) {
    F.rK = static_cast<int>(std::floor(c / (2.0 * M_PI)));   // N_per = 2 rK + 1
  } else {
    F.rK = static_cast<int>(std::ceil(c / h0)) + 1;          // |k_i| <= c + h0 (and a little beyond)
  }
  F.rnh = F.rK + 1;
  F.rnm = 2 * F.rK + 1;
  if (F.rnm > kMaxP) throw Error{DMK_ERR_UNSUPPORTED, "root mode count beyond the compiled maximum"};
  F.rmodes = static_cast<int64_t>(F.rnh) * F.rnm * F.rnm;

  // ---- box hierarchy from the leaves -------------------------------------------
  const int nl = T.n_leaf;
  std::vector<int32_t> lev(nl), cnt(nl), tst;
  std::vector<uint64_t> anc(nl);
  DMK_CUDA_TRY(cudaMemcpyAsync(lev.data(), T.leaf_level, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DMK_CUDA_TRY(cudaMemcpyAsync(cnt.data(), T.leaf_count, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DMK_CUDA_TRY(cudaMemcpyAsync(anc.data(), T.leaf_anchor, nl * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  if (T.sep) {
    tst.resize(nl + 1);
    DMK_CUDA_TRY(cudaMemcpyAsync(tst.data(), T.leaf_tstart, (nl + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> tcnt(nl);
  for (int i = 0; i < nl; ++i) tcnt[i] = T.sep ? tst[i + 1] - tst[i] : cnt[i];
  int maxlev = 0;
  for (int i = 0; i < nl; ++i) maxlev = std::max(maxlev, lev[i]);
  F.maxlev = maxlev;
  struct Box {
    int lev;
    int64_t c[3];
    uint64_t key;     // Morton key at its level
    int leaf = -1;
    int64_t src = 0, trg = 0;
    int child[8];
  };
  std::vector<std::unordered_map<uint64_t, int>> at(maxlev + 1);
  std::vector<Box> boxes;
  auto find_or_add = [&](int l, const int64_t* cc) {
    const uint64_t key = morton<3>(cc);
    auto it = at[l].find(key);
    if (it != at[l].end()) return it->second;
    Box b;
    b.lev = l;
    for (int a = 0; a < 3; ++a) b.c[a] = cc[a];
    b.key = key;
    for (int k = 0; k < 8; ++k) b.child[k] = -1;
    boxes.push_back(b);
    const int id = static_cast<int>(boxes.size()) - 1;
    at[l][key] = id;
    return id;
  };
  for (int i = 0; i < nl; ++i) {
    int64_t cc[3];
    leaf_coords<3>(anc[i], lev[i], T.M, cc);
    for (int l = lev[i]; l >= 0; --l) {
      int64_t ca[3] = {cc[0] >> (lev[i] - l), cc[1] >> (lev[i] - l), cc[2] >> (lev[i] - l)};
      const int id = find_or_add(l, ca);
      if (l == lev[i]) {
        boxes[id].leaf = i;
        boxes[id].src = cnt[i];
        boxes[id].trg = tcnt[i];
      }
    }
  }
  // order: by level, Morton within a level
  std::vector<int> order(boxes.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return boxes[a].lev != boxes[b].lev ? boxes[a].lev < boxes[b].lev : boxes[a].key < boxes[b].key;
  });
  std::vector<int> newid(boxes.size());
  for (size_t i = 0; i < order.size(); ++i) newid[order[i]] = static_cast<int>(i);
  {
    std::vector<Box> sorted(boxes.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = boxes[order[i]];
    boxes.swap(sorted);
    for (auto& m : at)
      for (auto& kv : m) kv.second = newid[kv.second];
  }
  const int nb = static_cast<int>(boxes.size());
  F.nbox = nb;
  // children and subtree counts (bottom-up)
  for (int i = nb - 1; i >= 0; --i) {
    Box& b = boxes[i];
    if (b.lev == 0) continue;
    int64_t pc[3] = {b.c[0] >> 1, b.c[1] >> 1, b.c[2] >> 1};
    const int par = at[b.lev - 1].at(morton<3>(pc));
    const int ch = static_cast<int>((b.c[0] & 1) | ((b.c[1] & 1) << 1) | ((b.c[2] & 1) << 2));
    boxes[par].child[ch] = i;
    boxes[par].src += b.src;
    boxes[par].trg += b.trg;
  }
  for (int i = 0; i < nb; ++i)
    if (boxes[i].leaf < 0)
      for (int k = 0; k < 8; ++k)
        if (boxes[i].child[k] < 0) throw Error{DMK_ERR_CUDA, "far field: incomplete box hierarchy"};
  // lists
  std::vector<int32_t> src_leaf, src_leaf_box, trg_leaf, trg_leaf_box, src_boxes, trg_boxes;
  std::vector<int> trg_index(nb, -1);
  for (int i = 0; i < nb; ++i) {
    const Box& b = boxes[i];
    if (b.src > 0) src_boxes.push_back(i);
    if (b.trg > 0) {
      trg_index[i] = static_cast<int>(trg_boxes.size());
      trg_boxes.push_back(i);
    }
    if (b.leaf >= 0 && b.src > 0) {
      src_leaf.push_back(b.leaf);
      src_leaf_box.push_back(i);
    }
    if (b.leaf >= 0 && b.trg > 0) {
      trg_leaf.push_back(b.leaf);
      trg_leaf_box.push_back(i);
    }
  }
  F.nsrc_box = static_cast<int>(src_boxes.size());
  F.ntrg_box = static_cast<int>(trg_boxes.size());
  F.nsrc_leaf = static_cast<int>(src_leaf.size());
  F.ntrg_leaf = static_cast<int>(trg_leaf.size());
  std::vector<int32_t> coll(static_cast<size_t>(F.ntrg_box) * 27, -1);
  for (int t = 0; t < F.ntrg_box; ++t) {
    const Box& b = boxes[trg_boxes[t]];
    const int64_t n = int64_t(1) << b.lev;
    for (int sl = 0; sl < 27; ++sl) {
      const int d[3] = {sl % 3 - 1, (sl / 3) % 3 - 1, sl / 9 - 1};
      int64_t cc[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        cc[a] = b.c[a] + d[a];
        if (o.periodic) cc[a] = ((cc[a] % n) + n) % n;
        else if (cc[a] < 0 || cc[a] >= n) ok = false;
      }
      if (!ok) continue;
      auto it = at[b.lev].find(morton<3>(cc));
      if (it == at[b.lev].end() || boxes[it->second].src == 0) continue;
      coll[static_cast<size_t>(t) * 27 + sl] = it->second;
    }
  }
  std::vector<BoxGeo> geo(nb);
  std::vector<int32_t> blev(nb);
  for (int i = 0; i < nb; ++i) {
    const double r = std::ldexp(1.0, -boxes[i].lev);
    geo[i] = BoxGeo{(boxes[i].c[0] + 0.5) * r, (boxes[i].c[1] + 0.5) * r, (boxes[i].c[2] + 0.5) * r, 0.5 * r};
    blev[i] = boxes[i].lev;
  }

  // ---- matrices and tables -------------------------------------------------------
  const int P = F.p;
  std::vector<double> nodes(P), bwt(P);
  for (int j = 0; j < P; ++j) {
    const double th = (2.0 * j + 1.0) * M_PI / (2.0 * P);
    nodes[j] = std::cos(th);
    bwt[j] = ((j & 1) ? -1.0 : 1.0) * std::sin(th);
  }
  auto lag = [&](double t, int j) {       // plain Lagrange product (host)
    double v = 1.0;
    for (int k = 0; k < P; ++k)
      if (k != j) v *= (t - nodes[k]) / (nodes[j] - nodes[k]);
    return v;
  };
  const bool f32 = F.fp32;
  std::vector<char> bank;
  auto put_real = [&](const std::vector<double>& v) {
    const size_t off = (bank.size() + 15) & ~size_t(15);
    bank.resize(off + v.size() * (f32 ? 4 : 8));
    for (size_t i = 0; i < v.size(); ++i) {
      if (f32) reinterpret_cast<float*>(bank.data() + off)[i] = static_cast<float>(v[i]);
      else reinterpret_cast<double*>(bank.data() + off)[i] = v[i];
    }
    return off;
  };
  auto put_cplx = [&](const std::vector<double>& re, const std::vector<double>& im) {
    const size_t off = (bank.size() + 15) & ~size_t(15);
    bank.resize(off + re.size() * (f32 ? 8 : 16));
    for (size_t i = 0; i < re.size(); ++i) {
      if (f32) {
        reinterpret_cast<float*>(bank.data() + off)[2 * i] = static_cast<float>(re[i]);
        reinterpret_cast<float*>(bank.data() + off)[2 * i + 1] = static_cast<float>(im[i]);
      } else {
        reinterpret_cast<double*>(bank.data() + off)[2 * i] = re[i];
        reinterpret_cast<double*>(bank.data() + off)[2 * i + 1] = im[i];
      }
    }
    return off;
  };
  // child -> parent anterpolation T_o[a][i] = L_a(((2o - 1) + xi_i) / 2), and the transposes
  for (int oo = 0; oo < 2; ++oo) {
    std::vector<double> Tm(P * P), Tt(P * P);
    for (int a = 0; a < P; ++a)
      for (int i = 0; i < P; ++i) {
        const double v = lag(((2 * oo - 1) + nodes[i]) / 2.0, a);
        Tm[a * P + i] = v;
        Tt[i * P + a] = v;
      }
    (oo == 0 ? F.m_T0 : F.m_T1) = put_real(Tm);
    (oo == 0 ? F.m_T0t : F.m_T1t) = put_real(Tt);
  }
  // plane-wave matrices: E[m][j] = e^{-i theta m xi_j}; F[a][m] = w_m e^{+i theta m xi_a}
  auto pw = [&](int lo, int n, double theta, bool eval, bool half, size_t* outm) {
    std::vector<double> re(static_cast<size_t>(n) * P), im(re.size());
    for (int mi = 0; mi < n; ++mi)
      for (int j = 0; j < P; ++j) {
        const int m = lo + mi;
        const double ph = theta * m * nodes[j];
        const double wgt = (eval && half && m > 0) ? 2.0 : 1.0;
        const size_t e = eval ? static_cast<size_t>(j) * n + mi : static_cast<size_t>(mi) * P + j;
        re[e] = wgt * std::cos(ph);
        im[e] = (eval ? 1.0 : -1.0) * wgt * std::sin(ph);
      }
    *outm = put_cplx(re, im);
  };
  const double th_l = M_PI / 3.0;
  pw(0, F.nh, th_l, false, true, &F.m_Eh);
  pw(-F.M, F.nm, th_l, false, false, &F.m_E);
  pw(0, F.nh, th_l, true, true, &F.m_Fh);
  pw(-F.M, F.nm, th_l, true, false, &F.m_F);
  const double th_r = o.periodic ? M_PI : 0.5 * h0;
  pw(0, F.rnh, th_r, false, true, &F.m_REh);
  pw(-F.rK, F.rnm, th_r, false, false, &F.m_RE);
  pw(0, F.rnh, th_r, true, true, &F.m_RFh);
  pw(-F.rK, F.rnm, th_r, true, false, &F.m_RF);
  // kernel tables by q = |m|^2
  GammaHat gh(c);
  {
    const int qmax = 3 * F.M * F.M;
    std::vector<double> tab(qmax + 1, 0.0);
    for (int q = 1; q <= qmax; ++q) {
      const double am = std::sqrt(static_cast<double>(q));
      const double dg = gh(M_PI * am / 3.0) - gh(2.0 * M_PI * am / 3.0);
      tab[q] = dg / (8.0 * M_PI * M_PI * M_PI * static_cast<double>(q) * q);
    }
    F.m_tab = put_real(tab);
    const int rq = 3 * F.rK * F.rK;
    std::vector<double> rt(rq + 1, 0.0);
    for (int q = 0; q <= rq; ++q) {
      const double am = std::sqrt(static_cast<double>(q));
      if (o.periodic) {
        if (q > 0) rt[q] = gh(2.0 * M_PI * am) / (4.0 * M_PI * M_PI * static_cast<double>(q) * q);
      } else {
        const double k = h0 * am;
        rt[q] = std::pow(h0 / (2.0 * M_PI), 3) * h0 * h0 * b_trunc_hat(k) * gh(k);
      }
    }
    F.m_rtab = put_real(rt);
    F.sT_root = o.periodic ? 2.0 * M_PI : h0;
    if (std::fabs(gh(0.0) - 1.0) > 1e-12) throw Error{DMK_ERR_CUDA, "window normalisation check failed"};
  }
  F.mats = p.arena.alloc<char>(bank.size());
  DMK_CUDA_TRY(cudaMemcpyAsync(F.mats, bank.data(), bank.size(), cudaMemcpyHostToDevice, s));
  F.nodes = upload(p, nodes);
  F.bw = upload(p, bwt);
  F.box_geo = upload(p, geo);
  F.box_level = upload(p, blev);
  {
    std::vector<int32_t> sl(src_leaf);
    sl.insert(sl.end(), src_leaf_box.begin(), src_leaf_box.end());
    F.src_leaf = upload(p, sl);
    std::vector<int32_t> tl(trg_leaf);
    tl.insert(tl.end(), trg_leaf_box.begin(), trg_leaf_box.end());
    F.trg_leaf = upload(p, tl);
  }
  F.src_box_list = upload(p, src_boxes);
  F.coll = upload(p, coll);
  F.root_box = upload(p, std::vector<int32_t>{0});

  // ---- scratch strides and job lists ---------------------------------------------------
  const int64_t p2 = static_cast<int64_t>(P) * P;
  const int nh = F.nh, nm = F.nm;
  int64_t st = 0;
  for (int64_t v : {p2 * nh, int64_t(P) * nh * nm, int64_t(nh) * nm * nm, int64_t(nm) * nm * P, int64_t(nm) * P * P,
                    p2 * F.rnh, int64_t(P) * F.rnh * F.rnm, int64_t(F.rnh) * F.rnm * F.rnm, int64_t(F.rnm) * F.rnm * P,
                    int64_t(F.rnm) * P * P})
    st = std::max(st, v);
  F.scr_stride = st;
  const int64_t P3 = F.p3;
  const int nc = F.ncomp;
  int64_t max_jobs = std::max<int64_t>(std::max(F.nsrc_box, F.ntrg_box), 1);
  // merges: parent at level l (non-leaf, with sources), per component
  for (int l = maxlev - 1; l >= 0; --l) {
    std::vector<RotJob> j1, j2, j3;
    int np = 0;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.src == 0) continue;
      for (int k = 0; k < nc; ++k) {
        const int64_t slotbase = (static_cast<int64_t>(np) * nc + k);      // per (parent, comp)
        for (int o12 = 0; o12 < 4; ++o12) {                                 // (o1, o2), stage 1 over o0
          const int c0 = b.child[0 | (o12 << 1)], c1 = b.child[1 | (o12 << 1)];
          RotJob J;
          J.x0 = boxes[c0].src ? (static_cast<int64_t>(c0) * nc + k) * P3 : -1;
          J.x1 = boxes[c1].src ? (static_cast<int64_t>(c1) * nc + k) * P3 : -1;
          if (J.x0 < 0 && J.x1 >= 0) {          // keep the zero input as x1
            J.x0 = J.x1;
            J.x1 = -1;
            J.a0 = 1;
            J.a1 = 0;
          } else {
            J.a0 = 0;
            J.a1 = 1;
          }
          if (J.x0 < 0) J.x0 = -1;
          J.y = (slotbase * 4 + o12) * P3;                                  // real elements in s1
          j1.push_back(J);
        }
        for (int o2 = 0; o2 < 2; ++o2) {
          RotJob J;
          J.x0 = (slotbase * 4 + (0 | (o2 << 1))) * P3;
          J.x1 = (slotbase * 4 + (1 | (o2 << 1))) * P3;
          J.a0 = 0;
          J.a1 = 1;
          J.y = (slotbase * 2 + o2) * P3;                                   // s2
          j2.push_back(J);
        }
        RotJob J;
        J.x0 = (slotbase * 2 + 0) * P3;
        J.x1 = (slotbase * 2 + 1) * P3;
        J.a0 = 0;
        J.a1 = 1;
        J.y = (static_cast<int64_t>(i) * nc + k) * P3;                      // q of the parent
        j3.push_back(J);
      }
      ++np;
    }
    if (np == 0) continue;
    F.merge_level.push_back(l);
    F.merge[0].push_back(make_launch(p, j1));
    F.merge[1].push_back(make_launch(p, j2));
    F.merge[2].push_back(make_launch(p, j3));
    max_jobs = std::max<int64_t>(max_jobs, (static_cast<int64_t>(np) * nc * 4 * P3 + 2 * st - 1) / (2 * st) + 1);
  }
  // interpolation: parent at level l (non-leaf, with targets) to its children with targets
  for (int l = 0; l < maxlev; ++l) {
    std::vector<RotJob> j1, j2, j3;
    int np = 0;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.trg == 0) continue;
      for (int k = 0; k < 3; ++k) {
        const int64_t slotbase = static_cast<int64_t>(np) * 3 + k;
        for (int o0 = 0; o0 < 2; ++o0) {
          RotJob J;
          J.x0 = (static_cast<int64_t>(i) * 3 + k) * P3;                    // pot of the parent
          J.x1 = -1;
          J.a0 = o0;
          J.a1 = 0;
          J.y = (slotbase * 2 + o0) * P3;                                   // s1
          j1.push_back(J);
        }
        for (int o01 = 0; o01 < 4; ++o01) {
          RotJob J;
          J.x0 = (slotbase * 2 + (o01 & 1)) * P3;
          J.x1 = -1;
          J.a0 = o01 >> 1;
          J.a1 = 0;
          J.y = (slotbase * 4 + o01) * P3;                                  // s2
          j2.push_back(J);
        }
        for (int ch = 0; ch < 8; ++ch) {
          const int cb = b.child[ch];
          if (boxes[cb].trg == 0) continue;
          RotJob J;
          J.x0 = (slotbase * 4 + (ch & 3)) * P3;
          J.x1 = -1;
          J.a0 = ch >> 2;
          J.a1 = 0;
          J.y = (static_cast<int64_t>(cb) * 3 + k) * P3;                    // pot of the child (+=)
          j3.push_back(J);
        }
      }
      ++np;
    }
    if (np == 0) continue;
    F.interp_level.push_back(l);
    F.interp[0].push_back(make_launch(p, j1));
    F.interp[1].push_back(make_launch(p, j2));
    F.interp[2].push_back(make_launch(p, j3));
    max_jobs = std::max<int64_t>(max_jobs, (static_cast<int64_t>(np) * 3 * 4 * P3 + 2 * st - 1) / (2 * st) + 1);
  }
  // outgoing: one job per source box (the component is the launch offset); eval: per target box
  {
    std::vector<RotJob> a1, a2, a3, e1, e2, e3;
    for (int jb = 0; jb < F.nsrc_box; ++jb) {
      const int b = src_boxes[jb];
      RotJob J;
      J.x1 = -1;
      J.a0 = 0;
      J.a1 = 0;
      J.x0 = static_cast<int64_t>(b) * nc * P3;
      J.y = jb * st;
      a1.push_back(J);
      J.x0 = jb * st;
      a2.push_back(J);
      a3.push_back(J);
    }
    for (int tb = 0; tb < F.ntrg_box; ++tb) {
      const int b = trg_boxes[tb];
      RotJob J;
      J.x1 = -1;
      J.a0 = 0;
      J.a1 = 0;
      J.x0 = static_cast<int64_t>(tb) * 3 * F.modes;
      J.y = tb * st;
      e1.push_back(J);
      J.x0 = tb * st;
      e2.push_back(J);
      J.y = static_cast<int64_t>(b) * 3 * P3;
      e3.push_back(J);
    }
    F.out1 = make_launch(p, a1);
    F.out2 = make_launch(p, a2);
    F.out3 = make_launch(p, a3);
    F.ev1 = make_launch(p, e1);
    F.ev2 = make_launch(p, e2);
    F.ev3 = make_launch(p, e3);
    RotJob J;
    J.x1 = -1;
    J.a0 = J.a1 = 0;
    J.x0 = 0;
    J.y = 0;
    std::vector<RotJob> one{J};
    F.r1 = make_launch(p, one);                 // x: q[root] (+ component offset)
    F.r2 = make_launch(p, one);
    F.r3 = make_launch(p, one);
    F.rv1 = make_launch(p, one);
    F.rv2 = make_launch(p, one);
    F.rv3 = make_launch(p, one);                // y: pot[root] (+ component offset), accumulate
  }
  // ---- big buffers -------------------------------------------------------------------
  const size_t er = elem_r(F), ec = 2 * er;
  auto big = [&](size_t bytes) {
    void* ptr = nullptr;
    DMK_CUDA_TRY(cudaMallocAsync(&ptr, std::max<size_t>(bytes, 256), s));
    F.bytes += bytes;
    return ptr;
  };
  F.q = big(static_cast<size_t>(nb) * nc * P3 * er);
  F.pot = big(static_cast<size_t>(nb) * 3 * P3 * er);
  F.O = big(static_cast<size_t>(nb) * 3 * F.modes * ec);
  F.I = big(static_cast<size_t>(std::max(F.ntrg_box, 1)) * 3 * F.modes * ec);
  F.s1 = big(static_cast<size_t>(max_jobs) * st * ec);
  F.s2 = big(static_cast<size_t>(max_jobs) * st * ec);
  F.rO = big(static_cast<size_t>(3) * F.rmodes * ec);
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  p.far = Fp.release();
}

void far_free(Plan& p) {
  FarState* F = p.far;
  if (!F) return;
  for (void** b : {&F->q, &F->pot, &F->O, &F->I, &F->s1, &F->s2, &F->rO})
    if (*b) cudaFreeAsync(*b, p.stream);
  delete F;                                   // small arrays live in the plan's arena
  p.far = nullptr;
}

size_t far_bytes(const Plan& p) { return p.far ? p.far->bytes : 0; }

namespace {

template <typename R>
void far_run_t(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u, cudaStream_t s) {
  using C = typename Cplx<R>::T;
  const FarState& F = *p.far;
  const DeviceTree& T = p.tree;
  const int P = F.p, nc = F.ncomp;
  const int64_t P3 = F.p3, p2 = static_cast<int64_t>(P) * P;
  const int nh = F.nh, nm = F.nm;
  const int64_t st = F.scr_stride;
  R* q = static_cast<R*>(F.q);
  R* pot = static_cast<R*>(F.pot);
  C* O = static_cast<C*>(F.O);
  C* I = static_cast<C*>(F.I);
  const char* mats = static_cast<const char*>(F.mats);
  // 1. leaf proxy charges
  if (F.nsrc_leaf > 0) {
    const size_t shm = (3 * kAntChunk * P + 3 * kAntChunk) * sizeof(R);
    auto kern = k_far_anterp<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    const int g0 = F.slot_f >= 0 ? 0 : 1;
    const int ng = (F.slot_f >= 0 ? 1 : 0) + (F.slot_t >= 0 ? 2 : 0);
    kern<<<dim3(F.nsrc_leaf, ng), 256, shm, s>>>(F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start, T.leaf_count, T.w,
                                                 T.N, T.perm, F.box_geo, d_f, d_g, d_n, g0, F.slot_f, F.slot_t, nc, q, P,
                                                 F.nodes, F.bw);
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
  }
  // 2. upward merges, finest parents first
  for (size_t i = 0; i < F.merge_level.size(); ++i) {
    launch_rot(p, F.merge[0][i], q, F.s1, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.merge[1][i], F.s1, F.s2, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.merge[2][i], F.s2, q, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
  }
  // 3. outgoing plane waves of every box with sources, contracted with the level kernel
  const R* tab = reinterpret_cast<const R*>(mats + F.m_tab);
  for (int k = 0; k < nc; ++k) {
    launch_rot(p, F.out1, q, F.s1, k * P3, 0, F.m_Eh, F.m_Eh, false, P, nh, static_cast<int>(p2), 0, 1, 1, 0, s);
    launch_rot(p, F.out2, F.s1, F.s2, 0, 0, F.m_E, F.m_E, false, P, nm, P * nh, 1, 1, 1, 0, s);
    launch_rot(p, F.out3, F.s2, F.s1, 0, 0, F.m_E, F.m_E, false, P, nm, nh * nm, 1, 1, 1, 0, s);
    const int comp = (F.slot_f >= 0 && k < 3) ? k : 3 + (k - (F.slot_t));
    const int64_t tot = static_cast<int64_t>(F.nsrc_box) * F.modes;
    k_far_contract<R><<<grid_for(tot, 256), 256, 0, s>>>(F.nsrc_box, F.src_box_list, F.box_level,
                                                         static_cast<const C*>(F.s1), st, O, comp, k == 0 ? 1 : 0, tab,
                                                         1.0, 1.0, 1, F.M, nh, nm);
    DMK_CUDA_TRY(cudaGetLastError());
    p.launches += 1;
  }
  // 4. incoming expansions (colleague sums) and their potential grids (written)
  {
    const int64_t tot = static_cast<int64_t>(F.ntrg_box) * 3 * F.modes;
    if (tot > 0) {
      k_far_colleague<R><<<grid_for(tot, 256), 256, 0, s>>>(F.ntrg_box, F.coll, O, I, F.M, nh, nm);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
    for (int k = 0; k < 3; ++k) {
      launch_rot(p, F.ev1, I, F.s1, k * F.modes, 0, F.m_Fh, F.m_Fh, false, nh, P, nm * nm, 1, 1, 1, 0, s);
      launch_rot(p, F.ev2, F.s1, F.s2, 0, 0, F.m_F, F.m_F, false, nm, P, nm * P, 1, 1, 1, 0, s);
      launch_rot(p, F.ev3, F.s2, pot, 0, k * P3, F.m_F, F.m_F, false, nm, P, static_cast<int>(p2), 1, 1, 0, 0, s);
    }
  }
  // 5. root: K_M,0 (periodic series or truncated free-space kernel) added to the root grid
  if (F.ntrg_box > 0 && F.nsrc_box > 0) {
    const int rnh = F.rnh, rnm = F.rnm;
    const R* rtab = reinterpret_cast<const R*>(mats + F.m_rtab);
    C* rO = static_cast<C*>(F.rO);
    for (int k = 0; k < nc; ++k) {
      launch_rot(p, F.r1, q, F.s1, k * P3, 0, F.m_REh, F.m_REh, false, P, rnh, static_cast<int>(p2), 0, 1, 1, 0, s);
      launch_rot(p, F.r2, F.s1, F.s2, 0, 0, F.m_RE, F.m_RE, false, P, rnm, P * rnh, 1, 1, 1, 0, s);
      launch_rot(p, F.r3, F.s2, F.s1, 0, 0, F.m_RE, F.m_RE, false, P, rnm, rnh * rnm, 1, 1, 1, 0, s);
      const int comp = (F.slot_f >= 0 && k < 3) ? k : 3 + (k - (F.slot_t));
      k_far_contract<R><<<grid_for(F.rmodes, 256), 256, 0, s>>>(1, F.root_box, F.box_level, static_cast<const C*>(F.s1),
                                                                st, rO, comp, k == 0 ? 1 : 0, rtab, 1.0, F.sT_root, 0,
                                                                F.rK, rnh, rnm);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
    for (int k = 0; k < 3; ++k) {
      launch_rot(p, F.rv1, rO, F.s1, k * F.rmodes, 0, F.m_RFh, F.m_RFh, false, rnh, P, rnm * rnm, 1, 1, 1, 0, s);
      launch_rot(p, F.rv2, F.s1, F.s2, 0, 0, F.m_RF, F.m_RF, false, rnm, P, rnm * P, 1, 1, 1, 0, s);
      launch_rot(p, F.rv3, F.s2, pot, 0, k * P3, F.m_RF, F.m_RF, false, rnm, P, static_cast<int>(p2), 1, 1, 0, 1, s);
    }
    if (!p.opts.periodic && F.slot_f >= 0) {
      k_far_corr<R><<<3, 256, 0, s>>>(q, F.slot_f, pot, P3);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
  }
  // 6. interpolation down the tree
  for (size_t i = 0; i < F.interp_level.size(); ++i) {
    launch_rot(p, F.interp[0][i], pot, F.s1, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.interp[1][i], F.s1, F.s2, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.interp[2][i], F.s2, pot, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 1, s);
  }
  // 7. leaf grids at the targets
  if (F.ntrg_leaf > 0) {
    const size_t shm = (3 * static_cast<size_t>(P) * kEvThreads + 3 * p2) * sizeof(R);
    auto kern = k_far_eval<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    if (T.sep)
      kern<<<F.ntrg_leaf, kEvThreads, shm, s>>>(F.trg_leaf, F.trg_leaf + F.ntrg_leaf, T.leaf_tstart, nullptr, T.tw, T.NT,
                                                T.tperm, F.box_geo, pot, P, F.nodes, F.bw, d_u);
    else
      kern<<<F.ntrg_leaf, kEvThreads, shm, s>>>(F.trg_leaf, F.trg_leaf + F.ntrg_leaf, T.leaf_start, T.leaf_count, T.w, T.N,
                                                T.perm, F.box_geo, pot, P, F.nodes, F.bw, d_u);
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
  }
}

}  // namespace

void far_run(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u, cudaStream_t s) {
  if (!p.far || !d_u || p.tree.N == 0) return;
  if (p.far->fp32) far_run_t<float>(p, d_f, d_g, d_n, d_u, s);
  else far_run_t<double>(p, d_f, d_g, d_n, d_u, s);
}

void far_info(const Plan& p, int32_t info[8]) {
  for (int i = 0; i < 8; ++i) info[i] = 0;
  const FarState* F = p.far;
  if (!F) return;
  info[0] = F->p;
  info[1] = 2 * F->M + 1;
  info[2] = F->rnm;
  info[3] = F->nbox;
  info[4] = F->nsrc_box;
  info[5] = F->ntrg_box;
  info[6] = F->maxlev;
  info[7] = F->fp32;
}

}  // namespace dmk
