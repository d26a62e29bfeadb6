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
// interpolation, outgoing and incoming plane waves, the root) run in the generic
// kernel k_rot, which contracts the slowest axis of a [n_in][rest] tensor with a
// small matrix and writes the result as [rest][n_out] (the contracted axis moves
// last, so three stages return the original axis order), or, in float32, in
// kernels that keep one box's (or one parent's) stages in shared memory.  Spectra
// keep m_0 >= 0 only (the potential is real).  Arithmetic is FP32 when the plan's
// pair terms are FP32 (MIXED at eps >= 2e-7), FP64 otherwise; in FP32 the two
// per-point contractions (leaf charges, leaf evaluation) run on the tcgen05
// tensor cores with split-TF32 products (tc.cuh).  The target velocities are
// accumulated in FP64.
#include "far_common.cuh"
#include "tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <type_traits>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

namespace dmk {

using namespace farc;

namespace {

constexpr int kRotTile = 64;       // rest columns per k_rot block
constexpr int kRotThreads = 256;
constexpr double kRTrunc = 2.7320508075688772;   // R = 1 + sqrt(3), Eq. (Btrunc_hat)

// one stage of a separable transform: Y[r][m] (=, +=) sum_j A[m][j] X[j][r] over the
// job's one or two inputs (the second with the second matrix), r < rest; complex
// arithmetic when X or A is complex, and the real part kept when Y is real
struct RotJob {
  int64_t x0, x1;   // element offsets into the launch's X base (x1 < 0: none; x0 < 0: zero input)
  int64_t y;        // element offset into the Y base
  int32_t a0, a1;   // matrix of each input (0 or 1)
};

// shared memory of k_rot: A transposed [nmat][n_in][n4] (n4 = n_out rounded up to 4,
// zero padded), X [nmat][n_in][kRotTile], Y [kRotTile][n_out]; each part 16-byte aligned
__host__ __device__ inline void rot_smem_layout(size_t bytesA, size_t bytesX, size_t* offX, size_t* offY) {
  *offX = align16(bytesA);
  *offY = *offX + align16(bytesX);
}


// MODE 0: write, 1: accumulate.  Each thread owns a 4 x 4 register tile: four
// consecutive columns r and four consecutive rows m; blockDim = 16 * (n4 / 4)
// rounded up to a warp multiple.
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
  const int nmat = two_mats ? 2 : 1;
  const int ninp = (J.x1 >= 0 && two_mats) ? 2 : 1;
  const int n4 = (n_out + 3) & ~3;
  size_t offX, offY;
  rot_smem_layout(nmat * n_in * n4 * sizeof(TA), nmat * n_in * kRotTile * sizeof(TX), &offX, &offY);
  TA* sA = reinterpret_cast<TA*>(smem);                                        // [nmat][n_in][n4]
  TX* sX = reinterpret_cast<TX*>(smem + offX);                                 // [nmat][n_in][kRotTile]
  TY* sY = reinterpret_cast<TY*>(smem + offY);                                 // [kRotTile][n_out]
  for (int i = threadIdx.x; i < nmat * n_in * n4; i += blockDim.x) {
    const int which = i / (n_in * n4), e = i - which * n_in * n4;
    const int j = e / n4, m = e - j * n4;
    TA v{};
    if (m < n_out) v = (which == 0 ? static_cast<const TA*>(A0) : static_cast<const TA*>(A1))[m * n_in + j];
    sA[i] = v;
  }
  const int ncol = min(kRotTile, rest - r0);
  for (int k = 0; k < ninp; ++k) {
    const int64_t xo = (k == 0 ? J.x0 : J.x1);
    const TX* X = static_cast<const TX*>(Xb) + xoff + xo;
    for (int i = threadIdx.x; i < n_in * kRotTile; i += blockDim.x) {
      const int j = i / kRotTile, c = i - j * kRotTile;
      TX v{};
      if (xo >= 0 && c < ncol) v = X[static_cast<int64_t>(j) * rest + r0 + c];
      sX[k * n_in * kRotTile + i] = v;
    }
  }
  __syncthreads();
  const int cq = threadIdx.x & 15, mc = threadIdx.x >> 4;
  if (mc < n4 / 4) {
    R ar[4][4], ai[4][4];        // [column][row]
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) ar[u][i] = ai[u][i] = R(0);
    for (int k = 0; k < ninp; ++k) {
      const int am = (k == 0 ? J.a0 : J.a1);
      const TA* Ak = sA + am * n_in * n4 + 4 * mc;
      const TX* Xk = sX + k * n_in * kRotTile + 4 * cq;
      for (int j = 0; j < n_in; ++j) {
        TA a[4];
        TX x[4];
        ld4(Ak + j * n4, a);
        ld4(Xk + j * kRotTile, x);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if constexpr (AC && XC) {
              ar[u][i] = fma(a[i].x, x[u].x, ar[u][i]);
              ar[u][i] = fma(-a[i].y, x[u].y, ar[u][i]);
              ai[u][i] = fma(a[i].x, x[u].y, ai[u][i]);
              ai[u][i] = fma(a[i].y, x[u].x, ai[u][i]);
            } else if constexpr (AC) {
              ar[u][i] = fma(a[i].x, x[u], ar[u][i]);
              ai[u][i] = fma(a[i].y, x[u], ai[u][i]);
            } else if constexpr (XC) {
              ar[u][i] = fma(a[i], x[u].x, ar[u][i]);
              ai[u][i] = fma(a[i], x[u].y, ai[u][i]);
            } else {
              ar[u][i] = fma(a[i], x[u], ar[u][i]);
            }
          }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = 4 * mc + i, c = 4 * cq + u;
        if (m < n_out) {
          TY out;
          if constexpr (YC) {
            out.x = ar[u][i];
            out.y = ai[u][i];
          } else {
            out = ar[u][i];
          }
          sY[c * n_out + m] = out;
        }
      }
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


// padded proxy order: the Lagrange rows and grid rows of the leaf kernels are PB
// long (zeros past p), PB a multiple of the c-chunk of the anterpolation (24 in
// float32, 12 in float64)
template <typename R> constexpr int ant_chunk() { return sizeof(R) == 4 ? 24 : 12; }
constexpr int kAntChunk = 64;
constexpr int kAntThreads = 320;

// Lagrange weights of every point of the listed leaves, once per evaluation:
// W[s][axis][PB] in sorted point order.  A thread forms one row (s, axis) with one
// reciprocal per node (L_j = (w_j / d_j) / sum_k w_k / d_k, exact at a node) into a
// shared-memory tile of kWRows rows; the tile then leaves in consecutive addresses
// (a leaf's rows are contiguous in W).
constexpr int kWRows = 256;
template <typename R>
__global__ void __launch_bounds__(kWRows) k_far_weights(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                        const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                                                        const double* __restrict__ w, int64_t N, const BoxGeo* __restrict__ box_geo,
                                                        int p, int PB, const R* __restrict__ nodes, const R* __restrict__ bw,
                                                        R* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sRow = reinterpret_cast<R*>(smem);                    // [kWRows][PB + 1]
  __shared__ R s_nodes[kMaxP], s_bw[kMaxP];
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  const int li = leaf_list[blockIdx.x];
  const BoxGeo geo = box_geo[leaf_box[blockIdx.x]];
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const double inv_half = 1.0 / geo.w;             // a power of two
  const int ld = PB + 1;
  R* Wl = W + static_cast<int64_t>(s0) * 3 * PB;
  for (int r0 = blockIdx.y * kWRows; r0 < 3 * ns; r0 += gridDim.y * kWRows) {   // a leaf's tiles over blockIdx.y
    const int nr = min(kWRows, 3 * ns - r0);
    __syncthreads();                               // nodes loaded; the previous tile written out
    if (threadIdx.x < nr) {
      const int row = r0 + threadIdx.x;
      const int sl = row / 3, ax = row - 3 * sl;
      const double ctr = ax == 0 ? geo.x : (ax == 1 ? geo.y : geo.z);
      const R t = static_cast<R>((w[ax * N + s0 + sl] - ctr) * inv_half);
      R* out = sRow + threadIdx.x * ld;
      R sum = R(0);
      int hit = -1;
      for (int j = 0; j < p; ++j) {
        const R d = t - s_nodes[j];
        R v = R(0);
        if (d == R(0)) hit = j;
        else v = s_bw[j] * recip<R>(d);
        out[j] = v;
        sum += v;
      }
      const R inv = hit >= 0 ? R(0) : recip<R>(sum);
      for (int j = 0; j < PB; ++j) out[j] = j < p ? (hit >= 0 ? (j == hit ? R(1) : R(0)) : out[j] * inv) : R(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * PB; i += blockDim.x) {
      const int r = i / PB, c = i - r * PB;
      Wl[static_cast<int64_t>(r0) * PB + i] = sRow[r * ld + c];
    }
  }
}

// leaf proxy charges: q[box][slot+k][a][b][c] = sum_s L_a(x_s) L_b(y_s) L_c(z_s) v_s,k
// for the three components of group grp0 + blockIdx.y (0: f; 1: rho_00, rho_11,
// rho_22; 2: rho_01, rho_02, rho_12 of the symmetric part of g (x) n).  A thread owns
// one (a, b) and a chunk of consecutive c; the leaf's weights stream through shared
// memory 32 sources at a time.
template <typename R>
__global__ void __launch_bounds__(kAntThreads, 2) k_far_anterp(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                            const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                                                            const R* __restrict__ W, const int32_t* __restrict__ perm,
                                                            const double* __restrict__ f, const double* __restrict__ g,
                                                            const double* __restrict__ nrm, int grp0, int slot_f, int slot_t,
                                                            int ncomp, R* __restrict__ q, int p, int PB) {
  constexpr int CB = ant_chunk<R>();
  extern __shared__ __align__(16) unsigned char smem[];
  R* sW = reinterpret_cast<R*>(smem);                          // [kAntChunk][3][PB]
  R* sV = sW + kAntChunk * 3 * PB;                             // [kAntChunk][4]
  const int li = leaf_list[blockIdx.x];
  const int box = leaf_box[blockIdx.x];
  const int grp = grp0 + blockIdx.y;
  const int slot = grp == 0 ? slot_f : slot_t + 3 * (grp - 1);
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const int nchunk = PB / CB;
  const int ntask = p * p * nchunk;
  const int64_t p3 = static_cast<int64_t>(p) * p * p;
  R* qb = q + (static_cast<int64_t>(box) * ncomp + slot) * p3;
  for (int t0 = blockIdx.z * blockDim.x; t0 < ntask; t0 += gridDim.z * blockDim.x) {
    const int task = t0 + threadIdx.x;
    const bool on = task < ntask;
    const int a = on ? task / (p * nchunk) : 0;
    const int rem = on ? task - a * p * nchunk : 0;
    const int b = rem / nchunk;
    const int c0 = (rem - b * nchunk) * CB;
    R acc[CB][3];
#pragma unroll
    for (int cc = 0; cc < CB; ++cc) acc[cc][0] = acc[cc][1] = acc[cc][2] = R(0);
    for (int sc = 0; sc < ns; sc += kAntChunk) {
      const int nc = min(kAntChunk, ns - sc);
      __syncthreads();
      const R* src = W + (static_cast<int64_t>(s0) + sc) * 3 * PB;
      for (int i = threadIdx.x; i < nc * 3 * PB; i += blockDim.x) sW[i] = src[i];
      for (int sl = threadIdx.x; sl < nc; sl += blockDim.x) {
        double v0, v1, v2;
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
        sV[sl * 4] = static_cast<R>(v0);
        sV[sl * 4 + 1] = static_cast<R>(v1);
        sV[sl * 4 + 2] = static_cast<R>(v2);
        sV[sl * 4 + 3] = R(0);
      }
      __syncthreads();
      if (on) {
        for (int sl = 0; sl < nc; ++sl) {
          const R* ws = sW + sl * 3 * PB;
          const R wab = ws[a] * ws[PB + b];
          R fv[4];
          ld4(sV + sl * 4, fv);
#pragma unroll
          for (int c4 = 0; c4 < CB / 4; ++c4) {
            R wc[4];
            ld4(ws + 2 * PB + c0 + 4 * c4, wc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const R wv = wab * wc[i];
              acc[4 * c4 + i][0] = fma(wv, fv[0], acc[4 * c4 + i][0]);
              acc[4 * c4 + i][1] = fma(wv, fv[1], acc[4 * c4 + i][1]);
              acc[4 * c4 + i][2] = fma(wv, fv[2], acc[4 * c4 + i][2]);
            }
          }
        }
      }
    }
    if (on) {
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
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

// listed target boxes from their 27 colleague slots (slot s: delta_a = ((s / 3^a) % 3) - 1):
// I[tlist[i]][k][m] = sum_slots phase O[colleague][k][m]   (used for the root)
template <typename R>
__global__ void k_far_colleague(int nlist, const int32_t* __restrict__ tlist, const int32_t* __restrict__ coll,
                                const typename Cplx<R>::T* __restrict__ O, typename Cplx<R>::T* __restrict__ I, int Mh,
                                int nh, int nm) {
  using C = typename Cplx<R>::T;
  const int64_t modes = static_cast<int64_t>(nh) * nm * nm;
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(nlist) * 3 * modes) return;
  const int li = static_cast<int>(idx / (3 * modes));
  const int64_t rem = idx - static_cast<int64_t>(li) * 3 * modes;
  const int k = static_cast<int>(rem / modes);
  const int64_t mi = rem - k * modes;
  const int tb = tlist[li];
  const int m0 = static_cast<int>(mi / (nm * nm));
  const int m1 = static_cast<int>((mi / nm) % nm) - Mh;
  const int m2 = static_cast<int>(mi % nm) - Mh;
  R sr = 0, si = 0;
  for (int s = 0; s < 27; ++s) {
    const int cb = coll[tb * 27 + s];
    if (cb < 0) continue;
    const int d0 = s % 3 - 1, d1 = (s / 3) % 3 - 1, d2 = s / 9 - 1;
    int e = (m0 * d0 + m1 * d1 + m2 * d2) % 3;
    if (e < 0) e += 3;
    const C o = O[(static_cast<int64_t>(cb) * 3 + k) * modes + mi];
    add_phased<R>(e, o.x, o.y, sr, si);
  }
  C r;
  r.x = sr;
  r.y = si;
  I[(static_cast<int64_t>(tb) * 3 + k) * modes + mi] = r;
}

// the eight children of one parent at once: their colleagues lie in the 4 x 4 x 4
// window of boxes at the children's level around them (window slot w = w0 + 4 w1 + 16 w2
// at position 2 c_parent - 1 + (w0, w1, w2)), so each window box is read once for all
// eight.  The phase of a colleague at offset delta factors over the axes,
// e^{-2 pi i m.delta/3} = prod_a f_a(delta_a), so the 27-term sums of the eight
// children are three passes of 3-term sums (axis 0, then 1, then 2).
// win[g][64]: box id or -1; chl[g][8]: target index of child o (o_a = bit a) or -1.
constexpr int kGrpThreads = 128;
template <typename R>
__global__ void __launch_bounds__(kGrpThreads) k_far_colleague_grp(const int32_t* __restrict__ win, const int32_t* __restrict__ chl,
                                                                   const typename Cplx<R>::T* __restrict__ O,
                                                                   typename Cplx<R>::T* __restrict__ I, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  __shared__ int s_win[64], s_ch[8];
  const int g = blockIdx.x, k = blockIdx.y;
  if (threadIdx.x < 64) s_win[threadIdx.x] = win[g * 64 + threadIdx.x];
  if (threadIdx.x < 8) s_ch[threadIdx.x] = chl[g * 8 + threadIdx.x];
  __syncthreads();
  const int64_t modes = static_cast<int64_t>(nh) * nm * nm;
  const int64_t mi = blockIdx.z * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (mi >= modes) return;
  const int m0 = static_cast<int>(mi / (nm * nm));
  const int m1 = static_cast<int>((mi / nm) % nm) - Mh;
  const int m2 = static_cast<int>(mi % nm) - Mh;
  R c0, s0, c1, s1, c2, s2;
  axis_phase<R>(m0, c0, s0);
  axis_phase<R>(m1, c1, s1);
  axis_phase<R>(m2, c2, s2);
  const C* Ok = O + static_cast<int64_t>(k) * modes + mi;
  // pass 0 (axis 0): t0[o0][w1][w2]
  R t0r[2][4][4], t0i[2][4][4];
#pragma unroll
  for (int w2 = 0; w2 < 4; ++w2)
#pragma unroll
    for (int w1 = 0; w1 < 4; ++w1) {
      R xr[4], xi[4];
#pragma unroll
      for (int w0 = 0; w0 < 4; ++w0) {
        const int cb = s_win[w0 + 4 * w1 + 16 * w2];
        xr[w0] = xi[w0] = R(0);
        if (cb >= 0) {
          const C v = Ok[static_cast<int64_t>(cb) * 3 * modes];
          xr[w0] = v.x;
          xi[w0] = v.y;
        }
      }
#pragma unroll
      for (int o0 = 0; o0 < 2; ++o0)
        sum3<R>(c0, s0, xr[o0], xi[o0], xr[o0 + 1], xi[o0 + 1], xr[o0 + 2], xi[o0 + 2], t0r[o0][w1][w2], t0i[o0][w1][w2]);
    }
  // pass 1 (axis 1): t1[o0][o1][w2]
  R t1r[2][2][4], t1i[2][2][4];
#pragma unroll
  for (int o0 = 0; o0 < 2; ++o0)
#pragma unroll
    for (int o1 = 0; o1 < 2; ++o1)
#pragma unroll
      for (int w2 = 0; w2 < 4; ++w2)
        sum3<R>(c1, s1, t0r[o0][o1][w2], t0i[o0][o1][w2], t0r[o0][o1 + 1][w2], t0i[o0][o1 + 1][w2],
                t0r[o0][o1 + 2][w2], t0i[o0][o1 + 2][w2], t1r[o0][o1][w2], t1i[o0][o1][w2]);
  // pass 2 (axis 2) and the writes
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int o0 = o & 1, o1 = (o >> 1) & 1, o2 = o >> 2;
    R yr, yi;
    sum3<R>(c2, s2, t1r[o0][o1][o2], t1i[o0][o1][o2], t1r[o0][o1][o2 + 1], t1i[o0][o1][o2 + 1],
            t1r[o0][o1][o2 + 2], t1i[o0][o1][o2 + 2], yr, yi);
    const int tb = s_ch[o];
    if (tb < 0) continue;
    C r;
    r.x = yr;
    r.y = yi;
    I[(static_cast<int64_t>(tb) * 3 + k) * modes + mi] = r;
  }
}

// ------------------------------------------------------------------ fused transforms
// One warp computes out(m, r) = sum_j A[j][m] X[xaddr(r) + j * sxj] for four
// consecutive m and RU rows r = base + 32 u + lane (so that a warp reads 32
// consecutive r), A transposed [n_j][n4] in shared memory (zero past n_m).  The
// warps of the block share the (m-quad, r-block) units of one contraction.
template <typename R, bool XC, bool AC, int RU, class XAddr, class Store>
__device__ __forceinline__ void warp_contract(const typename std::conditional<XC, typename Cplx<R>::T, R>::type* X,
                                              XAddr xaddr, int sxj, int n_j, int n_r,
                                              const typename std::conditional<AC, typename Cplx<R>::T, R>::type* AT,
                                              int n_m, Store store) {
  using C = typename Cplx<R>::T;
  using TX = typename std::conditional<XC, C, R>::type;
  using TA = typename std::conditional<AC, C, R>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int n4 = (n_m + 3) & ~3, nmq = n4 / 4, nrb = (n_r + 32 * RU - 1) / (32 * RU);
  for (int unit = warp; unit < nmq * nrb; unit += nwarp) {
    const int mq = unit % nmq, rb = unit / nmq;
    int64_t xo[RU];
    bool ok[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int r = rb * 32 * RU + 32 * u + lane;
      ok[u] = r < n_r;
      xo[u] = ok[u] ? xaddr(r) : 0;
    }
    R ar[RU][4], ai[RU][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) ar[u][i] = ai[u][i] = R(0);
    for (int j = 0; j < n_j; ++j) {
      TA a[4];
      ld4(AT + j * n4 + 4 * mq, a);
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const TX x = X[xo[u] + static_cast<int64_t>(j) * sxj];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if constexpr (AC && XC) {
            ar[u][i] = fma(a[i].x, x.x, ar[u][i]);
            ar[u][i] = fma(-a[i].y, x.y, ar[u][i]);
            ai[u][i] = fma(a[i].x, x.y, ai[u][i]);
            ai[u][i] = fma(a[i].y, x.x, ai[u][i]);
          } else if constexpr (AC) {
            ar[u][i] = fma(a[i].x, x, ar[u][i]);
            ai[u][i] = fma(a[i].y, x, ai[u][i]);
          } else if constexpr (XC) {
            ar[u][i] = fma(a[i], x.x, ar[u][i]);
            ai[u][i] = fma(a[i], x.y, ai[u][i]);
          } else {
            ar[u][i] = fma(a[i], x, ar[u][i]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = 4 * mq + i;
        if (ok[u] && m < n_m) store(m, rb * 32 * RU + 32 * u + lane, ar[u][i], ai[u][i]);
      }
  }
}

// transposed copy of a row-major [n_m][n_j] matrix into shared memory [n_j][n4]
template <typename T>
__device__ inline void load_AT(T* dst, const T* src, int n_m, int n_j) {
  const int n4 = (n_m + 3) & ~3;
  for (int i = threadIdx.x; i < n_j * n4; i += blockDim.x) {
    const int j = i / n4, m = i - j * n4;
    T v{};
    if (m < n_m) v = src[m * n_j + j];
    dst[i] = v;
  }
}

// shared-memory sizes of the fused transforms (bytes), one box per block
inline size_t fused_out_smem(int p, int nh, int nm, size_t er) {
  const size_t ec = 2 * er;
  const size_t mats = (static_cast<size_t>(p) * ((nh + 3) & ~3) + static_cast<size_t>(p) * ((nm + 3) & ~3)) * ec;
  const size_t y1 = static_cast<size_t>(p) * p * nh * ec;
  const size_t big = std::max(static_cast<size_t>(p) * p * p * er, static_cast<size_t>(p) * nh * nm * ec);
  return align16(mats) + align16(y1) + align16(big);
}
inline size_t fused_ev_smem(int p, int nh, int nm, size_t er) {
  const size_t ec = 2 * er;
  const size_t p4 = (p + 3) & ~3;
  const size_t mats = (static_cast<size_t>(nm) * p4 + static_cast<size_t>(nh) * p4) * ec;
  return align16(mats) + align16(static_cast<size_t>(nh) * nm * p * ec) + align16(static_cast<size_t>(nh) * p * p * ec);
}

// outgoing plane waves of one box, all components, in shared memory:
//   X = q[box][k] [a][b][c] -> Y1 [(b,c)][m0] -> Y2 [(c,m0)][m1] -> [(m0,m1)][m2],
// the last stage contracted with the level kernel into O[box][3][modes] (first
// component written, the others added)
template <typename R>
__global__ void __launch_bounds__(1024) k_far_out_fused(const int32_t* __restrict__ src_boxes, const int32_t* __restrict__ box_level,
                                                        const R* __restrict__ q, int ncomp, int slot_f, int slot_t,
                                                        const typename Cplx<R>::T* __restrict__ Eh,
                                                        const typename Cplx<R>::T* __restrict__ E, const R* __restrict__ tab,
                                                        typename Cplx<R>::T* __restrict__ O, int p, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nh4 = (nh + 3) & ~3, nm4 = (nm + 3) & ~3;
  C* sEh = reinterpret_cast<C*>(smem);                                  // [p][nh4]
  C* sE = sEh + p * nh4;                                                // [p][nm4]
  const size_t mats = align16((static_cast<size_t>(p) * nh4 + static_cast<size_t>(p) * nm4) * sizeof(C));
  C* sY1 = reinterpret_cast<C*>(smem + mats);                           // [p*p][nh]
  unsigned char* big = smem + mats + align16(static_cast<size_t>(p) * p * nh * sizeof(C));
  R* sX = reinterpret_cast<R*>(big);                                    // [p^3] (stage 1 input)
  C* sY2 = reinterpret_cast<C*>(big);                                   // [(c, m0)][nm] (stage 2 output)
  const int box = src_boxes[blockIdx.x];
  load_AT(sEh, Eh, nh, p);
  load_AT(sE, E, nm, p);
  const R h = static_cast<R>(2.0 * M_PI / 3.0 * static_cast<double>(1 << box_level[box]));
  const int p2 = p * p;
  const int64_t p3 = static_cast<int64_t>(p2) * p, modes = static_cast<int64_t>(nh) * nm * nm;
  C* Ob = O + static_cast<int64_t>(box) * 3 * modes;
  const bool raw3 = ncomp == 3 && slot_f == 0;   // Stokeslet alone: contract once after the three spectra
  for (int k = 0; k < ncomp; ++k) {
    const int comp = (slot_f >= 0 && k < 3) ? k : 3 + (k - slot_t);
    const R* qk = q + (static_cast<int64_t>(box) * ncomp + k) * p3;
    __syncthreads();
    for (int i = threadIdx.x; i < p3; i += blockDim.x) sX[i] = qk[i];
    __syncthreads();
    warp_contract<R, false, true, 2>(sX, [](int r) { return static_cast<int64_t>(r); }, p2, p, p2, sEh, nh,
                                     [&](int m, int r, R re, R im) { sY1[r * nh + m] = C{re, im}; });
    __syncthreads();
    warp_contract<R, true, true, 2>(sY1, [](int r) { return static_cast<int64_t>(r); }, p * nh, p, p * nh, sE, nm,
                                    [&](int m, int r, R re, R im) { sY2[r * nm + m] = C{re, im}; });
    __syncthreads();
    // stage 3 in chunks of rows (m0, m1), staged in the free Y1 buffer so that the
    // kernel contraction and the update of O run over consecutive modes
    const int rows = nh * nm;
    const int chunk = static_cast<int>((static_cast<size_t>(p) * p * nh) / nm);    // rows of nm modes that fit in Y1
    for (int r0 = 0; r0 < rows; r0 += chunk) {
      const int nr = min(chunk, rows - r0);
      warp_contract<R, true, true, 2>(sY2, [r0](int r) { return static_cast<int64_t>(r0 + r); }, nh * nm, p, nr, sE, nm,
                                      [&](int m, int r, R re, R im) { sY1[r * nm + m] = C{re, im}; });
      __syncthreads();
      if (raw3) {                    // Stokeslet alone: the raw spectrum of component k into O[box][k]
        for (int i = threadIdx.x; i < nr * nm; i += blockDim.x)
          Ob[k * modes + static_cast<int64_t>(r0) * nm + i] = sY1[i];
        __syncthreads();
        continue;
      }
      for (int i = threadIdx.x; i < nr * nm; i += blockDim.x) {
        const int r = r0 + i / nm, m = i - (i / nm) * nm;
        const C v = sY1[i];
        const int m0 = r / nm, m1 = r - m0 * nm - Mh, m2 = m - Mh;
        const R mv[3] = {R(m0), R(m1), R(m2)};
        const int qi = m0 * m0 + m1 * m1 + m2 * m2;
        const R t = tab[qi], qq = R(qi);
        const int64_t mi = static_cast<int64_t>(r) * nm + m;
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          R cr = R(0), ci = R(0);
          if (comp < 3) {
            cr = h * t * ((jj == comp ? qq : R(0)) - mv[jj] * mv[comp]);
          } else {
            const int cc = comp - 3;
            R w;
            if (cc < 3) {
              w = qq * (R(2) * (jj == cc ? mv[cc] : R(0)) + mv[jj]) - R(2) * mv[jj] * mv[cc] * mv[cc];
            } else {
              const int l = cc == 5 ? 1 : 0, n = cc == 3 ? 1 : 2;
              w = R(2) * qq * ((jj == l ? mv[n] : R(0)) + (jj == n ? mv[l] : R(0))) - R(4) * mv[jj] * mv[l] * mv[n];
            }
            ci = h * h * t * w;
          }
          C add;
          add.x = cr * v.x - ci * v.y;
          add.y = cr * v.y + ci * v.x;
          if (k == 0) {
            Ob[jj * modes + mi] = add;
          } else {
            C o = Ob[jj * modes + mi];
            o.x += add.x;
            o.y += add.y;
            Ob[jj * modes + mi] = o;
          }
        }
      }
      __syncthreads();
    }
  }
  if (raw3) {
    // O_j = h t(q) (q rho_j - m_j (m . rho)) in place over the box's modes
    __syncthreads();
    for (int64_t mi = threadIdx.x; mi < modes; mi += blockDim.x) {
      const int r = static_cast<int>(mi / nm), m = static_cast<int>(mi - static_cast<int64_t>(r) * nm);
      const int m0 = r / nm, m1 = r - m0 * nm - Mh, m2 = m - Mh;
      const int qi = m0 * m0 + m1 * m1 + m2 * m2;
      const R sc = h * tab[qi], qq = R(qi);
      const C x0 = Ob[mi], x1 = Ob[modes + mi], x2 = Ob[2 * modes + mi];
      const R dr = R(m0) * x0.x + R(m1) * x1.x + R(m2) * x2.x;
      const R di = R(m0) * x0.y + R(m1) * x1.y + R(m2) * x2.y;
      Ob[mi] = C{sc * (qq * x0.x - R(m0) * dr), sc * (qq * x0.y - R(m0) * di)};
      Ob[modes + mi] = C{sc * (qq * x1.x - R(m1) * dr), sc * (qq * x1.y - R(m1) * di)};
      Ob[2 * modes + mi] = C{sc * (qq * x2.x - R(m2) * dr), sc * (qq * x2.y - R(m2) * di)};
    }
  }
}

// child merge of one parent, one component per block (float32):
//   q[parent] = sum over children o of (T_o0 (x) T_o1 (x) T_o2) q[child o],
// with the sums over o0 and o1 taken after the first and second contractions
// (Y1 = sum_o0 T_o0 q[o], Z_o2 = sum_o1 T_o1 Y1, q = sum_o2 T_o2 Z_o2: 14 instead
// of 24 p^4 multiply-adds) in four p^3 buffers of shared memory; chl[g][8]: box
// id of child o (o_a = bit a) or -1 (no sources)
template <typename R>
__global__ void __launch_bounds__(1024) k_far_merge_fused(const int32_t* __restrict__ parents, const int32_t* __restrict__ chl,
                                                          R* __restrict__ q, int ncomp, const R* __restrict__ T0,
                                                          const R* __restrict__ T1, int p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p4 = (p + 3) & ~3, p2 = p * p;
  const int64_t p3 = static_cast<int64_t>(p2) * p;
  R* sT = reinterpret_cast<R*>(smem);                                   // [2][p][p4] transposed T_0, T_1
  R* sX = sT + 2 * p * p4;                                              // child charges; later the result
  R* sY = sX + p3;
  R* sZ = sY + p3;                                                      // [2][p^3]: Z_0, Z_1
  const int g = blockIdx.x, k = blockIdx.y;
  load_AT(sT, T0, p, p);
  load_AT(sT + p * p4, T1, p, p);
  int cz[2] = {0, 0};                                                   // contributions held in Z_o2
  auto id = [](int r) { return static_cast<int64_t>(r); };
  for (int o2 = 0; o2 < 2; ++o2)
    for (int o1 = 0; o1 < 2; ++o1) {
      int ny = 0;
      for (int o0 = 0; o0 < 2; ++o0) {
        const int cb = chl[g * 8 + (o0 | (o1 << 1) | (o2 << 2))];
        if (cb < 0) continue;
        const R* X = q + (static_cast<int64_t>(cb) * ncomp + k) * p3;
        __syncthreads();
        for (int i = threadIdx.x; i < p3; i += blockDim.x) sX[i] = X[i];
        __syncthreads();
        const bool first = ny == 0;
        warp_contract<R, false, false, 2>(sX, id, p2, p, p2, sT + o0 * p * p4, p, [&](int m, int r, R re, R) {
          if (first) sY[r * p + m] = re;
          else sY[r * p + m] += re;
        });
        ++ny;
      }
      if (ny == 0) continue;
      __syncthreads();
      R* Z = sZ + o2 * p3;
      const bool first = cz[o2] == 0;
      warp_contract<R, false, false, 2>(sY, id, p2, p, p2, sT + o1 * p * p4, p, [&](int m, int r, R re, R) {
        if (first) Z[r * p + m] = re;
        else Z[r * p + m] += re;
      });
      ++cz[o2];
    }
  __syncthreads();
  int nw = 0;
  for (int o2 = 0; o2 < 2; ++o2) {
    if (cz[o2] == 0) continue;
    const bool first = nw == 0;
    warp_contract<R, false, false, 2>(sZ + o2 * p3, id, p2, p, p2, sT + o2 * p * p4, p, [&](int m, int r, R re, R) {
      if (first) sX[r * p + m] = re;
      else sX[r * p + m] += re;
    });
    ++nw;
    __syncthreads();
  }
  R* Y = q + (static_cast<int64_t>(parents[g]) * ncomp + k) * p3;
  for (int i = threadIdx.x; i < p3; i += blockDim.x) Y[i] = nw ? sX[i] : R(0);
}

// interpolation of one parent's potential grid to its children, one component per
// block (float32): pot[child o] += (T_o0^T (x) T_o1^T (x) T_o2^T) pot[parent], the
// partial products shared (Z_o0 = T_o0^T pot, Y = T_o1^T Z_o0, child = T_o2^T Y);
// chl[g][8]: box id of child o or -1 (no targets)
template <typename R>
__global__ void __launch_bounds__(1024) k_far_interp_fused(const int32_t* __restrict__ parents, const int32_t* __restrict__ chl,
                                                           R* __restrict__ pot, const R* __restrict__ T0t,
                                                           const R* __restrict__ T1t, int p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p4 = (p + 3) & ~3, p2 = p * p;
  const int64_t p3 = static_cast<int64_t>(p2) * p;
  R* sT = reinterpret_cast<R*>(smem);
  R* sX = sT + 2 * p * p4;                                              // parent grid; later a child's result
  R* sY = sX + p3;
  R* sZ = sY + p3;                                                      // [2][p^3]: Z_0, Z_1
  const int g = blockIdx.x, k = blockIdx.y;
  load_AT(sT, T0t, p, p);
  load_AT(sT + p * p4, T1t, p, p);
  int need[2] = {0, 0};
  for (int o = 0; o < 8; ++o)
    if (chl[g * 8 + o] >= 0) need[o & 1] = 1;
  const R* Xg = pot + (static_cast<int64_t>(parents[g]) * 3 + k) * p3;
  for (int i = threadIdx.x; i < p3; i += blockDim.x) sX[i] = Xg[i];
  __syncthreads();
  auto id = [](int r) { return static_cast<int64_t>(r); };
  for (int o0 = 0; o0 < 2; ++o0) {
    if (!need[o0]) continue;
    R* Z = sZ + o0 * p3;
    warp_contract<R, false, false, 2>(sX, id, p2, p, p2, sT + o0 * p * p4, p,
                                      [&](int m, int r, R re, R) { Z[r * p + m] = re; });
  }
  for (int o0 = 0; o0 < 2; ++o0)
    for (int o1 = 0; o1 < 2; ++o1) {
      const int c0 = chl[g * 8 + (o0 | (o1 << 1))], c1 = chl[g * 8 + (o0 | (o1 << 1) | 4)];
      if (c0 < 0 && c1 < 0) continue;
      __syncthreads();
      warp_contract<R, false, false, 2>(sZ + o0 * p3, id, p2, p, p2, sT + o1 * p * p4, p,
                                        [&](int m, int r, R re, R) { sY[r * p + m] = re; });
      for (int o2 = 0; o2 < 2; ++o2) {
        const int cb = o2 ? c1 : c0;
        if (cb < 0) continue;
        __syncthreads();
        warp_contract<R, false, false, 2>(sY, id, p2, p, p2, sT + o2 * p * p4, p,
                                          [&](int m, int r, R re, R) { sX[r * p + m] = re; });
        __syncthreads();
        R* Yc = pot + (static_cast<int64_t>(cb) * 3 + k) * p3;
        for (int i = threadIdx.x; i < p3; i += blockDim.x) Yc[i] += sX[i];
      }
    }
}

inline size_t fused_tree_smem(int p, size_t er) {
  const size_t p4 = (p + 3) & ~3;
  return (2 * static_cast<size_t>(p) * p4 + 4 * static_cast<size_t>(p) * p * p) * er;
}

// potential grid of one target box from its incoming expansion, in shared memory:
//   I[tb][k] [(m0,m1)][m2] -> Y1 [(m0,m1)][c] -> Y2 [m0][b][c] -> Re [a][b][c] = pot[box][k]
// (the m0 >= 0 half carries the weights 1, 2, 2, ... in Fh)
template <typename R>
__global__ void __launch_bounds__(1024) k_far_ev_fused(const int32_t* __restrict__ trg_boxes,
                                                       const typename Cplx<R>::T* __restrict__ I,
                                                       const typename Cplx<R>::T* __restrict__ Fh,
                                                       const typename Cplx<R>::T* __restrict__ F, R* __restrict__ pot,
                                                       int p, int nh, int nm) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int p4 = (p + 3) & ~3;
  C* sF = reinterpret_cast<C*>(smem);                                   // [nm][p4]: F^T
  C* sFh = sF + nm * p4;                                                // [nh][p4]: Fh^T
  const size_t mats = align16((static_cast<size_t>(nm) * p4 + static_cast<size_t>(nh) * p4) * sizeof(C));
  C* sY1 = reinterpret_cast<C*>(smem + mats);                           // [(m0,m1)][p]
  C* sY2 = reinterpret_cast<C*>(smem + mats + align16(static_cast<size_t>(nh) * nm * p * sizeof(C)));   // [m0][b][c]
  const int tb = blockIdx.x;
  const int box = trg_boxes[tb];
  load_AT(sF, F, p, nm);
  load_AT(sFh, Fh, p, nh);
  const int p2 = p * p;
  const int64_t p3 = static_cast<int64_t>(p2) * p, modes = static_cast<int64_t>(nh) * nm * nm;
  for (int k = 0; k < 3; ++k) {
    const C* Ik = I + (static_cast<int64_t>(tb) * 3 + k) * modes;
    R* Pk = pot + (static_cast<int64_t>(box) * 3 + k) * p3;
    __syncthreads();
    warp_contract<R, true, true, 2>(Ik, [nm](int r) { return static_cast<int64_t>(r) * nm; }, 1, nm, nh * nm, sF, p,
                                    [&](int m, int r, R re, R im) { sY1[r * p + m] = C{re, im}; });
    __syncthreads();
    warp_contract<R, true, true, 2>(sY1, [p, nm](int r) { return static_cast<int64_t>(r / p) * nm * p + (r % p); }, p, nm,
                                    nh * p, sF, p,
                                    [&](int m, int r, R re, R im) { sY2[(r / p) * p2 + m * p + (r % p)] = C{re, im}; });
    __syncthreads();
    warp_contract<R, true, true, 2>(sY2, [](int r) { return static_cast<int64_t>(r); }, p2, nh, p2, sFh, p,
                                    [&](int m, int r, R re, R im) { Pk[static_cast<int64_t>(m) * p2 + r] = re; });
  }
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

// leaf evaluation: u[caller][k] += sum_abc L_a(x) L_b(y) L_c(z) pot[box][k][a][b][c].
// A block takes one chunk of at most kEvThreads targets of one leaf (item it:
// leaf list entry it_leaf[it], first target it_off[it]); a thread takes TT of
// them (slots tid + u * blockDim), their c-weights in registers (PB each, zero
// past p), so that every grid row read from shared memory serves TT targets.  The
// leaf's grid passes through shared memory one a-slab (3 x p x PB) at a time,
// double buffered: slab a + 1 is read into registers while slab a is used.
constexpr int kEvThreads = 128;
template <typename R, int PB, int TT>
__global__ void __launch_bounds__(kEvThreads) k_far_eval(const int32_t* __restrict__ it_leaf, const int32_t* __restrict__ it_off,
                                                         const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                         const int32_t* __restrict__ t_start, const int32_t* __restrict__ t_count,
                                                         const double* __restrict__ tw, int64_t NT, const int32_t* __restrict__ tperm,
                                                         const BoxGeo* __restrict__ box_geo, const R* __restrict__ pot, int p,
                                                         const R* __restrict__ nodes, const R* __restrict__ bw,
                                                         double* __restrict__ u) {
  constexpr int NTH = kEvThreads / TT;                   // threads of the block
  // slab entries per thread (p <= PB); prefetched into registers when that is few
  constexpr int kSlabPer = (3 * PB * PB + NTH - 1) / NTH;
  constexpr bool kPre = kSlabPer <= 32;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sL = reinterpret_cast<R*>(smem);                    // [2][p][kEvThreads] a- and b-weights per target slot
  R* sP = sL + 2 * p * kEvThreads;                       // [2 buffers][3][p][PB]
  __shared__ R s_nodes[kMaxP], s_bw[kMaxP];
  const int e = it_leaf[blockIdx.x];
  const int li = leaf_list[e];
  const int box = leaf_box[e];
  for (int j = threadIdx.x; j < p; j += NTH) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  const BoxGeo geo = box_geo[box];
  const double inv_half = 1.0 / geo.w;
  const int lt0 = t_start[li], lnt = t_count ? t_count[li] : t_start[li + 1] - lt0;
  const int t0 = lt0 + it_off[blockIdx.x];
  const int nt = min(kEvThreads, lnt - it_off[blockIdx.x]);
  const int64_t p2 = static_cast<int64_t>(p) * p, p3 = p2 * p;
  const int slab = 3 * p * PB;
  const R* P = pot + static_cast<int64_t>(box) * 3 * p3;
  __syncthreads();
  R cw[TT][PB];
  bool on[TT];
#pragma unroll
  for (int uu = 0; uu < TT; ++uu) {
    const int t = threadIdx.x + uu * NTH;
    on[uu] = t < nt;
#pragma unroll
    for (int j = 0; j < PB; ++j) cw[uu][j] = R(0);
    if (on[uu]) {
      for (int ax = 0; ax < 2; ++ax) {
        const double ctr = ax == 0 ? geo.x : geo.y;
        const R x = static_cast<R>((tw[ax * NT + t0 + t] - ctr) * inv_half);
        lagrange_row<R>(x, p, s_nodes, s_bw, sL + ax * p * kEvThreads + t, kEvThreads, p);
      }
      const R z = static_cast<R>((tw[2 * NT + t0 + t] - geo.z) * inv_half);
      R ssum = R(0);
      int hit = -1;
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        R v = R(0);
        if (j < p) {
          const R d = z - s_nodes[j];
          if (d == R(0)) hit = j;
          else v = s_bw[j] * recip<R>(d);
        }
        cw[uu][j] = v;
        ssum += v;
      }
      const R inv = hit >= 0 ? R(0) : recip<R>(ssum);
#pragma unroll
      for (int j = 0; j < PB; ++j) cw[uu][j] = hit >= 0 ? (j == hit ? R(1) : R(0)) : cw[uu][j] * inv;
    } else {
      for (int j = 0; j < p; ++j) sL[j * kEvThreads + t] = sL[(p + j) * kEvThreads + t] = R(0);
    }
  }
  // entry i of slab a: grid value (k, a, b, c) with i = (k p + b) PB + c (zero past p)
  auto slab_val = [&](int a, int i) {
    const int k = i / (p * PB);
    const int r = i - k * p * PB;
    const int b = r / PB, c = r - b * PB;
    return c < p ? P[k * p3 + a * p2 + b * p + c] : R(0);
  };
  R pre[kPre ? kSlabPer : 1];
  auto fetch = [&](int a) {
#pragma unroll
    for (int n = 0; n < (kPre ? kSlabPer : 1); ++n) {
      const int i = threadIdx.x + n * NTH;
      pre[n] = i < slab ? slab_val(a, i) : R(0);
    }
  };
  if constexpr (kPre) fetch(0);
  R acc[TT][3];
#pragma unroll
  for (int uu = 0; uu < TT; ++uu) acc[uu][0] = acc[uu][1] = acc[uu][2] = R(0);
  for (int a = 0; a < p; ++a) {
    R* buf = sP + (a & 1) * slab;
    if constexpr (kPre) {
#pragma unroll
      for (int n = 0; n < kSlabPer; ++n) {
        const int i = threadIdx.x + n * NTH;
        if (i < slab) buf[i] = pre[n];
      }
      __syncthreads();
      if (a + 1 < p) fetch(a + 1);
    } else {
      for (int i = threadIdx.x; i < slab; i += NTH) buf[i] = slab_val(a, i);
      __syncthreads();
    }
    R la[TT];
#pragma unroll
    for (int uu = 0; uu < TT; ++uu) la[uu] = sL[a * kEvThreads + threadIdx.x + uu * NTH];
    for (int b = 0; b < p; ++b) {
      const R* row = buf + b * PB;
      R r[TT][3];
#pragma unroll
      for (int uu = 0; uu < TT; ++uu) r[uu][0] = r[uu][1] = r[uu][2] = R(0);
#pragma unroll
      for (int c4 = 0; c4 < PB / 4; ++c4) {
        R v0[4], v1[4], v2[4];
        ld4(row + 4 * c4, v0);
        ld4(row + p * PB + 4 * c4, v1);
        ld4(row + 2 * p * PB + 4 * c4, v2);
#pragma unroll
        for (int uu = 0; uu < TT; ++uu)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            r[uu][0] = fma(cw[uu][4 * c4 + i], v0[i], r[uu][0]);
            r[uu][1] = fma(cw[uu][4 * c4 + i], v1[i], r[uu][1]);
            r[uu][2] = fma(cw[uu][4 * c4 + i], v2[i], r[uu][2]);
          }
      }
#pragma unroll
      for (int uu = 0; uu < TT; ++uu) {
        const R lab = la[uu] * sL[(p + b) * kEvThreads + threadIdx.x + uu * NTH];
        acc[uu][0] = fma(lab, r[uu][0], acc[uu][0]);
        acc[uu][1] = fma(lab, r[uu][1], acc[uu][1]);
        acc[uu][2] = fma(lab, r[uu][2], acc[uu][2]);
      }
    }
  }
#pragma unroll
  for (int uu = 0; uu < TT; ++uu)
    if (on[uu]) {
      const int64_t o = tperm[t0 + threadIdx.x + uu * NTH];
      u[o * 3] += static_cast<double>(acc[uu][0]);
      u[o * 3 + 1] += static_cast<double>(acc[uu][1]);
      u[o * 3 + 2] += static_cast<double>(acc[uu][2]);
    }
}

// ------------------------------------------------------------------ tensor-core leaf kernels
// The float32 far field's two per-point contractions on tcgen05 (kind::tf32, split
// TF32 products, D in tensor memory; tc.cuh).  Several blocks share an SM (their MMAs
// and their operand forming interleave); within a block the next stage's inputs
// arrive by cp.async while the current one is formed and multiplied.  Warp 0 waits on
// the MMAs' mbarrier while the other warps wait at the block barrier.  A wait that runs
// out sets ST_TC_TIMEOUT in the plan's status word, ends the block's work, waits once
// more for the MMAs in flight and frees the tensor memory.
constexpr int kTcThreads = 256;
constexpr int kTcK = 32;                            // sources per operand stage (four K = 8 steps)
constexpr int kTcSbo = (kTcK / 4) * 128;            // 8-row group stride of those operands (bytes)
constexpr long long kTcWaitCycles = 4000000000LL;   // about 2 s of SM clock
constexpr size_t kSmemPerSM = 228 * 1024;

// densities of the component groups per source in sorted point order, float32:
// Vs[gi][s] = (v0, v1, v2, 0) for the gi-th present group (0: f; 1: rho_00, rho_11,
// rho_22; 2: rho_01, rho_02, rho_12 of the symmetric part of g (x) n)
__global__ void k_far_values(const int32_t* __restrict__ perm, const double* __restrict__ f, const double* __restrict__ g,
                             const double* __restrict__ nrm, int64_t N, int grp0, int ng, float4* __restrict__ Vs) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (s >= N) return;
  const int64_t o = perm[s];
  for (int gi = 0; gi < ng; ++gi) {
    const int grp = grp0 + gi;
    double v0, v1, v2;
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
    Vs[gi * N + s] = make_float4(static_cast<float>(v0), static_cast<float>(v1), static_cast<float>(v2), 0.f);
  }
}

// shared memory of the leaf-charge kernel: one operand buffer (A hi/lo [128][kTcK],
// B hi/lo [NP][kTcK]) and two source stages (weights [kTcK][3][PB], densities
// [kTcK][4], 128-byte aligned); at least a quarter of the SM so that at most three
// blocks (384 TMEM columns) share one
inline size_t anterp_tc_op_bytes(int NP) { return 2 * 128 * kTcK * 4 + 2 * static_cast<size_t>(NP) * kTcK * 4; }
inline size_t anterp_tc_stage_floats(int PB) { return static_cast<size_t>(kTcK) * 3 * PB + kTcK * 4; }
inline size_t anterp_tc_smem(int NP, int PB) {
  const size_t need = anterp_tc_op_bytes(NP) + 2 * anterp_tc_stage_floats(PB) * 4 + 128;
  return std::max({need, kSmemPerSM / 4 + 1024, 128 * static_cast<size_t>(NP + 1) * 4});
}

// leaf proxy charges: per leaf and component group, Q[(a,b)][(k,c)] = sum_s A[(a,b)][s] B[(k,c)][s]
// with A = L_a(x_s) L_b(y_s) and B = L_c(z_s) v_s,k.  A block owns one tile of 128
// rows (a, b) and all 3p columns (padded to NP, a multiple of 16, <= 128) in tensor
// memory; the tiles of one leaf are consecutive blocks, so they run side by side and
// read the leaf's weights once from HBM (then from L2).  Per stage of kTcK sources,
// warps 0-3 form row tid of A and warps 4-7 row tid - 128 of B from the stage's
// weights and densities, which arrive one stage ahead by two TMA tile loads
// (tmW: W as [N][3 PB], tmV: Vs as [groups N][4]) on the stage's mbarrier.  The
// result leaves through shared memory in the layout q[box][slot + k][a][b][c].
__global__ void __launch_bounds__(kTcThreads) k_far_anterp_tc(const __grid_constant__ CUtensorMap tmW,
                                                              const __grid_constant__ CUtensorMap tmV,
                                                              const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                              const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                                                              int64_t N, int slot_f, int slot_t, int ncomp, float* __restrict__ q,
                                                              int p, int PB, int NP, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t opA = 128 * kTcK * 4, opB = static_cast<size_t>(NP) * kTcK * 4;
  const int stW = kTcK * 3 * PB;                                       // weight floats of one stage
  const int stF = stW + kTcK * 4;                                      // floats of one stage
  unsigned char* sAh = smem;
  unsigned char* sAl = sAh + opA;
  unsigned char* sBh = sAl + opA;
  unsigned char* sBl = sBh + opB;
  float* stage0;
  {
    const uint32_t a = tc::smem_u32(sBl + opB);
    stage0 = reinterpret_cast<float*>(sBl + opB + ((128u - (a & 127u)) & 127u));   // TMA destinations: 128-byte aligned
  }
  __shared__ __align__(8) uint64_t mbar, mbst[2];
  __shared__ uint32_t tbase;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nmt = (p * p + 127) / 128;
  const int leaf = blockIdx.x / nmt, mt = blockIdx.x - leaf * nmt;   // a leaf's row tiles run side by side
  const int li = leaf_list[leaf], box = leaf_box[leaf];
  const int gi = blockIdx.y;
  const int grp = (slot_f >= 0 ? 0 : 1) + gi;
  const int slot = grp == 0 ? slot_f : slot_t + 3 * (grp - 1);
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const int p2 = p * p;
  const int64_t p3 = static_cast<int64_t>(p2) * p;
  const bool arole = tid < 128;
  const int rr = arole ? tid : tid - 128;
  const int R = mt * 128 + rr;
  // weight offsets of this thread's row within a source's [3][PB] block (zero row: none)
  int w0 = -1, w1 = -1;
  if (arole && R < p2) {                                               // row (a, b) of A: L_a(x) L_b(y)
    w0 = R / p;
    w1 = PB + (R - w0 * p);
  } else if (!arole && rr < 3 * p) {                                   // row (k, c) of B: L_c(z) v_k
    w0 = 2 * PB + rr % p;
    w1 = rr / p;
  }
  const bool forms = arole || rr < NP;
  const int nchunk = (ns + kTcK - 1) / kTcK;
  auto stage_in = [&](int ch) {                                        // thread 0: the TMA loads of stage ch
    float* sw = stage0 + (ch & 1) * stF;
    const int y = s0 + ch * kTcK;
    tc::expect_tx(&mbst[ch & 1], static_cast<uint32_t>(stF) * 4u);
    tc::tma_load_2d(sw, &tmW, 0, y, &mbst[ch & 1]);
    tc::tma_load_2d(sw + stW, &tmV, 0, static_cast<int>(gi * N) + y, &mbst[ch & 1]);
  };
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_init(&mbst[0], 1);
    tc::mbar_init(&mbst[1], 1);
    fail = 0;
    if (nchunk > 0) stage_in(0);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 128);
  tc::sync_tc();
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  unsigned char* dh = arole ? sAh : sBh;
  unsigned char* dl = arole ? sAl : sBl;
  int issued = 0, staged = nchunk > 0 ? 1 : 0;
  for (int ch = 0; ch < nchunk; ++ch) {
    if (ch + 1 < nchunk) {                                             // its stage was last read while forming ch - 1
      if (tid == 0) stage_in(ch + 1);
      ++staged;
    }
    if (!tc::mbar_wait(&mbst[ch & 1], (ch >> 1) & 1, kTcWaitCycles)) atomicExch(&fail, 1);
    if (ch >= 1 && warp == 0)                                          // the operands were read by the MMAs of ch - 1
      if (!tc::mbar_wait(&mbar, (ch - 1) & 1, kTcWaitCycles)) atomicExch(&fail, 1);
    const int ncnt = min(kTcK, ns - ch * kTcK);
    float* sw = stage0 + (ch & 1) * stF;
    if (ncnt < kTcK) {                                                 // a leaf's last stage: sources past it read as zero
      for (int i = ncnt * 3 * PB + tid; i < stW; i += kTcThreads) sw[i] = 0.f;
      for (int i = ncnt * 4 + tid; i < kTcK * 4; i += kTcThreads) sw[stW + i] = 0.f;
    }
    __syncthreads();
    if (fail) break;
    if (forms) {
#pragma unroll 4
      for (int s4 = 0; s4 < kTcK / 4; ++s4) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int sl = 4 * s4 + j;
          const float* ws = sw + sl * 3 * PB;
          const float v = w0 < 0 ? 0.f : ws[w0] * (arole ? ws[w1] : sw[stW + sl * 4 + w1]);
          tc::split_tf32_fast(v, h[j], l[j]);
        }
        const int o = tc::kmajor_off(rr, 4 * s4, kTcSbo);
        *reinterpret_cast<uint4*>(dh + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(dl + o) = make_uint4(l[0], l[1], l[2], l[3]);
      }
    }
    tc::fence_async_smem();
    tc::sync_tc();
    if (tid == 0) {
      const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t ko = kk * 256;                                  // two core matrices along K per step
        tc::mma_tf32x3(tmem, tc::smem_desc(ah + ko, kTcSbo), tc::smem_desc(al + ko, kTcSbo),
                       tc::smem_desc(bh + ko, kTcSbo), tc::smem_desc(bl + ko, kTcSbo), idesc,
                       (ch > 0 || kk > 0) ? 1u : 0u);
      }
      tc::commit(&mbar);
    }
    ++issued;
  }
  if (issued > 0 && !fail && warp == 0)
    if (!tc::mbar_wait(&mbar, (issued - 1) & 1, kTcWaitCycles)) atomicExch(&fail, 1);
  tc::sync_tc();
  if (!fail && issued > 0) {
    // D rows (a, b) x columns (k, c) through shared memory (the operand buffer is free):
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 and the column blocks of parity w / 4
    float* sD = reinterpret_cast<float*>(smem);                       // [128][NP + 1]
    const int lanew = warp & 3, half = warp >> 2, row = 32 * lanew + (tid & 31);
    for (int cb = half; cb < NP / 16; cb += 2) {
      float v[16];
      tc::ld16(tmem + (static_cast<uint32_t>(32 * lanew) << 16) + cb * 16, v);
      tc::ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) sD[row * (NP + 1) + cb * 16 + j] = v[j];
    }
    __syncthreads();
    const int R0 = mt * 128, nrow = min(128, p2 - R0);
    float* qb = q + (static_cast<int64_t>(box) * ncomp + slot) * p3 + static_cast<int64_t>(R0) * p;
    for (int i = tid; i < 3 * nrow * p; i += kTcThreads) {
      const int k = i / (nrow * p), rem = i - k * nrow * p;
      const int r = rem / p, c = rem - r * p;
      qb[k * p3 + rem] = sD[r * (NP + 1) + k * p + c];
    }
  } else if (fail) {
    if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    if (issued > 0 && warp == 0) tc::mbar_wait(&mbar, (issued - 1) & 1, kTcWaitCycles);
    if (staged > 0) tc::mbar_wait(&mbst[(staged - 1) & 1], ((staged - 1) >> 1) & 1, kTcWaitCycles);   // the last TMA load
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// grid rows (k, a) of one MMA block of the leaf evaluation: RB rows of RW columns b,
// N = RB RW <= 256 and a multiple of 16
constexpr int eval_tc_rows(int rw) {
  int rb = 256 / rw;
  while ((rb * rw) % 16) --rb;
  return rb;
}
// shared memory of the leaf evaluation: A hi/lo [128][RW], B hi/lo [NB][RW], the staged
// grid rows [RB][p^2], the a-weights [p][128] and the partial sums [128][3]; at least a
// third of the SM, so that at most two blocks (512 TMEM columns) share one
template <int RW>
size_t eval_tc_smem_t(int p) {
  const size_t nb = static_cast<size_t>(eval_tc_rows(RW)) * RW;
  const size_t need = 2 * 128 * RW * 4 + 2 * nb * RW * 4 + static_cast<size_t>(eval_tc_rows(RW)) * p * p * 4 +
                      static_cast<size_t>(p) * 128 * 4 + 128 * 3 * 4;
  return std::max(need, kSmemPerSM / 3 + 1024);
}

// leaf evaluation: a block takes one chunk of at most 128 targets of one leaf (item
// it_leaf / it_off, target t in TMEM lane t).  For each block j of RB grid rows (k, a)
// the MMA forms V[t][(k,a,b)] = sum_c L_c(z_t) P[k][a][b][c] (K = c and the b of each
// row padded to RW), and the threads reduce u_k(t) += L_a(x_t) sum_b L_b(y_t) V[t][(k,a,b)]
// (threads t and t + 128 split the block's rows); block j + 1's grid rows arrive by
// cp.async during the MMAs of block j.
template <int RW>
__global__ void __launch_bounds__(kTcThreads) k_far_eval_tc(const int32_t* __restrict__ it_leaf, const int32_t* __restrict__ it_off,
                                                            const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                            const int32_t* __restrict__ t_start, const int32_t* __restrict__ t_count,
                                                            const double* __restrict__ tw, int64_t NT, const int32_t* __restrict__ tperm,
                                                            const BoxGeo* __restrict__ box_geo, const float* __restrict__ pot, int p,
                                                            const float* __restrict__ nodes, const float* __restrict__ bw,
                                                            double* __restrict__ u, int* __restrict__ status) {
  constexpr int KP = RW;                         // K = c padded like the rows
  constexpr int SBO = (KP / 4) * 128;
  constexpr int RB = eval_tc_rows(RW);
  constexpr int NB = RB * RW;
  constexpr int RH = (RB + 1) / 2;               // rows of a block reduced by threads 0..127
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr size_t opA = 128 * KP * 4, opB = static_cast<size_t>(NB) * KP * 4;
  unsigned char* sAh = smem;                                  // [128][KP]: L_c(z_t)
  unsigned char* sAl = sAh + opA;
  unsigned char* sBh = sAl + opA;                             // [NB][KP]: grid rows
  unsigned char* sBl = sBh + opB;
  float* sP = reinterpret_cast<float*>(sBl + opB);            // [RB][p^2]: staged grid rows
  const int p2 = p * p;
  float* sLa = sP + RB * p2;                                  // [p][128]: L_a(x_t)
  float* sRed = sLa + p * 128;                                // [128][3]
  __shared__ float s_nodes[kMaxP], s_bw[kMaxP];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int t = tid & 127, half = tid >> 7;
  const int e = it_leaf[blockIdx.x];
  const int li = leaf_list[e];
  const int box = leaf_box[e];
  const float* P = pot + static_cast<int64_t>(box) * 3 * p2 * p;
  const int nrows = 3 * p;
  const int nblk = (nrows + RB - 1) / RB;
  auto stage_in = [&](int j) {                   // grid rows j RB .. of the leaf into sP
    const int r0 = j * RB, nr = min(RB, nrows - r0);
    const float* src = P + static_cast<int64_t>(r0) * p2;
    for (int i = tid; i < nr * p2; i += kTcThreads) tc::cp_async4(sP + i, src + i);
    tc::cp_async_commit();
  };
  stage_in(0);
  for (int j = tid; j < p; j += kTcThreads) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    fail = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 256);
  tc::sync_tc();
  const BoxGeo geo = box_geo[box];
  const double inv_half = 1.0 / geo.w;
  const int lt0 = t_start[li], lnt = t_count ? t_count[li] : t_start[li + 1] - lt0;
  const int t0 = lt0 + it_off[blockIdx.x];
  const int nt = min(128, lnt - it_off[blockIdx.x]);
  const bool on = t < nt;
  // b-weights in registers (both halves); a-weights and the c-row of A from half 0
  float lb[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) lb[j] = 0.f;
  if (on) {
    const float y = static_cast<float>((tw[NT + t0 + t] - geo.y) * inv_half);
    float sy = 0.f;
    int hy = -1;
#pragma unroll
    for (int j = 0; j < RW; ++j) {
      float v = 0.f;
      if (j < p) {
        const float d = y - s_nodes[j];
        if (d == 0.f) hy = j;
        else v = s_bw[j] * __frcp_rn(d);
      }
      lb[j] = v;
      sy += v;
    }
    const float iy = hy >= 0 ? 0.f : __frcp_rn(sy);
#pragma unroll
    for (int j = 0; j < RW; ++j) lb[j] = hy >= 0 ? (j == hy ? 1.f : 0.f) : lb[j] * iy;
  }
  if (half == 0) {
    float lc[RW];
#pragma unroll
    for (int j = 0; j < RW; ++j) lc[j] = 0.f;
    if (on) {
      const float x = static_cast<float>((tw[t0 + t] - geo.x) * inv_half);
      lagrange_row<float>(x, p, s_nodes, s_bw, sLa + t, 128, p);
      const float z = static_cast<float>((tw[2 * NT + t0 + t] - geo.z) * inv_half);
      float sz = 0.f;
      int hz = -1;
#pragma unroll
      for (int j = 0; j < RW; ++j) {
        float v = 0.f;
        if (j < p) {
          const float d = z - s_nodes[j];
          if (d == 0.f) hz = j;
          else v = s_bw[j] * __frcp_rn(d);
        }
        lc[j] = v;
        sz += v;
      }
      const float iz = hz >= 0 ? 0.f : __frcp_rn(sz);
#pragma unroll
      for (int j = 0; j < RW; ++j) lc[j] = hz >= 0 ? (j == hz ? 1.f : 0.f) : lc[j] * iz;
    } else {
      for (int j = 0; j < p; ++j) sLa[j * 128 + t] = 0.f;
    }
#pragma unroll
    for (int c4 = 0; c4 < KP / 4; ++c4) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) tc::split_tf32_fast(lc[4 * c4 + j], h[j], l[j]);
      const int o = tc::kmajor_off(t, 4 * c4, SBO);
      *reinterpret_cast<uint4*>(sAh + o) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(sAl + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::idesc_tf32(128, NB);
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
  float acc[3] = {0.f, 0.f, 0.f};
  tc::cp_async_wait<0>();
  __syncthreads();
  int issued = 0;
  for (int j = 0; j < nblk; ++j) {
    const int r0 = j * RB;
    // block j as the B operand: n = (row, b), K = c; consecutive threads take consecutive n
    for (int i = tid; i < NB * (KP / 4); i += kTcThreads) {
      const int c4 = i / NB, n = i - c4 * NB;
      const int rl = n / RW, b = n - rl * RW;
      const bool ok = r0 + rl < nrows && b < p;
      uint32_t h[4], l[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = 4 * c4 + jj;
        tc::split_tf32_fast(ok && c < p ? sP[rl * p2 + b * p + c] : 0.f, h[jj], l[jj]);
      }
      const int o = tc::kmajor_off(n, 4 * c4, SBO);
      *reinterpret_cast<uint4*>(sBh + o) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(sBl + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    tc::fence_async_smem();
    tc::sync_tc();                               // sP consumed, B visible, the previous D read
    if (j + 1 < nblk) stage_in(j + 1);
    if (tid == 0) {
      const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
#pragma unroll
      for (int kk = 0; kk < KP / 8; ++kk) {
        const uint32_t ko = kk * 256;
        tc::mma_tf32x3(tmem, tc::smem_desc(ah + ko, SBO), tc::smem_desc(al + ko, SBO), tc::smem_desc(bh + ko, SBO),
                       tc::smem_desc(bl + ko, SBO), idesc, kk > 0 ? 1u : 0u);
      }
      tc::commit(&mbar);
    }
    ++issued;
    if (warp == 0)
      if (!tc::mbar_wait(&mbar, (issued - 1) & 1, kTcWaitCycles)) atomicExch(&fail, 1);
    tc::cp_async_wait<0>();
    tc::sync_tc();
    if (fail) break;
    // reduce block j: rows [0, RH) by threads 0..127, [RH, RB) by 128..255
    for (int rr = half * RH; rr < (half ? RB : RH); ++rr) {
      const int r = r0 + rr;
      if (r >= nrows) break;
      float v[RW];
#pragma unroll
      for (int c = 0; c + 16 <= RW; c += 16) tc::ld16(lane_base + rr * RW + c, v + c);
      if constexpr (RW % 16 != 0) tc::ld8(lane_base + rr * RW + (RW - 8), v + (RW - 8));
      tc::ld_wait();
      float s = 0.f;
#pragma unroll
      for (int b = 0; b < RW; ++b) s = fmaf(lb[b], v[b], s);
      const int k = r / p, a = r - k * p;
      const float w = sLa[a * 128 + t] * s;
      if (k == 0) acc[0] += w;
      else if (k == 1) acc[1] += w;
      else acc[2] += w;
    }
  }
  if (fail) {
    if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    if (warp == 0 && issued > 0) tc::mbar_wait(&mbar, (issued - 1) & 1, kTcWaitCycles);
  } else {
    if (half == 1) {
      sRed[t * 3] = acc[0];
      sRed[t * 3 + 1] = acc[1];
      sRed[t * 3 + 2] = acc[2];
    }
    __syncthreads();
    if (half == 0 && on) {
      const int64_t o = tperm[t0 + t];
      u[o * 3] += static_cast<double>(acc[0] + sRed[t * 3]);
      u[o * 3 + 1] += static_cast<double>(acc[1] + sRed[t * 3 + 1]);
      u[o * 3 + 2] += static_cast<double>(acc[2] + sRed[t * 3 + 2]);
    }
  }
  tc::cp_async_wait<0>();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// the failure path of the tensor-core kernels on purpose, without a fault: tensor
// memory allocated, an mbarrier that nothing arrives on, the bounded wait running
// out after max_cycles, the status bit, the tensor memory freed
__global__ void k_tc_wait_selftest(int* __restrict__ status, long long max_cycles) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  tc::sync_tc();
  if (warp == 0 && !tc::mbar_wait(&mbar, 0, max_cycles) && threadIdx.x == 0) atomicOr(status, ST_TC_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 32);
}

// ------------------------------------------------------------------ host side

// B-hat^R(k) in 3D, Eq. (Btrunc_hat); Taylor series of the bracket near k = 0
double b_trunc_hat(double k) {
  const double x = k * kRTrunc;
  if (x > 1e-2) return (1.0 + 0.5 * std::cos(x) - 1.5 * std::sin(x) / x) / (k * k * k * k);
  const double R4 = kRTrunc * kRTrunc * kRTrunc * kRTrunc;
  return R4 * (1.0 / 120.0 - x * x / 2520.0 + x * x * x * x / 120960.0);
}


// matrix bank of a parameter set (Chebyshev points, child matrices, plane-wave
// matrices, kernel tables): built once per process for each set
struct BankKey {
  int p, M, rK, periodic, fp32;
  double c;
  bool operator==(const BankKey& o) const {
    return p == o.p && M == o.M && rK == o.rK && periodic == o.periodic && fp32 == o.fp32 && c == o.c;
  }
};
struct CachedBank {
  std::vector<char> bank;
  size_t off[16];
  double sT_root;
};
std::mutex g_bank_mu;
std::vector<std::pair<BankKey, std::shared_ptr<const CachedBank>>> g_banks;
std::shared_ptr<const CachedBank> find_bank(const BankKey& k) {
  std::lock_guard<std::mutex> lk(g_bank_mu);
  for (auto& e : g_banks)
    if (e.first == k) return e.second;
  return nullptr;
}
void store_bank(const BankKey& k, std::shared_ptr<const CachedBank> b) {
  std::lock_guard<std::mutex> lk(g_bank_mu);
  g_banks.emplace_back(k, std::move(b));
}

struct RotLaunch {
  RotJob* jobs = nullptr;   // device
  int n = 0;
};


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
  int PB = 0;                        // padded proxy order of the leaf kernels
  size_t m_nodes = 0, m_bw = 0;      // Chebyshev points and barycentric weights in the bank
  void* W = nullptr;                 // [N][3][PB] Lagrange weights of the sources
  int32_t* src_leaf = nullptr;       // [nsrc_leaf] leaf index, then box id at + nsrc_leaf
  int32_t* trg_leaf = nullptr;
  int32_t* src_box_list = nullptr;   // boxes with sources (outgoing jobs order)
  int32_t* trg_box_list = nullptr;   // boxes with targets (incoming order)
  int n_ev_items = 0;                // leaf-evaluation work items: chunks of at most kEvThreads targets
  int32_t* ev_item_leaf = nullptr;   // index into the target-leaf list
  int32_t* ev_item_off = nullptr;    // first target of the chunk within its leaf
  int fused = 0;                     // 1: float32 transforms of a box in one kernel (shared memory fits)
  int tc = 0;                        // 1: float32 leaf charges and leaf evaluation on the tensor cores
  int tc_NP = 0, tc_RW = 0;          // their padded column count (3p) and row width (p)
  void* Vs = nullptr;                // [groups][N] float4 densities of the sources (tensor-core charges)
  int w_tiles = 1;                   // tiles of kWRows weight rows of the largest source leaf
  CUtensorMap tmW{}, tmV{};          // TMA maps of W as [N][3 PB] and of Vs as [groups N][4], 32-row boxes
  size_t fused_out_bytes = 0, fused_ev_bytes = 0;
  int32_t* coll = nullptr;           // [27] colleague slots of the root
  int32_t* root_tlist = nullptr;     // {target index of the root}
  int ngrp = 0;                      // parents whose children hold targets
  int32_t* grp_win = nullptr;        // [ngrp][64]
  int32_t* grp_ch = nullptr;         // [ngrp][8]
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
  // the same per level for the fused float32 kernels: parents and their 8 children
  int fused_tree = 0;
  size_t fused_tree_bytes = 0;
  std::vector<int32_t*> mf_par, mf_ch, if_par, if_ch;
  std::vector<int> mf_n, if_n;
  RotLaunch out1, out2, out3, ev1, ev2, ev3, r1, r2, r3, rv1, rv2, rv3;
  size_t bytes = 0;
  Far2State* d2 = nullptr;           // the 2D far field (far2d.cu) in place of all of the above
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
  const int n4 = (n_out + 3) & ~3;
  rot_smem_layout((two_mats ? 2 : 1) * n_in * n4 * sa, (two_mats ? 2 : 1) * n_in * kRotTile * sx, &offX, &offY);
  const size_t shm = offY + kRotTile * n_out * sy;
  const dim3 grid(L.n, (rest + kRotTile - 1) / kRotTile);
  const int nthr = ((16 * (n4 / 4) + 31) / 32) * 32;
  const char* base = static_cast<const char*>(F.mats);
  const void* A0 = base + matA0;
  const void* A1 = base + matA1;
  const int tm = two_mats ? 1 : 0;
#define DMK_ROT(XC_, AC_, YC_, MODE_)                                                                         \
  do {                                                                                                        \
    auto kern = k_rot<R, XC_, AC_, YC_, MODE_>;                                                               \
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm))); \
    kern<<<grid, nthr, shm, s>>>(L.jobs, X, Y, xoff, yoff, A0, A1, tm, n_in, n_out, rest);                   \
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

RotLaunch make_launch(Uploader& up, const std::vector<RotJob>& jobs) {
  RotLaunch L;
  L.n = static_cast<int>(jobs.size());
  if (L.n) L.jobs = up.put(jobs);
  return L;
}

}  // namespace

namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the
// driver library); null when the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}
// a row-major float32 [rows][inner] array read in boxes of 32 rows (inner x 4 bytes a
// multiple of 16, at most 256 elements)
bool encode_rows(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || rows == 0 || inner > 256 || (inner * 4) % 16) return false;
  const cuuint64_t dim[2] = {inner, rows};
  const cuuint64_t stride[1] = {inner * 4};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(inner), static_cast<cuuint32_t>(kTcK)};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dim, stride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void far_setup(Plan& p) {
  if (p.opts.dim == 2) {
    auto Fp = std::make_unique<FarState>();
    Fp->d2 = far2d_setup(p);
    p.far = Fp.release();
    return;
  }
  const DeviceTree& T = p.tree;
  const dmk_stokes_opts_t& o = p.opts;
  cudaStream_t s = p.stream;
  auto Fp = std::make_unique<FarState>();
  FarState& F = *Fp;
  Uploader up(p);
  F.fp32 = fp32_pair_terms(o) ? 1 : 0;
  const double c = p.tables.c;
  const int tcp = static_cast<int>(std::lround(3.0 * c / M_PI));
  F.p = table2_p(o.eps, o.kernels);
  if (o.bandlimit > 0) F.p = std::max(F.p, static_cast<int>(std::ceil(1.3 * tcp)));
  F.M = tcp - 1;                                   // N1 = 2 (3c/pi) - 1 modes a side
  F.nh = F.M + 1;
  F.nm = 2 * F.M + 1;
  if (F.p > 60 || F.nm > kMaxP) throw Error{DMK_ERR_UNSUPPORTED, "far-field order beyond the compiled maximum"};
  {
    const int cb = F.fp32 ? ant_chunk<float>() : ant_chunk<double>();
    F.PB = ((F.p + cb - 1) / cb) * cb;
    if (F.fp32 && F.PB > 48) throw Error{DMK_ERR_UNSUPPORTED, "far-field order beyond the compiled maximum"};
  }
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
  {
    int64_t mx = 1;
    for (int32_t li : src_leaf) mx = std::max<int64_t>(mx, cnt[li]);
    F.w_tiles = static_cast<int>(std::min<int64_t>((3 * mx + kWRows - 1) / kWRows, 65535));
  }
  F.ntrg_leaf = static_cast<int>(trg_leaf.size());
  // 27 colleague slots of the root (target index 0: boxes are sorted by level); the
  // other boxes take their colleagues from their parent's window below
  std::vector<int32_t> coll(27, -1);
  for (int t = 0; t < std::min(F.ntrg_box, 1); ++t) {
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
  // parent groups for the colleague sums of every non-root target box
  std::vector<int32_t> gwin, gch;
  for (int i = 0; i < nb; ++i) {
    const Box& b = boxes[i];
    if (b.leaf >= 0 || b.trg == 0) continue;
    const int l = b.lev + 1;
    const int64_t n = int64_t(1) << l;
    for (int w = 0; w < 64; ++w) {
      const int64_t wd[3] = {w & 3, (w >> 2) & 3, w >> 4};
      int64_t cc[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        cc[a] = 2 * b.c[a] - 1 + wd[a];
        if (o.periodic) cc[a] = ((cc[a] % n) + n) % n;
        else if (cc[a] < 0 || cc[a] >= n) ok = false;
      }
      int id = -1;
      if (ok) {
        auto it = at[l].find(morton<3>(cc));
        if (it != at[l].end() && boxes[it->second].src > 0) id = it->second;
      }
      gwin.push_back(id);
    }
    for (int ch = 0; ch < 8; ++ch) gch.push_back(trg_index[b.child[ch]]);
  }
  F.ngrp = static_cast<int>(gch.size() / 8);
  F.grp_win = up.put(gwin);
  F.grp_ch = up.put(gch);
  F.root_tlist = up.put(std::vector<int32_t>{trg_index[0]});
  std::vector<BoxGeo> geo(nb);
  std::vector<int32_t> blev(nb);
  for (int i = 0; i < nb; ++i) {
    const double r = std::ldexp(1.0, -boxes[i].lev);
    geo[i] = BoxGeo{(boxes[i].c[0] + 0.5) * r, (boxes[i].c[1] + 0.5) * r, (boxes[i].c[2] + 0.5) * r, 0.5 * r};
    blev[i] = boxes[i].lev;
  }

  // ---- matrices and tables (depend on the parameters only; kept per process) ----
  const int P = F.p;
  const BankKey bkey{F.p, F.M, F.rK, o.periodic, F.fp32, c};
  std::shared_ptr<const CachedBank> cached = find_bank(bkey);
  std::vector<char> bank;
  if (cached) {
    bank = cached->bank;
    const size_t* m = cached->off;
    F.m_nodes = m[0]; F.m_bw = m[1]; F.m_T0 = m[2]; F.m_T1 = m[3]; F.m_T0t = m[4]; F.m_T1t = m[5];
    F.m_Eh = m[6]; F.m_E = m[7]; F.m_Fh = m[8]; F.m_F = m[9]; F.m_REh = m[10]; F.m_RE = m[11];
    F.m_RFh = m[12]; F.m_RF = m[13]; F.m_tab = m[14]; F.m_rtab = m[15];
    F.sT_root = cached->sT_root;
  } else {
    MatBank mb;
    mb.f32 = F.fp32;
    std::vector<double> nodes, bwt;
    cheb_nodes_bw(P, nodes, bwt);
    auto put_real = [&](const std::vector<double>& v) { return mb.put_real(v); };
    F.m_nodes = put_real(nodes);
    F.m_bw = put_real(bwt);
    // child -> parent anterpolation T_o[a][i] = L_a(((2o - 1) + xi_i) / 2), and the transposes
    for (int oo = 0; oo < 2; ++oo) {
      std::vector<double> Tm(P * P), Tt(P * P);
      for (int a = 0; a < P; ++a)
        for (int i = 0; i < P; ++i) {
          const double v = lagrange_host(nodes, ((2 * oo - 1) + nodes[i]) / 2.0, a);
          Tm[a * P + i] = v;
          Tt[i * P + a] = v;
        }
      (oo == 0 ? F.m_T0 : F.m_T1) = put_real(Tm);
      (oo == 0 ? F.m_T0t : F.m_T1t) = put_real(Tt);
    }
    // plane-wave matrices: E[m][j] = e^{-i theta m xi_j}; F[a][m] = w_m e^{+i theta m xi_a}
    const double th_l = M_PI / 3.0;
    F.m_Eh = mb.plane_wave(nodes, 0, F.nh, th_l, false, true);
    F.m_E = mb.plane_wave(nodes, -F.M, F.nm, th_l, false, false);
    F.m_Fh = mb.plane_wave(nodes, 0, F.nh, th_l, true, true);
    F.m_F = mb.plane_wave(nodes, -F.M, F.nm, th_l, true, false);
    const double th_r = o.periodic ? M_PI : 0.5 * h0;
    F.m_REh = mb.plane_wave(nodes, 0, F.rnh, th_r, false, true);
    F.m_RE = mb.plane_wave(nodes, -F.rK, F.rnm, th_r, false, false);
    F.m_RFh = mb.plane_wave(nodes, 0, F.rnh, th_r, true, true);
    F.m_RF = mb.plane_wave(nodes, -F.rK, F.rnm, th_r, true, false);
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
    bank = std::move(mb.bytes);
    auto cb = std::make_shared<CachedBank>();
    cb->bank = bank;
    const size_t offs[16] = {F.m_nodes, F.m_bw, F.m_T0, F.m_T1, F.m_T0t, F.m_T1t, F.m_Eh, F.m_E,
                             F.m_Fh, F.m_F, F.m_REh, F.m_RE, F.m_RFh, F.m_RF, F.m_tab, F.m_rtab};
    for (int i = 0; i < 16; ++i) cb->off[i] = offs[i];
    cb->sT_root = F.sT_root;
    store_bank(bkey, cb);
  }
  F.mats = up.put(bank);
  F.box_geo = up.put(geo);
  F.box_level = up.put(blev);
  {
    std::vector<int32_t> sl(src_leaf);
    sl.insert(sl.end(), src_leaf_box.begin(), src_leaf_box.end());
    F.src_leaf = up.put(sl);
    std::vector<int32_t> tl(trg_leaf);
    tl.insert(tl.end(), trg_leaf_box.begin(), trg_leaf_box.end());
    F.trg_leaf = up.put(tl);
  }
  F.src_box_list = up.put(src_boxes);
  F.trg_box_list = up.put(trg_boxes);
  {
    std::vector<int32_t> il, io;
    for (size_t e = 0; e < trg_leaf.size(); ++e) {
      const int nt = tcnt[trg_leaf[e]];
      for (int off = 0; off < nt; off += kEvThreads) {
        il.push_back(static_cast<int32_t>(e));
        io.push_back(off);
      }
    }
    F.n_ev_items = static_cast<int>(il.size());
    F.ev_item_leaf = up.put(il);
    F.ev_item_off = up.put(io);
  }
  if (F.fp32) {
    F.fused_out_bytes = fused_out_smem(F.p, F.nh, F.nm, sizeof(float));
    F.fused_ev_bytes = fused_ev_smem(F.p, F.nh, F.nm, sizeof(float));
    int dev_smem = 0;
    DMK_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device));
    F.fused = (std::max(F.fused_out_bytes, F.fused_ev_bytes) <= static_cast<size_t>(dev_smem)) ? 1 : 0;
    F.fused_tree_bytes = fused_tree_smem(F.p, sizeof(float));
    F.fused_tree = F.fused_tree_bytes <= static_cast<size_t>(dev_smem) ? 1 : 0;
    // tensor cores for the leaf kernels unless DMK_STOKES_FAR_TC=0 (the FP32-pipe kernels then run)
    const char* env = std::getenv("DMK_STOKES_FAR_TC");
    F.tc_NP = ((3 * F.p + 15) / 16) * 16;
    F.tc_RW = std::max(16, ((F.p + 7) / 8) * 8);
    F.tc = (!(env && env[0] == '0') && F.tc_NP <= 128 && F.tc_RW <= 40 &&
            anterp_tc_smem(F.tc_NP, F.PB) <= static_cast<size_t>(dev_smem)) ? 1 : 0;
  }
  F.coll = up.put(coll);
  F.root_box = up.put(std::vector<int32_t>{0});

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
  // the generic stage kernels (and their job lists and scratch) serve what the fused
  // float32 kernels do not: the root always, the boxes when the fused kernels are off
  int64_t max_jobs = F.fused ? 1 : std::max<int64_t>(std::max(F.nsrc_box, F.ntrg_box), 1);
  // merges: parent at level l (non-leaf, with sources), per component
  for (int l = maxlev - 1; l >= 0; --l) {
    std::vector<RotJob> j1, j2, j3;
    std::vector<int32_t> fpar, fch;
    int np = 0;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.src == 0) continue;
      fpar.push_back(i);
      for (int ch = 0; ch < 8; ++ch) fch.push_back(boxes[b.child[ch]].src ? b.child[ch] : -1);
      if (F.fused_tree) {
        ++np;
        continue;
      }
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
    F.mf_par.push_back(up.put(fpar));
    F.mf_ch.push_back(up.put(fch));
    F.mf_n.push_back(np);
    F.merge_level.push_back(l);
    F.merge[0].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j1));
    F.merge[1].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j2));
    F.merge[2].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j3));
    if (!F.fused_tree)
      max_jobs = std::max<int64_t>(max_jobs, (static_cast<int64_t>(np) * nc * 4 * P3 + 2 * st - 1) / (2 * st) + 1);
  }
  // interpolation: parent at level l (non-leaf, with targets) to its children with targets
  for (int l = 0; l < maxlev; ++l) {
    std::vector<RotJob> j1, j2, j3;
    std::vector<int32_t> fpar, fch;
    int np = 0;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.trg == 0) continue;
      fpar.push_back(i);
      for (int ch = 0; ch < 8; ++ch) fch.push_back(boxes[b.child[ch]].trg ? b.child[ch] : -1);
      if (F.fused_tree) {
        ++np;
        continue;
      }
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
    F.if_par.push_back(up.put(fpar));
    F.if_ch.push_back(up.put(fch));
    F.if_n.push_back(np);
    F.interp_level.push_back(l);
    F.interp[0].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j1));
    F.interp[1].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j2));
    F.interp[2].push_back(F.fused_tree ? RotLaunch{} : make_launch(up, j3));
    if (!F.fused_tree)
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
    if (!F.fused) {
      F.out1 = make_launch(up, a1);
      F.out2 = make_launch(up, a2);
      F.out3 = make_launch(up, a3);
      F.ev1 = make_launch(up, e1);
      F.ev2 = make_launch(up, e2);
      F.ev3 = make_launch(up, e3);
    }
    RotJob J;
    J.x1 = -1;
    J.a0 = J.a1 = 0;
    J.x0 = 0;
    J.y = 0;
    // one job at offset 0 for every root stage: q[root], the scratch, pot[root] (+ component offsets)
    const RotLaunch one = make_launch(up, std::vector<RotJob>{J});
    F.r1 = F.r2 = F.r3 = F.rv1 = F.rv2 = F.rv3 = one;
  }
  up.flush();
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
  F.W = big(static_cast<size_t>(std::max<int64_t>(T.N, 1)) * 3 * F.PB * er);
  if (F.tc) {
    F.Vs = big(static_cast<size_t>(std::max<int64_t>(T.N, 1)) * (F.ncomp / 3) * sizeof(float4));
    if (T.N > 0 && !(encode_rows(&F.tmW, F.W, 3 * static_cast<uint64_t>(F.PB), static_cast<uint64_t>(T.N)) &&
                     encode_rows(&F.tmV, F.Vs, 4, static_cast<uint64_t>(T.N) * (F.ncomp / 3))))
      F.tc = 0;                      // no tensor maps here: the FP32-pipe leaf kernels
  }
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  p.far = Fp.release();
}

void far_free(Plan& p) {
  FarState* F = p.far;
  if (!F) return;
  if (F->d2) far2d_free(p, F->d2);
  for (void** b : {&F->q, &F->pot, &F->O, &F->I, &F->s1, &F->s2, &F->rO, &F->W, &F->Vs})
    if (*b) cudaFreeAsync(*b, p.stream);
  delete F;                                   // small arrays live in the plan's arena
  p.far = nullptr;
}

size_t far_bytes(const Plan& p) { return p.far ? (p.far->d2 ? far2d_bytes(*p.far->d2) : p.far->bytes) : 0; }

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
  const R* nodes = reinterpret_cast<const R*>(mats + F.m_nodes);
  const R* bw = reinterpret_cast<const R*>(mats + F.m_bw);
  const int PB = F.PB;
  // stage boundaries for dmk_stokes_eval_traced (events 2..9; 0 and 1 bracket the near pass)
  auto mark = [&](int i) {
    if (p.trace) DMK_CUDA_TRY(cudaEventRecord(p.trace[i], s));
  };
  // 1. Lagrange weights of the sources, leaf proxy charges
  if (F.nsrc_leaf > 0) {
    R* W = static_cast<R*>(F.W);
    const size_t wshm = static_cast<size_t>(kWRows) * (PB + 1) * sizeof(R);
    DMK_CUDA_TRY(cudaFuncSetAttribute(k_far_weights<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(wshm)));
    k_far_weights<R><<<dim3(F.nsrc_leaf, F.w_tiles), kWRows, wshm, s>>>(F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start, T.leaf_count, T.w,
                                                 T.N, F.box_geo, P, PB, nodes, bw, W);
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
    const int g0 = F.slot_f >= 0 ? 0 : 1;
    const int ng = (F.slot_f >= 0 ? 1 : 0) + (F.slot_t >= 0 ? 2 : 0);
    if constexpr (sizeof(R) == 4) {
      if (F.tc) {
        float4* Vs = static_cast<float4*>(F.Vs);
        k_far_values<<<grid_for(T.N, 256), 256, 0, s>>>(T.perm, d_f, d_g, d_n, T.N, g0, ng, Vs);
        DMK_CUDA_TRY(cudaGetLastError());
        ++p.launches;
        const size_t shm_tc = anterp_tc_smem(F.tc_NP, PB);
        DMK_CUDA_TRY(cudaFuncSetAttribute(k_far_anterp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(shm_tc)));
        const unsigned nmt = static_cast<unsigned>((P * P + 127) / 128);
        k_far_anterp_tc<<<dim3(F.nsrc_leaf * nmt, ng), kTcThreads, shm_tc, s>>>(
            F.tmW, F.tmV, F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start, T.leaf_count, T.N, F.slot_f, F.slot_t,
            nc, q, P, PB, F.tc_NP, p.status);
        DMK_CUDA_TRY(cudaGetLastError());
        ++p.launches;
      }
    }
  }
  if (F.nsrc_leaf > 0 && !(F.tc && sizeof(R) == 4)) {
    R* W = static_cast<R*>(F.W);
    const size_t shm = (static_cast<size_t>(kAntChunk) * 3 * PB + 4 * kAntChunk) * sizeof(R);
    auto kern = k_far_anterp<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    const int ntask = P * P * (PB / ant_chunk<R>());
    // the (a, b, c-chunk) tasks of a leaf spread over nz blocks of nthr threads
    const int nz = (ntask + kAntThreads - 1) / kAntThreads;
    const int nthr = (((ntask + nz - 1) / nz + 31) / 32) * 32;
    const int g0 = F.slot_f >= 0 ? 0 : 1;
    const int ng = (F.slot_f >= 0 ? 1 : 0) + (F.slot_t >= 0 ? 2 : 0);
    kern<<<dim3(F.nsrc_leaf, ng, nz), nthr, shm, s>>>(F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start, T.leaf_count, W,
                                                  T.perm, d_f, d_g, d_n, g0, F.slot_f, F.slot_t, nc, q, P, PB);
    DMK_CUDA_TRY(cudaGetLastError());
    p.launches += 1;
  }
  mark(2);
  // 2. upward merges, finest parents first
  const bool ftree = F.fused_tree && sizeof(R) == 4;
  if constexpr (sizeof(R) == 4) {
    if (ftree) {
      auto kern = k_far_merge_fused<R>;
      DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(F.fused_tree_bytes)));
      for (size_t i = 0; i < F.merge_level.size(); ++i) {
        kern<<<dim3(F.mf_n[i], nc), 1024, F.fused_tree_bytes, s>>>(F.mf_par[i], F.mf_ch[i], q, nc,
                                                                   reinterpret_cast<const R*>(mats + F.m_T0),
                                                                   reinterpret_cast<const R*>(mats + F.m_T1), P);
        DMK_CUDA_TRY(cudaGetLastError());
        ++p.launches;
      }
    }
  }
  for (size_t i = 0; i < (ftree ? 0 : F.merge_level.size()); ++i) {
    launch_rot(p, F.merge[0][i], q, F.s1, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.merge[1][i], F.s1, F.s2, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.merge[2][i], F.s2, q, 0, 0, F.m_T0, F.m_T1, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
  }
  mark(3);
  // 3. outgoing plane waves of every box with sources, contracted with the level kernel
  const R* tab = reinterpret_cast<const R*>(mats + F.m_tab);
  const bool fused = F.fused && sizeof(R) == 4;
  if constexpr (sizeof(R) == 4) {
    if (fused && F.nsrc_box > 0) {
      auto kern = k_far_out_fused<R>;
      DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(F.fused_out_bytes)));
      kern<<<F.nsrc_box, 1024, F.fused_out_bytes, s>>>(F.src_box_list, F.box_level, q, nc, F.slot_f, F.slot_t,
                                                       reinterpret_cast<const C*>(mats + F.m_Eh),
                                                       reinterpret_cast<const C*>(mats + F.m_E), tab, O, P, F.M, nh, nm);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
  }
  for (int k = 0; k < (fused ? 0 : nc); ++k) {
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
  mark(4);
  // 4. incoming expansions (colleague sums) and their potential grids (written)
  {
    if (F.ntrg_box > 0) {
      k_far_colleague<R><<<grid_for(3 * F.modes, 256), 256, 0, s>>>(1, F.root_tlist, F.coll, O, I, F.M, nh, nm);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
    if (F.ngrp > 0) {
      const dim3 grid(F.ngrp, 3, static_cast<unsigned>((F.modes + kGrpThreads - 1) / kGrpThreads));
      k_far_colleague_grp<R><<<grid, kGrpThreads, 0, s>>>(F.grp_win, F.grp_ch, O, I, F.M, nh, nm);
      DMK_CUDA_TRY(cudaGetLastError());
      ++p.launches;
    }
    mark(5);
    if constexpr (sizeof(R) == 4) {
      if (fused && F.ntrg_box > 0) {
        auto kern = k_far_ev_fused<R>;
        DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(F.fused_ev_bytes)));
        kern<<<F.ntrg_box, 1024, F.fused_ev_bytes, s>>>(F.trg_box_list, I, reinterpret_cast<const C*>(mats + F.m_Fh),
                                                        reinterpret_cast<const C*>(mats + F.m_F), pot, P, nh, nm);
        DMK_CUDA_TRY(cudaGetLastError());
        ++p.launches;
      }
    }
    for (int k = 0; k < (fused ? 0 : 3); ++k) {
      launch_rot(p, F.ev1, I, F.s1, k * F.modes, 0, F.m_Fh, F.m_Fh, false, nh, P, nm * nm, 1, 1, 1, 0, s);
      launch_rot(p, F.ev2, F.s1, F.s2, 0, 0, F.m_F, F.m_F, false, nm, P, nm * P, 1, 1, 1, 0, s);
      launch_rot(p, F.ev3, F.s2, pot, 0, k * P3, F.m_F, F.m_F, false, nm, P, static_cast<int>(p2), 1, 1, 0, 0, s);
    }
  }
  mark(6);
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
  mark(7);
  // 6. interpolation down the tree
  if constexpr (sizeof(R) == 4) {
    if (ftree) {
      auto kern = k_far_interp_fused<R>;
      DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(F.fused_tree_bytes)));
      for (size_t i = 0; i < F.interp_level.size(); ++i) {
        kern<<<dim3(F.if_n[i], 3), 1024, F.fused_tree_bytes, s>>>(F.if_par[i], F.if_ch[i], pot,
                                                                  reinterpret_cast<const R*>(mats + F.m_T0t),
                                                                  reinterpret_cast<const R*>(mats + F.m_T1t), P);
        DMK_CUDA_TRY(cudaGetLastError());
        ++p.launches;
      }
    }
  }
  for (size_t i = 0; i < (ftree ? 0 : F.interp_level.size()); ++i) {
    launch_rot(p, F.interp[0][i], pot, F.s1, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.interp[1][i], F.s1, F.s2, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 0, s);
    launch_rot(p, F.interp[2][i], F.s2, pot, 0, 0, F.m_T0t, F.m_T1t, true, P, P, static_cast<int>(p2), 0, 0, 0, 1, s);
  }
  mark(8);
  // 7. leaf grids at the targets
  if (F.n_ev_items > 0) {
    const size_t shm = (2 * static_cast<size_t>(P) * kEvThreads + 2 * 3 * static_cast<size_t>(P) * PB) * sizeof(R);
    auto go = [&](auto kern, int tt) {
      const int nth = kEvThreads / tt;
      DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
      if (T.sep)
        kern<<<F.n_ev_items, nth, shm, s>>>(F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                                                   T.leaf_tstart, nullptr, T.tw, T.NT, T.tperm, F.box_geo, pot, P,
                                                   nodes, bw, d_u);
      else
        kern<<<F.n_ev_items, nth, shm, s>>>(F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                                                   T.leaf_start, T.leaf_count, T.w, T.N, T.perm, F.box_geo, pot, P,
                                                   nodes, bw, d_u);
    };
    if constexpr (sizeof(R) == 4) {
      if (F.tc) {
        auto go_tc = [&](auto kern, size_t shm_tc) {
          DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm_tc)));
          if (T.sep)
            kern<<<F.n_ev_items, kTcThreads, shm_tc, s>>>(F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                                                   T.leaf_tstart, nullptr, T.tw, T.NT, T.tperm, F.box_geo, pot, P, nodes,
                                                   bw, d_u, p.status);
          else
            kern<<<F.n_ev_items, kTcThreads, shm_tc, s>>>(F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                                                   T.leaf_start, T.leaf_count, T.w, T.N, T.perm, F.box_geo, pot, P, nodes,
                                                   bw, d_u, p.status);
        };
        switch (F.tc_RW) {
          case 16: go_tc(k_far_eval_tc<16>, eval_tc_smem_t<16>(P)); break;
          case 24: go_tc(k_far_eval_tc<24>, eval_tc_smem_t<24>(P)); break;
          case 32: go_tc(k_far_eval_tc<32>, eval_tc_smem_t<32>(P)); break;
          default: go_tc(k_far_eval_tc<40>, eval_tc_smem_t<40>(P)); break;
        }
      } else if (PB == 24) go(k_far_eval<R, 24, 2>, 2);
      else go(k_far_eval<R, 48, 1>, 1);
    } else {
      switch (PB) {
        case 12: go(k_far_eval<R, 12, 1>, 1); break;
        case 24: go(k_far_eval<R, 24, 1>, 1); break;
        case 36: go(k_far_eval<R, 36, 1>, 1); break;
        case 48: go(k_far_eval<R, 48, 1>, 1); break;
        default: go(k_far_eval<R, 60, 1>, 1); break;
      }
    }
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
  }
  mark(9);
}

}  // namespace

bool tc_wait_selftest(cudaStream_t s) {
  int* d = nullptr;
  int h = 0;
  DMK_CUDA_TRY(cudaMallocAsync(&d, sizeof(int), s));
  DMK_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int), s));
  k_tc_wait_selftest<<<1, 128, 0, s>>>(d, 2000000LL);      // about 1 ms of SM clock
  DMK_CUDA_TRY(cudaGetLastError());
  DMK_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  DMK_CUDA_TRY(cudaFreeAsync(d, s));
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  return (h & ST_TC_TIMEOUT) != 0;
}

void far_run(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u, cudaStream_t s) {
  if (!p.far || !d_u || p.tree.N == 0) return;
  if (p.far->d2) far2d_run(p, *p.far->d2, d_f, d_g, d_n, d_u, s);
  else if (p.far->fp32) far_run_t<float>(p, d_f, d_g, d_n, d_u, s);
  else far_run_t<double>(p, d_f, d_g, d_n, d_u, s);
}

void far_info(const Plan& p, int32_t info[8]) {
  for (int i = 0; i < 8; ++i) info[i] = 0;
  const FarState* F = p.far;
  if (!F) return;
  if (F->d2) {
    far2d_info(*F->d2, info);
    return;
  }
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
