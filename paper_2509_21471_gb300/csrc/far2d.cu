// DMK far field in 2D (components = ALL): the steps of the 3D path on p x p proxy
// grids with N1 x N1 plane waves, 9 colleagues and the App. B kernels.
//
// Sec. 6.1 Steps 1(c), 2, 3, Sec. 6.2 and App. B, with the parameters of Table 2:
//   * box B at level l (side r_l = 2^-l, centre c_B) carries the p x p grid
//     z = c_B + (r_l / 2) (xi_a, xi_b), xi the Chebyshev points of the first kind;
//   * upward pass: leaf proxy charges q_j = sum_s L_j(x_s) rho_s with rho = f (two
//     components) for the Stokeslet and the symmetric part of g (x) n (rho_00,
//     rho_11, rho_01) for the stresslet; a parent takes its children's charges;
//   * level-l plane waves k = h m, h = 2 pi / (3 r_l), m_0 in [0, M], m_1 in [-M, M]
//     (the potential is real, so the m_0 < 0 half is the conjugate):
//         O_B(m) = (h / 2 pi)^2 K-hat_D,l(hm) . sum_j q_j e^{-i h m.(z_j - c_B)},
//     B-hat of K_D,l = (gamma-hat(k r_{l+1}) - gamma-hat(k r_l)) / k^4.  With q = |m|^2
//     the Stokeslet part is t(q) (q rho_j - m_j m.rho), t = dgamma / (4 pi^2 q^2), the
//     same at every level (the powers of h cancel in 2D), and the stresslet part
//     carries one factor h;
//   * colleagues C = B + delta: I_B(m) = sum_C e^{-2 pi i m.delta / 3} O_C(m), and
//     pot_B(z) += Re sum_m e^{i h m.(z - c_B)} I_B(m) (weights 1, 2, 2, ... on m_0);
//   * root: the periodic Fourier series of K_M,0 over k = 2 pi kappa, or the
//     truncated kernel B-hat^R gamma-hat of Eq. (Btrunc_hat) with R = 1 + sqrt 2 by
//     the trapezoidal rule with spacing h0 = 2 pi / (2 + 2 sqrt 2), plus the constant
//     K_corr = (1 - log R) / (4 pi) times sum f for the free-space Stokeslet (Sec. 5.3);
//   * downward pass: parents interpolate their grids to their children; leaves
//     evaluate their grids at their targets.
//
// GPU layout.  A 2D box is small (p^2 grid values, (M + 1)(2M + 1) modes), so every
// transform of a box runs in one block from shared memory: outgoing waves with the
// kernel contraction, incoming grids, child merges and interpolation (one block per
// parent), colleague sums (one block per parent for its four children, the phases
// separable over the two axes).  Arithmetic is FP32 when the plan's pair terms are
// FP32 (MIXED at eps >= 2e-7), FP64 otherwise; target velocities accumulate in FP64.
#include "far_common.cuh"

#include <memory>
#include <unordered_map>

namespace dmk {

using namespace farc;

namespace {

constexpr double kRTrunc2 = 2.4142135623730951;   // R = 1 + sqrt(2)
constexpr int kBox2Threads = 256;                 // threads of the per-box kernels
constexpr int kAnt2Chunk = 64;                    // sources per shared-memory pass
constexpr int kEv2Threads = 128;                  // targets per leaf-evaluation block

// Lagrange weights of every point of the listed leaves: W[s][axis][PB] (zero past p)
template <typename R>
__global__ void k_far2_weights(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                               const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                               const double* __restrict__ w, int64_t N, const BoxGeo* __restrict__ box_geo, int p,
                               int PB, const R* __restrict__ nodes, const R* __restrict__ bw, R* __restrict__ W) {
  __shared__ R s_nodes[kMaxP], s_bw[kMaxP];
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  __syncthreads();
  const int li = leaf_list[blockIdx.x];
  const BoxGeo geo = box_geo[leaf_box[blockIdx.x]];
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const double inv_half = 1.0 / geo.w;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < 2 * ns; i += gridDim.y * blockDim.x) {   // rows over blockIdx.y
    const int sl = i >> 1, ax = i & 1;
    const int64_t si = s0 + sl;
    const R t = static_cast<R>((w[ax * N + si] - (ax == 0 ? geo.x : geo.y)) * inv_half);
    lagrange_row<R>(t, p, s_nodes, s_bw, W + (si * 2 + ax) * PB, 1, PB);
  }
}

// leaf proxy charges q[box][slot + k][a][b] = sum_s L_a(x_s) L_b(y_s) v_s,k for the
// components of group blockIdx.y (0: f_0, f_1 at slot_f; 1: rho_00, rho_11, rho_01 at
// slot_t).  A thread owns one a and four consecutive b; the leaf's weights stream
// through shared memory kAnt2Chunk sources at a time.
template <typename R>
__global__ void __launch_bounds__(512) k_far2_anterp(const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                     const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_count,
                                                     const R* __restrict__ W, const int32_t* __restrict__ perm,
                                                     const double* __restrict__ f, const double* __restrict__ g,
                                                     const double* __restrict__ nrm, int grp0, int slot_f, int slot_t,
                                                     int ncomp, R* __restrict__ q, int p, int PB) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sW = reinterpret_cast<R*>(smem);                 // [kAnt2Chunk][2][PB]
  R* sV = sW + kAnt2Chunk * 2 * PB;                   // [kAnt2Chunk][4]
  const int li = leaf_list[blockIdx.x];
  const int box = leaf_box[blockIdx.x];
  const int grp = grp0 + blockIdx.y;
  const int slot = grp == 0 ? slot_f : slot_t;
  const int nk = grp == 0 ? 2 : 3;
  const int s0 = leaf_start[li], ns = leaf_count[li];
  const int nb4 = PB / 4, ntask = p * nb4;
  const int64_t p2 = static_cast<int64_t>(p) * p;
  R* qb = q + (static_cast<int64_t>(box) * ncomp + slot) * p2;
  for (int t0 = 0; t0 < ntask; t0 += blockDim.x) {
    const int task = t0 + threadIdx.x;
    const bool on = task < ntask;
    const int a = on ? task / nb4 : 0;
    const int b0 = on ? (task - a * nb4) * 4 : 0;
    R acc[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = R(0);
    for (int sc = 0; sc < ns; sc += kAnt2Chunk) {
      const int nc = min(kAnt2Chunk, ns - sc);
      __syncthreads();
      const R* src = W + (static_cast<int64_t>(s0) + sc) * 2 * PB;
      for (int i = threadIdx.x; i < nc * 2 * PB; i += blockDim.x) sW[i] = src[i];
      for (int sl = threadIdx.x; sl < nc; sl += blockDim.x) {
        const int64_t o = perm[s0 + sc + sl];
        double v0, v1, v2 = 0.0;
        if (grp == 0) {
          v0 = f[o * 2];
          v1 = f[o * 2 + 1];
        } else {
          const double g0 = g[o * 2], g1 = g[o * 2 + 1], n0 = nrm[o * 2], n1 = nrm[o * 2 + 1];
          v0 = g0 * n0;
          v1 = g1 * n1;
          v2 = 0.5 * (g0 * n1 + g1 * n0);
        }
        sV[sl * 4] = static_cast<R>(v0);
        sV[sl * 4 + 1] = static_cast<R>(v1);
        sV[sl * 4 + 2] = static_cast<R>(v2);
        sV[sl * 4 + 3] = R(0);
      }
      __syncthreads();
      if (on) {
        for (int sl = 0; sl < nc; ++sl) {
          const R* ws = sW + sl * 2 * PB;
          const R wa = ws[a];
          R wb[4], fv[4];
          ld4(ws + PB + b0, wb);
          ld4(sV + sl * 4, fv);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const R wv = wa * wb[i];
            acc[i][0] = fma(wv, fv[0], acc[i][0]);
            acc[i][1] = fma(wv, fv[1], acc[i][1]);
            acc[i][2] = fma(wv, fv[2], acc[i][2]);
          }
        }
      }
    }
    if (on) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = b0 + i;
        if (b < p)
          for (int k = 0; k < nk; ++k) qb[k * p2 + static_cast<int64_t>(a) * p + b] = acc[i][k];
      }
    }
  }
}

// the kernel contraction of one component's spectrum x at mode (m0, m1), q = |m|^2:
//   Stokeslet component l (comp 0, 1):          O_j += sS t (q delta_jl - m_j m_l) x
//   stresslet component G (comp 2, 3, 4 = 00, 11, 01 + 10):
//                                               O_j += i sT t [q ((G + G^T) m + m tr G)_j - 2 m_j m.G.m] x
template <typename R>
__device__ __forceinline__ void contract2(int comp, R m0, R m1, R qq, R sS, R sT, R t, R xr, R xi, R* o_r, R* o_i) {
  const R mv[2] = {m0, m1};
  if (comp < 2) {
    const R s = sS * t;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const R c = s * ((j == comp ? qq : R(0)) - mv[j] * mv[comp]);
      o_r[j] = fma(c, xr, o_r[j]);
      o_i[j] = fma(c, xi, o_i[j]);
    }
  } else {
    const R s = sT * t;
    const int cc = comp - 2;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      R v;
      if (cc < 2) v = qq * (R(2) * (j == cc ? mv[cc] : R(0)) + mv[j]) - R(2) * mv[j] * mv[cc] * mv[cc];
      else v = R(2) * qq * (j == 0 ? mv[1] : mv[0]) - R(4) * mv[j] * mv[0] * mv[1];
      const R c = s * v;          // O_j += i c x
      o_r[j] = fma(-c, xi, o_r[j]);
      o_i[j] = fma(c, xr, o_i[j]);
    }
  }
}

// outgoing plane waves of one box (block g of the list), all components, in shared memory:
//   Y[m0][b] = sum_a Eh[m0][a] q[a][b];  S[m0][m1] = sum_b E[m1][b] Y[m0][b],
// contracted with the kernel table and written to O[g or box][2][nh * nm].  Level boxes:
// table tab, sS = 1, sT = h = 2 pi 2^l / 3; the root (root = 1): its table and factors.
inline size_t out2_smem(int p, int nh, int nm, size_t er) {
  const size_t ec = 2 * er;
  return align16(static_cast<size_t>(nh) * p * ec) + align16(static_cast<size_t>(p) * nm * ec) +
         align16(static_cast<size_t>(p) * p * er) + align16(static_cast<size_t>(nh) * p * ec) +
         align16(2 * static_cast<size_t>(nh) * nm * ec);
}
template <typename R>
__global__ void __launch_bounds__(kBox2Threads) k_far2_out(const int32_t* __restrict__ boxes, const int32_t* __restrict__ box_level,
                                                           const R* __restrict__ q, int ncomp, int slot_f, int slot_t,
                                                           const typename Cplx<R>::T* __restrict__ Eh,
                                                           const typename Cplx<R>::T* __restrict__ E, const R* __restrict__ tab,
                                                           typename Cplx<R>::T* __restrict__ O, int root, double sS_root,
                                                           double sT_root, int p, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t ec = sizeof(C);
  C* sEh = reinterpret_cast<C*>(smem);                                                  // [nh][p]
  unsigned char* ptr = smem + align16(static_cast<size_t>(nh) * p * ec);
  C* sET = reinterpret_cast<C*>(ptr);                                                   // [p][nm]: E transposed
  ptr += align16(static_cast<size_t>(p) * nm * ec);
  R* sX = reinterpret_cast<R*>(ptr);                                                    // [p][p]
  ptr += align16(static_cast<size_t>(p) * p * sizeof(R));
  C* sY = reinterpret_cast<C*>(ptr);                                                    // [nh][p]
  ptr += align16(static_cast<size_t>(nh) * p * ec);
  C* sO = reinterpret_cast<C*>(ptr);                                                    // [2][nh * nm]
  const int box = boxes[blockIdx.x];
  for (int i = threadIdx.x; i < nh * p; i += blockDim.x) sEh[i] = Eh[i];
  for (int i = threadIdx.x; i < p * nm; i += blockDim.x) {
    const int j = i / nm, m = i - j * nm;
    sET[i] = E[m * p + j];
  }
  R sS, sT;
  if (root) {
    sS = static_cast<R>(sS_root);
    sT = static_cast<R>(sT_root);
  } else {
    sS = R(1);
    sT = static_cast<R>(2.0 * M_PI / 3.0 * ldexp(1.0, box_level[box]));    // h at the level (up to 31 in 2D)
  }
  const int p2 = p * p, modes = nh * nm;
  for (int k = 0; k < ncomp; ++k) {
    const int comp = (slot_f >= 0 && k < 2) ? k : 2 + (k - slot_t);
    const R* qk = q + (static_cast<int64_t>(box) * ncomp + k) * p2;
    __syncthreads();
    for (int i = threadIdx.x; i < p2; i += blockDim.x) sX[i] = qk[i];
    __syncthreads();
    for (int i = threadIdx.x; i < nh * p; i += blockDim.x) {
      const int m0 = i / p, b = i - m0 * p;
      const C* e = sEh + m0 * p;
      R yr = R(0), yi = R(0);
      for (int a = 0; a < p; ++a) {
        const R x = sX[a * p + b];
        yr = fma(e[a].x, x, yr);
        yi = fma(e[a].y, x, yi);
      }
      sY[i] = C{yr, yi};
    }
    __syncthreads();
    for (int mi = threadIdx.x; mi < modes; mi += blockDim.x) {
      const int m0 = mi / nm, m1i = mi - m0 * nm;
      const C* y = sY + m0 * p;
      R sr = R(0), si = R(0);
      for (int b = 0; b < p; ++b) {
        const C e = sET[b * nm + m1i], v = y[b];
        sr = fma(e.x, v.x, sr);
        sr = fma(-e.y, v.y, sr);
        si = fma(e.x, v.y, si);
        si = fma(e.y, v.x, si);
      }
      const int m1 = m1i - Mh;
      const int qi = m0 * m0 + m1 * m1;
      R o_r[2] = {R(0), R(0)}, o_i[2] = {R(0), R(0)};
      if (k > 0) {
        o_r[0] = sO[mi].x;
        o_i[0] = sO[mi].y;
        o_r[1] = sO[modes + mi].x;
        o_i[1] = sO[modes + mi].y;
      }
      contract2<R>(comp, R(m0), R(m1), R(qi), sS, sT, tab[qi], sr, si, o_r, o_i);
      sO[mi] = C{o_r[0], o_i[0]};
      sO[modes + mi] = C{o_r[1], o_i[1]};
    }
  }
  __syncthreads();
  C* Ob = O + (root ? int64_t(0) : static_cast<int64_t>(box) * 2 * modes);
  for (int i = threadIdx.x; i < 2 * modes; i += blockDim.x) Ob[i] = sO[i];
}

// incoming expansion of the root from its 9 colleague slots (slot s: delta = (s % 3 - 1, s / 3 - 1))
template <typename R>
__global__ void k_far2_colleague_root(const int32_t* __restrict__ coll, const typename Cplx<R>::T* __restrict__ O,
                                      typename Cplx<R>::T* __restrict__ I, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  const int modes = nh * nm;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * modes) return;
  const int k = idx / modes, mi = idx - k * modes;
  const int m0 = mi / nm, m1 = mi % nm - Mh;
  R sr = R(0), si = R(0);
  for (int s = 0; s < 9; ++s) {
    const int cb = coll[s];
    if (cb < 0) continue;
    int e = (m0 * (s % 3 - 1) + m1 * (s / 3 - 1)) % 3;
    if (e < 0) e += 3;
    const C o = O[(static_cast<int64_t>(cb) * 2 + k) * modes + mi];
    add_phased<R>(e, o.x, o.y, sr, si);
  }
  I[k * modes + mi] = C{sr, si};    // the root is target index 0 (boxes sorted by level)
}

// the four children of one parent at once: their colleagues lie in the 4 x 4 window of
// boxes at the children's level (slot w = w0 + 4 w1 at position 2 c_parent - 1 + (w0, w1)),
// summed in two passes of 3-term sums (axis 0, then axis 1).  win[g][16]: box id or -1;
// chl[g][4]: target index of child o (o_a = bit a) or -1.
template <typename R>
__global__ void __launch_bounds__(128) k_far2_colleague_grp(const int32_t* __restrict__ win, const int32_t* __restrict__ chl,
                                                            const typename Cplx<R>::T* __restrict__ O,
                                                            typename Cplx<R>::T* __restrict__ I, int Mh, int nh, int nm) {
  using C = typename Cplx<R>::T;
  __shared__ int s_win[16], s_ch[4];
  const int g = blockIdx.x, k = blockIdx.y;
  if (threadIdx.x < 16) s_win[threadIdx.x] = win[g * 16 + threadIdx.x];
  if (threadIdx.x < 4) s_ch[threadIdx.x] = chl[g * 4 + threadIdx.x];
  __syncthreads();
  const int modes = nh * nm;
  const int mi = blockIdx.z * blockDim.x + threadIdx.x;
  if (mi >= modes) return;
  const int m0 = mi / nm, m1 = mi % nm - Mh;
  R c0, s0, c1, s1;
  axis_phase<R>(m0, c0, s0);
  axis_phase<R>(m1, c1, s1);
  const C* Ok = O + static_cast<int64_t>(k) * modes + mi;
  R tr[2][4], ti[2][4];
#pragma unroll
  for (int w1 = 0; w1 < 4; ++w1) {
    R xr[4], xi[4];
#pragma unroll
    for (int w0 = 0; w0 < 4; ++w0) {
      const int cb = s_win[w0 + 4 * w1];
      xr[w0] = xi[w0] = R(0);
      if (cb >= 0) {
        const C v = Ok[static_cast<int64_t>(cb) * 2 * modes];
        xr[w0] = v.x;
        xi[w0] = v.y;
      }
    }
#pragma unroll
    for (int o0 = 0; o0 < 2; ++o0)
      sum3<R>(c0, s0, xr[o0], xi[o0], xr[o0 + 1], xi[o0 + 1], xr[o0 + 2], xi[o0 + 2], tr[o0][w1], ti[o0][w1]);
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int o0 = o & 1, o1 = o >> 1;
    R yr, yi;
    sum3<R>(c1, s1, tr[o0][o1], ti[o0][o1], tr[o0][o1 + 1], ti[o0][o1 + 1], tr[o0][o1 + 2], ti[o0][o1 + 2], yr, yi);
    const int tb = s_ch[o];
    if (tb >= 0) I[(static_cast<int64_t>(tb) * 2 + k) * modes + mi] = C{yr, yi};
  }
}

// potential grid of one box from an incoming expansion:
//   Z[m0][b] = sum_m1 F[b][m1] I[m0][m1];  pot[box][k][a][b] (=, +=) Re sum_m0 Fh[a][m0] Z[m0][b]
// (Fh carries the weights 1, 2, 2, ... of the m0 >= 0 half).  I of list entry g at
// I + g * 2 * nh * nm (the root: g = 0).
inline size_t ev2_smem(int p, int nh, int nm, size_t er) {
  const size_t ec = 2 * er;
  return align16(static_cast<size_t>(nm) * p * ec) + align16(static_cast<size_t>(p) * nh * ec) +
         align16(static_cast<size_t>(nh) * nm * ec) + align16(static_cast<size_t>(nh) * p * ec);
}
template <typename R>
__global__ void __launch_bounds__(kBox2Threads) k_far2_ev(const int32_t* __restrict__ boxes, const typename Cplx<R>::T* __restrict__ I,
                                                          const typename Cplx<R>::T* __restrict__ Fh,
                                                          const typename Cplx<R>::T* __restrict__ F, R* __restrict__ pot,
                                                          int accumulate, int p, int nh, int nm) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t ec = sizeof(C);
  C* sFT = reinterpret_cast<C*>(smem);                                                  // [nm][p]: F transposed
  unsigned char* ptr = smem + align16(static_cast<size_t>(nm) * p * ec);
  C* sFh = reinterpret_cast<C*>(ptr);                                                   // [p][nh]
  ptr += align16(static_cast<size_t>(p) * nh * ec);
  C* sI = reinterpret_cast<C*>(ptr);                                                    // [nh][nm]
  ptr += align16(static_cast<size_t>(nh) * nm * ec);
  C* sZ = reinterpret_cast<C*>(ptr);                                                    // [nh][p]
  const int box = boxes[blockIdx.x];
  for (int i = threadIdx.x; i < nm * p; i += blockDim.x) {
    const int m = i / p, j = i - m * p;
    sFT[i] = F[j * nm + m];
  }
  for (int i = threadIdx.x; i < p * nh; i += blockDim.x) sFh[i] = Fh[i];
  const int p2 = p * p, modes = nh * nm;
  for (int k = 0; k < 2; ++k) {
    const C* Ik = I + (static_cast<int64_t>(blockIdx.x) * 2 + k) * modes;
    __syncthreads();
    for (int i = threadIdx.x; i < modes; i += blockDim.x) sI[i] = Ik[i];
    __syncthreads();
    for (int i = threadIdx.x; i < nh * p; i += blockDim.x) {
      const int m0 = i / p, b = i - m0 * p;
      const C* x = sI + m0 * nm;
      R zr = R(0), zi = R(0);
      for (int m1 = 0; m1 < nm; ++m1) {
        const C e = sFT[m1 * p + b], v = x[m1];
        zr = fma(e.x, v.x, zr);
        zr = fma(-e.y, v.y, zr);
        zi = fma(e.x, v.y, zi);
        zi = fma(e.y, v.x, zi);
      }
      sZ[i] = C{zr, zi};
    }
    __syncthreads();
    R* Pk = pot + (static_cast<int64_t>(box) * 2 + k) * p2;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      const int a = i / p, b = i - a * p;
      const C* e = sFh + a * nh;
      R v = R(0);
      for (int m0 = 0; m0 < nh; ++m0) {
        const C z = sZ[m0 * p + b];
        v = fma(e[m0].x, z.x, v);
        v = fma(-e[m0].y, z.y, v);
      }
      if (accumulate) Pk[i] += v;
      else Pk[i] = v;
    }
  }
}

// child merge of one parent (block g), one component per blockIdx.y:
//   q[parent] = sum_o (T_o0 (x) T_o1) q[child o]:  Y[a][j] = sum_i T_o0[a][i] X[i][j],
//   Q[a][b] += sum_j T_o1[b][j] Y[a][j]  (T_o^T[j][b] = T_o[b][j] read for the second stage);
// chl[g][4]: box id of child o or -1 (no sources)
inline size_t tree2_smem(int p, size_t er) { return (4 * static_cast<size_t>(p) * p + 3 * static_cast<size_t>(p) * p) * er; }
template <typename R>
__global__ void __launch_bounds__(kBox2Threads) k_far2_merge(const int32_t* __restrict__ parents, const int32_t* __restrict__ chl,
                                                             R* __restrict__ q, int ncomp, const R* __restrict__ T0,
                                                             const R* __restrict__ T1, const R* __restrict__ T0t,
                                                             const R* __restrict__ T1t, int p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p2 = p * p;
  R* sT = reinterpret_cast<R*>(smem);       // T0, T1, T0^T, T1^T
  R* sX = sT + 4 * p2;
  R* sY = sX + p2;
  R* sQ = sY + p2;
  const int g = blockIdx.x, k = blockIdx.y;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) {
    sT[i] = T0[i];
    sT[p2 + i] = T1[i];
    sT[2 * p2 + i] = T0t[i];
    sT[3 * p2 + i] = T1t[i];
  }
  bool first = true;
  for (int o = 0; o < 4; ++o) {
    const int cb = chl[g * 4 + o];
    if (cb < 0) continue;
    const R* A = sT + (o & 1) * p2;                   // T_o0 [a][i]
    const R* Bt = sT + (2 + (o >> 1)) * p2;           // T_o1^T [j][b]
    const R* X = q + (static_cast<int64_t>(cb) * ncomp + k) * p2;
    __syncthreads();
    for (int i = threadIdx.x; i < p2; i += blockDim.x) sX[i] = X[i];
    __syncthreads();
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      const int a = i / p, j = i - a * p;
      R v = R(0);
      for (int ii = 0; ii < p; ++ii) v = fma(A[a * p + ii], sX[ii * p + j], v);
      sY[i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      const int a = i / p, b = i - a * p;
      R v = R(0);
      for (int j = 0; j < p; ++j) v = fma(Bt[j * p + b], sY[a * p + j], v);
      sQ[i] = first ? v : sQ[i] + v;
    }
    first = false;
  }
  R* Y = q + (static_cast<int64_t>(parents[g]) * ncomp + k) * p2;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) Y[i] = first ? R(0) : sQ[i];
}

// interpolation of one parent's potential grid to its children (block g, component
// blockIdx.y):  Y_o0[i][b] = sum_a T_o0[a][i] P[a][b];  pot[child o][i][j] += sum_b T_o1[b][j] Y_o0[i][b];
// chl[g][4]: box id of child o or -1 (no targets)
template <typename R>
__global__ void __launch_bounds__(kBox2Threads) k_far2_interp(const int32_t* __restrict__ parents, const int32_t* __restrict__ chl,
                                                              R* __restrict__ pot, const R* __restrict__ T0,
                                                              const R* __restrict__ T1, int p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p2 = p * p;
  R* sT = reinterpret_cast<R*>(smem);       // T0, T1
  R* sP = sT + 2 * p2;
  R* sY = sP + p2;                          // [2][p2]
  const int g = blockIdx.x, k = blockIdx.y;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) {
    sT[i] = T0[i];
    sT[p2 + i] = T1[i];
  }
  const R* P = pot + (static_cast<int64_t>(parents[g]) * 2 + k) * p2;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) sP[i] = P[i];
  __syncthreads();
  int need[2] = {0, 0};
  for (int o = 0; o < 4; ++o)
    if (chl[g * 4 + o] >= 0) need[o & 1] = 1;
  for (int o0 = 0; o0 < 2; ++o0) {
    if (!need[o0]) continue;
    const R* A = sT + o0 * p2;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      const int ii = i / p, b = i - ii * p;
      R v = R(0);
      for (int a = 0; a < p; ++a) v = fma(A[a * p + ii], sP[a * p + b], v);
      sY[o0 * p2 + i] = v;
    }
  }
  __syncthreads();
  for (int o = 0; o < 4; ++o) {
    const int cb = chl[g * 4 + o];
    if (cb < 0) continue;
    const R* Y = sY + (o & 1) * p2;
    const R* B = sT + (o >> 1) * p2;
    R* Pc = pot + (static_cast<int64_t>(cb) * 2 + k) * p2;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      const int ii = i / p, j = i - ii * p;
      R v = R(0);
      for (int b = 0; b < p; ++b) v = fma(B[b * p + j], Y[ii * p + b], v);
      Pc[i] += v;
    }
  }
}

// free-space Stokeslet constant K_corr sum_s f_s = K_corr sum_j q_root,j (the Lagrange
// basis sums to one) added to the root potential grid, component blockIdx.x
template <typename R>
__global__ void k_far2_corr(const R* __restrict__ q_root, int slot_f, R* __restrict__ pot_root, int p2, double kcorr) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) s += static_cast<double>(q_root[(slot_f + k) * p2 + i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const R add = static_cast<R>(red[0] * kcorr);
  for (int i = threadIdx.x; i < p2; i += blockDim.x) pot_root[k * p2 + i] += add;
}

// leaf evaluation: u[caller][k] += sum_ab L_a(x) L_b(y) pot[box][k][a][b].  A block
// takes one chunk of at most kEv2Threads targets of one leaf (item: leaf list entry
// it_leaf, first target it_off); a thread takes one target, its b-weights in
// registers (PB, zero past p), its a-weights in shared memory; the leaf's two grids
// sit in shared memory as rows of PB.
template <typename R, int PB>
__global__ void __launch_bounds__(kEv2Threads) k_far2_eval(const int32_t* __restrict__ it_leaf, const int32_t* __restrict__ it_off,
                                                           const int32_t* __restrict__ leaf_list, const int32_t* __restrict__ leaf_box,
                                                           const int32_t* __restrict__ t_start, const int32_t* __restrict__ t_count,
                                                           const double* __restrict__ tw, int64_t NT, const int32_t* __restrict__ tperm,
                                                           const BoxGeo* __restrict__ box_geo, const R* __restrict__ pot, int p,
                                                           const R* __restrict__ nodes, const R* __restrict__ bw,
                                                           double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sP = reinterpret_cast<R*>(smem);                    // [2][p][PB]
  R* sL = sP + 2 * p * PB;                               // [p][kEv2Threads] a-weights
  __shared__ R s_nodes[kMaxP], s_bw[kMaxP];
  const int e = it_leaf[blockIdx.x];
  const int li = leaf_list[e];
  const int box = leaf_box[e];
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    s_nodes[j] = nodes[j];
    s_bw[j] = bw[j];
  }
  const int64_t p2 = static_cast<int64_t>(p) * p;
  const R* P = pot + static_cast<int64_t>(box) * 2 * p2;
  for (int i = threadIdx.x; i < 2 * p * PB; i += blockDim.x) {
    const int kr = i / PB, c = i - kr * PB;             // kr = k p + a
    sP[i] = c < p ? P[static_cast<int64_t>(kr) * p + c] : R(0);
  }
  __syncthreads();
  const BoxGeo geo = box_geo[box];
  const double inv_half = 1.0 / geo.w;
  const int lt0 = t_start[li], lnt = t_count ? t_count[li] : t_start[li + 1] - lt0;
  const int t0 = lt0 + it_off[blockIdx.x];
  const int nt = min(kEv2Threads, lnt - it_off[blockIdx.x]);
  const int t = threadIdx.x;
  const bool on = t < nt;
  R cw[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) cw[j] = R(0);
  if (on) {
    const R x = static_cast<R>((tw[t0 + t] - geo.x) * inv_half);
    lagrange_row<R>(x, p, s_nodes, s_bw, sL + t, kEv2Threads, p);
    const R y = static_cast<R>((tw[NT + t0 + t] - geo.y) * inv_half);
    R ssum = R(0);
    int hit = -1;
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      R v = R(0);
      if (j < p) {
        const R d = y - s_nodes[j];
        if (d == R(0)) hit = j;
        else v = s_bw[j] * recip<R>(d);
      }
      cw[j] = v;
      ssum += v;
    }
    const R inv = hit >= 0 ? R(0) : recip<R>(ssum);
#pragma unroll
    for (int j = 0; j < PB; ++j) cw[j] = hit >= 0 ? (j == hit ? R(1) : R(0)) : cw[j] * inv;
  } else {
    for (int j = 0; j < p; ++j) sL[j * kEv2Threads + t] = R(0);
  }
  R acc0 = R(0), acc1 = R(0);
  for (int a = 0; a < p; ++a) {
    const R* row0 = sP + a * PB;
    const R* row1 = sP + (p + a) * PB;
    R r0 = R(0), r1 = R(0);
#pragma unroll
    for (int c4 = 0; c4 < PB / 4; ++c4) {
      R v0[4], v1[4];
      ld4(row0 + 4 * c4, v0);
      ld4(row1 + 4 * c4, v1);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        r0 = fma(cw[4 * c4 + i], v0[i], r0);
        r1 = fma(cw[4 * c4 + i], v1[i], r1);
      }
    }
    const R la = sL[a * kEv2Threads + t];
    acc0 = fma(la, r0, acc0);
    acc1 = fma(la, r1, acc1);
  }
  if (on) {
    const int64_t o = tperm[t0 + t];
    u[o * 2] += static_cast<double>(acc0);
    u[o * 2 + 1] += static_cast<double>(acc1);
  }
}

// B-hat^R(k) in 2D, Eq. (Btrunc_hat): (1 - J0(Rk) - (Rk / 2) J1(Rk)) / k^4.  For
// x = Rk < 1/2 the bracket is summed from the power series of J0 and J1,
// sum_{n >= 2} (-1)^n (n - 1) (x/2)^{2n} / (n!)^2, which avoids the cancellation.
double b_trunc_hat_2d(double k) {
  const double x = k * kRTrunc2;
  if (x >= 0.5) return (1.0 - ::j0(x) - 0.5 * x * ::j1(x)) / (k * k * k * k);
  const double R4 = kRTrunc2 * kRTrunc2 * kRTrunc2 * kRTrunc2;
  // bracket / x^4 = sum_{n >= 2} (-1)^n (n - 1) x^{2n - 4} / (4^n (n!)^2)
  double sum = 0.0, term = 1.0 / 16.0 / 4.0;      // n = 2: 1 / (4^2 (2!)^2)
  const double x2 = x * x;
  for (int n = 2; n < 20; ++n) {
    sum += ((n & 1) ? -1.0 : 1.0) * (n - 1) * term;
    term *= x2 / (4.0 * (n + 1) * (n + 1));
  }
  return R4 * sum;
}

// the evaluation kernel for a padded order
template <typename R>
void launch_eval2(int PB, int nitems, size_t shm, cudaStream_t s, const int32_t* il, const int32_t* io,
                  const int32_t* ll, const int32_t* lb, const int32_t* ts, const int32_t* tc, const double* tw, int64_t NT,
                  const int32_t* tp, const BoxGeo* geo, const R* pot, int p, const R* nodes, const R* bw, double* u) {
  auto go = [&](auto kern) {
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    kern<<<nitems, kEv2Threads, shm, s>>>(il, io, ll, lb, ts, tc, tw, NT, tp, geo, pot, p, nodes, bw, u);
  };
  switch (PB) {
    case 12: go(k_far2_eval<R, 12>); break;
    case 24: go(k_far2_eval<R, 24>); break;
    case 36: go(k_far2_eval<R, 36>); break;
    case 48: go(k_far2_eval<R, 48>); break;
    default: go(k_far2_eval<R, 60>); break;
  }
}

}  // namespace

struct Far2State {
  int fp32 = 1;
  int p = 0, M = 0, nh = 0, nm = 0, PB = 0;   // level modes: m_0 in [0, M], m_1 in [-M, M]
  int rK = 0, rnh = 0, rnm = 0;               // root modes
  int ncomp = 0, slot_f = -1, slot_t = -1;
  int nbox = 0, maxlev = 0, nsrc_box = 0, ntrg_box = 0, nsrc_leaf = 0, ntrg_leaf = 0;
  int ngrp = 0, n_ev_items = 0;
  int w_tiles = 1;                   // blocks of 128 weight rows of the largest source leaf
  int64_t p2 = 0, modes = 0, rmodes = 0;
  double sT_root = 1.0;
  BoxGeo* box_geo = nullptr;
  int32_t* box_level = nullptr;
  int32_t* src_leaf = nullptr;       // [nsrc_leaf] leaf index, then box id at + nsrc_leaf
  int32_t* trg_leaf = nullptr;
  int32_t* src_box_list = nullptr;
  int32_t* trg_box_list = nullptr;
  int32_t* ev_item_leaf = nullptr;
  int32_t* ev_item_off = nullptr;
  int32_t* coll = nullptr;           // [9] colleague slots of the root
  int32_t* grp_win = nullptr;        // [ngrp][16]
  int32_t* grp_ch = nullptr;         // [ngrp][4]
  int32_t* root_box = nullptr;       // {0}
  std::vector<int32_t*> mf_par, mf_ch, if_par, if_ch;   // per level: parents and their 4 children
  std::vector<int> mf_n, if_n;
  void* mats = nullptr;
  size_t m_nodes = 0, m_bw = 0, m_T0 = 0, m_T1 = 0, m_T0t = 0, m_T1t = 0, m_Eh = 0, m_E = 0, m_Fh = 0, m_F = 0;
  size_t m_REh = 0, m_RE = 0, m_RFh = 0, m_RF = 0, m_tab = 0, m_rtab = 0;
  size_t out_bytes = 0, ev_bytes = 0, rout_bytes = 0, rev_bytes = 0, tree_bytes = 0;
  void* q = nullptr;                 // [nbox][ncomp][p^2] R
  void* pot = nullptr;               // [nbox][2][p^2] R
  void* O = nullptr;                 // [nbox][2][modes] C
  void* I = nullptr;                 // [ntrg_box][2][modes] C
  void* rO = nullptr;                // [2][rmodes] C
  void* W = nullptr;                 // [N][2][PB] R
  size_t bytes = 0;
};

Far2State* far2d_setup(Plan& p) {
  const DeviceTree& T = p.tree;
  const dmk_stokes_opts_t& o = p.opts;
  cudaStream_t s = p.stream;
  auto Fp = std::make_unique<Far2State>();
  Far2State& F = *Fp;
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
  F.PB = ((F.p + 11) / 12) * 12;
  F.p2 = static_cast<int64_t>(F.p) * F.p;
  F.modes = static_cast<int64_t>(F.nh) * F.nm;
  const bool wS = o.kernels & DMK_KERNEL_STOKESLET, wT = o.kernels & DMK_KERNEL_STRESSLET;
  F.slot_f = wS ? 0 : -1;
  F.slot_t = wT ? (wS ? 2 : 0) : -1;
  F.ncomp = (wS ? 2 : 0) + (wT ? 3 : 0);
  const double h0 = 2.0 * M_PI / (2.0 + 2.0 * std::sqrt(2.0));
  if (o.periodic) F.rK = static_cast<int>(std::floor(c / (2.0 * M_PI)));   // N_per = 2 rK + 1
  else F.rK = static_cast<int>(std::ceil(c / h0)) + 1;                       // |k_i| <= c + h0 (and a little beyond)
  F.rnh = F.rK + 1;
  F.rnm = 2 * F.rK + 1;
  if (F.rnm > kMaxP) throw Error{DMK_ERR_UNSUPPORTED, "root mode count beyond the compiled maximum"};
  F.rmodes = static_cast<int64_t>(F.rnh) * F.rnm;

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
    int64_t c[2];
    uint64_t key;
    int leaf = -1;
    int64_t src = 0, trg = 0;
    int child[4];
  };
  std::vector<std::unordered_map<uint64_t, int>> at(maxlev + 1);
  std::vector<Box> boxes;
  auto find_or_add = [&](int l, const int64_t* cc) {
    const uint64_t key = morton<2>(cc);
    auto it = at[l].find(key);
    if (it != at[l].end()) return it->second;
    Box b;
    b.lev = l;
    b.c[0] = cc[0];
    b.c[1] = cc[1];
    b.key = key;
    for (int k = 0; k < 4; ++k) b.child[k] = -1;
    boxes.push_back(b);
    const int id = static_cast<int>(boxes.size()) - 1;
    at[l][key] = id;
    return id;
  };
  for (int i = 0; i < nl; ++i) {
    int64_t cc[2];
    leaf_coords<2>(anc[i], lev[i], T.M, cc);
    for (int l = lev[i]; l >= 0; --l) {
      const int64_t ca[2] = {cc[0] >> (lev[i] - l), cc[1] >> (lev[i] - l)};
      const int id = find_or_add(l, ca);
      if (l == lev[i]) {
        boxes[id].leaf = i;
        boxes[id].src = cnt[i];
        boxes[id].trg = tcnt[i];
      }
    }
  }
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
  for (int i = nb - 1; i >= 0; --i) {
    Box& b = boxes[i];
    if (b.lev == 0) continue;
    const int64_t pc[2] = {b.c[0] >> 1, b.c[1] >> 1};
    const int par = at[b.lev - 1].at(morton<2>(pc));
    const int ch = static_cast<int>((b.c[0] & 1) | ((b.c[1] & 1) << 1));
    boxes[par].child[ch] = i;
    boxes[par].src += b.src;
    boxes[par].trg += b.trg;
  }
  for (int i = 0; i < nb; ++i)
    if (boxes[i].leaf < 0)
      for (int k = 0; k < 4; ++k)
        if (boxes[i].child[k] < 0) throw Error{DMK_ERR_CUDA, "far field: incomplete box hierarchy"};
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
  {
    int64_t mx = 1;
    for (int32_t li : src_leaf) mx = std::max<int64_t>(mx, cnt[li]);
    F.w_tiles = static_cast<int>(std::min<int64_t>((2 * mx + 127) / 128, 65535));
  }
  auto lookup = [&](int l, const int64_t* raw, int* id) {
    const int64_t n = int64_t(1) << l;
    int64_t cc[2];
    for (int a = 0; a < 2; ++a) {
      cc[a] = raw[a];
      if (o.periodic) cc[a] = ((cc[a] % n) + n) % n;
      else if (cc[a] < 0 || cc[a] >= n) return;
    }
    auto it = at[l].find(morton<2>(cc));
    if (it != at[l].end() && boxes[it->second].src > 0) *id = it->second;
  };
  // the root's 9 colleague slots (images in the periodic case)
  std::vector<int32_t> coll(9, -1);
  if (F.ntrg_box > 0)
    for (int sl = 0; sl < 9; ++sl) {
      const int64_t raw[2] = {sl % 3 - 1, sl / 3 - 1};
      int id = -1;
      lookup(0, raw, &id);
      coll[sl] = id;
    }
  // parent groups for the colleague sums of every non-root target box
  std::vector<int32_t> gwin, gch;
  for (int i = 0; i < nb; ++i) {
    const Box& b = boxes[i];
    if (b.leaf >= 0 || b.trg == 0) continue;
    for (int w = 0; w < 16; ++w) {
      const int64_t raw[2] = {2 * b.c[0] - 1 + (w & 3), 2 * b.c[1] - 1 + (w >> 2)};
      int id = -1;
      lookup(b.lev + 1, raw, &id);
      gwin.push_back(id);
    }
    for (int ch = 0; ch < 4; ++ch) gch.push_back(trg_index[b.child[ch]]);
  }
  F.ngrp = static_cast<int>(gch.size() / 4);
  std::vector<BoxGeo> geo(nb);
  std::vector<int32_t> blev(nb);
  for (int i = 0; i < nb; ++i) {
    const double r = std::ldexp(1.0, -boxes[i].lev);
    geo[i] = BoxGeo{(boxes[i].c[0] + 0.5) * r, (boxes[i].c[1] + 0.5) * r, 0.0, 0.5 * r};
    blev[i] = boxes[i].lev;
  }
  // merges (parents with sources, finest level first) and interpolation (parents with
  // targets, coarsest first): parents and their four children
  for (int l = maxlev - 1; l >= 0; --l) {
    std::vector<int32_t> par, ch;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.src == 0) continue;
      par.push_back(i);
      for (int k = 0; k < 4; ++k) ch.push_back(boxes[b.child[k]].src ? b.child[k] : -1);
    }
    if (par.empty()) continue;
    F.mf_par.push_back(up.put(par));
    F.mf_ch.push_back(up.put(ch));
    F.mf_n.push_back(static_cast<int>(par.size()));
  }
  for (int l = 0; l < maxlev; ++l) {
    std::vector<int32_t> par, ch;
    for (int i = 0; i < nb; ++i) {
      const Box& b = boxes[i];
      if (b.lev != l || b.leaf >= 0 || b.trg == 0) continue;
      par.push_back(i);
      for (int k = 0; k < 4; ++k) ch.push_back(boxes[b.child[k]].trg ? b.child[k] : -1);
    }
    if (par.empty()) continue;
    F.if_par.push_back(up.put(par));
    F.if_ch.push_back(up.put(ch));
    F.if_n.push_back(static_cast<int>(par.size()));
  }

  // ---- matrices and tables --------------------------------------------------------
  const int P = F.p;
  MatBank bank;
  bank.f32 = F.fp32;
  std::vector<double> nodes, bwt;
  cheb_nodes_bw(P, nodes, bwt);
  F.m_nodes = bank.put_real(nodes);
  F.m_bw = bank.put_real(bwt);
  // child -> parent anterpolation T_o[a][i] = L_a(((2o - 1) + xi_i) / 2) and the transposes
  for (int oo = 0; oo < 2; ++oo) {
    std::vector<double> Tm(P * P), Tt(P * P);
    for (int a = 0; a < P; ++a)
      for (int i = 0; i < P; ++i) {
        const double v = lagrange_host(nodes, ((2 * oo - 1) + nodes[i]) / 2.0, a);
        Tm[a * P + i] = v;
        Tt[i * P + a] = v;
      }
    (oo == 0 ? F.m_T0 : F.m_T1) = bank.put_real(Tm);
    (oo == 0 ? F.m_T0t : F.m_T1t) = bank.put_real(Tt);
  }
  const double th_l = M_PI / 3.0;                 // h (z - c_B) = pi xi / 3 at every level
  F.m_Eh = bank.plane_wave(nodes, 0, F.nh, th_l, false, true);
  F.m_E = bank.plane_wave(nodes, -F.M, F.nm, th_l, false, false);
  F.m_Fh = bank.plane_wave(nodes, 0, F.nh, th_l, true, true);
  F.m_F = bank.plane_wave(nodes, -F.M, F.nm, th_l, true, false);
  const double th_r = o.periodic ? M_PI : 0.5 * h0;
  F.m_REh = bank.plane_wave(nodes, 0, F.rnh, th_r, false, true);
  F.m_RE = bank.plane_wave(nodes, -F.rK, F.rnm, th_r, false, false);
  F.m_RFh = bank.plane_wave(nodes, 0, F.rnh, th_r, true, true);
  F.m_RF = bank.plane_wave(nodes, -F.rK, F.rnm, th_r, true, false);
  {
    GammaHat gh(c);
    if (std::fabs(gh(0.0) - 1.0) > 1e-12) throw Error{DMK_ERR_CUDA, "window normalisation check failed"};
    // level table by q = |m|^2: (gamma-hat(pi |m| / 3) - gamma-hat(2 pi |m| / 3)) / (4 pi^2 q^2)
    const int qmax = 2 * F.M * F.M;
    std::vector<double> tab(qmax + 1, 0.0);
    for (int q = 1; q <= qmax; ++q) {
      const double am = std::sqrt(static_cast<double>(q));
      tab[q] = (gh(M_PI * am / 3.0) - gh(2.0 * M_PI * am / 3.0)) / (4.0 * M_PI * M_PI * static_cast<double>(q) * q);
    }
    F.m_tab = bank.put_real(tab);
    // root table: periodic gamma-hat(2 pi |kappa|) / (4 pi^2 q^2), kappa != 0;
    // free space (h0 / 2 pi)^2 h0^2 B-hat^R(h0 |m|) gamma-hat(h0 |m|)
    const int rq = 2 * F.rK * F.rK;
    std::vector<double> rt(rq + 1, 0.0);
    for (int q = 0; q <= rq; ++q) {
      const double am = std::sqrt(static_cast<double>(q));
      if (o.periodic) {
        if (q > 0) rt[q] = gh(2.0 * M_PI * am) / (4.0 * M_PI * M_PI * static_cast<double>(q) * q);
      } else {
        const double k = h0 * am;
        rt[q] = (h0 / (2.0 * M_PI)) * (h0 / (2.0 * M_PI)) * h0 * h0 * b_trunc_hat_2d(k) * gh(k);
      }
    }
    F.m_rtab = bank.put_real(rt);
    F.sT_root = o.periodic ? 2.0 * M_PI : h0;
  }
  F.mats = up.put(bank.bytes);
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
      for (int off = 0; off < nt; off += kEv2Threads) {
        il.push_back(static_cast<int32_t>(e));
        io.push_back(off);
      }
    }
    F.n_ev_items = static_cast<int>(il.size());
    F.ev_item_leaf = up.put(il);
    F.ev_item_off = up.put(io);
  }
  F.coll = up.put(coll);
  F.grp_win = up.put(gwin);
  F.grp_ch = up.put(gch);
  F.root_box = up.put(std::vector<int32_t>{0});
  const size_t er = F.fp32 ? sizeof(float) : sizeof(double), ec = 2 * er;
  F.out_bytes = out2_smem(P, F.nh, F.nm, er);
  F.ev_bytes = ev2_smem(P, F.nh, F.nm, er);
  F.rout_bytes = out2_smem(P, F.rnh, F.rnm, er);
  F.rev_bytes = ev2_smem(P, F.rnh, F.rnm, er);
  F.tree_bytes = tree2_smem(P, er);
  {
    int dev_smem = 0;
    DMK_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device));
    const size_t need = std::max({F.out_bytes, F.ev_bytes, F.rout_bytes, F.rev_bytes, F.tree_bytes});
    if (need > static_cast<size_t>(dev_smem)) throw Error{DMK_ERR_UNSUPPORTED, "2D far field: shared memory too small"};
  }
  up.flush();
  // ---- big buffers -------------------------------------------------------------------
  auto big = [&](size_t bytes) {
    void* ptr = nullptr;
    DMK_CUDA_TRY(cudaMallocAsync(&ptr, std::max<size_t>(bytes, 256), s));
    F.bytes += bytes;
    return ptr;
  };
  F.q = big(static_cast<size_t>(nb) * F.ncomp * F.p2 * er);
  F.pot = big(static_cast<size_t>(nb) * 2 * F.p2 * er);
  F.O = big(static_cast<size_t>(nb) * 2 * F.modes * ec);
  F.I = big(static_cast<size_t>(std::max(F.ntrg_box, 1)) * 2 * F.modes * ec);
  F.rO = big(static_cast<size_t>(2) * F.rmodes * ec);
  F.W = big(static_cast<size_t>(std::max<int64_t>(T.N, 1)) * 2 * F.PB * er);
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  return Fp.release();
}

void far2d_free(Plan& p, Far2State* F) {
  if (!F) return;
  for (void** b : {&F->q, &F->pot, &F->O, &F->I, &F->rO, &F->W})
    if (*b) cudaFreeAsync(*b, p.stream);
  delete F;                                   // small arrays live in the plan's arena
}

size_t far2d_bytes(const Far2State& F) { return F.bytes; }

void far2d_info(const Far2State& F, int32_t info[8]) {
  info[0] = F.p;
  info[1] = F.nm;
  info[2] = F.rnm;
  info[3] = F.nbox;
  info[4] = F.nsrc_box;
  info[5] = F.ntrg_box;
  info[6] = F.maxlev;
  info[7] = F.fp32;
}

namespace {

template <typename R>
void far2d_run_t(const Plan& p, const Far2State& F, const double* d_f, const double* d_g, const double* d_n, double* d_u,
                 cudaStream_t s) {
  using C = typename Cplx<R>::T;
  const DeviceTree& T = p.tree;
  const int P = F.p, nc = F.ncomp, PB = F.PB;
  const int p2 = static_cast<int>(F.p2);
  R* q = static_cast<R*>(F.q);
  R* pot = static_cast<R*>(F.pot);
  C* O = static_cast<C*>(F.O);
  C* I = static_cast<C*>(F.I);
  const char* mats = static_cast<const char*>(F.mats);
  auto mat_r = [&](size_t off) { return reinterpret_cast<const R*>(mats + off); };
  auto mat_c = [&](size_t off) { return reinterpret_cast<const C*>(mats + off); };
  const R* nodes = mat_r(F.m_nodes);
  const R* bw = mat_r(F.m_bw);
  auto mark = [&](int i) {
    if (p.trace) DMK_CUDA_TRY(cudaEventRecord(p.trace[i], s));
  };
  auto check = [&]() {
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
  };
  // 1. Lagrange weights of the sources, leaf proxy charges
  if (F.nsrc_leaf > 0) {
    R* W = static_cast<R*>(F.W);
    k_far2_weights<R><<<dim3(F.nsrc_leaf, F.w_tiles), 128, 0, s>>>(F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start, T.leaf_count, T.w,
                                                  T.N, F.box_geo, P, PB, nodes, bw, W);
    check();
    const size_t shm = (static_cast<size_t>(kAnt2Chunk) * 2 * PB + 4 * kAnt2Chunk) * sizeof(R);
    const int ntask = P * (PB / 4);
    const int nthr = std::min(512, ((ntask + 31) / 32) * 32);
    const int g0 = F.slot_f >= 0 ? 0 : 1;
    const int ng = (F.slot_f >= 0 ? 1 : 0) + (F.slot_t >= 0 ? 1 : 0);
    DMK_CUDA_TRY(cudaFuncSetAttribute(k_far2_anterp<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    k_far2_anterp<R><<<dim3(F.nsrc_leaf, ng), nthr, shm, s>>>(F.src_leaf, F.src_leaf + F.nsrc_leaf, T.leaf_start,
                                                               T.leaf_count, W, T.perm, d_f, d_g, d_n, g0, F.slot_f,
                                                               F.slot_t, nc, q, P, PB);
    check();
  }
  mark(2);
  // 2. upward merges, finest parents first
  {
    auto kern = k_far2_merge<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F.tree_bytes)));
    for (size_t i = 0; i < F.mf_n.size(); ++i) {
      kern<<<dim3(F.mf_n[i], nc), kBox2Threads, F.tree_bytes, s>>>(F.mf_par[i], F.mf_ch[i], q, nc, mat_r(F.m_T0),
                                                                   mat_r(F.m_T1), mat_r(F.m_T0t), mat_r(F.m_T1t), P);
      check();
    }
  }
  mark(3);
  // 3. outgoing plane waves of every box with sources, contracted with the level kernel
  if (F.nsrc_box > 0) {
    auto kern = k_far2_out<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F.out_bytes)));
    kern<<<F.nsrc_box, kBox2Threads, F.out_bytes, s>>>(F.src_box_list, F.box_level, q, nc, F.slot_f, F.slot_t,
                                                       mat_c(F.m_Eh), mat_c(F.m_E), mat_r(F.m_tab), O, 0, 1.0, 1.0, P,
                                                       F.M, F.nh, F.nm);
    check();
  }
  mark(4);
  // 4. incoming expansions (colleague sums) and their potential grids (written)
  if (F.ntrg_box > 0) {
    k_far2_colleague_root<R><<<grid_for(2 * F.modes, 128), 128, 0, s>>>(F.coll, O, I, F.M, F.nh, F.nm);
    check();
    if (F.ngrp > 0) {
      const dim3 grid(F.ngrp, 2, static_cast<unsigned>((F.modes + 127) / 128));
      k_far2_colleague_grp<R><<<grid, 128, 0, s>>>(F.grp_win, F.grp_ch, O, I, F.M, F.nh, F.nm);
      check();
    }
  }
  mark(5);
  if (F.ntrg_box > 0) {
    auto kern = k_far2_ev<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F.ev_bytes)));
    kern<<<F.ntrg_box, kBox2Threads, F.ev_bytes, s>>>(F.trg_box_list, I, mat_c(F.m_Fh), mat_c(F.m_F), pot, 0, P, F.nh,
                                                      F.nm);
    check();
  }
  mark(6);
  // 5. root: K_M,0 (periodic series or truncated free-space kernel) added to the root grid
  if (F.ntrg_box > 0 && F.nsrc_box > 0) {
    C* rO = static_cast<C*>(F.rO);
    auto ko = k_far2_out<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(ko, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F.rout_bytes)));
    ko<<<1, kBox2Threads, F.rout_bytes, s>>>(F.root_box, F.box_level, q, nc, F.slot_f, F.slot_t, mat_c(F.m_REh),
                                             mat_c(F.m_RE), mat_r(F.m_rtab), rO, 1, 1.0, F.sT_root, P, F.rK, F.rnh,
                                             F.rnm);
    check();
    auto ke = k_far2_ev<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(F.rev_bytes)));
    ke<<<1, kBox2Threads, F.rev_bytes, s>>>(F.root_box, rO, mat_c(F.m_RFh), mat_c(F.m_RF), pot, 1, P, F.rnh, F.rnm);
    check();
    if (!p.opts.periodic && F.slot_f >= 0) {
      k_far2_corr<R><<<2, 256, 0, s>>>(q, F.slot_f, pot, p2, (1.0 - std::log(kRTrunc2)) / (4.0 * M_PI));
      check();
    }
  }
  mark(7);
  // 6. interpolation down the tree
  {
    const size_t shm = 5 * F.p2 * sizeof(R);     // T0, T1, the parent grid, Y_0, Y_1
    auto kern = k_far2_interp<R>;
    DMK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
    for (size_t i = 0; i < F.if_n.size(); ++i) {
      kern<<<dim3(F.if_n[i], 2), kBox2Threads, shm, s>>>(F.if_par[i], F.if_ch[i], pot, mat_r(F.m_T0), mat_r(F.m_T1), P);
      check();
    }
  }
  mark(8);
  // 7. leaf grids at the targets
  if (F.n_ev_items > 0) {
    const size_t shm = (2 * static_cast<size_t>(P) * PB + static_cast<size_t>(P) * kEv2Threads) * sizeof(R);
    if (T.sep)
      launch_eval2<R>(PB, F.n_ev_items, shm, s, F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                      T.leaf_tstart, nullptr, T.tw, T.NT, T.tperm, F.box_geo, pot, P, nodes, bw, d_u);
    else
      launch_eval2<R>(PB, F.n_ev_items, shm, s, F.ev_item_leaf, F.ev_item_off, F.trg_leaf, F.trg_leaf + F.ntrg_leaf,
                      T.leaf_start, T.leaf_count, T.w, T.N, T.perm, F.box_geo, pot, P, nodes, bw, d_u);
    check();
  }
  mark(9);
}

}  // namespace

void far2d_run(const Plan& p, const Far2State& F, const double* d_f, const double* d_g, const double* d_n, double* d_u,
               cudaStream_t s) {
  if (F.fp32) far2d_run_t<float>(p, F, d_f, d_g, d_n, d_u, s);
  else far2d_run_t<double>(p, F, d_f, d_g, d_n, d_u, s);
}

}  // namespace dmk
