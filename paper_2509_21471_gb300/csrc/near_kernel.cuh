// Near-field (residual + self) kernels, 2D and 3D.
//
// Sec. 5.2, Eqs. (res_stokeslet), (Soffdiag), (res_stresslet), (T-offd), with
// the length-scale remark closing Sec. 5.2 (real-space functions at rho = r/nu).
// Every pair term has the form
//   S_R f     = [A f + C (x.f) x] / (8 pi)
//   T_R:(g n) = [D (g (x.n) + x (g.n) + n (x.g)) + E x (x.g)(x.n)] / (8 pi)
// 3D, with the even polynomials gS, hS, pT, qT of s = rho^2 (tables.h):
//   A = 1/r + gS/nu,  C = 1/r^3 + hS/(nu r^2),
//   D = pT/(nu r^2),  E = -6 (1/r^5 + qT/(nu r^4)).
// 2D (App. B functions m_d, m_o, m_td, m_to at unit scale, scaled by nu):
//   A = -log rho^2 - m_d,  C = 2/r^2 - m_o/nu^2,
//   D = -m_td/nu^2,        E = -8/r^4 + 6 m_to/nu^4.
// Self terms (Eq. (S_self); App. B.1 in 2D): 3D -phi(0)/(2 pi nu_t) f_t,
// 2D (-m_d(0) + 2 log nu_t) f_t / (8 pi).
//
// Gradient (3D Stokeslet; derivative of Eq. (res_stokeslet), tree held fixed):
//   d_m (S_R f)_j = A1 x_m f_j + C1 x_m x_j (x.f) + C (delta_jm (x.f) + x_j f_m)
//   A1 = (-1/r^3 + 2 gS'/nu^3) / 8pi,
//   C1 = (-3/r^5 + 2 hS'/(nu^3 r^2) - 2 hS/(nu r^4)) / 8pi,   ' = d/ds.
//
// Work decomposition: one warp per target tile (<= 32 points of one leaf, one
// target per lane).  The warp walks its leaf's near list (leaf X, image offset
// q, scale nu = 2^-(min(L_B, L_X)+1)), skips source tiles whose bounding box
// is farther than nu from the target tile's box and stages the surviving
// source tiles in shared memory.  MIXED: every lane tests its target against
// each staged source and evaluates the pairs with 0 < r^2 < nu^2.  FP64:
// batches of tiles are staged, each lane marks its candidate pairs with a
// cheap FP32 test (with a margin) and then decides and evaluates only those.
//
// MIXED: coordinates are FP32 offsets from the leaf centre; a source is moved
// into the target leaf's frame by the exact dyadic offset (c_X - c_B - q),
// computed in integers.  Pair terms are FP32 (3D: rsqrt + one Newton step),
// each source tile's partial sum is added to a two-sum (hi, lo) accumulator.
// FP64: coordinates are the in-cell FP64 values; the pair displacement is
// (w_t - w_s) + q and r^2 = (dx*dx + dy*dy) [+ dz*dz] without fused
// operations, so the r < nu decision is the same as in a plain FP64 evaluation.
#pragma once
#include "common.cuh"

namespace dmk {

constexpr int kPolyCap = 32;

struct NearParams {
  int64_t N;
  int n_tile;
  int M;
  const int32_t* tile_leaf;
  const int32_t* tile_start;
  const int32_t* tile_count;
  const float4* tile_lo;
  const float4* tile_hi;
  const uint64_t* leaf_anchor;
  const int32_t* leaf_level;
  const int32_t* leaf_tile0;
  const int32_t* leaf_ntile;
  const int32_t* near_off;
  const int32_t* near_leaf;
  const int32_t* near_q;
  const int32_t* perm;
  const float4* rel;     // leaf-relative FP32 coordinates (sorted; z = 0 in 2D)
  const double* w;       // FP64 in-cell coordinates, SoA [D][N] (sorted)
  const float4* f32;     // mixed, sorted Stokeslet forces, [NR][N] (column k at k*N)
  const float4* g32;     // mixed, sorted stresslet strengths
  const float4* n32;     // mixed, sorted orientations, .w = g.n
  const double* f64;     // FP64 sorted forces SoA [NR][D][N]
  const double* g64;     // FP64 sorted strengths SoA [D][N]
  const double* n64;     // FP64 sorted orientations SoA [D][N] (+ [D] g.n)
  const double* f_orig;  // caller's forces [N][D][n_rhs] (self term)
  double* u;             // [N][D][n_rhs] caller order (may be null for grad-only)
  double* gradu;         // [N][3][3] caller order
  double* acc;           // sorted FP64 accumulator [N][D] (symmetric Stokeslet pass), zeroed
  // targets of the one-sided passes: the points themselves (same_set = 1,
  // every ttile_* / t* array equals its source counterpart) or separate targets
  int same_set;
  int n_ttile;
  int64_t NT;
  const int32_t* ttile_leaf;
  const int32_t* ttile_start;
  const int32_t* ttile_count;
  const float4* ttile_lo;
  const float4* ttile_hi;
  const float4* trel;    // FP32 leaf-relative target coordinates
  const double* tw;      // FP64 in-cell target coordinates, SoA [D][NT]
  const int32_t* tperm;  // sorted target -> caller's target index
  int* close_flag;       // per target tile, zeroed: set where a nearly coincident pair was skipped
  int* close_count;      // skipped pairs queued (zeroed; may exceed close_cap)
  int4* close_q;         // queued pairs: (target, source, near-list entry, L_B | both << 8), sorted indices
  int close_cap;
  double self_base;      // 3D: -phi(0)/(2 pi); 2D: -m_d(0)/(8 pi)
  int n_rhs;             // force columns of the caller's arrays
  float2 c32p[3][kPolyCap];   // FP32 pairs (gS, hS), (pT, qT), (gS', hS')
  double c64[P_COUNT][kPolyCap];
};

template <int NT, typename T>
__device__ __forceinline__ T horner(const T (&c)[kPolyCap], T t) {
  T v = c[NT - 1];
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) v = fma(v, t, c[k]);
  return v;
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

constexpr double kInv8Pi = 0.039788735772973836;   // 1 / (8 pi)
constexpr double kLn2 = 0.6931471805599453;

// self-term coefficient of a target in a leaf at level LB (nu_t = 2^-(LB+1))
template <int D>
__device__ __forceinline__ double self_coeff(const NearParams& P, int LB) {
  if (D == 3) return P.self_base * ldexp(1.0, LB + 1);
  return P.self_base - 2.0 * (LB + 1) * kLn2 * kInv8Pi;        // + 2 log(nu_t) / (8 pi)
}

// ------------------------------------------------ nearly coincident pairs
// FP32 and float-float pair terms start from leaf-relative coordinates whose
// rounding error (about 2^-23 h in FP32 for a leaf of side h, 2^-48 h in
// float-float) is a relative error 2^-23 h / r of the displacement x: for
// nearly coincident points it would dominate the pair term, which is also the
// largest one (S_R -> S as r -> 0, App. A.1).  The FP32 kernels skip the pairs
// with r^2 <= kClose32 nu^2 (r <= nu/32: beyond it x carries at most ~8e-6
// relative error) and the float-float kernel those with r^2 <= kCloseFF nu^2
// (r <= nu/1024); k_near_close (near_close.cuh) then evaluates them with
// close_pair_fp64: x = (w_t - w_s) + q from the FP64 in-cell coordinates and
// the pair terms with the FP64 kernel's arithmetic.
constexpr float kClose32 = 0x1p-10f;
constexpr float kCloseFF = 0x1p-20f;

// it: sorted target index (coordinates P.tw), is: sorted source index (P.w).
// Densities of one point: [0, 3) Stokeslet force, [3, 6) stresslet strength
// g, [6, 9) orientation n, [9] g.n.  out (zeroed by the caller): [0, 3) target
// side of the velocity, [3, 12) of the gradient (grad[j*3+m] = d_m u_j);
// [12, 15), [15, 24) the source side (only if both): S_R is even, T_R and
// grad S_R odd.  Terms without the 1/(8 pi) factor, as in the kernels.
constexpr int kClosePairOut = 24;
template <int D, int KM, bool GRAD>
__device__ __noinline__ void close_pair_fp64(const NearParams& P, int64_t it, int64_t is, const double* q,
                                             double nuinv, const double* sd, const double* td, bool both,
                                             double* out) {
  const int64_t N = P.N;
  double x[3] = {0.0, 0.0, 0.0};
  double r2 = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    x[a] = __dadd_rn(__dsub_rn(P.tw[a * P.NT + it], P.w[a * N + is]), q[a]);
    r2 = __dadd_rn(r2, __dmul_rn(x[a], x[a]));
  }
  const double nu2inv = nuinv * nuinv;
  const double rho2 = r2 * nu2inv;
  if (!(rho2 < 1.0 && r2 > 0.0)) return;
  const double t = fma(2.0, rho2, -1.0);
  double ri = 0.0, ri2, logr2 = 0.0;
  if (D == 3) {
    ri = 1.0 / sqrt(r2);
    ri2 = ri * ri;
  } else {
    ri2 = 1.0 / r2;
    logr2 = log(rho2);
  }
  const double dx = x[0], dy = x[1], dz = x[2];
  if (KM & 1) {
    const double g = horner<kPolyCap>(P.c64[P_GS], t);
    const double h = horner<kPolyCap>(P.c64[P_HS], t);
    double A, C;
    if (D == 3) {
      A = fma(g, nuinv, ri);
      C = ri2 * fma(h, nuinv, ri);
    } else {
      A = -logr2 - g;
      C = fma(-h, nu2inv, 2.0 * ri2);
    }
    double A1 = 0.0, C1 = 0.0;
    if (GRAD) {
      const double dg = horner<kPolyCap>(P.c64[P_DGS], t);
      const double dh = horner<kPolyCap>(P.c64[P_DHS], t);
      const double nu3i = nuinv * nuinv * nuinv;
      const double ri3 = ri2 * ri;
      A1 = fma(2.0 * dg, nu3i, -ri3);
      C1 = fma(-3.0 * ri3, ri2, ri2 * fma(2.0 * dh, nu3i, -2.0 * h * nuinv * ri2));
    }
    for (int side = 0; side < (both ? 2 : 1); ++side) {
      const double* fv = side ? td : sd;               // target side: the source's force
      const double sgn = side ? -1.0 : 1.0;            // grad S_R is odd
      double* o = out + 12 * side;
      const double xf = fma(dx, fv[0], fma(dy, fv[1], dz * fv[2]));
      const double Cx = C * xf;
      o[0] += fma(A, fv[0], Cx * dx);
      o[1] += fma(A, fv[1], Cx * dy);
      if (D == 3) o[2] += fma(A, fv[2], Cx * dz);
      if (GRAD) {
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const double a1 = fma(A1, fv[jj], C1 * x[jj] * xf);
#pragma unroll
          for (int mm = 0; mm < 3; ++mm) {
            double v = fma(a1, x[mm], C * x[jj] * fv[mm]);
            if (jj == mm) v = fma(C, xf, v);
            o[3 + jj * 3 + mm] += sgn * v;
          }
        }
      }
    }
  }
  if (KM & 2) {
    const double pt = horner<kPolyCap>(P.c64[P_PT], t);
    const double qt = horner<kPolyCap>(P.c64[P_QT], t);
    double Dc, Ec;
    if (D == 3) {
      Dc = pt * nuinv * ri2;
      Ec = -6.0 * ri2 * ri2 * fma(qt, nuinv, ri);
    } else {
      Dc = -pt * nu2inv;
      Ec = fma(6.0 * qt, nu2inv * nu2inv, -8.0 * ri2 * ri2);
    }
    for (int side = 0; side < (both ? 2 : 1); ++side) {
      const double* dv = side ? td : sd;
      const double sgn = side ? -1.0 : 1.0;            // T_R is odd
      double* o = out + 12 * side;
      const double xn = fma(dx, dv[6], fma(dy, dv[7], dz * dv[8]));
      const double xg = fma(dx, dv[3], fma(dy, dv[4], dz * dv[5]));
      const double Ex = Ec * xg * xn + Dc * dv[9];
#pragma unroll
      for (int a = 0; a < D; ++a) o[a] += sgn * fma(Dc, fma(dv[3 + a], xn, dv[6 + a] * xg), Ex * x[a]);
    }
  }
}

// Queues a skipped nearly coincident pair (target t, source s, sorted
// indices) of near-list entry e of the target leaf (level LB); both: the pair
// gives the source its side too (symmetric passes).  Beyond the capacity only
// the count grows, and the tiles' marks take over (k_near_close).
__device__ __forceinline__ void close_push(const NearParams& P, int64_t t, int64_t s, int e, int LB, bool both) {
  const int k = atomicAdd(P.close_count, 1);
  if (k < P.close_cap)
    P.close_q[k] = make_int4(static_cast<int>(t), static_cast<int>(s), e, LB | (both ? 256 : 0));
}

// two-sum accumulator (hi, lo) += v for an FP64 value v
__device__ __forceinline__ void two_sum_add_d(float& hi, float& lo, double v) {
  const float vh = __double2float_rn(v);
  two_sum_add(hi, lo, vh);
  lo += __double2float_rn(v - static_cast<double>(vh));
}

// ------------------------------------------------------ tile traversal
// Per near-list entry of the target leaf B: the source leaf X, its image
// offset q, the residual scale nu = 2^-(min(L_B, L_X) + 1) and the exact dyadic
// offset (c_X - c_B - q) that moves X's leaf-relative FP32 coordinates into B's
// frame (computed in integers; exact in FP32 for neighbouring leaves).
struct Entry {
  int X;
  float off[3];
  float nuinv;   // 1/nu (power of two)
  float nu2;
  double q[3];
};

template <int D>
__device__ __forceinline__ Entry make_entry(const NearParams& P, int e, int LB, const int64_t* cB) {
  Entry E;
  E.X = P.near_leaf[e];
  const int32_t qp = P.near_q[e];
  const int LX = P.leaf_level[E.X];
  const int Lmin = min(LB, LX), Lmax = max(LB, LX);
  E.nuinv = ldexpf(1.f, Lmin + 1);
  const float nu = ldexpf(1.f, -(Lmin + 1));
  E.nu2 = nu * nu;
  int64_t cX[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[E.X], LX, P.M, cX);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E.q[a] = 0.0;
    E.off[a] = 0.f;
    if (a < D) {
      const int qa = unpack_q(qp, a);
      E.q[a] = static_cast<double>(qa);
      const int64_t v = ((2 * cX[a] + 1) << (Lmax - LX)) - ((2 * cB[a] + 1) << (Lmax - LB)) -
                        (static_cast<int64_t>(qa) << (Lmax + 1));
      E.off[a] = ldexpf(static_cast<float>(v), -(Lmax + 1));
    }
  }
  return E;
}

// true if source tile U can hold a pair closer than nu to the target tile
__device__ __forceinline__ bool tile_near(const NearParams& P, int U, const Entry& E, float4 tlo, float4 thi) {
  const float4 slo = P.tile_lo[U], shi = P.tile_hi[U];
  const float gx = fmaxf(fmaxf(slo.x + E.off[0] - thi.x, tlo.x - (shi.x + E.off[0])), 0.f);
  const float gy = fmaxf(fmaxf(slo.y + E.off[1] - thi.y, tlo.y - (shi.y + E.off[1])), 0.f);
  const float gz = fmaxf(fmaxf(slo.z + E.off[2] - thi.z, tlo.z - (shi.z + E.off[2])), 0.f);
  return gx * gx + gy * gy + gz * gz < E.nu2 * 1.0001f;
}

// The source tiles Ub + lane (< Uend) of a near leaf that can hold a pair
// closer than nu to the target tile, tested by the whole warp at once (one
// tile per lane) and returned as a bit mask over [Ub, Ub + 32).
__device__ __forceinline__ uint32_t near_tile_mask(const NearParams& P, int Ub, int Uend, const Entry& E,
                                                   float4 tlo, float4 thi, int lane) {
  const int U = Ub + lane;
  return __ballot_sync(0xffffffffu, U < Uend && tile_near(P, U, E, tlo, thi));
}

// Candidate bits of one staged tile for this lane's target: bit j is set when
// |x_t|^2 + (|s_j|^2 - nu'^2) - 2 x_t.s_j < 0, with the slot holding
// (-2 s, |s|^2 - nu'^2), nu'^2 = nu^2 (1 + 2^-12).  The margin is far above
// the rounding error of this expanded form (~2e-6 nu^2 for coordinates within
// ~3 nu of the leaf centre), so no pair with r < nu is missed; the exact
// r < nu decision is taken again on the candidates.
__device__ __forceinline__ uint32_t candidate_bits(const float4* __restrict__ slots, float4 xt, float tt) {
  uint32_t bits = 0u;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float4 a = slots[j];
    const float r2m = fmaf(a.x, xt.x, fmaf(a.y, xt.y, fmaf(a.z, xt.z, tt + a.w)));
    bits |= (r2m < 0.f) ? (1u << j) : 0u;
  }
  return bits;
}

// Walks the set bits of up to four 32-bit words in order; slot index in idx.
struct BitWalker {
  uint32_t m0, m1, m2, m3;
  int base;
  __device__ __forceinline__ bool next(int& idx) {
    if ((m0 | m1 | m2 | m3) == 0u) return false;
    while (m0 == 0u) {
      m0 = m1;
      m1 = m2;
      m2 = m3;
      m3 = 0u;
      base += 32;
    }
    idx = base + __ffs(m0) - 1;
    m0 &= m0 - 1u;
    return true;
  }
};

// ---------------------------------------------------------------- mixed
// Each surviving source tile is staged in shared memory (moved into the
// target leaf's frame).  Every lane first tests its target against all 32
// staged sources with the expanded form |x_t|^2 + (|s|^2 - nu'^2) - 2 x_t.s,
// two sources per packed FP32x2 FMA, and collects the signs into a bit mask
// (bit j: source j is a candidate).  The warp then walks the union of the
// lanes' masks; for each source in it every lane takes the exact FP32 test
// r^2 < nu^2 and the lanes inside the cutoff evaluate the pair.  The kernel
// polynomials are evaluated in pairs ((gS, hS), (pT, qT), (gS', hS')) by packed
// Horner.  The tile's partial sums are added to a two-sum (hi, lo) accumulator.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int NT>
__device__ __forceinline__ float2 horner2(const float2 (&c)[kPolyCap], float t) {
  const float2 tt = f2(t, t);
  float2 v = c[NT - 1];
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) v = __ffma2_rn(v, tt, c[k]);
  return v;
}

// bit j of the result is the sign of (|x_t|^2 + w_j + a_j . x_t), j = 0..31,
// from the test rows of one staged tile (x, y, z, w as float[32] each)
__device__ __forceinline__ uint32_t candidate_mask(const float4 (&rows)[4][8], float4 xt, float tt) {
  const float2 X = f2(xt.x, xt.x), Y = f2(xt.y, xt.y), Z = f2(xt.z, xt.z), T = f2(tt, tt);
  uint32_t bits = 0u;
#pragma unroll
  for (int q = 7; q >= 0; --q) {
    const float4 ax = rows[0][q], ay = rows[1][q], az = rows[2][q], aw = rows[3][q];
    const float2 hi = __ffma2_rn(f2(ax.z, ax.w), X,
                                 __ffma2_rn(f2(ay.z, ay.w), Y, __ffma2_rn(f2(az.z, az.w), Z, __fadd2_rn(f2(aw.z, aw.w), T))));
    const float2 lo = __ffma2_rn(f2(ax.x, ax.y), X,
                                 __ffma2_rn(f2(ay.x, ay.y), Y, __ffma2_rn(f2(az.x, az.y), Z, __fadd2_rn(f2(aw.x, aw.y), T))));
    bits = __funnelshift_l(__float_as_uint(hi.y), bits, 1);   // source 4q+3
    bits = __funnelshift_l(__float_as_uint(hi.x), bits, 1);
    bits = __funnelshift_l(__float_as_uint(lo.y), bits, 1);
    bits = __funnelshift_l(__float_as_uint(lo.x), bits, 1);   // source 4q
  }
  return bits;
}

// One warp (target tile) per block, at least 24 resident per SM: the
// 16-column variant then runs with ~80 registers and some spilled to L1,
// which measured 14 % faster on GB300 than its natural 142 registers (12
// resident warps).  The one-column variants fit below the limit anyway.
constexpr int kMixWarps = 1;
template <int D, int KM, bool GRAD, int NT, int NR>
__global__ void __launch_bounds__(32 * kMixWarps, 24 / kMixWarps) k_near_mixed(const __grid_constant__ NearParams P) {
  static_assert(NR == 1 || (KM == 1 && !GRAD), "several force columns: Stokeslet velocity only");
  static_assert(D == 3 || !GRAD, "the gradient kernel is 3D");
  constexpr bool COMP = (NR == 1);                     // two-sum accumulation
  constexpr int W = kMixWarps;
  __shared__ float4 s_tst[W][4][8];                    // test rows: -2 s (x, y, z), |s|^2 - nu'^2
  __shared__ float4 s_pos[W][kTile];                   // s (x, y, z) in the target leaf's frame
  constexpr int NP = (NR > 1) ? NR / 2 : 1;          // force columns in packed pairs (NR > 1)
  __shared__ float4 s_f[(KM & 1) ? W : 1][1][kTile];
  __shared__ float4 s_fxy[(NR > 1) ? W : 1][NP][kTile];  // (x_k, x_k+1, y_k, y_k+1)
  __shared__ float2 s_fz[(NR > 1) ? W : 1][NP][kTile];   // (z_k, z_k+1)
  __shared__ float4 s_g[(KM & 2) ? W : 1][kTile];
  __shared__ float4 s_n[(KM & 2) ? W : 1][kTile];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * W + wid;               // target tile
  if (tile >= P.n_ttile) return;
  const int64_t N = P.N;
  const int B = P.ttile_leaf[tile];
  const int t0 = P.ttile_start[tile], nt = P.ttile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.ttile_lo[tile], thi = P.ttile_hi[tile];
  const bool on = lane < nt;
  const float4 xt = on ? P.trel[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  // |x_t|^2; +inf for an empty lane makes every candidate test fail
  const float tt = on ? fmaf(xt.x, xt.x, fmaf(xt.y, xt.y, xt.z * xt.z)) : __int_as_float(0x7f800000);
  float* const rowx = reinterpret_cast<float*>(s_tst[wid][0]);
  float* const rowy = reinterpret_cast<float*>(s_tst[wid][1]);
  float* const rowz = reinterpret_cast<float*>(s_tst[wid][2]);
  float* const roww = reinterpret_cast<float*>(s_tst[wid][3]);

  float uh[1][3], ul[COMP ? 3 : 1];
  uh[0][0] = uh[0][1] = uh[0][2] = 0.f;
  float2 uh2[NP][3];
#pragma unroll
  for (int k = 0; k < NP; ++k) uh2[k][0] = uh2[k][1] = uh2[k][2] = f2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < (COMP ? 3 : 1); ++a) ul[a] = 0.f;
  float Gh[GRAD ? 9 : 1], Gl[GRAD ? 9 : 1];
#pragma unroll
  for (int k = 0; k < (GRAD ? 9 : 1); ++k) Gh[k] = Gl[k] = 0.f;

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float nu2 = E.nu2, nuinv = E.nuinv;
    const float nu2inv = nuinv * nuinv;
    const float nu2m = nu2 * (1.f + 0x1p-12f);
    const float thr = nu2 * kClose32;                  // nearly coincident: k_near_close
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane); tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      __syncwarp();
      if (lane < ns) {
        const float4 r = P.rel[s0 + lane];
        const float sx = r.x + E.off[0], sy = r.y + E.off[1], sz = r.z + E.off[2];
        rowx[lane] = -2.f * sx;
        rowy[lane] = -2.f * sy;
        rowz[lane] = -2.f * sz;
        roww[lane] = fmaf(sx, sx, fmaf(sy, sy, sz * sz)) - nu2m;
        s_pos[wid][lane] = make_float4(sx, sy, sz, 0.f);
        if (KM & 1) {
          if (NR == 1) {
            s_f[(KM & 1) ? wid : 0][0][lane] = P.f32[s0 + lane];
          } else {
#pragma unroll
            for (int kp = 0; kp < NP; ++kp) {
              const float4 fa = P.f32[(2 * kp) * N + s0 + lane], fb = P.f32[(2 * kp + 1) * N + s0 + lane];
              s_fxy[(NR > 1) ? wid : 0][kp][lane] = make_float4(fa.x, fb.x, fa.y, fb.y);
              s_fz[(NR > 1) ? wid : 0][kp][lane] = f2(fa.z, fb.z);
            }
          }
        }
        if (KM & 2) {
          s_g[(KM & 2) ? wid : 0][lane] = P.g32[s0 + lane];
          s_n[(KM & 2) ? wid : 0][lane] = P.n32[s0 + lane];
        }
      } else {
        rowx[lane] = rowy[lane] = rowz[lane] = 0.f;
        roww[lane] = __int_as_float(0x7f800000);      // never a candidate
      }
      __syncwarp();
      // candidate test (margin 2^-12 nu^2, far above its rounding error), then
      // the exact test r^2 < nu^2 for the sources some lane marked
      uint32_t m = __reduce_or_sync(0xffffffffu, candidate_mask(s_tst[wid], xt, tt));
      float p[1][3] = {{0.f, 0.f, 0.f}};
      float pg[GRAD ? 9 : 1];
#pragma unroll
      for (int k = 0; k < (GRAD ? 9 : 1); ++k) pg[k] = 0.f;
      float rmin = __int_as_float(0x7f800000);         // smallest r^2 of the staged tile
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        const float4 sp = s_pos[wid][j];
        const float dx = xt.x - sp.x, dy = xt.y - sp.y, dz = xt.z - sp.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        rmin = fminf(rmin, r2);
        if (!(r2 < nu2 && r2 > thr)) continue;         // r^2 <= thr: queued below
        const float rho2 = r2 * nu2inv;
        const float t = fmaf(2.f, rho2, -1.f);
        float ri = 0.f, ri2, logr2 = 0.f;
        if (D == 3) {
          ri = rsqrtf(r2);
          ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);      // one Newton step
          ri2 = ri * ri;
        } else {
          ri2 = __frcp_rn(r2);
          logr2 = __logf(rho2);
        }
        if (KM & 1) {
          const float2 gh = horner2<NT>(P.c32p[0], t);
          float A, C;
          if (D == 3) {
            A = fmaf(gh.x, nuinv, ri);
            C = ri2 * fmaf(gh.y, nuinv, ri);
          } else {
            A = -logr2 - gh.x;
            C = fmaf(-gh.y, nu2inv, 2.f * ri2);
          }
          float2 dgh = f2(0.f, 0.f);
          if (GRAD) dgh = horner2<NT>(P.c32p[2], t);
          if (NR > 1) {
            // several columns: the kernel terms once, applied to two columns per
            // packed FP32x2 instruction
            const float2 A2 = f2(A, A), C2 = f2(C, C), dx2 = f2(dx, dx), dy2 = f2(dy, dy), dz2 = f2(dz, dz);
#pragma unroll
            for (int kp = 0; kp < NP; ++kp) {
              const float4 fxy = s_fxy[(NR > 1) ? wid : 0][kp][j];
              const float2 fx2 = f2(fxy.x, fxy.y), fy2 = f2(fxy.z, fxy.w), fz2 = s_fz[(NR > 1) ? wid : 0][kp][j];
              const float2 Cx2 = __fmul2_rn(C2, __ffma2_rn(dx2, fx2, __ffma2_rn(dy2, fy2, __fmul2_rn(dz2, fz2))));
              uh2[kp][0] = __ffma2_rn(A2, fx2, __ffma2_rn(Cx2, dx2, uh2[kp][0]));
              uh2[kp][1] = __ffma2_rn(A2, fy2, __ffma2_rn(Cx2, dy2, uh2[kp][1]));
              if (D == 3) uh2[kp][2] = __ffma2_rn(A2, fz2, __ffma2_rn(Cx2, dz2, uh2[kp][2]));
            }
          }
#pragma unroll
          for (int k = 0; k < (NR == 1 ? 1 : 0); ++k) {
            const float4 fs = s_f[(KM & 1) ? wid : 0][0][j];
            const float xf = fmaf(dx, fs.x, fmaf(dy, fs.y, dz * fs.z));
            const float Cx = C * xf;
            p[k][0] = fmaf(A, fs.x, fmaf(Cx, dx, p[k][0]));
            p[k][1] = fmaf(A, fs.y, fmaf(Cx, dy, p[k][1]));
            if (D == 3) p[k][2] = fmaf(A, fs.z, fmaf(Cx, dz, p[k][2]));
            if (GRAD) {
              const float nu3i = nuinv * nuinv * nuinv;
              const float ri3 = ri2 * ri;
              const float A1 = fmaf(2.f * dgh.x, nu3i, -ri3);
              const float C1 = fmaf(-3.f * ri3, ri2, ri2 * fmaf(2.f * dgh.y, nu3i, -2.f * gh.y * nuinv * ri2));
              const float xv[3] = {dx, dy, dz};
              const float fv[3] = {fs.x, fs.y, fs.z};
#pragma unroll
              for (int jj = 0; jj < 3; ++jj) {
                const float a1 = fmaf(A1, fv[jj], C1 * xv[jj] * xf);
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) {
                  float v = fmaf(a1, xv[mm], C * xv[jj] * fv[mm]);
                  if (jj == mm) v = fmaf(C, xf, v);
                  pg[jj * 3 + mm] += v;
                }
              }
            }
          }
        }
        if (KM & 2) {
          const float2 pq = horner2<NT>(P.c32p[1], t);
          const float4 gs = s_g[(KM & 2) ? wid : 0][j];
          const float4 nsv = s_n[(KM & 2) ? wid : 0][j];
          const float xn = fmaf(dx, nsv.x, fmaf(dy, nsv.y, dz * nsv.z));
          const float xg = fmaf(dx, gs.x, fmaf(dy, gs.y, dz * gs.z));
          float Dc, Ec;
          if (D == 3) {
            Dc = pq.x * nuinv * ri2;
            Ec = -6.f * ri2 * ri2 * fmaf(pq.y, nuinv, ri);
          } else {
            Dc = -pq.x * nu2inv;
            Ec = fmaf(6.f * pq.y, nu2inv * nu2inv, -8.f * ri2 * ri2);
          }
          const float Ex = Ec * xg * xn + Dc * nsv.w;      // coefficient of x
          p[0][0] += fmaf(Dc, fmaf(gs.x, xn, nsv.x * xg), Ex * dx);
          p[0][1] += fmaf(Dc, fmaf(gs.y, xn, nsv.y * xg), Ex * dy);
          if (D == 3) p[0][2] += fmaf(Dc, fmaf(gs.z, xn, nsv.z * xg), Ex * dz);
        }
      }
      if (COMP) {
#pragma unroll
        for (int a = 0; a < D; ++a) two_sum_add(uh[0][a], ul[a], p[0][a]);
      }
      if (GRAD) {
#pragma unroll
        for (int k = 0; k < 9; ++k) two_sum_add(Gh[k], Gl[k], pg[k]);
      }
      // skipped nearly coincident pairs mark T for k_near_close (on T's own
      // tile the self pair, r = 0, always triggers the scan and is left out);
      // this one-sided pass stays bitwise reproducible, so they are not queued
      if (__any_sync(0xffffffffu, on && rmin <= thr)) {
        bool any = false;
        if (on)
          for (int j = 0; j < ns; ++j) {
            const float4 sp = s_pos[wid][j];
            const float dx = xt.x - sp.x, dy = xt.y - sp.y, dz = xt.z - sp.z;
            any |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= thr && !(P.same_set && U == tile && j == lane);
          }
        if (__any_sync(0xffffffffu, any) && lane == 0) P.close_flag[tile] = 1;
      }
    }
  }
  if (!on) return;
  const int64_t o = P.tperm[t0 + lane];
  const double sc = P.same_set ? self_coeff<D>(P, LB) : 0.0;   // separate targets: no self term
  const int nr = P.n_rhs;
  if (P.u) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k >= nr) break;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double v = (NR == 1) ? static_cast<double>(uh[0][a])
                             : static_cast<double>((k & 1) ? uh2[k >> 1][a].y : uh2[k >> 1][a].x);
        if (COMP) v += static_cast<double>(ul[a]);
        v *= kInv8Pi;
        const int64_t q = (o * D + a) * nr + k;
        if ((KM & 1) && P.same_set) v += sc * P.f_orig[q];
        P.u[q] = v;
      }
    }
  }
  if (GRAD) {
#pragma unroll
    for (int k = 0; k < 9; ++k)
      P.gradu[o * 9 + k] = (static_cast<double>(Gh[k]) + static_cast<double>(Gl[k])) * kInv8Pi;
  }
}

// ------------------------------------------- mixed, Stokeslet, one column
// The residual Stokeslet is even, S_R(-x) = S_R(x), and the pair rule and
// scale nu_ts are symmetric, so one evaluation of a pair serves both points:
// u_t += S_R(x) f_s and u_s += S_R(x) f_t with x = x_t - x_s.  The warp of
// target tile T takes the source tiles U > T of its near list (the warp of U
// skips T) and the tile itself (U = T, target side only, every ordered pair).
// Same FP32 arithmetic and candidate test as k_near_mixed; the source side of
// each union source is summed over the warp by shuffles into the lane that
// owns the source slot, and both sides are added to an FP64 accumulator in
// sorted order (atomically), finished by k_near_sym_finish.
constexpr int kSymWarps = 1;                           // warps (target tiles) per block
template <int D, int NT>
__global__ void __launch_bounds__(32 * kSymWarps, 28 / kSymWarps) k_near_sym(const __grid_constant__ NearParams P, double* __restrict__ acc) {
  __shared__ float4 s_tst[kSymWarps][4][8];
  __shared__ float4 s_pos[kSymWarps][kTile];
  __shared__ float4 s_f[kSymWarps][kTile];
  __shared__ float s_q[kSymWarps][kTile * 3];          // source side of the staged tile
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kSymWarps + wid;
  if (tile >= P.n_tile) return;
#pragma unroll
  for (int a = 0; a < 3; ++a) s_q[wid][lane * 3 + a] = 0.f;
  const int64_t N = P.N;
  const int B = P.tile_leaf[tile];
  const int t0 = P.tile_start[tile], nt = P.tile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.tile_lo[tile], thi = P.tile_hi[tile];
  const bool on = lane < nt;
  const float4 xt = on ? P.rel[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 ft = on ? P.f32[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float tt = on ? fmaf(xt.x, xt.x, fmaf(xt.y, xt.y, xt.z * xt.z)) : __int_as_float(0x7f800000);
  float* const rowx = reinterpret_cast<float*>(s_tst[wid][0]);
  float* const rowy = reinterpret_cast<float*>(s_tst[wid][1]);
  float* const rowz = reinterpret_cast<float*>(s_tst[wid][2]);
  float* const roww = reinterpret_cast<float*>(s_tst[wid][3]);
  float uh[3] = {0.f, 0.f, 0.f}, ul[3] = {0.f, 0.f, 0.f};

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float nu2 = E.nu2, nuinv = E.nuinv;
    const float nu2inv = nuinv * nuinv;
    const float nu2m = nu2 * (1.f + 0x1p-12f);
    const float thr = nu2 * kClose32;                  // nearly coincident: k_near_close
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    if (U1 <= tile) continue;                          // every tile of X precedes T
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane) & __ballot_sync(0xffffffffu, Ub + lane >= tile);
         tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      const bool sym = U != tile;
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      __syncwarp();
      if (lane < ns) {
        const float4 r = P.rel[s0 + lane];
        const float sx = r.x + E.off[0], sy = r.y + E.off[1], sz = r.z + E.off[2];
        rowx[lane] = -2.f * sx;
        rowy[lane] = -2.f * sy;
        rowz[lane] = -2.f * sz;
        roww[lane] = fmaf(sx, sx, fmaf(sy, sy, sz * sz)) - nu2m;
        s_pos[wid][lane] = make_float4(sx, sy, sz, 0.f);
        s_f[wid][lane] = P.f32[s0 + lane];
      } else {
        rowx[lane] = rowy[lane] = rowz[lane] = 0.f;
        roww[lane] = __int_as_float(0x7f800000);
      }
      __syncwarp();
      uint32_t m = __reduce_or_sync(0xffffffffu, candidate_mask(s_tst[wid], xt, tt));
      float p[3] = {0.f, 0.f, 0.f};                    // target side, this tile
      // One pair (this lane's target, staged source j): adds the target side
      // to p and returns the source side (A f_t + C (x.f_t) x) in c.  Pairs
      // with r^2 <= thr are left to k_near_close.
      auto pair = [&](int j, float (&c)[3]) -> float {
        const float4 sp = s_pos[wid][j];
        const float dx = xt.x - sp.x, dy = xt.y - sp.y, dz = xt.z - sp.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool inside = r2 < nu2 && r2 > thr;
        const float rr = inside ? r2 : nu2;            // finite stand-in for the other lanes
        const float rho2 = rr * nu2inv;
        const float t = fmaf(2.f, rho2, -1.f);
        const float2 gh = horner2<NT>(P.c32p[0], t);
        float A, C;
        if (D == 3) {
          float ri = rsqrtf(rr);
          ri = ri * fmaf(-0.5f * rr, ri * ri, 1.5f);      // one Newton step
          A = fmaf(gh.x, nuinv, ri);
          C = ri * ri * fmaf(gh.y, nuinv, ri);
        } else {
          A = -__logf(rho2) - gh.x;
          C = fmaf(-gh.y, nu2inv, 2.f * __frcp_rn(rr));
        }
        A = inside ? A : 0.f;
        C = inside ? C : 0.f;
        const float4 fs = s_f[wid][j];
        const float Cx = C * fmaf(dx, fs.x, fmaf(dy, fs.y, dz * fs.z));
        p[0] = fmaf(A, fs.x, fmaf(Cx, dx, p[0]));
        p[1] = fmaf(A, fs.y, fmaf(Cx, dy, p[1]));
        if (D == 3) p[2] = fmaf(A, fs.z, fmaf(Cx, dz, p[2]));
        const float Ct = C * fmaf(dx, ft.x, fmaf(dy, ft.y, dz * ft.z));
        c[0] = fmaf(A, ft.x, Ct * dx);
        c[1] = fmaf(A, ft.y, Ct * dy);
        c[2] = D == 3 ? fmaf(A, ft.z, Ct * dz) : 0.f;
        return r2;
      };
      // skipped nearly coincident pairs (r^2 <= thr) mark the tiles of both
      // points for k_near_close: the smallest r^2 of the staged tile, or on
      // T's own tile the count of pairs at r^2 <= thr (the self pair is one)
      bool skipped;
      if (!sym) {
        float c[3];
        int ncl = 0;
        while (m) {
          const int j = __ffs(m) - 1;
          m &= m - 1u;
          ncl += (pair(j, c) <= thr) ? 1 : 0;
        }
        skipped = on && ncl > 1;
      } else {
        float rmin = __int_as_float(0x7f800000);
        // The source sides of two consecutive sources (2 x 3 components,
        // padded to 4) are summed over the warp together by a transposing
        // butterfly: each exchange halves the values a lane keeps, so 7
        // shuffles sum all six, leaving the total of (source s, component a)
        // in lane 16 s + 4 a, which stores it in the source's slot.
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        const int a_own = (b3 ? 2 : 0) + (b2 ? 1 : 0);
        auto reduce2 = [&](const float (&c0)[3], const float (&c1)[3], int j0, int j1) {
          float x[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {                  // keep source b4
            const float send = b4 ? c0[a] : c1[a];
            x[a] = (b4 ? c1[a] : c0[a]) + __shfl_xor_sync(0xffffffffu, send, 16);
          }
          // keep components {0, 1} (b3 = 0) or {2, pad} (b3 = 1)
          const float y0 = (b3 ? x[2] : x[0]) + __shfl_xor_sync(0xffffffffu, b3 ? x[0] : x[2], 8);
          const float y1 = (b3 ? 0.f : x[1]) + __shfl_xor_sync(0xffffffffu, b3 ? x[1] : 0.f, 8);
          float z = (b2 ? y1 : y0) + __shfl_xor_sync(0xffffffffu, b2 ? y0 : y1, 4);
          z += __shfl_xor_sync(0xffffffffu, z, 2);
          z += __shfl_xor_sync(0xffffffffu, z, 1);
          const int js = b4 ? j1 : j0;
          if ((lane & 3) == 0 && a_own < 3 && js >= 0) s_q[wid][js * 3 + a_own] = z;   // each slot once per tile
        };
        int jp = -1;                                     // source held back for the next round
        float cp[3] = {0.f, 0.f, 0.f};
        while (m) {
          const int j = __ffs(m) - 1;
          m &= m - 1u;
          float c[3];
          rmin = fminf(rmin, pair(j, c));
          if (jp < 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) cp[a] = c[a];
            jp = j;
            continue;
          }
          reduce2(cp, c, jp, j);
          jp = -1;
        }
        if (jp >= 0) {
          const float z3[3] = {0.f, 0.f, 0.f};
          reduce2(cp, z3, jp, -1);
        }
        skipped = rmin <= thr;
      }
      if (__any_sync(0xffffffffu, skipped)) {
        if (lane == 0) {
          P.close_flag[tile] = 1;
          P.close_flag[U] = 1;
        }
        // queue them (same FP32 arithmetic as the pair path)
        if (on)
          for (int j = 0; j < ns; ++j) {
            const float4 sp = s_pos[wid][j];
            const float dx = xt.x - sp.x, dy = xt.y - sp.y, dz = xt.z - sp.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= thr && (sym || j != lane))
              close_push(P, t0 + lane, s0 + j, e, LB, sym);
          }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) two_sum_add(uh[a], ul[a], p[a]);
      __syncwarp();
      if (sym && lane < ns) {
        float q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          q[a] = s_q[wid][lane * 3 + a];
          s_q[wid][lane * 3 + a] = 0.f;
        }
        if (q[0] != 0.f || q[1] != 0.f || q[2] != 0.f)
#pragma unroll
          for (int a = 0; a < D; ++a) atomicAdd(acc + (static_cast<int64_t>(s0) + lane) * D + a, static_cast<double>(q[a]));
      }
    }
  }
  if (on)
#pragma unroll
    for (int a = 0; a < D; ++a)
      atomicAdd(acc + (static_cast<int64_t>(t0) + lane) * D + a, static_cast<double>(uh[a]) + static_cast<double>(ul[a]));
  (void)N;
}

// u (caller order) = acc / (8 pi) [+ Stokeslet self term], one warp per tile
template <int D, int KM>
__global__ void k_near_sym_finish(const __grid_constant__ NearParams P, const double* __restrict__ acc) {
  const int tile = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= P.n_tile || lane >= P.tile_count[tile]) return;
  const int64_t i = P.tile_start[tile] + lane;
  const int64_t o = P.perm[i];
  const double sc = (KM & 1) ? self_coeff<D>(P, P.leaf_level[P.tile_leaf[tile]]) : 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double v = acc[i * D + a] * kInv8Pi;
    if (KM & 1) v += sc * P.f_orig[o * D + a];
    P.u[o * D + a] = v;
  }
}

// ----------------------------------------------------------------- FP64
// Same traversal and FP32 candidate test; every candidate is then decided
// exactly in FP64 with the oracle's operation order.
template <int D, int KM, bool GRAD, int NT, int NR>
struct Fp64Shape {
  static constexpr int NB = (NR == 1) ? ((KM == 1 && !GRAD) ? 4 : 2) : 1;   // staged tiles per batch
  static constexpr int WPB = (NR > 4) ? 2 : 4;                       // warps per block
};

template <int D, int KM, bool GRAD, int NT, int NR>
__global__ void __launch_bounds__(32 * Fp64Shape<D, KM, GRAD, NT, NR>::WPB) k_near_fp64(const __grid_constant__ NearParams P) {
  static_assert(NR == 1 || (KM == 1 && !GRAD), "several force columns: velocity only");
  static_assert(D == 3 || !GRAD, "the gradient kernel is 3D");
  constexpr int NB = Fp64Shape<D, KM, GRAD, NT, NR>::NB;
  constexpr int WPB = Fp64Shape<D, KM, GRAD, NT, NR>::WPB;
  constexpr int NS = NB * kTile;
  constexpr int NF = D + ((KM & 1) ? D * NR : 0) + ((KM & 2) ? 2 * D + 1 : 0);
  constexpr int Z = (D == 3) ? 2 : 0;   // index of the z row where one exists
  __shared__ float4 sA[WPB][NS];
  __shared__ double sD[WPB][NF][NS];
  __shared__ double sQ[WPB][NB][4];                  // per staged tile: q, 1/nu
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * WPB + wid;             // target tile
  if (tile >= P.n_ttile) return;
  const int64_t N = P.N;
  const int B = P.ttile_leaf[tile];
  const int t0 = P.ttile_start[tile], nt = P.ttile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.ttile_lo[tile], thi = P.ttile_hi[tile];
  const bool on = lane < nt;
  const float4 xt = on ? P.trel[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float tt = fmaf(xt.x, xt.x, fmaf(xt.y, xt.y, xt.z * xt.z));
  double wt[3] = {0.0, 0.0, 0.0};
  if (on)
#pragma unroll
    for (int a = 0; a < D; ++a) wt[a] = P.tw[a * P.NT + t0 + lane];

  double acc[NR][3];
#pragma unroll
  for (int k = 0; k < NR; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0;
  double G[GRAD ? 9 : 1];
#pragma unroll
  for (int k = 0; k < (GRAD ? 9 : 1); ++k) G[k] = 0.0;

  // Symmetric pass (one column, no gradient): the warp of target tile T takes
  // the source tiles U >= T; for U > T each pair also gives the source its
  // contribution (S_R even, T_R odd), from the target's densities s_td.
  constexpr bool SYM64 = (NR == 1 && !GRAD);
  constexpr int NTD = ((KM & 1) ? D : 0) + ((KM & 2) ? 2 * D + 1 : 0);
  __shared__ double s_td[SYM64 ? WPB : 1][SYM64 ? NTD : 1][kTile];
  __shared__ int s_s0[SYM64 ? WPB : 1][NB];           // per staged tile: first point, -1 if U == T
  const int tw = SYM64 ? wid : 0;
  if (SYM64 && P.acc) {
    int k = 0;
    if (KM & 1)
#pragma unroll
      for (int a = 0; a < D; ++a) s_td[tw][k++][lane] = on ? P.f64[a * N + t0 + lane] : 0.0;
    if (KM & 2) {
#pragma unroll
      for (int a = 0; a < D; ++a) s_td[tw][k++][lane] = on ? P.g64[a * N + t0 + lane] : 0.0;
#pragma unroll
      for (int a = 0; a < D + 1; ++a) s_td[tw][k++][lane] = on ? P.n64[a * N + t0 + lane] : 0.0;
    }
  }

  // One candidate pair (target coordinates w3, staged source slot idx):
  // decided and evaluated in FP64 with the oracle's operation order; the
  // contributions are added to a (velocity, [NR][3]) and gr (gradient).
  auto pair = [&](const double (&w3)[3], int idx, double (&a)[NR][3], double (&gr)[GRAD ? 9 : 1], int tl,
                  double (&sr)[3]) {
    const double* q = sQ[wid][idx >> 5];
    const double dx = __dadd_rn(__dsub_rn(w3[0], sD[wid][0][idx]), q[0]);
    const double dy = __dadd_rn(__dsub_rn(w3[1], sD[wid][1][idx]), q[1]);
    double dz = 0.0, r2;
    if (D == 3) {
      dz = __dadd_rn(__dsub_rn(w3[2], sD[wid][Z][idx]), q[2]);
      r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    } else {
      r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    }
    const double nuinv = q[3];
    const double nu2inv = nuinv * nuinv;
    const double rho2 = r2 * nu2inv;                  // exact: nuinv is a power of two
    if (!(rho2 < 1.0 && r2 > 0.0)) return;
    const double t = fma(2.0, rho2, -1.0);
    double ri = 0.0, ri2, logr2 = 0.0;
    if (D == 3) {
      ri = 1.0 / sqrt(r2);
      ri2 = ri * ri;
    } else {
      ri2 = 1.0 / r2;
      logr2 = log(rho2);
    }
    int k = D;
    if (KM & 1) {
      const double g = horner<NT>(P.c64[P_GS], t);
      const double h = horner<NT>(P.c64[P_HS], t);
      double A, C;
      if (D == 3) {
        A = fma(g, nuinv, ri);
        C = ri2 * fma(h, nuinv, ri);
      } else {
        A = -logr2 - g;
        C = fma(-h, nu2inv, 2.0 * ri2);
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const double fx = sD[wid][k][idx], fy = sD[wid][k + 1][idx];
        const double fz = (D == 3) ? sD[wid][k + Z][idx] : 0.0;
        k += D;
        const double xf = fma(dx, fx, fma(dy, fy, dz * fz));
        const double Cx = C * xf;
        a[c][0] = fma(A, fx, fma(Cx, dx, a[c][0]));
        a[c][1] = fma(A, fy, fma(Cx, dy, a[c][1]));
        if (D == 3) a[c][2] = fma(A, fz, fma(Cx, dz, a[c][2]));
        if (SYM64 && tl >= 0) {
          // S_R is even: the source gets S_R(x) f_t
          const double tfx = s_td[tw][0][tl], tfy = s_td[tw][1][tl], tfz = (D == 3) ? s_td[tw][Z][tl] : 0.0;
          const double Ct = C * fma(dx, tfx, fma(dy, tfy, dz * tfz));
          sr[0] += fma(A, tfx, Ct * dx);
          sr[1] += fma(A, tfy, Ct * dy);
          if (D == 3) sr[2] += fma(A, tfz, Ct * dz);
        }
        if (GRAD) {
          const double dg = horner<NT>(P.c64[P_DGS], t);
          const double dh = horner<NT>(P.c64[P_DHS], t);
          const double nu3i = nuinv * nuinv * nuinv;
          const double ri3 = ri2 * ri;
          const double A1 = fma(2.0 * dg, nu3i, -ri3);
          const double C1 = fma(-3.0 * ri3, ri2, ri2 * fma(2.0 * dh, nu3i, -2.0 * h * nuinv * ri2));
          const double xv[3] = {dx, dy, dz};
          const double fv[3] = {fx, fy, fz};
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            const double a1 = fma(A1, fv[jj], C1 * xv[jj] * xf);
#pragma unroll
            for (int mm = 0; mm < 3; ++mm) {
              double v = fma(a1, xv[mm], C * xv[jj] * fv[mm]);
              if (jj == mm) v = fma(C, xf, v);
              gr[jj * 3 + mm] += v;
            }
          }
        }
      }
    }
    if (KM & 2) {
      const double pt = horner<NT>(P.c64[P_PT], t);
      const double qt = horner<NT>(P.c64[P_QT], t);
      const double gx_ = sD[wid][k][idx], gy_ = sD[wid][k + 1][idx];
      const double gz_ = (D == 3) ? sD[wid][k + Z][idx] : 0.0;
      const double nx = sD[wid][k + D][idx], ny = sD[wid][k + D + 1][idx];
      const double nz = (D == 3) ? sD[wid][k + D + Z][idx] : 0.0;
      const double gn = sD[wid][k + 2 * D][idx];
      const double xn = fma(dx, nx, fma(dy, ny, dz * nz));
      const double xg = fma(dx, gx_, fma(dy, gy_, dz * gz_));
      double Dc, Ec;
      if (D == 3) {
        Dc = pt * nuinv * ri2;
        Ec = -6.0 * ri2 * ri2 * fma(qt, nuinv, ri);
      } else {
        Dc = -pt * nu2inv;
        Ec = fma(6.0 * qt, nu2inv * nu2inv, -8.0 * ri2 * ri2);
      }
      const double Ex = Ec * xg * xn + Dc * gn;
      a[0][0] += fma(Dc, fma(gx_, xn, nx * xg), Ex * dx);
      a[0][1] += fma(Dc, fma(gy_, xn, ny * xg), Ex * dy);
      if (D == 3) a[0][2] += fma(Dc, fma(gz_, xn, nz * xg), Ex * dz);
      if (GRAD) {
        // derivative of u_j = Dc V_j + Ec x_j (x.g)(x.n), V = g (x.n) + x (g.n) + n (x.g):
        //   d_m u_j = D1 x_m V_j + Dc (g_j n_m + delta_jm (g.n) + n_j g_m)
        //           + E1 x_m x_j (x.g)(x.n) + Ec (delta_jm (x.g)(x.n) + x_j (g_m (x.n) + (x.g) n_m)),
        // D1 = Dc'/r = 2 pT'/(nu^3 r^2) - 2 pT/(nu r^4),
        // E1 = Ec'/r = -6 (-5/r^7 + 2 qT'/(nu^3 r^4) - 4 qT/(nu r^6))   (' = d/ds, s = rho^2)
        const double dpt = horner<NT>(P.c64[P_DPT], t);
        const double dqt = horner<NT>(P.c64[P_DQT], t);
        const double nu3i = nuinv * nuinv * nuinv;
        const double ri4 = ri2 * ri2;
        const double D1 = fma(2.0 * dpt, nu3i * ri2, -2.0 * pt * nuinv * ri4);
        const double E1 = -6.0 * fma(-5.0 * ri4 * ri2, ri, fma(2.0 * dqt, nu3i * ri4, -4.0 * qt * nuinv * ri4 * ri2));
        const double xv[3] = {dx, dy, dz};
        const double gv[3] = {gx_, gy_, gz_};
        const double nv[3] = {nx, ny, nz};
        const double xgn = xg * xn;
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const double Vj = fma(gv[jj], xn, fma(xv[jj], gn, nv[jj] * xg));
          const double c1 = fma(D1, Vj, E1 * xv[jj] * xgn);
#pragma unroll
          for (int mm = 0; mm < 3; ++mm) {
            double v = fma(c1, xv[mm], Dc * fma(gv[jj], nv[mm], nv[jj] * gv[mm]));
            v = fma(Ec * xv[jj], fma(gv[mm], xn, xg * nv[mm]), v);
            if (jj == mm) v += fma(Dc, gn, Ec * xgn);
            gr[jj * 3 + mm] += v;
          }
        }
      }
      if (SYM64 && tl >= 0) {
        // T_R is odd: the source gets -T_R(x) : (g_t n_t)
        const int kg = (KM & 1) ? D : 0;
        const double tgx = s_td[tw][kg][tl], tgy = s_td[tw][kg + 1][tl];
        const double tgz = (D == 3) ? s_td[tw][kg + Z][tl] : 0.0;
        const double tnx = s_td[tw][kg + D][tl], tny = s_td[tw][kg + D + 1][tl];
        const double tnz = (D == 3) ? s_td[tw][kg + D + Z][tl] : 0.0;
        const double tgn = s_td[tw][kg + 2 * D][tl];
        const double xnt = fma(dx, tnx, fma(dy, tny, dz * tnz));
        const double xgt = fma(dx, tgx, fma(dy, tgy, dz * tgz));
        const double Ext = Ec * xgt * xnt + Dc * tgn;
        sr[0] -= fma(Dc, fma(tgx, xnt, tnx * xgt), Ext * dx);
        sr[1] -= fma(Dc, fma(tgy, xnt, tny * xgt), Ext * dy);
        if (D == 3) sr[2] -= fma(Dc, fma(tgz, xnt, tnz * xgt), Ext * dz);
      }
    }
  };

  // NR == 1: the warp's candidate pairs are queued (grouped by target) and
  // evaluated 32 at a time by all lanes, so the FP64 pair path runs on full
  // warps; each lane then adds its own target's results.  NR > 1: every lane
  // walks its own candidates.
  constexpr int NO = GRAD ? 12 : D;
  constexpr int Q = (NR == 1) ? ((KM == 3 && D == 3) ? 32 : 64) : 1;   // queued pairs per round (48 KB limit)
  __shared__ double s_wt[(NR == 1) ? WPB : 1][3][kTile];
  __shared__ uint16_t s_q[(NR == 1) ? WPB : 1][Q];
  __shared__ double s_r[(NR == 1) ? WPB : 1][(NR == 1) ? NO : 1][Q];
  if (NR == 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) s_wt[(NR == 1) ? wid : 0][c][lane] = wt[c];

  int nb = 0;
  auto flush = [&]() {
    __syncwarp();
    uint32_t m[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int w = 0; w < NB; ++w)
      if (w < nb) m[w] = on ? candidate_bits(&sA[wid][w * kTile], xt, tt) : 0u;
    if (NR == 1) {
      const int qw = (NR == 1) ? wid : 0;
      int cnt = 0;
#pragma unroll
      for (int w = 0; w < NB; ++w) cnt += __popc(m[w]);
      int off = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off -= cnt;
      for (int base = 0; base < total; base += Q) {
        {   // queue this lane's entries with index in [base, base + Q)
          int i = off;
#pragma unroll
          for (int w = 0; w < NB; ++w) {
            uint32_t bm = m[w];
            if (i + __popc(bm) <= base) {
              i += __popc(bm);
              continue;
            }
            while (bm && i < base + Q) {
              const int j = __ffs(bm) - 1;
              bm &= bm - 1u;
              if (i >= base) s_q[qw][i - base] = static_cast<uint16_t>((lane << 7) | (w * kTile + j));
              ++i;
            }
          }
        }
        __syncwarp();
        const int n = min(Q, total - base);
        for (int q0 = 0; q0 < n; q0 += 32) {
          const int qi = q0 + lane;
          if (qi >= n) continue;
          const int ent = s_q[qw][qi];
          const int tl = ent >> 7;
          const double w3[3] = {s_wt[qw][0][tl], s_wt[qw][1][tl], s_wt[qw][2][tl]};
          double a[NR][3] = {};
          double gr[GRAD ? 9 : 1] = {};
          double sr[3] = {0.0, 0.0, 0.0};
          const int idx = ent & 127;
          const int ss0 = (SYM64 && P.acc) ? s_s0[tw][idx >> 5] : -1;
          pair(w3, idx, a, gr, ss0 >= 0 ? tl : -1, sr);
          if (SYM64 && ss0 >= 0 && (sr[0] != 0.0 || sr[1] != 0.0 || sr[2] != 0.0))
#pragma unroll
            for (int c = 0; c < D; ++c) atomicAdd(P.acc + (static_cast<int64_t>(ss0) + (idx & 31)) * D + c, sr[c]);
#pragma unroll
          for (int c = 0; c < D; ++c) s_r[qw][c % NO][qi] = a[0][c];
          if (GRAD)
#pragma unroll
            for (int c = 0; c < 9; ++c) s_r[qw][(D + c) % NO][qi] = gr[c];
        }
        __syncwarp();
        const int i0 = max(off, base), i1 = min(off + cnt, base + Q);
        for (int i = i0; i < i1; ++i) {
#pragma unroll
          for (int c = 0; c < D; ++c) acc[0][c] += s_r[qw][c % NO][i - base];
          if (GRAD)
#pragma unroll
            for (int c = 0; c < 9; ++c) G[c] += s_r[qw][(D + c) % NO][i - base];
        }
        __syncwarp();
      }
    } else {
      BitWalker bw{m[0], m[1], m[2], m[3], 0};
      int idx;
      double sr[3];
      while (bw.next(idx)) pair(wt, idx, acc, G, -1, sr);
    }
    __syncwarp();
    nb = 0;
  };

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float nu2m = E.nu2 * (1.f + 0x1p-12f);
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    const bool sym = SYM64 && P.acc;
    if (sym && U1 <= tile) continue;
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane) &
                       (sym ? __ballot_sync(0xffffffffu, Ub + lane >= tile) : 0xffffffffu);
         tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      if (nb == NB) flush();
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      const int slot = nb * kTile + lane;
      if (lane == 0) {
        if (SYM64) s_s0[tw][nb] = (sym && U != tile) ? s0 : -1;
        sQ[wid][nb][0] = E.q[0];
        sQ[wid][nb][1] = E.q[1];
        sQ[wid][nb][2] = E.q[2];
        sQ[wid][nb][3] = static_cast<double>(E.nuinv);
      }
      if (lane < ns) {
        const int64_t sidx = s0 + lane;
        const float4 r = P.rel[sidx];
        const float sx = r.x + E.off[0], sy = r.y + E.off[1], sz = r.z + E.off[2];
        sA[wid][slot] = make_float4(-2.f * sx, -2.f * sy, -2.f * sz, fmaf(sx, sx, fmaf(sy, sy, sz * sz)) - nu2m);
        int k = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) sD[wid][k++][slot] = P.w[a * N + sidx];
        if (KM & 1)
#pragma unroll
          for (int a = 0; a < D * NR; ++a) sD[wid][k++][slot] = P.f64[a * N + sidx];
        if (KM & 2) {
#pragma unroll
          for (int a = 0; a < D; ++a) sD[wid][k++][slot] = P.g64[a * N + sidx];
#pragma unroll
          for (int a = 0; a < D + 1; ++a) sD[wid][k++][slot] = P.n64[a * N + sidx];
        }
      } else {
        sA[wid][slot] = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
      }
      ++nb;
    }
  }
  if (nb > 0) flush();

  if (!on) return;
  if (SYM64 && P.acc) {
    // both sides meet in the sorted accumulator, finished by k_near_sym_finish
#pragma unroll
    for (int a = 0; a < D; ++a) atomicAdd(P.acc + (static_cast<int64_t>(t0) + lane) * D + a, acc[0][a]);
    return;
  }
  const int64_t o = P.tperm[t0 + lane];
  const double sc = P.same_set ? self_coeff<D>(P, LB) : 0.0;   // separate targets: no self term
  const int nr = P.n_rhs;
  if (P.u) {
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      if (c >= nr) break;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double v = acc[c][a] * kInv8Pi;
        const int64_t q = (o * D + a) * nr + c;
        if ((KM & 1) && P.same_set) v += sc * P.f_orig[q];
        P.u[q] = v;
      }
    }
  }
  if (GRAD) {
#pragma unroll
    for (int k = 0; k < 9; ++k) P.gradu[o * 9 + k] = G[k] * kInv8Pi;
  }
}

// The symmetric FP32 pass (P.acc set) leaves its sums in P.acc: the caller
// adds the nearly coincident pairs (k_near_close) and finishes with
// k_near_sym_finish.
template <int D, int KM, bool GRAD, int NT, int NR>
void run_near_mixed(const NearParams& P, cudaStream_t s) {
  if constexpr (KM == 1 && !GRAD && NR == 1) {
    if (P.acc && P.u) {
      k_near_sym<D, NT><<<(P.n_tile + kSymWarps - 1) / kSymWarps, 32 * kSymWarps, 0, s>>>(P, P.acc);
      return;
    }
  }
  k_near_mixed<D, KM, GRAD, NT, NR><<<(P.n_ttile + kMixWarps - 1) / kMixWarps, 32 * kMixWarps, 0, s>>>(P);
}
template <int D, int KM, bool GRAD, int NT, int NR>
void run_near_fp64(const NearParams& P, cudaStream_t s) {
  constexpr int WPB = Fp64Shape<D, KM, GRAD, NT, NR>::WPB;
  k_near_fp64<D, KM, GRAD, NT, NR><<<(P.n_ttile + WPB - 1) / WPB, 32 * WPB, 0, s>>>(P);
  if (NR == 1 && !GRAD && P.acc) k_near_sym_finish<D, KM><<<(P.n_tile + 7) / 8, 256, 0, s>>>(P, P.acc);
}

// instantiation lists (near_mixed*.cu, near_fp64*.cu): (dim, kernels, gradient, NT, NR)
#define DMK_FOR_EACH_VARIANT_3D(M, NT) \
  M(3, 1, false, NT, 1) M(3, 2, false, NT, 1) M(3, 3, false, NT, 1) M(3, 1, true, NT, 1) \
  M(3, 1, false, NT, 4) M(3, 1, false, NT, 16)
// FP64 only: the stresslet gradient (every precision takes FP64 pair terms for it)
#define DMK_FOR_EACH_VARIANT_3D_FP64(M, NT) \
  DMK_FOR_EACH_VARIANT_3D(M, NT) M(3, 2, true, NT, 1) M(3, 3, true, NT, 1)
#define DMK_FOR_EACH_VARIANT_2D(M, NT) \
  M(2, 1, false, NT, 1) M(2, 2, false, NT, 1) M(2, 3, false, NT, 1) M(2, 1, false, NT, 4) M(2, 1, false, NT, 16)

#define DMK_NT_MIXED(X) X(8) X(10) X(12) X(13) X(14) X(16)   // FP32 pair terms: eps >= 2e-7
#define DMK_NT_FP64(X) X(16) X(20) X(24) X(28) X(32)

}  // namespace dmk
