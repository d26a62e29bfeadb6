// Float-float near-field kernel (2D and 3D): the MIXED path for eps below the
// FP32 floor of the pair terms.
//
// GB300 runs FP64 at about 1/74 of its FP32 FMA rate, so the tight-tolerance
// pair terms are evaluated in float-float (FF) arithmetic: every quantity is an
// unevaluated sum hi + lo of two floats (about 48 significant bits), built from
// the error-free transformations two-sum (Knuth) and two-product by FMA
// (exact product error fma(a, b, -ab)).  The formulas are those of the FP64
// kernel (Sec. 5.2, Eqs. (res_stokeslet), (Soffdiag), (res_stresslet),
// (T-offd) with the length-scale remark closing Sec. 5.2):
//   S_R f     = [A f + C (x.f) x] / (8 pi),   A = 1/r + gS/nu,  C = (1/r + hS/nu)/r^2
//   T_R:(g n) = [D (g (x.n) + x (g.n) + n (x.g)) + E x (x.g)(x.n)] / (8 pi),
//               D = pT/(nu r^2),  E = -6 (1/r + qT/nu)/r^4
// with gS, hS, pT, qT polynomials in t = 2 rho^2 - 1 whose FP64 coefficients
// are split into FF pairs and evaluated two at a time by packed FP32x2 Horner.
// In 2D (App. B functions m_d, m_o, m_td, m_to in the same tables):
//   A = -log rho^2 - m_d,  C = 2/r^2 - m_o/nu^2,  D = -m_td/nu^2,
//   E = -8/r^4 + 6 m_to/nu^4,
// with log rho^2 in FF by argument reduction and the atanh series.
//
// Inputs in FF: leaf-relative coordinates (rel + rel_lo, the FP32 residual of
// the FP64 offset from the leaf centre), forces, strengths and orientations
// (FP64 values split as hi + lo).  1/r is FP32 rsqrt refined by one Newton step
// in FF.  Candidate pairs come from the FP32 test of the mixed kernel (on the hi
// parts, margin 2^-12 nu^2); the cutoff r < nu is then decided on the FF r^2.
//
// Work decomposition: one warp per target tile.  Each surviving source tile is
// staged in shared memory; each lane marks its candidate sources in a bit mask;
// the candidate (target, source) pairs of the warp are written to a shared
// queue (grouped by target) and evaluated 32 at a time by all lanes, so the
// expensive FF pair evaluation runs on full warps whatever the geometry; each
// lane then adds the results of its own target's pairs to its FF accumulator.
#pragma once
#include "near_kernel.cuh"

namespace dmk {

struct FFParams {
  const float4* rel_lo;  // FP32 residual of the leaf-relative coordinates (sorted)
  const float4* f_hi;    // sorted forces, hi / lo
  const float4* f_lo;
  const float4* g_hi;    // sorted stresslet strengths, hi / lo
  const float4* g_lo;
  const float4* n_hi;    // sorted orientations, hi / lo; .w = g.n hi / lo
  const float4* n_lo;
  float2 chi[3][kPolyCap];   // (gS, hS), (pT, qT), (gS', hS'): hi parts of the FP64 coefficients
  float2 clo[3][kPolyCap];   // lo parts
};

// ------------------------------------------------------------ FF helpers
// Round-to-nearest intrinsics throughout so that no operation is contracted.
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float s) {        // s a power of two: exact
  return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {         // b any float
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ double ff_to_double(ff a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// packed pair of FF numbers (two polynomials at once)
struct ff2 {
  float2 hi, lo;
};

// Horner for two polynomials in FF with packed FP32x2 operations; the running
// value is kept unnormalised between steps (its lo part stays within a few
// ulp of hi), normalised once at the end.
template <int NT>
__device__ __forceinline__ ff2 horner_ff2(const float2 (&chi)[kPolyCap], const float2 (&clo)[kPolyCap], ff t) {
  const float2 th = make_float2(t.hi, t.hi), tl = make_float2(t.lo, t.lo);
  float2 vh = chi[NT - 1], vl = clo[NT - 1];
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) {
    const float2 p = __fmul2_rn(vh, th);
    float2 e = __ffma2_rn(vh, th, make_float2(-p.x, -p.y));
    e = __ffma2_rn(vh, tl, e);
    e = __ffma2_rn(vl, th, e);
    const float2 c = chi[k];
    const float2 s = __fadd2_rn(p, c);
    const float2 bb = sub2(s, p);
    const float2 err = __fadd2_rn(sub2(p, sub2(s, bb)), sub2(c, bb));
    vh = s;
    vl = __fadd2_rn(err, __fadd2_rn(e, clo[k]));
  }
  const ff a = fast_two_sum(vh.x, vl.x), b = fast_two_sum(vh.y, vl.y);
  return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}

// 1/sqrt(r2) in FF: FP32 rsqrt y, then y (1 + d/2) with d = 1 - r2 y^2 from an
// FF product (relative error ~2^-44 from the one Newton step)
__device__ __forceinline__ ff ff_rsqrt(ff r2) {
  const float y = rsqrtf(r2.hi);
  const float y2 = __fmul_rn(y, y);
  const ff yy = {y2, fmaf(y, y, -y2)};
  const ff q = ff_mul(r2, yy);
  const float d = __fsub_rn(__fsub_rn(1.f, q.hi), q.lo);
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), d));
}

// 1/r2 in FF: FP32 reciprocal y, then y (1 + d) with d = 1 - r2 y (one Newton step)
__device__ __forceinline__ ff ff_rcp(ff r2) {
  const float y = __frcp_rn(r2.hi);
  const ff q = ff_mul_f(r2, y);
  const float d = __fsub_rn(__fsub_rn(1.f, q.hi), q.lo);
  return fast_two_sum(y, __fmul_rn(y, d));
}

// log(x) in FF for 0 < x (normalised FF): x = 2^e m with m in [sqrt(1/2),
// sqrt(2)); log m = 2 atanh(s), s = (m - 1)/(m + 1), |s| < 0.172, summed as
// 2 s sum_k s^(2k)/(2k+1) (terms k >= 4 in FP32: they are below 1e-7 of the
// sum), plus e log 2 with log 2 in FF.
__device__ __forceinline__ ff ff_log(ff x) {
  int e;
  float m0 = frexpf(x.hi, &e);                          // x.hi = m0 2^e, m0 in [1/2, 1)
  if (m0 < 0.70710678f) --e;
  const float sc = ldexpf(1.f, -e);                      // exact
  const ff m = {__fmul_rn(x.hi, sc), __fmul_rn(x.lo, sc)};
  const ff num = fast_two_sum(__fsub_rn(m.hi, 1.f), m.lo);    // m.hi - 1 exact (Sterbenz)
  const ff den = ff_add(m, {1.f, 0.f});
  const float q1 = __fdiv_rn(num.hi, den.hi);
  const ff rr = ff_add(num, ff_neg(ff_mul_f(den, q1)));
  const ff sv = fast_two_sum(q1, __fdiv_rn(rr.hi, den.hi));
  const ff z = ff_mul(sv, sv);
  // FP32 tail: sum_{k>=4} z^(k-4)/(2k+1), k = 4..10
  float tail = 1.f / 21.f;
  tail = fmaf(tail, z.hi, 1.f / 19.f);
  tail = fmaf(tail, z.hi, 1.f / 17.f);
  tail = fmaf(tail, z.hi, 1.f / 15.f);
  tail = fmaf(tail, z.hi, 1.f / 13.f);
  tail = fmaf(tail, z.hi, 1.f / 11.f);
  tail = fmaf(tail, z.hi, 1.f / 9.f);
  // FF steps k = 3, 2, 1, 0
  constexpr double c7 = 1.0 / 7.0, c5 = 1.0 / 5.0, c3 = 1.0 / 3.0;
  ff v = {tail, 0.f};
  v = ff_add(ff_mul(v, z), {static_cast<float>(c7), static_cast<float>(c7 - static_cast<double>(static_cast<float>(c7)))});
  v = ff_add(ff_mul(v, z), {static_cast<float>(c5), static_cast<float>(c5 - static_cast<double>(static_cast<float>(c5)))});
  v = ff_add(ff_mul(v, z), {static_cast<float>(c3), static_cast<float>(c3 - static_cast<double>(static_cast<float>(c3)))});
  v = ff_add(ff_mul(v, z), {1.f, 0.f});
  constexpr double ln2 = 0.6931471805599453094;
  const ff l2 = {static_cast<float>(ln2), static_cast<float>(ln2 - static_cast<double>(static_cast<float>(ln2)))};
  return ff_add(ff_scale(ff_mul(sv, v), 2.f), ff_mul_f(l2, static_cast<float>(e)));
}

// Source position in the target leaf's frame in FF: (rel + off) + rel_lo,
// with off the exact dyadic offset of the source leaf (hi parts in ph, lo in pl).
__device__ __forceinline__ void ff_source_pos(float4 r, float4 rl, const float (&off)[3], float4& ph, float4& pl) {
  const ff sx = two_sum(r.x, off[0]), sy = two_sum(r.y, off[1]), sz = two_sum(r.z, off[2]);
  const ff px = fast_two_sum(sx.hi, __fadd_rn(sx.lo, rl.x));
  const ff py = fast_two_sum(sy.hi, __fadd_rn(sy.lo, rl.y));
  const ff pz = fast_two_sum(sz.hi, __fadd_rn(sz.lo, rl.z));
  ph = make_float4(px.hi, py.hi, pz.hi, 0.f);
  pl = make_float4(px.lo, py.lo, pz.lo, 0.f);
}

// FF displacement x = target - source (target th + tl, source ph + pl) and r^2;
// the float-float kernel and k_near_close decide "nearly coincident" on the
// same r^2.hi, so they split the pairs exactly.
template <int D>
__device__ __forceinline__ ff ff_disp_r2(float4 th, float4 tl, float4 ph, float4 pl, ff& dx, ff& dy, ff& dz) {
  dx = two_sum(th.x, -ph.x);
  dy = two_sum(th.y, -ph.y);
  dz = {0.f, 0.f};
  dx = fast_two_sum(dx.hi, __fadd_rn(dx.lo, __fsub_rn(tl.x, pl.x)));
  dy = fast_two_sum(dy.hi, __fadd_rn(dy.lo, __fsub_rn(tl.y, pl.y)));
  ff r2 = ff_add(ff_mul(dx, dx), ff_mul(dy, dy));
  if (D == 3) {
    dz = two_sum(th.z, -ph.z);
    dz = fast_two_sum(dz.hi, __fadd_rn(dz.lo, __fsub_rn(tl.z, pl.z)));
    r2 = ff_add(r2, ff_mul(dz, dz));
  }
  return r2;
}

// ------------------------------------------------------------------ kernel
// GRAD (Stokeslet only) adds the velocity gradient, the derivative of
// Eq. (res_stokeslet) with the tree held fixed:
//   d_m (S_R f)_j = A1 x_m f_j + C1 x_m x_j (x.f) + C (delta_jm (x.f) + x_j f_m)
//   A1 = -1/r^3 + 2 gS'/nu^3,  C1 = -3/r^5 + (2 hS'/nu^3 - 2 hS/(nu r^2))/r^2.
// warps (target tiles) per block: measured best on GB300 (3D 4, 2D 1)
template <int D> constexpr int kFFWarps = (D == 3) ? 4 : 1;
template <int D, int KM, bool GRAD, int NT>
__global__ void __launch_bounds__(32 * kFFWarps<D>) k_near_ff(const __grid_constant__ NearParams P,
                                                           const __grid_constant__ FFParams F) {
  static_assert(!GRAD || (KM == 1 && D == 3), "the gradient kernel is the 3D Stokeslet's");
  constexpr int NO = GRAD ? 12 : D;                  // outputs per pair: u (D) [+ grad u (9)]
  constexpr int kFFQueue = GRAD ? 64 : 128;          // candidate pairs evaluated per round (per warp)
  constexpr int W = kFFWarps<D>;
  __shared__ float4 s_tst[W][4][8];                  // FP32 test rows (as in the mixed kernel)
  __shared__ float4 s_ph[W][kTile], s_pl[W][kTile];  // source position in the target frame, FF
  __shared__ float4 s_ah[W][kTile], s_al[W][kTile];  // Stokeslet force / stresslet strength, FF
  __shared__ float4 s_nh[(KM & 2) ? W : 1][kTile], s_nl[(KM & 2) ? W : 1][kTile];   // orientation, .w = g.n
  __shared__ float4 s_bh[(KM == 3) ? W : 1][kTile], s_bl[(KM == 3) ? W : 1][kTile];  // stresslet strength if both
  __shared__ float4 s_th[W][kTile], s_tl[W][kTile];  // targets, FF
  __shared__ uint16_t s_q[W][kFFQueue];              // queue: target lane << 5 | source slot
  __shared__ float2 s_r[W][NO][kFFQueue];            // per queued pair: contributions (hi, lo)
  // symmetric pass: the targets' densities for the source side of each pair
  // (the gradient of the source is minus the derivative at x: grad S_R is odd)
  constexpr bool SYM = true;
  __shared__ float4 s_tfh[(SYM && (KM & 1)) ? W : 1][kTile], s_tfl[(SYM && (KM & 1)) ? W : 1][kTile];
  __shared__ float4 s_tgh[(SYM && (KM & 2)) ? W : 1][kTile], s_tgl[(SYM && (KM & 2)) ? W : 1][kTile];
  __shared__ float4 s_tnh[(SYM && (KM & 2)) ? W : 1][kTile], s_tnl[(SYM && (KM & 2)) ? W : 1][kTile];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * W + wid;
  if (tile >= P.n_tile) return;
  const int B = P.tile_leaf[tile];
  const int t0 = P.tile_start[tile], nt = P.tile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.tile_lo[tile], thi = P.tile_hi[tile];
  const bool on = lane < nt;
  const float4 xt = on ? P.rel[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float tt = on ? fmaf(xt.x, xt.x, fmaf(xt.y, xt.y, xt.z * xt.z)) : __int_as_float(0x7f800000);
  s_th[wid][lane] = xt;
  s_tl[wid][lane] = on ? F.rel_lo[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (SYM) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int ws = SYM ? wid : 0;
    if (KM & 1) {
      s_tfh[(KM & 1) ? ws : 0][lane] = on ? F.f_hi[t0 + lane] : z4;
      s_tfl[(KM & 1) ? ws : 0][lane] = on ? F.f_lo[t0 + lane] : z4;
    }
    if (KM & 2) {
      s_tgh[(KM & 2) ? ws : 0][lane] = on ? F.g_hi[t0 + lane] : z4;
      s_tgl[(KM & 2) ? ws : 0][lane] = on ? F.g_lo[t0 + lane] : z4;
      s_tnh[(KM & 2) ? ws : 0][lane] = on ? F.n_hi[t0 + lane] : z4;
      s_tnl[(KM & 2) ? ws : 0][lane] = on ? F.n_lo[t0 + lane] : z4;
    }
  }
  float* const rowx = reinterpret_cast<float*>(s_tst[wid][0]);
  float* const rowy = reinterpret_cast<float*>(s_tst[wid][1]);
  float* const rowz = reinterpret_cast<float*>(s_tst[wid][2]);
  float* const roww = reinterpret_cast<float*>(s_tst[wid][3]);
  ff acc[NO];
#pragma unroll
  for (int a = 0; a < NO; ++a) acc[a] = {0.f, 0.f};

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float nu2 = E.nu2, nuinv = E.nuinv;
    const float nu2inv = nuinv * nuinv;
    const float nu2m = nu2 * (1.f + 0x1p-12f);
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    // symmetric pass: the source tiles U >= T (T's own tile: target side only)
    if (SYM && U1 <= tile) continue;
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane) &
                       (SYM ? __ballot_sync(0xffffffffu, Ub + lane >= tile) : 0xffffffffu);
         tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      const bool both = SYM && U != tile;              // source side too
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      __syncwarp();
      if (lane < ns) {
        const int64_t si = s0 + lane;
        float4 ph, pl;
        ff_source_pos(P.rel[si], F.rel_lo[si], E.off, ph, pl);
        s_ph[wid][lane] = ph;
        s_pl[wid][lane] = pl;
        rowx[lane] = -2.f * ph.x;
        rowy[lane] = -2.f * ph.y;
        rowz[lane] = -2.f * ph.z;
        roww[lane] = fmaf(ph.x, ph.x, fmaf(ph.y, ph.y, ph.z * ph.z)) - nu2m;
        if (KM & 1) {
          s_ah[wid][lane] = F.f_hi[si];
          s_al[wid][lane] = F.f_lo[si];
        }
        if (KM & 2) {
          if (KM == 3) {
            s_bh[(KM == 3) ? wid : 0][lane] = F.g_hi[si];
            s_bl[(KM == 3) ? wid : 0][lane] = F.g_lo[si];
          } else {
            s_ah[wid][lane] = F.g_hi[si];
            s_al[wid][lane] = F.g_lo[si];
          }
          s_nh[(KM & 2) ? wid : 0][lane] = F.n_hi[si];
          s_nl[(KM & 2) ? wid : 0][lane] = F.n_lo[si];
        }
      } else {
        rowx[lane] = rowy[lane] = rowz[lane] = 0.f;
        roww[lane] = __int_as_float(0x7f800000);      // never a candidate
      }
      __syncwarp();
      // candidates of this lane's target; the warp's list grouped by target
      uint32_t bits = candidate_mask(s_tst[wid], xt, tt);
      const int cnt = __popc(bits);
      int off = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off -= cnt;                                       // exclusive prefix
      for (int base = 0; base < total; base += kFFQueue) {
        // queue the entries [base, base + kFFQueue) of the warp's list
        {
          uint32_t b = bits;
          int i = off;
          for (; b && i < base; ++i) b &= b - 1u;
          for (; b && i < base + kFFQueue; ++i) {
            const int j = __ffs(b) - 1;
            b &= b - 1u;
            s_q[wid][i - base] = static_cast<uint16_t>((lane << 5) | j);
          }
        }
        __syncwarp();
        const int n = min(kFFQueue, total - base);
        for (int q0 = 0; q0 < n; q0 += 32) {
          const int qi = q0 + lane;
          if (qi >= n) continue;
          const int ent = s_q[wid][qi];
          const int tl = ent >> 5, j = ent & 31;
          ff dx, dy, dz;
          const ff r2 = ff_disp_r2<D>(s_th[wid][tl], s_tl[wid][tl], s_ph[wid][j], s_pl[wid][j], dx, dy, dz);
          float2 res[NO];
#pragma unroll
          for (int a = 0; a < NO; ++a) res[a] = make_float2(0.f, 0.f);
          // nearly coincident pairs (r^2 <= kCloseFF nu^2) are left to
          // k_near_close (FP64); they mark the tiles of both points
          const bool inside = (r2.hi < nu2 || (r2.hi == nu2 && r2.lo < 0.f)) && (r2.hi > nu2 * kCloseFF);
          if (r2.hi <= nu2 * kCloseFF && (both || tl != j)) {
            P.close_flag[tile] = 1;
            if (both) P.close_flag[U] = 1;
            close_push(P, t0 + tl, s0 + j, e, LB, both);
          }
          if (inside) {
            const ff rho2 = ff_scale(r2, nu2inv);
            // t = 2 rho^2 - 1; the FP32 difference is not exact for rho^2 < 1/4
            const ff t0 = two_sum(__fmul_rn(2.f, rho2.hi), -1.f);
            const ff t = fast_two_sum(t0.hi, __fadd_rn(t0.lo, __fmul_rn(2.f, rho2.lo)));
            ff ri = {0.f, 0.f}, ri2, logr2 = {0.f, 0.f};
            if (D == 3) {
              ri = ff_rsqrt(r2);
              ri2 = ff_mul(ri, ri);
            } else {
              ri2 = ff_rcp(r2);
              logr2 = ff_log(rho2);
            }
            const ff xv[3] = {dx, dy, dz};
            ff out[NO];
            ff src[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};   // source side (symmetric pass)
            ff srcg[GRAD ? 9 : 1];                             // source side of the gradient
#pragma unroll
            for (int a = 0; a < (GRAD ? 9 : 1); ++a) srcg[a] = {0.f, 0.f};
            if (KM & 1) {
              const ff2 gh = horner_ff2<NT>(F.chi[0], F.clo[0], t);
              ff A, C;
              if (D == 3) {
                A = ff_add(ri, ff_scale({gh.hi.x, gh.lo.x}, nuinv));
                C = ff_mul(ri2, ff_add(ri, ff_scale({gh.hi.y, gh.lo.y}, nuinv)));
              } else {
                A = ff_neg(ff_add(logr2, {gh.hi.x, gh.lo.x}));
                C = ff_add(ff_scale(ri2, 2.f), ff_neg(ff_scale({gh.hi.y, gh.lo.y}, nu2inv)));
              }
              const float4 fh = s_ah[wid][j], fl = s_al[wid][j];
              const ff fv[3] = {{fh.x, fl.x}, {fh.y, fl.y}, {fh.z, fl.z}};
              ff xf = ff_add(ff_mul(dx, fv[0]), ff_mul(dy, fv[1]));
              if (D == 3) xf = ff_add(xf, ff_mul(dz, fv[2]));
              const ff Cx = ff_mul(C, xf);
#pragma unroll
              for (int a = 0; a < D; ++a) out[a] = ff_add(ff_mul(A, fv[a]), ff_mul(Cx, xv[a]));
              if (SYM && both) {
                // S_R is even: u_s += S_R(x) f_t
                const float4 th4 = s_tfh[(SYM && (KM & 1)) ? wid : 0][tl];
                const float4 tl4 = s_tfl[(SYM && (KM & 1)) ? wid : 0][tl];
                const ff ftv[3] = {{th4.x, tl4.x}, {th4.y, tl4.y}, {th4.z, tl4.z}};
                ff xft = ff_add(ff_mul(dx, ftv[0]), ff_mul(dy, ftv[1]));
                if (D == 3) xft = ff_add(xft, ff_mul(dz, ftv[2]));
                const ff Cxt = ff_mul(C, xft);
#pragma unroll
                for (int a = 0; a < D; ++a) src[a] = ff_add(ff_mul(A, ftv[a]), ff_mul(Cxt, xv[a]));
              }
              if (GRAD) {
                const ff2 dgh = horner_ff2<NT>(F.chi[2], F.clo[2], t);
                const float nu3i = nuinv * nuinv * nuinv;
                const ff ri3 = ff_mul(ri2, ri);
                const ff A1 = ff_add(ff_scale({dgh.hi.x, dgh.lo.x}, 2.f * nu3i), ff_neg(ri3));
                const ff hnr = ff_mul(ff_scale({gh.hi.y, gh.lo.y}, 2.f * nuinv), ri2);
                const ff C1 = ff_add(ff_mul_f(ff_mul(ri3, ri2), -3.f),
                                     ff_mul(ri2, ff_add(ff_scale({dgh.hi.y, dgh.lo.y}, 2.f * nu3i), ff_neg(hnr))));
                const ff Cxf = ff_mul(C, xf);
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                  const ff a1 = ff_add(ff_mul(A1, fv[jj]), ff_mul(ff_mul(C1, xv[jj]), xf));
                  const ff cx = ff_mul(C, xv[jj]);
#pragma unroll
                  for (int mm = 0; mm < 3; ++mm) {
                    ff v = ff_add(ff_mul(a1, xv[mm]), ff_mul(cx, fv[mm]));
                    if (jj == mm) v = ff_add(v, Cxf);
                    out[3 + jj * 3 + mm] = v;
                  }
                }
                if (SYM && both) {
                  // the source's gradient: minus the same expression with f_t
                  const float4 th4 = s_tfh[(SYM && (KM & 1)) ? wid : 0][tl];
                  const float4 tl4 = s_tfl[(SYM && (KM & 1)) ? wid : 0][tl];
                  const ff ftv[3] = {{th4.x, tl4.x}, {th4.y, tl4.y}, {th4.z, tl4.z}};
                  const ff xft = ff_add(ff_add(ff_mul(dx, ftv[0]), ff_mul(dy, ftv[1])), ff_mul(dz, ftv[2]));
                  const ff Cxft = ff_mul(C, xft);
#pragma unroll
                  for (int jj = 0; jj < 3; ++jj) {
                    const ff a1 = ff_add(ff_mul(A1, ftv[jj]), ff_mul(ff_mul(C1, xv[jj]), xft));
                    const ff cx = ff_mul(C, xv[jj]);
#pragma unroll
                    for (int mm = 0; mm < 3; ++mm) {
                      ff v = ff_add(ff_mul(a1, xv[mm]), ff_mul(cx, ftv[mm]));
                      if (jj == mm) v = ff_add(v, Cxft);
                      srcg[jj * 3 + mm] = ff_neg(v);
                    }
                  }
                }
              }
            } else {
#pragma unroll
              for (int a = 0; a < D; ++a) out[a] = {0.f, 0.f};
            }
            if (KM & 2) {
              const ff2 pq = horner_ff2<NT>(F.chi[1], F.clo[1], t);
              const float4 gh4 = (KM == 3) ? s_bh[(KM == 3) ? wid : 0][j] : s_ah[wid][j];
              const float4 gl4 = (KM == 3) ? s_bl[(KM == 3) ? wid : 0][j] : s_al[wid][j];
              const float4 nh4 = s_nh[(KM & 2) ? wid : 0][j], nl4 = s_nl[(KM & 2) ? wid : 0][j];
              const ff gv[3] = {{gh4.x, gl4.x}, {gh4.y, gl4.y}, {gh4.z, gl4.z}};
              const ff nv[3] = {{nh4.x, nl4.x}, {nh4.y, nl4.y}, {nh4.z, nl4.z}};
              const ff gn = {nh4.w, nl4.w};
              ff xn = ff_add(ff_mul(dx, nv[0]), ff_mul(dy, nv[1]));
              ff xg = ff_add(ff_mul(dx, gv[0]), ff_mul(dy, gv[1]));
              if (D == 3) {
                xn = ff_add(xn, ff_mul(dz, nv[2]));
                xg = ff_add(xg, ff_mul(dz, gv[2]));
              }
              ff Dc, Ec;
              if (D == 3) {
                Dc = ff_mul(ff_scale({pq.hi.x, pq.lo.x}, nuinv), ri2);
                Ec = ff_mul_f(ff_mul(ff_mul(ri2, ri2), ff_add(ri, ff_scale({pq.hi.y, pq.lo.y}, nuinv))), -6.f);
              } else {
                Dc = ff_neg(ff_scale({pq.hi.x, pq.lo.x}, nu2inv));
                Ec = ff_add(ff_scale(ff_mul(ri2, ri2), -8.f),
                            ff_mul_f(ff_scale({pq.hi.y, pq.lo.y}, nu2inv * nu2inv), 6.f));
              }
              // E (x.g)(x.n) + D (g.n): coefficient of x
              const ff Ex = ff_add(ff_mul(Ec, ff_mul(xg, xn)), ff_mul(Dc, gn));
#pragma unroll
              for (int a = 0; a < D; ++a) {
                const ff sym = ff_add(ff_mul(gv[a], xn), ff_mul(nv[a], xg));
                out[a] = ff_add(out[a], ff_add(ff_mul(Dc, sym), ff_mul(Ex, xv[a])));
              }
              if (SYM && both) {
                // T_R is odd: u_s -= T_R(x) : (g_t n_t)
                const int ws = (SYM && (KM & 2)) ? wid : 0;
                const float4 gh5 = s_tgh[ws][tl], gl5 = s_tgl[ws][tl], nh5 = s_tnh[ws][tl], nl5 = s_tnl[ws][tl];
                const ff gt[3] = {{gh5.x, gl5.x}, {gh5.y, gl5.y}, {gh5.z, gl5.z}};
                const ff ntv[3] = {{nh5.x, nl5.x}, {nh5.y, nl5.y}, {nh5.z, nl5.z}};
                const ff gnt = {nh5.w, nl5.w};
                ff xnt = ff_add(ff_mul(dx, ntv[0]), ff_mul(dy, ntv[1]));
                ff xgt = ff_add(ff_mul(dx, gt[0]), ff_mul(dy, gt[1]));
                if (D == 3) {
                  xnt = ff_add(xnt, ff_mul(dz, ntv[2]));
                  xgt = ff_add(xgt, ff_mul(dz, gt[2]));
                }
                const ff Ext = ff_add(ff_mul(Ec, ff_mul(xgt, xnt)), ff_mul(Dc, gnt));
#pragma unroll
                for (int a = 0; a < D; ++a) {
                  const ff st = ff_add(ff_mul(gt[a], xnt), ff_mul(ntv[a], xgt));
                  src[a] = ff_add(src[a], ff_neg(ff_add(ff_mul(Dc, st), ff_mul(Ext, xv[a]))));
                }
              }
            }
            if (SYM && both) {
#pragma unroll
              for (int a = 0; a < D; ++a) atomicAdd(P.acc + (static_cast<int64_t>(s0) + j) * NO + a, ff_to_double(src[a]));
              if (GRAD)
#pragma unroll
                for (int a = 0; a < 9; ++a) atomicAdd(P.acc + (static_cast<int64_t>(s0) + j) * NO + 3 + a, ff_to_double(srcg[a]));
            }
#pragma unroll
            for (int a = 0; a < NO; ++a) res[a] = make_float2(out[a].hi, out[a].lo);
          }
#pragma unroll
          for (int a = 0; a < NO; ++a) s_r[wid][a][qi] = res[a];
        }
        __syncwarp();
        // this lane's own entries of the round
        const int i0 = max(off, base), i1 = min(off + cnt, base + kFFQueue);
        for (int i = i0; i < i1; ++i) {
#pragma unroll
          for (int a = 0; a < NO; ++a) {
            const float2 v = s_r[wid][a][i - base];
            acc[a] = ff_add(acc[a], {v.x, v.y});
          }
        }
        __syncwarp();
      }
    }
  }
  if (!on) return;
  // both sides meet in the sorted FP64 accumulator (NO values per point),
  // finished by k_near_sym_finish / k_near_sym_finish_grad
#pragma unroll
  for (int a = 0; a < NO; ++a) atomicAdd(P.acc + (static_cast<int64_t>(t0) + lane) * NO + a, ff_to_double(acc[a]));
  (void)LB;
}

// velocity (if asked) and gradient from the accumulator of the symmetric
// gradient pass: u at [0, 3), grad u at [3, 12) per sorted point
template <int D>
__global__ void k_near_sym_finish_grad(const __grid_constant__ NearParams P, const double* __restrict__ acc) {
  static_assert(D == 3, "the gradient is 3D");
  const int tile = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= P.n_tile || lane >= P.tile_count[tile]) return;
  const int64_t i = P.tile_start[tile] + lane;
  const int64_t o = P.perm[i];
  if (P.u) {
    const double sc = self_coeff<3>(P, P.leaf_level[P.tile_leaf[tile]]);
#pragma unroll
    for (int a = 0; a < 3; ++a) P.u[o * 3 + a] = acc[i * 12 + a] * kInv8Pi + sc * P.f_orig[o * 3 + a];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) P.gradu[o * 9 + k] = acc[i * 12 + 3 + k] * kInv8Pi;
}

// Leaves its sums in P.acc: the caller adds the nearly coincident pairs
// (k_near_close) and finishes with k_near_sym_finish(_grad).
template <int D, int KM, bool GRAD, int NT>
void run_near_ff(const NearParams& P, const FFParams& F, cudaStream_t s) {
  k_near_ff<D, KM, GRAD, NT><<<(P.n_tile + kFFWarps<D> - 1) / kFFWarps<D>, 32 * kFFWarps<D>, 0, s>>>(P, F);
}

#define DMK_FOR_EACH_FF(M, NT)                                                    \
  M(3, 1, false, NT) M(3, 2, false, NT) M(3, 3, false, NT) M(3, 1, true, NT)     \
  M(2, 1, false, NT) M(2, 2, false, NT) M(2, 3, false, NT)

}  // namespace dmk
