// Adjoint of the 3D near-field Stokeslet (reverse mode of u = S_R f with the
// tree, hence every residual scale nu_ts, held fixed).
//
// For L = sum_t w_t . u_t with u_t = sum_{s near t} S_R(x_t - x_s) f_s + self:
//   dL/df_s = v_s = sum_t S_R(x_s - x_t) w_t + self(w_s)    (S_R even and symmetric)
//   dL/dx_t = sum_s G(w_t, f_s; x) + G(f_t, w_s; x),         x = x_t - x_s,
// where G(a, b; x)_m = sum_j a_j d_m (S_R b)_j.  With S_R b = A b + C (x.b) x
// (the pair terms of Eq. (res_stokeslet); A, C, and A1 = A'/r, C1 = C'/r as in
// the gradient kernels):
//   G(a, b; x) = [A1 (a.b) + C1 (x.a)(x.b)] x + C [a (x.b) + b (x.a)].
// G is odd in x and symmetric in (a, b), so the pair's contribution to the
// source is minus its contribution to the target, and v is symmetric as in
// the forward pass: one evaluation serves both points (the symmetric pass of
// the forward kernels).  The self term of v is the forward self term applied
// to w; the self term does not depend on x.
//
// One kernel, two arithmetics: float-float pair terms (MIXED plans, all eps)
// with nearly coincident pairs (r <= nu/1024) in FP64, or FP64 throughout
// (FP64 plans).  Traversal as in k_near_ff: one warp per target tile, source
// tiles U >= T of its near list staged in shared memory, candidate pairs by
// the FP32 test, queued and evaluated 32 at a time by the whole warp.  Both
// sides meet in an FP64 accumulator [N][6] (v, dL/dx) in sorted order.
#pragma once
#include <type_traits>

#include "near_ff.cuh"

namespace dmk {

struct AdjParams {
  // float-float inputs (sorted): coordinate residuals, forces f and cotangents w
  const float4* rel_lo;
  const float4* f_hi;
  const float4* f_lo;
  const float4* w_hi;
  const float4* w_lo;
  // FP64 inputs (sorted SoA [3][N]): forces and cotangents
  const double* f64;
  const double* w64;
  const double* w_orig;   // caller's cotangents [N][3] (self term of v)
  double* v;              // [N][3] caller order: dL/df
  double* gx;             // [N][3] caller order: dL/dx
  double* acc;            // [N][6] sorted, zeroed
  float2 chi[3][kPolyCap];   // (gS, hS), (gS', hS') FF coefficients (rows 0 and 2 used)
  float2 clo[3][kPolyCap];
};

// One pair in FP64: x = (w_t - w_s) + q (the FP64 kernel's decision r < nu),
// densities ft, wt of the target and fs, ws of the source.  out[0, 3) target
// v, [3, 6) target dL/dx; with both, [6, 9) source v, [9, 12) source dL/dx.
// Terms without the 1/(8 pi) factor.
template <int D>
__device__ __noinline__ void adj_pair_fp64(const NearParams& P, int64_t it, int64_t is, const double* q, double nuinv,
                                           const double* ft, const double* wt, const double* fs, const double* ws,
                                           bool both, double* out) {
  const int64_t N = P.N;
  double x[3];
  double r2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = __dadd_rn(__dsub_rn(P.w[a * N + it], P.w[a * N + is]), q[a]);
    r2 = __dadd_rn(r2, __dmul_rn(x[a], x[a]));
  }
  const double rho2 = r2 * (nuinv * nuinv);
  if (!(rho2 < 1.0 && r2 > 0.0)) return;
  const double t = fma(2.0, rho2, -1.0);
  const double ri = 1.0 / sqrt(r2);
  const double ri2 = ri * ri, ri3 = ri2 * ri;
  const double g = horner<kPolyCap>(P.c64[P_GS], t);
  const double h = horner<kPolyCap>(P.c64[P_HS], t);
  const double dg = horner<kPolyCap>(P.c64[P_DGS], t);
  const double dh = horner<kPolyCap>(P.c64[P_DHS], t);
  const double nu3i = nuinv * nuinv * nuinv;
  const double A = fma(g, nuinv, ri);
  const double C = ri2 * fma(h, nuinv, ri);
  const double A1 = fma(2.0 * dg, nu3i, -ri3);
  const double C1 = fma(-3.0 * ri3, ri2, ri2 * fma(2.0 * dh, nu3i, -2.0 * h * nuinv * ri2));
  auto dot = [](const double* a, const double* b) { return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2])); };
  const double xwt = dot(x, wt), xfs = dot(x, fs), xft = dot(x, ft), xws = dot(x, ws);
  const double ab = dot(wt, fs) + dot(ft, ws);
  const double sc = fma(A1, ab, C1 * fma(xwt, xfs, xft * xws));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double gm = fma(sc, x[a], C * (fma(wt[a], xfs, fs[a] * xwt) + fma(ft[a], xws, ws[a] * xft)));
    out[a] += fma(A, ws[a], C * xws * x[a]);
    out[3 + a] += gm;
    if (both) {
      out[6 + a] += fma(A, wt[a], C * xwt * x[a]);
      out[9 + a] -= gm;
    }
  }
}

// FF dot product of two FF 3-vectors
__device__ __forceinline__ ff ff_dot3(const ff (&a)[3], const ff (&b)[3]) {
  return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

constexpr int kAdjQueue = 64;   // candidate pairs per round (per warp)
constexpr int kAdjWarps = 4;

template <bool FFP, int NT>
__global__ void __launch_bounds__(32 * kAdjWarps) k_near_adj(const __grid_constant__ NearParams P,
                                                            const __grid_constant__ AdjParams J) {
  constexpr int W = kAdjWarps;
  constexpr int Q = kAdjQueue;
  using R = typename std::conditional<FFP, float2, double>::type;   // queued result type
  __shared__ float4 s_tst[W][4][8];
  // staged sources: FF (position hi / lo, f hi / lo, w hi / lo) or FP64 (f, w)
  __shared__ float4 s_ff[FFP ? W : 1][6][kTile];
  __shared__ double s_d64[FFP ? 1 : W][6][kTile];
  // the tile's targets: FF (position hi / lo, f hi / lo, w hi / lo) or FP64 (f, w)
  __shared__ float4 s_tff[FFP ? W : 1][6][kTile];
  __shared__ double s_t64[FFP ? 1 : W][6][kTile];
  __shared__ uint16_t s_q[W][Q];
  __shared__ R s_r[W][6][Q];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * W + wid;
  if (tile >= P.n_tile) return;
  const int64_t N = P.N;
  const int B = P.tile_leaf[tile];
  const int t0 = P.tile_start[tile], nt = P.tile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<3>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.tile_lo[tile], thi = P.tile_hi[tile];
  const bool on = lane < nt;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 xt = on ? P.rel[t0 + lane] : z4;
  const float tt = on ? fmaf(xt.x, xt.x, fmaf(xt.y, xt.y, xt.z * xt.z)) : __int_as_float(0x7f800000);
  if (FFP) {
    const int k = FFP ? wid : 0;
    s_tff[k][0][lane] = xt;
    s_tff[k][1][lane] = on ? J.rel_lo[t0 + lane] : z4;
    s_tff[k][2][lane] = on ? J.f_hi[t0 + lane] : z4;
    s_tff[k][3][lane] = on ? J.f_lo[t0 + lane] : z4;
    s_tff[k][4][lane] = on ? J.w_hi[t0 + lane] : z4;
    s_tff[k][5][lane] = on ? J.w_lo[t0 + lane] : z4;
  } else {
    const int k = FFP ? 0 : wid;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_t64[k][a][lane] = on ? J.f64[a * N + t0 + lane] : 0.0;
      s_t64[k][3 + a][lane] = on ? J.w64[a * N + t0 + lane] : 0.0;
    }
  }
  float* const rowx = reinterpret_cast<float*>(s_tst[wid][0]);
  float* const rowy = reinterpret_cast<float*>(s_tst[wid][1]);
  float* const rowz = reinterpret_cast<float*>(s_tst[wid][2]);
  float* const roww = reinterpret_cast<float*>(s_tst[wid][3]);
  ff accf[6];
  double accd[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    accf[a] = {0.f, 0.f};
    accd[a] = 0.0;
  }

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<3>(P, e, LB, cB);
    const float nu2 = E.nu2, nuinv = E.nuinv;
    const float nu2inv = nuinv * nuinv;
    const float nu2m = nu2 * (1.f + 0x1p-12f);
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    if (U1 <= tile) continue;                          // every tile of X precedes T
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane) & __ballot_sync(0xffffffffu, Ub + lane >= tile);
         tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      const bool both = U != tile;                     // source side too
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      __syncwarp();
      if (lane < ns) {
        const int64_t si = s0 + lane;
        const float4 r = P.rel[si];
        float px = r.x + E.off[0], py = r.y + E.off[1], pz = r.z + E.off[2];
        if (FFP) {
          const int k = FFP ? wid : 0;
          const float4 rl = J.rel_lo[si];
          const ff sx = two_sum(r.x, E.off[0]), sy = two_sum(r.y, E.off[1]), sz = two_sum(r.z, E.off[2]);
          const ff fx = fast_two_sum(sx.hi, __fadd_rn(sx.lo, rl.x));
          const ff fy = fast_two_sum(sy.hi, __fadd_rn(sy.lo, rl.y));
          const ff fz = fast_two_sum(sz.hi, __fadd_rn(sz.lo, rl.z));
          px = fx.hi, py = fy.hi, pz = fz.hi;
          s_ff[k][0][lane] = make_float4(fx.hi, fy.hi, fz.hi, 0.f);
          s_ff[k][1][lane] = make_float4(fx.lo, fy.lo, fz.lo, 0.f);
          s_ff[k][2][lane] = J.f_hi[si];
          s_ff[k][3][lane] = J.f_lo[si];
          s_ff[k][4][lane] = J.w_hi[si];
          s_ff[k][5][lane] = J.w_lo[si];
        } else {
          const int k = FFP ? 0 : wid;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            s_d64[k][a][lane] = J.f64[a * N + si];
            s_d64[k][3 + a][lane] = J.w64[a * N + si];
          }
        }
        rowx[lane] = -2.f * px;
        rowy[lane] = -2.f * py;
        rowz[lane] = -2.f * pz;
        roww[lane] = fmaf(px, px, fmaf(py, py, pz * pz)) - nu2m;
      } else {
        rowx[lane] = rowy[lane] = rowz[lane] = 0.f;
        roww[lane] = __int_as_float(0x7f800000);      // never a candidate
      }
      __syncwarp();
      const uint32_t bits = candidate_mask(s_tst[wid], xt, tt);
      const int cnt = __popc(bits);
      int off = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off -= cnt;
      for (int base = 0; base < total; base += Q) {
        {
          uint32_t b = bits;
          int i = off;
          for (; b && i < base; ++i) b &= b - 1u;
          for (; b && i < base + Q; ++i) {
            const int j = __ffs(b) - 1;
            b &= b - 1u;
            s_q[wid][i - base] = static_cast<uint16_t>((lane << 5) | j);
          }
        }
        __syncwarp();
        const int n = min(Q, total - base);
        for (int q0 = 0; q0 < n; q0 += 32) {
          const int qi = q0 + lane;
          if (qi >= n) continue;
          const int ent = s_q[wid][qi];
          const int tl = ent >> 5, j = ent & 31;
          double o[12] = {};
          bool done64 = !FFP;
          R res[6];
          if constexpr (FFP) {
            const int k = FFP ? wid : 0;
            const float4 th = s_tff[k][0][tl], tlw = s_tff[k][1][tl];
            const float4 ph = s_ff[k][0][j], pl = s_ff[k][1][j];
            ff dx = two_sum(th.x, -ph.x), dy = two_sum(th.y, -ph.y), dz = two_sum(th.z, -ph.z);
            dx = fast_two_sum(dx.hi, __fadd_rn(dx.lo, __fsub_rn(tlw.x, pl.x)));
            dy = fast_two_sum(dy.hi, __fadd_rn(dy.lo, __fsub_rn(tlw.y, pl.y)));
            dz = fast_two_sum(dz.hi, __fadd_rn(dz.lo, __fsub_rn(tlw.z, pl.z)));
            const ff r2 = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
            for (int a = 0; a < 6; ++a) res[a] = R{};
            const bool close = r2.hi <= nu2 * kCloseFF;
            const bool inside = !close && (r2.hi < nu2 || (r2.hi == nu2 && r2.lo < 0.f)) && (r2.hi > 0.f);
            done64 = close;
            if (inside) {
              const ff rho2 = ff_scale(r2, nu2inv);
              const ff tq = two_sum(__fmul_rn(2.f, rho2.hi), -1.f);
              const ff t = fast_two_sum(tq.hi, __fadd_rn(tq.lo, __fmul_rn(2.f, rho2.lo)));
              const ff ri = ff_rsqrt(r2);
              const ff ri2 = ff_mul(ri, ri);
              const ff ri3 = ff_mul(ri2, ri);
              const ff2 gh = horner_ff2<NT>(J.chi[0], J.clo[0], t);
              const ff2 dgh = horner_ff2<NT>(J.chi[2], J.clo[2], t);
              const float nu3i = nuinv * nuinv * nuinv;
              const ff A = ff_add(ri, ff_scale({gh.hi.x, gh.lo.x}, nuinv));
              const ff C = ff_mul(ri2, ff_add(ri, ff_scale({gh.hi.y, gh.lo.y}, nuinv)));
              const ff A1 = ff_add(ff_scale({dgh.hi.x, dgh.lo.x}, 2.f * nu3i), ff_neg(ri3));
              const ff hnr = ff_mul(ff_scale({gh.hi.y, gh.lo.y}, 2.f * nuinv), ri2);
              const ff C1 = ff_add(ff_mul_f(ff_mul(ri3, ri2), -3.f),
                                   ff_mul(ri2, ff_add(ff_scale({dgh.hi.y, dgh.lo.y}, 2.f * nu3i), ff_neg(hnr))));
              const float4 tfh = s_tff[k][2][tl], tfl = s_tff[k][3][tl], twh = s_tff[k][4][tl], twl = s_tff[k][5][tl];
              const float4 sfh = s_ff[k][2][j], sfl = s_ff[k][3][j], swh = s_ff[k][4][j], swl = s_ff[k][5][j];
              const ff xv[3] = {dx, dy, dz};
              const ff ft[3] = {{tfh.x, tfl.x}, {tfh.y, tfl.y}, {tfh.z, tfl.z}};
              const ff wt[3] = {{twh.x, twl.x}, {twh.y, twl.y}, {twh.z, twl.z}};
              const ff fs[3] = {{sfh.x, sfl.x}, {sfh.y, sfl.y}, {sfh.z, sfl.z}};
              const ff ws[3] = {{swh.x, swl.x}, {swh.y, swl.y}, {swh.z, swl.z}};
              const ff xwt = ff_dot3(xv, wt), xfs = ff_dot3(xv, fs), xft = ff_dot3(xv, ft), xws = ff_dot3(xv, ws);
              const ff ab = ff_add(ff_dot3(wt, fs), ff_dot3(ft, ws));
              const ff sc = ff_add(ff_mul(A1, ab), ff_mul(C1, ff_add(ff_mul(xwt, xfs), ff_mul(xft, xws))));
              const ff Cxws = ff_mul(C, xws), Cxwt = ff_mul(C, xwt);
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                const ff gm = ff_add(ff_mul(sc, xv[a]),
                                     ff_mul(C, ff_add(ff_add(ff_mul(wt[a], xfs), ff_mul(fs[a], xwt)),
                                                      ff_add(ff_mul(ft[a], xws), ff_mul(ws[a], xft)))));
                const ff vt = ff_add(ff_mul(A, ws[a]), ff_mul(Cxws, xv[a]));
                res[a] = make_float2(vt.hi, vt.lo);
                res[3 + a] = make_float2(gm.hi, gm.lo);
                if (both) {
                  const ff vs = ff_add(ff_mul(A, wt[a]), ff_mul(Cxwt, xv[a]));
                  o[6 + a] = ff_to_double(vs);
                  o[9 + a] = -ff_to_double(gm);
                }
              }
              if (both)
#pragma unroll
                for (int a = 0; a < 6; ++a) atomicAdd(J.acc + (static_cast<int64_t>(s0) + j) * 6 + a, o[6 + a]);
            }
          }
          if (done64) {
            // FP64 pair (FP64 plans; nearly coincident pairs of float-float plans)
            double ft[3], wt[3], fs[3], ws[3];
            if (FFP) {
              const int k = FFP ? wid : 0;
              const float4 a0 = s_tff[k][2][tl], a1 = s_tff[k][3][tl], b0 = s_tff[k][4][tl], b1 = s_tff[k][5][tl];
              const float4 c0 = s_ff[k][2][j], c1 = s_ff[k][3][j], d0 = s_ff[k][4][j], d1 = s_ff[k][5][j];
              ft[0] = static_cast<double>(a0.x) + a1.x, ft[1] = static_cast<double>(a0.y) + a1.y,
              ft[2] = static_cast<double>(a0.z) + a1.z;
              wt[0] = static_cast<double>(b0.x) + b1.x, wt[1] = static_cast<double>(b0.y) + b1.y,
              wt[2] = static_cast<double>(b0.z) + b1.z;
              fs[0] = static_cast<double>(c0.x) + c1.x, fs[1] = static_cast<double>(c0.y) + c1.y,
              fs[2] = static_cast<double>(c0.z) + c1.z;
              ws[0] = static_cast<double>(d0.x) + d1.x, ws[1] = static_cast<double>(d0.y) + d1.y,
              ws[2] = static_cast<double>(d0.z) + d1.z;
            } else {
              const int k = FFP ? 0 : wid;
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                ft[a] = s_t64[k][a][tl];
                wt[a] = s_t64[k][3 + a][tl];
                fs[a] = s_d64[k][a][j];
                ws[a] = s_d64[k][3 + a][j];
              }
            }
            adj_pair_fp64<3>(P, t0 + tl, s0 + j, E.q, static_cast<double>(nuinv), ft, wt, fs, ws, both, o);
            if (both)
#pragma unroll
              for (int a = 0; a < 6; ++a) atomicAdd(J.acc + (static_cast<int64_t>(s0) + j) * 6 + a, o[6 + a]);
#pragma unroll
            for (int a = 0; a < 6; ++a) {
              if constexpr (FFP) {
                const float hh = __double2float_rn(o[a]);
                res[a] = make_float2(hh, __double2float_rn(o[a] - static_cast<double>(hh)));
              } else {
                res[a] = o[a];
              }
            }
          }
#pragma unroll
          for (int a = 0; a < 6; ++a) s_r[wid][a][qi] = res[a];
        }
        __syncwarp();
        const int i0 = max(off, base), i1 = min(off + cnt, base + Q);
        for (int i = i0; i < i1; ++i) {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            if constexpr (FFP) {
              const float2 v = s_r[wid][a][i - base];
              accf[a] = ff_add(accf[a], {v.x, v.y});
            } else {
              accd[a] += s_r[wid][a][i - base];
            }
          }
        }
        __syncwarp();
      }
    }
  }
  if (!on) return;
#pragma unroll
  for (int a = 0; a < 6; ++a)
    atomicAdd(J.acc + (static_cast<int64_t>(t0) + lane) * 6 + a, FFP ? ff_to_double(accf[a]) : accd[a]);
}

// v = acc[0, 3) / (8 pi) + self term of w, dL/dx = acc[3, 6) / (8 pi), caller order
template <int D>
__global__ void k_adj_finish(const __grid_constant__ NearParams P, const __grid_constant__ AdjParams J) {
  const int tile = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= P.n_tile || lane >= P.tile_count[tile]) return;
  const int64_t i = P.tile_start[tile] + lane;
  const int64_t o = P.perm[i];
  const double sc = self_coeff<3>(P, P.leaf_level[P.tile_leaf[tile]]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    J.v[o * 3 + a] = J.acc[i * 6 + a] * kInv8Pi + sc * J.w_orig[o * 3 + a];
    J.gx[o * 3 + a] = J.acc[i * 6 + 3 + a] * kInv8Pi;
  }
}

template <bool FFP, int NT>
void run_near_adj(const NearParams& P, const AdjParams& J, cudaStream_t s) {
  k_near_adj<FFP, NT><<<(P.n_tile + kAdjWarps - 1) / kAdjWarps, 32 * kAdjWarps, 0, s>>>(P, J);
  k_adj_finish<3><<<(P.n_tile + 7) / 8, 256, 0, s>>>(P, J);
}

}  // namespace dmk
