// Nearly coincident pairs of the MIXED near-field passes, in FP64.
//
// The FP32 kernels (k_near_sym, k_near_mixed) skip every pair with
// r^2 <= kClose32 nu^2 and the float-float kernel (k_near_ff) every pair with
// r^2 <= kCloseFF nu^2, decided on their own r^2 (FP32, or the hi part of the
// float-float r^2).  Leaf-relative coordinates cannot resolve those pairs
// (their rounding is a relative error ~2^-23 h / r of x in FP32), and they
// carry the largest terms (S_R -> S as r -> 0, App. A.1).  This kernel finds
// them again with the same arithmetic, so every pair goes to exactly one of
// the two kernels, and evaluates them with close_pair_fp64: x = (w_t - w_s) + q
// from the FP64 in-cell coordinates, FP64 pair terms, FP64 densities of the
// caller.
//
// The pair kernels mark the target tiles holding a point of a skipped pair
// (P.close_flag); the symmetric passes (whose sums meet in FP64 atomics
// anyway) also queue every skipped pair (P.close_q, usually a few per thousand
// points) and k_close_queue evaluates the queue, one thread per pair.  The
// one-sided pass (bitwise reproducible), and a symmetric pass whose queue
// overflowed (many coincident points), take k_near_close instead: one warp
// per marked tile, one target per lane, walks the tile's whole near list
// (target side of every ordered pair, as in a one-sided pass), staging only the
// source tiles whose bounding box comes within the close radius (nu/32 or
// nu/1024); unmarked tiles return at once.  Each lane owns its target's
// outputs and adds its pairs in a fixed order, without atomics.
#pragma once
#include "near_ff.cuh"

namespace dmk {

struct CloseParams {
  const float4* rel_lo;   // float-float plans: coordinate residuals (sorted)
  const double* f;        // caller's forces [N][D][n_rhs]
  const double* g;        // caller's stresslet strengths [N][D]
  const double* n;        // caller's orientations [N][D]
  double* acc;            // sorted accumulator (stride values per point), or null: add to P.u (and P.gradu)
  int stride;             // values per point of acc: D, or 12 with the gradient
  float scale;            // kClose32 or kCloseFF
};

// squared gap between the target tile's box and source tile U's box (moved
// into the target leaf's frame), as tile_near forms it
__device__ __forceinline__ float tile_gap2(const NearParams& P, int U, const Entry& E, float4 tlo, float4 thi) {
  const float4 slo = P.tile_lo[U], shi = P.tile_hi[U];
  const float gx = fmaxf(fmaxf(slo.x + E.off[0] - thi.x, tlo.x - (shi.x + E.off[0])), 0.f);
  const float gy = fmaxf(fmaxf(slo.y + E.off[1] - thi.y, tlo.y - (shi.y + E.off[1])), 0.f);
  const float gz = fmaxf(fmaxf(slo.z + E.off[2] - thi.z, tlo.z - (shi.z + E.off[2])), 0.f);
  return gx * gx + gy * gy + gz * gz;
}

constexpr int kCloseWarps = 4;

template <int D, int KM, bool GRAD, bool FFC>
__global__ void __launch_bounds__(32 * kCloseWarps) k_near_close(const __grid_constant__ NearParams P,
                                                                const __grid_constant__ CloseParams C) {
  static_assert(!GRAD || (KM == 1 && D == 3), "the gradient is the 3D Stokeslet's");
  __shared__ float4 s_ph[kCloseWarps][kTile];
  __shared__ float4 s_pl[FFC ? kCloseWarps : 1][kTile];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kCloseWarps + wid;
  if (C.acc && *P.close_count <= P.close_cap) return;   // symmetric pass, queue complete: k_close_queue
  if (tile >= P.n_ttile || !P.close_flag[tile]) return;  // no skipped pair has a point in this tile
  const int B = P.ttile_leaf[tile];
  const int t0 = P.ttile_start[tile], nt = P.ttile_count[tile];
  const int LB = P.leaf_level[B];
  int64_t cB[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[B], LB, P.M, cB);
  const float4 tlo = P.ttile_lo[tile], thi = P.ttile_hi[tile];
  const bool on = lane < nt;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 xt = on ? P.trel[t0 + lane] : z4;
  const float4 xl = (FFC && on) ? C.rel_lo[t0 + lane] : z4;   // float-float plans have no separate targets
  const int64_t it = t0 + lane;
  const int64_t o = on ? P.tperm[it] : 0;
  const int nr = P.n_rhs;

  const int e1 = P.near_off[B + 1];
  for (int e = P.near_off[B]; e < e1; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float thr = E.nu2 * C.scale;
    const float thr_tile = thr * 1.01f;               // box gaps in FP32: a margin far above their rounding
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = __ballot_sync(0xffffffffu, Ub + lane < U1 && tile_gap2(P, Ub + lane, E, tlo, thi) <= thr_tile);
         tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      __syncwarp();
      if (lane < ns) {
        const float4 r = P.rel[s0 + lane];
        if (FFC) {
          float4 ph, pl;
          ff_source_pos(r, C.rel_lo[s0 + lane], E.off, ph, pl);
          s_ph[wid][lane] = ph;
          s_pl[FFC ? wid : 0][lane] = pl;
        } else {
          // the FP32 kernels' staged source position, same expression
          const float sx = r.x + E.off[0], sy = r.y + E.off[1], sz = r.z + E.off[2];
          s_ph[wid][lane] = make_float4(sx, sy, sz, 0.f);
        }
      }
      __syncwarp();
      if (on) {
        for (int j = 0; j < ns; ++j) {
          const int64_t is = s0 + j;
          if (P.same_set && is == it) continue;        // the target itself (its images are never close)
          float r2;
          if (FFC) {
            ff dx, dy, dz;
            r2 = ff_disp_r2<D>(xt, xl, s_ph[wid][j], s_pl[FFC ? wid : 0][j], dx, dy, dz).hi;
          } else {
            const float4 sp = s_ph[wid][j];
            const float dx = xt.x - sp.x, dy = xt.y - sp.y, dz = xt.z - sp.z;
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          }
          if (!(r2 <= thr)) continue;
          const int64_t os = P.perm[is];
          double sd[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
          if (KM & 2) {
            for (int a = 0; a < D; ++a) {
              sd[3 + a] = C.g[os * D + a];
              sd[6 + a] = C.n[os * D + a];
              sd[9] += sd[3 + a] * sd[6 + a];
            }
          }
          for (int k = 0; k < ((KM & 1) ? nr : 1); ++k) {
            if (KM & 1)
              for (int a = 0; a < D; ++a) sd[a] = C.f[(os * D + a) * nr + k];
            double out[kClosePairOut];
            for (int a = 0; a < kClosePairOut; ++a) out[a] = 0.0;
            if (k == 0) close_pair_fp64<D, KM, GRAD>(P, it, is, E.q, static_cast<double>(E.nuinv), sd, sd, false, out);
            else close_pair_fp64<D, 1, false>(P, it, is, E.q, static_cast<double>(E.nuinv), sd, sd, false, out);
            if (C.acc) {
              for (int a = 0; a < D; ++a) C.acc[it * C.stride + a] += out[a];
              if (GRAD)
                for (int m = 0; m < 9; ++m) C.acc[it * C.stride + 3 + m] += out[3 + m];
            } else {
              for (int a = 0; a < D; ++a) P.u[(o * D + a) * nr + k] += out[a] * kInv8Pi;
              if (GRAD)
                for (int m = 0; m < 9; ++m) P.gradu[o * 9 + m] += out[3 + m] * kInv8Pi;
            }
            if (KM & 2)
              for (int a = 3; a < 10; ++a) sd[a] = 0.0;   // the stresslet once, with the first column
          }
        }
      }
    }
  }
}

// The queued pairs of a symmetric pass, one thread each: the FP64 pair, its
// target side and its source side, added atomically to the accumulator (a
// point may be in several pairs).
template <int D, int KM, bool GRAD>
__global__ void __launch_bounds__(128) k_close_queue(const __grid_constant__ NearParams P,
                                                     const __grid_constant__ CloseParams C) {
  const int cnt = *P.close_count;
  if (cnt > P.close_cap) return;                        // overflow: k_near_close takes the marked tiles
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const int4 qe = P.close_q[i];
  const int64_t it = qe.x, is = qe.y;
  const int e = qe.z, LB = qe.w & 255;
  const bool both = (qe.w >> 8) & 1;
  const int X = P.near_leaf[e];
  const int Lmin = min(LB, P.leaf_level[X]);
  const double nuinv = ldexp(1.0, Lmin + 1);
  double q[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < D; ++a) q[a] = static_cast<double>(unpack_q(P.near_q[e], a));
  const int64_t ot = P.perm[it], os = P.perm[is];
  const int nr = P.n_rhs;
  double sd[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double td[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (KM & 2)
    for (int a = 0; a < D; ++a) {
      sd[3 + a] = C.g[os * D + a], sd[6 + a] = C.n[os * D + a], sd[9] += sd[3 + a] * sd[6 + a];
      td[3 + a] = C.g[ot * D + a], td[6 + a] = C.n[ot * D + a], td[9] += td[3 + a] * td[6 + a];
    }
  for (int k = 0; k < ((KM & 1) ? nr : 1); ++k) {
    if (KM & 1)
      for (int a = 0; a < D; ++a) {
        sd[a] = C.f[(os * D + a) * nr + k];
        td[a] = C.f[(ot * D + a) * nr + k];
      }
    double out[kClosePairOut];
    for (int a = 0; a < kClosePairOut; ++a) out[a] = 0.0;
    if (k == 0) close_pair_fp64<D, KM, GRAD>(P, it, is, q, nuinv, sd, td, both, out);
    else close_pair_fp64<D, 1, false>(P, it, is, q, nuinv, sd, td, both, out);
    if (C.acc) {
      for (int a = 0; a < D; ++a) {
        atomicAdd(C.acc + it * C.stride + a, out[a]);
        if (both) atomicAdd(C.acc + is * C.stride + a, out[12 + a]);
      }
      if (GRAD)
        for (int m = 0; m < 9; ++m) {
          atomicAdd(C.acc + it * C.stride + 3 + m, out[3 + m]);
          if (both) atomicAdd(C.acc + is * C.stride + 3 + m, out[15 + m]);
        }
    }
    if (KM & 2)
      for (int a = 3; a < 10; ++a) sd[a] = td[a] = 0.0;   // the stresslet once, with the first column
  }
}

template <int D, int KM, bool GRAD, bool FFC>
void run_near_close(const NearParams& P, const CloseParams& C, cudaStream_t s) {
  if (C.acc) {
    const int cap_blocks = (P.close_cap + 127) / 128;
    k_close_queue<D, KM, GRAD><<<cap_blocks > 0 ? cap_blocks : 1, 128, 0, s>>>(P, C);
  }
  k_near_close<D, KM, GRAD, FFC><<<(P.n_ttile + kCloseWarps - 1) / kCloseWarps, 32 * kCloseWarps, 0, s>>>(P, C);
}

// (dim, kernels, gradient, float-float coordinates)
#define DMK_FOR_EACH_CLOSE(M)                                                              \
  M(3, 1, false, false) M(3, 2, false, false) M(3, 3, false, false) M(2, 1, false, false) \
  M(2, 2, false, false) M(2, 3, false, false) M(3, 1, false, true) M(3, 2, false, true)   \
  M(3, 3, false, true) M(3, 1, true, true) M(2, 1, false, true) M(2, 2, false, true)       \
  M(2, 3, false, true)

}  // namespace dmk
