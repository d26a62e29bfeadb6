// Near-field dispatch, density permutation, the periodic stresslet zero mode
// and the useful-pair count (2D and 3D).
#include "near_adj.cuh"
#include "near_close.cuh"

namespace dmk {

#define DMK_EXT_M(D, KM, GR, NT, NR) \
  extern template void run_near_mixed<D, KM, GR, NT, NR>(const NearParams&, cudaStream_t);
#define DMK_EXT_D(D, KM, GR, NT, NR) \
  extern template void run_near_fp64<D, KM, GR, NT, NR>(const NearParams&, cudaStream_t);
#define DMK_EXT_M_NT(NT) DMK_FOR_EACH_VARIANT_3D(DMK_EXT_M, NT) DMK_FOR_EACH_VARIANT_2D(DMK_EXT_M, NT)
#define DMK_EXT_D_NT(NT) DMK_FOR_EACH_VARIANT_3D_FP64(DMK_EXT_D, NT) DMK_FOR_EACH_VARIANT_2D(DMK_EXT_D, NT)
DMK_NT_MIXED(DMK_EXT_M_NT)
DMK_NT_FP64(DMK_EXT_D_NT)
#define DMK_EXT_F(D, KM, GR, NT) \
  extern template void run_near_ff<D, KM, GR, NT>(const NearParams&, const FFParams&, cudaStream_t);
#define DMK_EXT_F_NT(NT) DMK_FOR_EACH_FF(DMK_EXT_F, NT)
DMK_NT_FP64(DMK_EXT_F_NT)
#define DMK_EXT_A(NT) extern template void run_near_adj<true, NT>(const NearParams&, const AdjParams&, cudaStream_t);
DMK_NT_FP64(DMK_EXT_A)
extern template void run_near_adj<false, 16>(const NearParams&, const AdjParams&, cudaStream_t);
#define DMK_EXT_C(D, KM, GR, FFC) \
  extern template void run_near_close<D, KM, GR, FFC>(const NearParams&, const CloseParams&, cudaStream_t);
DMK_FOR_EACH_CLOSE(DMK_EXT_C)

namespace {

// sorted FP32 copy of a [N][D] FP64 array: out[i] = in[perm[i]] (z = 0 in 2D)
template <int D>
__global__ void k_perm_f32(int64_t N, const int32_t* __restrict__ perm, const double* __restrict__ in,
                           float4* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  float v[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < D; ++a) v[a] = static_cast<float>(in[o * D + a]);
  out[i] = make_float4(v[0], v[1], v[2], 0.f);
}

// sorted orientation vectors with .w = g.n (g.n in FP64, then rounded)
template <int D>
__global__ void k_perm_n32(int64_t N, const int32_t* __restrict__ perm, const double* __restrict__ g,
                           const double* __restrict__ n, float4* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  double gn = 0.0;
  float v[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < D; ++a) {
    gn += g[o * D + a] * n[o * D + a];
    v[a] = static_cast<float>(n[o * D + a]);
  }
  out[i] = make_float4(v[0], v[1], v[2], static_cast<float>(gn));
}

// sorted FP32 force columns: out[k*N + i] = f[perm[i]][:][k] (k < nr; zero up to NR)
template <int D>
__global__ void k_perm_f32_cols(int64_t N, int nr, int NR, const int32_t* __restrict__ perm,
                                const double* __restrict__ f, float4* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  for (int k = 0; k < NR; ++k) {
    float v[3] = {0.f, 0.f, 0.f};
    if (k < nr)
      for (int a = 0; a < D; ++a) v[a] = static_cast<float>(f[(o * D + a) * nr + k]);
    out[k * N + i] = make_float4(v[0], v[1], v[2], 0.f);
  }
}

// sorted FP64 force columns: out[(k*D + a)*N + i] = f[perm[i]][a][k]
template <int D>
__global__ void k_perm_f64_cols(int64_t N, int nr, int NR, const int32_t* __restrict__ perm,
                                const double* __restrict__ f, double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  for (int k = 0; k < NR; ++k)
    for (int a = 0; a < D; ++a) out[(k * D + a) * N + i] = k < nr ? f[(o * D + a) * nr + k] : 0.0;
}

// sorted SoA FP64 copy: out[a*N + i] = in[perm[i]*D + a]
__global__ void k_perm_soa(int64_t N, int D, const int32_t* __restrict__ perm, const double* __restrict__ in,
                           double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  for (int a = 0; a < D; ++a) out[a * N + i] = in[o * D + a];
}

__global__ void k_gn64(int64_t N, int D, const double* __restrict__ g, double* __restrict__ n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int a = 0; a < D; ++a) s += g[a * N + i] * n[a * N + i];
  n[D * N + i] = s;
}

// Periodic stresslet k = 0 term (Sec. 5.3, after Eq. (ewald_far)):
//   u0(x_t) = -sum_s (w_t - w_s)(g_s . n_s) = -( w_t G - W ),
//   G = sum_s g_s.n_s,  W = sum_s w_s (g_s.n_s), per system.
// Points are sorted by system, so a warp almost always holds one system: its
// four partial sums are then reduced by shuffles and added by one lane.
__global__ void k_zero_reduce(int64_t N, int D, const double* __restrict__ w, const double* __restrict__ n64,
                              const int32_t* __restrict__ psys, double* __restrict__ sums) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool on = i < N;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  int sys = -1;
  if (on) {
    sys = psys[i];
    v[0] = n64[D * N + i];
    for (int a = 0; a < D; ++a) v[1 + a] = w[a * N + i] * v[0];
  }
  const int sys0 = __shfl_sync(0xffffffffu, sys, 0);
  const bool uniform = __all_sync(0xffffffffu, !on || sys == sys0);
  if (uniform) {
    for (int k = 0; k < 4; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0 && sys0 >= 0)
      for (int k = 0; k < 1 + D; ++k) atomicAdd(sums + 4 * sys0 + k, v[k]);
  } else if (on) {
    for (int k = 0; k < 1 + D; ++k) atomicAdd(sums + 4 * sys + k, v[k]);
  }
}

// at the targets: N, w, perm are the targets' (the sums are the sources')
// (and its gradient d_m u0_j = -delta_jm G, if gradu is given)
__global__ void k_zero_apply(int64_t N, int D, const double* __restrict__ w, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ psys, const double* __restrict__ sums,
                             double* __restrict__ u, double* __restrict__ gradu) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* s = sums + 4 * (psys ? psys[i] : 0);   // psys null: one system (separate targets)
  int64_t o = perm[i];
  if (u)
    for (int a = 0; a < D; ++a) u[o * D + a] -= w[a * N + i] * s[0] - s[1 + a];
  if (gradu)
    for (int a = 0; a < D; ++a) gradu[o * D * D + a * (D + 1)] -= s[0];
}

// FP32 residual of the leaf-relative coordinates: rel_lo = (w - c) - rel, so
// that rel + rel_lo carries the FP64 offset from the leaf centre c in FF.
// One warp per tile, as the plan's rel is computed.
template <int D>
__global__ void k_rel_lo(const __grid_constant__ NearParams P, float4* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= P.n_tile || lane >= P.tile_count[warp]) return;
  const int leaf = P.tile_leaf[warp];
  const int lev = P.leaf_level[leaf];
  int64_t c[3] = {0, 0, 0};
  leaf_coords<D>(P.leaf_anchor[leaf], lev, P.M, c);
  const double h = ldexp(1.0, -lev);
  const int64_t i = P.tile_start[warp] + lane;
  const float4 r = P.rel[i];
  const float rv[3] = {r.x, r.y, r.z};
  float v[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < D; ++a) {
    const double centre = (static_cast<double>(c[a]) + 0.5) * h;
    v[a] = __double2float_rn((P.w[a * P.N + i] - centre) - static_cast<double>(rv[a]));
  }
  out[i] = make_float4(v[0], v[1], v[2], 0.f);
}

// sorted FF split of a [N][D] FP64 array (hi = rounded value, lo = rounded
// remainder; z = 0 in 2D); with n != nullptr, .w holds the split of g.n (g = in)
template <int D>
__global__ void k_split_ff(int64_t N, const int32_t* __restrict__ perm, const double* __restrict__ in,
                           const double* __restrict__ n, float4* __restrict__ hi, float4* __restrict__ lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t o = perm[i];
  const double* src = n ? n : in;
  float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
  double gn = 0.0;
  for (int a = 0; a < D; ++a) {
    const double v = src[o * D + a];
    h[a] = __double2float_rn(v);
    l[a] = __double2float_rn(v - static_cast<double>(h[a]));
    if (n) gn += in[o * D + a] * n[o * D + a];
  }
  h[3] = __double2float_rn(gn);
  l[3] = __double2float_rn(gn - static_cast<double>(h[3]));
  hi[i] = make_float4(h[0], h[1], h[2], h[3]);
  lo[i] = make_float4(l[0], l[1], l[2], l[3]);
}

// Number of pairs (t, s) with 0 < r2 < nu_ts^2, decided in float64 exactly as
// the FP64 kernel does.  Source tiles are culled by bounding box and single
// sources by an FP32 test with the kernels' margin before the FP64 decision.
template <int D>
__global__ void k_count_useful(const __grid_constant__ NearParams P, unsigned long long* out) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * 4 + wid;                // target tile
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
  double wt[3] = {0.0, 0.0, 0.0};
  if (on)
    for (int a = 0; a < D; ++a) wt[a] = P.tw[a * P.NT + t0 + lane];
  unsigned long long cnt = 0;
  for (int e = P.near_off[B]; e < P.near_off[B + 1]; ++e) {
    const Entry E = make_entry<D>(P, e, LB, cB);
    const float nu2m = E.nu2 * (1.f + 0x1p-12f);
    const double nu2 = static_cast<double>(E.nu2);
    const int U0 = P.leaf_tile0[E.X], U1 = U0 + P.leaf_ntile[E.X];
    for (int Ub = U0; Ub < U1; Ub += 32)
    for (uint32_t tm = near_tile_mask(P, Ub, U1, E, tlo, thi, lane); tm; tm &= tm - 1u) {
      const int U = Ub + __ffs(tm) - 1;
      if (!on) continue;
      const int s0 = P.tile_start[U], ns = P.tile_count[U];
      for (int j = 0; j < ns; ++j) {
        const float4 r = P.rel[s0 + j];
        const float dx = xt.x - (r.x + E.off[0]), dy = xt.y - (r.y + E.off[1]), dz = xt.z - (r.z + E.off[2]);
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= nu2m) continue;
        // (dx*dx + dy*dy) [+ dz*dz], unfused, as in the FP64 kernel
        double r2 = 0.0;
        for (int a = 0; a < D; ++a) {
          const double d = __dadd_rn(__dsub_rn(wt[a], P.w[a * N + s0 + j]), E.q[a]);
          r2 = __dadd_rn(r2, __dmul_rn(d, d));
        }
        if (r2 < nu2 && r2 > 0.0) ++cnt;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0 && cnt) atomicAdd(out, cnt);
}

// MIXED precision evaluates pair terms in FP32 only where that meets the
// requested tolerance: its relative l2 error is set by FP32 rounding of the
// pair terms (about 1e-7 to 2e-6 on clustered points), so below eps = 2e-7 the
// pair terms are taken in FP64 (the FP32 candidate filter is kept).
// There (one force column) the pair terms, and the gradient, are evaluated in
// float-float (k_near_ff), which GB300 runs far faster than FP64; several
// force columns take FP64 pair terms.
bool fp32_pairs(const dmk_stokes_opts_t& o) { return fp32_pair_terms(o); }
bool ff_pairs(const dmk_stokes_opts_t& o) {
  return o.precision == DMK_PRECISION_MIXED && o.eps < kFp32PairMinEps && o.n_rhs == 1;
}

// workspace: [FP32 sorted densities (fp32 pairs)] [FP64 sorted densities]
// [FF split densities] [FP64 accumulator of the symmetric FP64 pass]
// [FP64 accumulator of the symmetric float-float gradient pass, 12 per point]
// [MIXED: count of the skipped nearly coincident pairs, then one mark per tile
// (at most one tile per point)] [MIXED: their queue, close_cap(N) entries]
struct WsLayout {
  size_t f64_off, ff_off, acc_off, accg_off, flag_off, queue_off, bytes;
};
// capacity of the queue of skipped nearly coincident pairs (16 bytes each)
int64_t close_cap(int64_t N) { return std::max<int64_t>(1024, N / 4); }
WsLayout ws_layout(const dmk_stokes_opts_t& o, int64_t N, int64_t NT) {
  const int NR = padded_rhs(o.n_rhs);
  WsLayout L;
  L.f64_off = fp32_pairs(o) ? std::max(3, NR) * N * sizeof(float4) : 0;
  L.ff_off = L.f64_off + std::max(3 + 3 + 4, 3 * NR) * N * sizeof(double);
  L.acc_off = L.ff_off + (ff_pairs(o) ? 7 * N * sizeof(float4) : 0);
  const bool fp64_sym = o.precision == DMK_PRECISION_FP64 && o.n_rhs == 1;
  L.accg_off = L.acc_off + (fp64_sym ? 3 * N * sizeof(double) : 0);
  L.flag_off = L.accg_off + ((ff_pairs(o) && o.dim == 3) ? 12 * N * sizeof(double) : 0);
  const int64_t NP = std::max(N, NT);                 // tiles: at most one per point or target
  L.queue_off = L.flag_off + (o.precision == DMK_PRECISION_MIXED ? ((NP + 2) * sizeof(int) + 15) / 16 * 16 : 0);
  L.bytes = L.queue_off + (o.precision == DMK_PRECISION_MIXED ? close_cap(N) * sizeof(int4) : 0);
  return L;
}

int pick_nt(const int* set, int n, int need) {
  for (int i = 0; i < n; ++i)
    if (set[i] >= need) return set[i];
  return -1;
}

void dispatch(bool mixed, int dim, int km, bool grad, int nt, int nr, const NearParams& P, cudaStream_t s) {
#define DMK_CASE_M(D, KM, GR, NT, NR)                                                  \
  if (mixed && dim == D && km == KM && grad == GR && nt == NT && nr == NR) {           \
    run_near_mixed<D, KM, GR, NT, NR>(P, s);                                           \
    return;                                                                            \
  }
#define DMK_CASE_D(D, KM, GR, NT, NR)                                                  \
  if (!mixed && dim == D && km == KM && grad == GR && nt == NT && nr == NR) {          \
    run_near_fp64<D, KM, GR, NT, NR>(P, s);                                            \
    return;                                                                            \
  }
#define DMK_CASE_M_NT(NT) DMK_FOR_EACH_VARIANT_3D(DMK_CASE_M, NT) DMK_FOR_EACH_VARIANT_2D(DMK_CASE_M, NT)
#define DMK_CASE_D_NT(NT) DMK_FOR_EACH_VARIANT_3D_FP64(DMK_CASE_D, NT) DMK_FOR_EACH_VARIANT_2D(DMK_CASE_D, NT)
  DMK_NT_MIXED(DMK_CASE_M_NT)
  DMK_NT_FP64(DMK_CASE_D_NT)
  throw Error{DMK_ERR_UNSUPPORTED, "no compiled near-field kernel for this configuration"};
}

void dispatch_ff(int dim, int km, bool grad, int nt, const NearParams& P, const FFParams& F, cudaStream_t s) {
#define DMK_CASE_F(D, KM, GR, NT)                                 \
  if (dim == D && km == KM && grad == GR && nt == NT) {           \
    run_near_ff<D, KM, GR, NT>(P, F, s);                          \
    return;                                                       \
  }
#define DMK_CASE_F_NT(NT) DMK_FOR_EACH_FF(DMK_CASE_F, NT)
  DMK_NT_FP64(DMK_CASE_F_NT)
  throw Error{DMK_ERR_UNSUPPORTED, "no compiled float-float kernel for this configuration"};
}

void dispatch_close(int dim, int km, bool grad, bool ffc, const NearParams& P, const CloseParams& C,
                    cudaStream_t s) {
#define DMK_CASE_C(D, KM, GR, FFC)                                        \
  if (dim == D && km == KM && grad == GR && ffc == FFC) {                 \
    run_near_close<D, KM, GR, FFC>(P, C, s);                              \
    return;                                                               \
  }
  DMK_FOR_EACH_CLOSE(DMK_CASE_C)
  throw Error{DMK_ERR_UNSUPPORTED, "no compiled close-pair kernel for this configuration"};
}

// u (caller order) from the sorted accumulator of a symmetric pass
void finish_sym(int dim, int km, bool grad, const NearParams& P, cudaStream_t s) {
  const unsigned g = (P.n_tile + 7) / 8;
  if (grad) k_near_sym_finish_grad<3><<<g, 256, 0, s>>>(P, P.acc);
  else if (dim == 3 && km == 1) k_near_sym_finish<3, 1><<<g, 256, 0, s>>>(P, P.acc);
  else if (dim == 3 && km == 2) k_near_sym_finish<3, 2><<<g, 256, 0, s>>>(P, P.acc);
  else if (dim == 3 && km == 3) k_near_sym_finish<3, 3><<<g, 256, 0, s>>>(P, P.acc);
  else if (dim == 2 && km == 1) k_near_sym_finish<2, 1><<<g, 256, 0, s>>>(P, P.acc);
  else if (dim == 2 && km == 2) k_near_sym_finish<2, 2><<<g, 256, 0, s>>>(P, P.acc);
  else k_near_sym_finish<2, 3><<<g, 256, 0, s>>>(P, P.acc);
}

NearParams tree_params(const Plan& p) {
  const DeviceTree& T = p.tree;
  NearParams P{};
  P.N = T.N;
  P.n_tile = T.n_tile;
  P.M = T.M;
  P.tile_leaf = T.tile_leaf;
  P.tile_start = T.tile_start;
  P.tile_count = T.tile_count;
  P.tile_lo = T.tile_lo;
  P.tile_hi = T.tile_hi;
  P.leaf_anchor = T.leaf_anchor;
  P.leaf_level = T.leaf_level;
  P.leaf_tile0 = T.leaf_tile0;
  P.leaf_ntile = T.leaf_ntile;
  P.near_off = T.near_off;
  P.near_leaf = T.near_leaf;
  P.near_q = T.near_q;
  P.perm = T.perm;
  P.rel = T.rel;
  P.w = T.w;
  // targets of the one-sided passes
  P.same_set = T.sep ? 0 : 1;
  P.n_ttile = T.sep ? T.n_ttile : T.n_tile;
  P.NT = T.sep ? T.NT : T.N;
  P.ttile_leaf = T.sep ? T.ttile_leaf : T.tile_leaf;
  P.ttile_start = T.sep ? T.ttile_start : T.tile_start;
  P.ttile_count = T.sep ? T.ttile_count : T.tile_count;
  P.ttile_lo = T.sep ? T.ttile_lo : T.tile_lo;
  P.ttile_hi = T.sep ? T.ttile_hi : T.tile_hi;
  P.trel = T.sep ? T.trel : T.rel;
  P.tw = T.sep ? T.tw : T.w;
  P.tperm = T.sep ? T.tperm : T.perm;
  return P;
}

// sorted copies of the densities in the workspace
template <int D>
void perm_densities(const Plan& p, bool mixed, bool ff, int km, int nr, int NR, const double* d_f,
                    const double* d_g, const double* d_n, char* ws, NearParams& P, cudaStream_t s) {
  const DeviceTree& T = p.tree;
  const int64_t N = T.N;
  const int B = 256;
  if (mixed) {
    float4* f32 = reinterpret_cast<float4*>(ws);
    float4* g32 = f32 + N;
    float4* n32 = g32 + N;
    if (km & 1) {
      k_perm_f32_cols<D><<<grid_for(N, B), B, 0, s>>>(N, nr, NR, T.perm, d_f, f32);
      ++p.launches;
    }
    if (km & 2) {
      k_perm_f32<D><<<grid_for(N, B), B, 0, s>>>(N, T.perm, d_g, g32);
      ++p.launches;
      k_perm_n32<D><<<grid_for(N, B), B, 0, s>>>(N, T.perm, d_g, d_n, n32);
      ++p.launches;
    }
    P.f32 = f32;
    P.g32 = g32;
    P.n32 = n32;
  }
  double* f64 = reinterpret_cast<double*>(ws + ws_layout(p.opts, N, T.sep ? T.NT : N).f64_off);
  double* g64 = f64 + 3 * N;
  double* n64 = g64 + 3 * N;
  const bool need64 = (!mixed && !ff) || ((km & 2) && p.opts.periodic);
  if (need64) {
    if ((km & 1) && !mixed && !ff) {
      k_perm_f64_cols<D><<<grid_for(N, B), B, 0, s>>>(N, nr, NR, T.perm, d_f, f64);
      ++p.launches;
    }
    if (km & 2) {
      k_perm_soa<<<grid_for(N, B), B, 0, s>>>(N, D, T.perm, d_g, g64);
      ++p.launches;
      k_perm_soa<<<grid_for(N, B), B, 0, s>>>(N, D, T.perm, d_n, n64);
      ++p.launches;
      k_gn64<<<grid_for(N, B), B, 0, s>>>(N, D, g64, n64);
      ++p.launches;
    }
  }
  P.f64 = f64;
  P.g64 = g64;
  P.n64 = n64;
}

// FF inputs: rel_lo and the hi / lo split of the sorted densities
FFParams ff_inputs(const Plan& p, int km, const double* d_f, const double* d_g, const double* d_n, float4* base,
                   const NearParams& P, cudaStream_t s) {
  const DeviceTree& T = p.tree;
  const int64_t N = T.N;
  const int B = 256;
  FFParams F{};
  F.rel_lo = base;
  F.f_hi = base + N;
  F.f_lo = base + 2 * N;
  F.g_hi = base + 3 * N;
  F.g_lo = base + 4 * N;
  F.n_hi = base + 5 * N;
  F.n_lo = base + 6 * N;
  const bool d3 = p.opts.dim == 3;
  const unsigned gt = grid_for(int64_t(T.n_tile) * 32, 256), gp = grid_for(N, B);
  if (T.n_tile > 0) {
    if (d3) k_rel_lo<3><<<gt, 256, 0, s>>>(P, base);
    else k_rel_lo<2><<<gt, 256, 0, s>>>(P, base);
    ++p.launches;
  }
  if (km & 1) {
    if (d3) k_split_ff<3><<<gp, B, 0, s>>>(N, T.perm, d_f, nullptr, base + N, base + 2 * N);
    else k_split_ff<2><<<gp, B, 0, s>>>(N, T.perm, d_f, nullptr, base + N, base + 2 * N);
    ++p.launches;
  }
  if (km & 2) {
    if (d3) {
      k_split_ff<3><<<gp, B, 0, s>>>(N, T.perm, d_g, nullptr, base + 3 * N, base + 4 * N);
      k_split_ff<3><<<gp, B, 0, s>>>(N, T.perm, d_g, d_n, base + 5 * N, base + 6 * N);
    } else {
      k_split_ff<2><<<gp, B, 0, s>>>(N, T.perm, d_g, nullptr, base + 3 * N, base + 4 * N);
      k_split_ff<2><<<gp, B, 0, s>>>(N, T.perm, d_g, d_n, base + 5 * N, base + 6 * N);
    }
    p.launches += 2;
  }
  const KernelTables& tb = p.tables;
  auto c64 = [&](int id, int k) { return k < tb.n64[id] ? tb.p64[id][k] : 0.0; };
  auto hi = [](double v) { return static_cast<float>(v); };
  auto lo = [](double v) { return static_cast<float>(v - static_cast<double>(static_cast<float>(v))); };
  const int pairs[3][2] = {{P_GS, P_HS}, {P_PT, P_QT}, {P_DGS, P_DHS}};
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < kPolyCap; ++k) {
      F.chi[q][k] = make_float2(hi(c64(pairs[q][0], k)), hi(c64(pairs[q][1], k)));
      F.clo[q][k] = make_float2(lo(c64(pairs[q][0], k)), lo(c64(pairs[q][1], k)));
    }
  return F;
}

}  // namespace

void launch_near(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u,
                 double* d_gradu, cudaStream_t s) {
  launch_near_ws(p, d_f, d_g, d_n, d_u, d_gradu, s, p.fsorted, p.reduce_buf, p.aux);
}

// MIXED gradients take float-float pair terms at every eps: the FP32 gradient
// terms (1/r^3) carry a relative l2 error of ~2e-5, above 10 eps at eps = 1e-6.
// A plan with FP32 pair terms then keeps the float-float inputs and the
// accumulator of the gradient pass in a workspace of its own (aux), allocated
// on the first gradient or adjoint call.
bool ff_grad_aux(const dmk_stokes_opts_t& o) { return fp32_pair_terms(o) && o.n_rhs == 1; }

size_t aux_bytes_grad(const dmk_stokes_opts_t& o, int64_t N) {
  return ff_grad_aux(o) ? static_cast<size_t>(N) * (7 * sizeof(float4) + 12 * sizeof(double)) + 512 : 0;
}
size_t aux_bytes_adjoint(const dmk_stokes_opts_t& o, int64_t N) {
  const size_t in = o.precision == DMK_PRECISION_MIXED ? 5 * sizeof(float4) : 6 * sizeof(double);
  return static_cast<size_t>(N) * (in + 6 * sizeof(double)) + 512;
}

void launch_near_ws(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u,
                    double* d_gradu, cudaStream_t s, void* workspace, double* reduce_buf, void* aux) {
  const DeviceTree& T = p.tree;
  const int64_t N = T.N;
  const int D = p.opts.dim;
  const int km = (d_f ? 1 : 0) | (d_g ? 2 : 0);
  const bool grad = d_gradu != nullptr;
  const bool sep = T.sep != 0;                          // separate targets: one-sided passes only
  // the stresslet gradient takes FP64 pair terms in every precision
  const bool grad64 = grad && (km & 2);
  const bool grad_aux = grad && ff_grad_aux(p.opts) && !sep && !grad64;   // float-float gradient of an FP32 plan
  const bool mixed = fp32_pairs(p.opts) && !grad_aux && !(sep && grad) && !grad64;
  // the float-float kernels are symmetric passes; with separate targets MIXED
  // below eps 2e-7 (and its gradient) takes FP64 pair terms
  const bool ff = ((ff_pairs(p.opts) && (d_u || grad)) || grad_aux) && !sep && !grad64;
  if (grad && D != 3) throw Error{DMK_ERR_UNSUPPORTED, "the gradient is provided in 3D"};
  if (grad_aux && !aux) throw Error{DMK_ERR_INVALID_ARG, "gradient workspace missing"};
  if (N == 0) {
    // no sources: separate targets see nothing
    if (sep && T.NT > 0) {
      if (d_u) DMK_CUDA_TRY(cudaMemsetAsync(d_u, 0, sizeof(double) * T.NT * D * p.opts.n_rhs, s));
      if (grad) DMK_CUDA_TRY(cudaMemsetAsync(d_gradu, 0, sizeof(double) * T.NT * 9, s));
    }
    return;
  }
  const int B = 256;
  const int nr = p.opts.n_rhs;
  const int NR = padded_rhs(nr);

  NearParams P = tree_params(p);
  P.f_orig = d_f;
  P.u = d_u;
  P.gradu = d_gradu;
  // 3D: -phi(0)/(2 pi) (times 1/nu_t in the kernel); 2D: -m_d(0)/(8 pi) (plus 2 log(nu_t)/(8 pi))
  P.self_base = (D == 3) ? -p.tables.phi0 / (2.0 * M_PI) : -p.tables.self2d_m0 / (8.0 * M_PI);
  P.n_rhs = nr;

  char* ws = static_cast<char*>(workspace);
  // float-float inputs and the symmetric gradient accumulator: in the plan's
  // workspace for float-float plans, in aux for the gradient of an FP32 plan
  const WsLayout WL = ws_layout(p.opts, N, T.sep ? T.NT : N);
  float4* ffbase = grad_aux ? static_cast<float4*>(aux) : reinterpret_cast<float4*>(ws + WL.ff_off);
  double* accg = grad_aux ? reinterpret_cast<double*>(static_cast<char*>(aux) + 7 * N * sizeof(float4))
                          : reinterpret_cast<double*>(ws + WL.accg_off);
  if (D == 3) perm_densities<3>(p, mixed, ff, km, nr, NR, d_f, d_g, d_n, ws, P, s);
  else perm_densities<2>(p, mixed, ff, km, nr, NR, d_f, d_g, d_n, ws, P, s);
  DMK_CUDA_TRY(cudaGetLastError());

  const KernelTables& tb = p.tables;
  int need = 1;
  const int ids[4] = {(km & 1) ? P_GS : -1, (km & 1) ? P_HS : -1, (km & 2) ? P_PT : -1, (km & 2) ? P_QT : -1};
  for (int id : ids)
    if (id >= 0) need = std::max(need, mixed ? tb.n32[id] : tb.n64[id]);
  if (grad && (km & 1))
    need = std::max(need, std::max(mixed ? tb.n32[P_DGS] : tb.n64[P_DGS], mixed ? tb.n32[P_DHS] : tb.n64[P_DHS]));
  if (grad && (km & 2)) need = std::max(need, std::max(tb.n64[P_DPT], tb.n64[P_DQT]));
  static const int kSetM[] = {8, 10, 12, 13, 14, 16};
  static const int kSetD[] = {16, 20, 24, 28, 32};
  int nt = mixed ? pick_nt(kSetM, 6, need) : pick_nt(kSetD, 5, need);
  if (nt < 0) throw Error{DMK_ERR_UNSUPPORTED, "kernel table longer than the compiled kernels"};
  for (int id = 0; id < P_COUNT; ++id)   // FP64 tables of every path (nearly coincident pairs included)
    if (tb.n64[id] > kPolyCap) throw Error{DMK_ERR_UNSUPPORTED, "FP64 kernel table longer than the kernels hold"};
  for (int id = 0; id < P_COUNT; ++id)
    for (int k = 0; k < kPolyCap; ++k) P.c64[id][k] = k < tb.n64[id] ? tb.p64[id][k] : 0.0;
  auto c32 = [&](int id, int k) { return k < tb.n32[id] ? tb.p32[id][k] : 0.f; };
  for (int k = 0; k < kPolyCap; ++k) {
    P.c32p[0][k] = make_float2(c32(P_GS, k), c32(P_HS, k));
    P.c32p[1][k] = make_float2(c32(P_PT, k), c32(P_QT, k));
    P.c32p[2][k] = make_float2(c32(P_DGS, k), c32(P_DHS, k));
  }
  if (P.n_ttile > 0 && T.n_tile > 0) {
    const bool fp64_sym = !mixed && !ff && NR == 1 && !grad && d_u && !sep;
    if (ff && grad) {
      // symmetric float-float gradient pass: velocity and gradient accumulated
      // both ways, 12 values per point
      P.acc = accg;
      DMK_CUDA_TRY(cudaMemsetAsync(P.acc, 0, sizeof(double) * 12 * N, s));
      ++p.launches;                                   // the finishing kernel
    } else if ((mixed && km == 1 && !grad && NR == 1 && d_u && !sep) || (ff && !grad) || fp64_sym) {
      // symmetric passes (FP32 Stokeslet; float-float and FP64 Stokeslet and
      // stresslet): both points of a pair from one evaluation, summed in a
      // zeroed FP64 accumulator (FP32 / FF: the first 3N doubles of the FP64
      // density region, which these paths leave unused; FP64: its own region)
      const WsLayout L = ws_layout(p.opts, N, T.sep ? T.NT : N);
      P.acc = reinterpret_cast<double*>(ws + (fp64_sym ? L.acc_off : L.f64_off));
      DMK_CUDA_TRY(cudaMemsetAsync(P.acc, 0, sizeof(double) * D * N, s));
      ++p.launches;                                   // the finishing kernel
    }
    const bool sym32 = mixed && km == 1 && !grad && NR == 1 && d_u && !sep;   // k_near_sym (P.acc set above)
    if (ff || mixed) {
      P.close_count = reinterpret_cast<int*>(ws + WL.flag_off);
      P.close_flag = P.close_count + 2;             // [1] unused
      P.close_q = reinterpret_cast<int4*>(ws + WL.queue_off);
      P.close_cap = static_cast<int>(close_cap(N));
      DMK_CUDA_TRY(cudaMemsetAsync(P.close_count, 0, sizeof(int) * (P.n_ttile + 2), s));
    }
    CloseParams C{};
    C.f = d_f;
    C.g = d_g;
    C.n = d_n;
    if (ff) {
      const FFParams F = ff_inputs(p, km, d_f, d_g, d_n, ffbase, P, s);
      dispatch_ff(D, km, grad, nt, P, F, s);
      C.rel_lo = F.rel_lo;
      C.acc = P.acc;
      C.stride = grad ? 12 : D;
      C.scale = kCloseFF;
    } else {
      dispatch(mixed, D, km, grad, nt, NR, P, s);
      C.acc = sym32 ? P.acc : nullptr;
      C.stride = D;
      C.scale = kClose32;
    }
    ++p.launches;
    if (ff || mixed) {
      // nearly coincident pairs in FP64, then the symmetric passes' finish
      dispatch_close(D, km, grad, ff, P, C, s);
      p.launches += 2;
      if (ff || sym32) finish_sym(D, km, grad, P, s);
    }
    DMK_CUDA_TRY(cudaGetLastError());
  }

  if ((km & 2) && p.opts.periodic && (d_u || grad)) {
    DMK_CUDA_TRY(cudaMemsetAsync(reduce_buf, 0, 4 * sizeof(double) * T.n_sys, s));
    k_zero_reduce<<<grid_for(N, B), B, 0, s>>>(N, D, T.w, P.n64, T.point_sys, reduce_buf);
    ++p.launches;
    if (sep) k_zero_apply<<<grid_for(T.NT, B), B, 0, s>>>(T.NT, D, T.tw, T.tperm, nullptr, reduce_buf, d_u, d_gradu);
    else k_zero_apply<<<grid_for(N, B), B, 0, s>>>(N, D, T.w, T.perm, T.point_sys, reduce_buf, d_u, d_gradu);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
  }
}

// Adjoint pass (near_adj.cuh): v = S[w] (dL/df) and dL/dx for the 3D
// Stokeslet, one force column.  MIXED plans: float-float pair terms; FP64
// plans: FP64.  aux holds the sorted inputs and the [N][6] accumulator.
void launch_adjoint(const Plan& p, const double* d_f, const double* d_w, double* d_v, double* d_gx, cudaStream_t s,
                    void* aux) {
  const DeviceTree& T = p.tree;
  const int64_t N = T.N;
  if (N == 0) return;
  if (!aux) throw Error{DMK_ERR_INVALID_ARG, "adjoint workspace missing"};
  const bool ffp = p.opts.precision == DMK_PRECISION_MIXED;
  const int B = 256;
  NearParams P = tree_params(p);
  P.self_base = -p.tables.phi0 / (2.0 * M_PI);
  P.n_rhs = 1;
  const KernelTables& tb = p.tables;
  for (int id = 0; id < P_COUNT; ++id) {
    if (tb.n64[id] > kPolyCap) throw Error{DMK_ERR_UNSUPPORTED, "FP64 kernel table longer than the kernels hold"};
    for (int k = 0; k < kPolyCap; ++k) P.c64[id][k] = k < tb.n64[id] ? tb.p64[id][k] : 0.0;
  }
  AdjParams J{};
  char* base = static_cast<char*>(aux);
  const size_t in_bytes = static_cast<size_t>(N) * (ffp ? 5 * sizeof(float4) : 6 * sizeof(double));
  J.acc = reinterpret_cast<double*>(base + ((in_bytes + 255) & ~size_t(255)));
  J.w_orig = d_w;
  J.v = d_v;
  J.gx = d_gx;
  const unsigned gp = grid_for(N, B);
  if (ffp) {
    float4* b4 = reinterpret_cast<float4*>(base);
    J.rel_lo = b4;
    J.f_hi = b4 + N;
    J.f_lo = b4 + 2 * N;
    J.w_hi = b4 + 3 * N;
    J.w_lo = b4 + 4 * N;
    if (T.n_tile > 0) {
      k_rel_lo<3><<<grid_for(int64_t(T.n_tile) * 32, 256), 256, 0, s>>>(P, b4);
      ++p.launches;
    }
    k_split_ff<3><<<gp, B, 0, s>>>(N, T.perm, d_f, nullptr, b4 + N, b4 + 2 * N);
    k_split_ff<3><<<gp, B, 0, s>>>(N, T.perm, d_w, nullptr, b4 + 3 * N, b4 + 4 * N);
    p.launches += 2;
    auto c64 = [&](int id, int k) { return k < tb.n64[id] ? tb.p64[id][k] : 0.0; };
    auto hi = [](double v) { return static_cast<float>(v); };
    auto lo = [](double v) { return static_cast<float>(v - static_cast<double>(static_cast<float>(v))); };
    const int pairs[3][2] = {{P_GS, P_HS}, {P_PT, P_QT}, {P_DGS, P_DHS}};
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < kPolyCap; ++k) {
        J.chi[q][k] = make_float2(hi(c64(pairs[q][0], k)), hi(c64(pairs[q][1], k)));
        J.clo[q][k] = make_float2(lo(c64(pairs[q][0], k)), lo(c64(pairs[q][1], k)));
      }
  } else {
    double* b8 = reinterpret_cast<double*>(base);
    J.f64 = b8;
    J.w64 = b8 + 3 * N;
    k_perm_soa<<<gp, B, 0, s>>>(N, 3, T.perm, d_f, b8);
    k_perm_soa<<<gp, B, 0, s>>>(N, 3, T.perm, d_w, b8 + 3 * N);
    p.launches += 2;
  }
  DMK_CUDA_TRY(cudaMemsetAsync(J.acc, 0, sizeof(double) * 6 * N, s));
  if (T.n_tile > 0) {
    int need = 1;
    for (int id : {P_GS, P_HS, P_DGS, P_DHS}) need = std::max(need, tb.n64[id]);
    static const int kSetD[] = {16, 20, 24, 28, 32};
    const int nt = pick_nt(kSetD, 5, need);
    if (nt < 0) throw Error{DMK_ERR_UNSUPPORTED, "kernel table longer than the compiled kernels"};
    if (!ffp) {
      run_near_adj<false, 16>(P, J, s);
    } else {
      switch (nt) {
#define DMK_CASE_A(NT) \
  case NT:             \
    run_near_adj<true, NT>(P, J, s); \
    break;
        DMK_NT_FP64(DMK_CASE_A)
        default:
          throw Error{DMK_ERR_UNSUPPORTED, "no compiled adjoint kernel for this table length"};
      }
    }
    p.launches += 2;
  }
  DMK_CUDA_TRY(cudaGetLastError());
}

int64_t count_useful_pairs(const Plan& p) {
  const DeviceTree& T = p.tree;
  const NearParams P = tree_params(p);
  if (T.N == 0 || P.n_ttile == 0) return 0;
  unsigned long long* d = dalloc<unsigned long long>(1, p.stream);
  DMK_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), p.stream));
  if (p.opts.dim == 3) k_count_useful<3><<<(P.n_ttile + 3) / 4, 128, 0, p.stream>>>(P, d);
  else k_count_useful<2><<<(P.n_ttile + 3) / 4, 128, 0, p.stream>>>(P, d);
  ++p.launches;
  DMK_CUDA_TRY(cudaGetLastError());
  unsigned long long h = 0;
  DMK_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, p.stream));
  DMK_CUDA_TRY(cudaStreamSynchronize(p.stream));
  dfree(d, p.stream);
  return static_cast<int64_t>(h);
}

size_t eval_workspace_bytes(const dmk_stokes_opts_t& o, int64_t N, int64_t NT) { return ws_layout(o, N, NT).bytes; }

}  // namespace dmk
