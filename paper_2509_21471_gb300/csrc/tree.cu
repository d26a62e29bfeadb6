// GPU adaptive, level-restricted quad/oct-tree with near lists and tiles.
//
// Sec. 6.1 Step 1: (a) split boxes until a leaf holds at most n_s points;
// (b) level-restrict: leaves that share a boundary point differ by at most one
// level (in the periodic case across the wrap too, Fig. 2 / Sec. 6.2).
// Near list of a leaf = the leaves sharing a boundary point with it (colleague,
// coarse and fine neighbours, itself included), with periodic image offsets q
// (pair displacement (w_t - w_s) + q).  This is the FMM list 1 of the remark
// after Step 4.
//
// Representation: a linear quad/oct-tree.  Points are sorted by Morton key of
// their finest-level cell (M = 21 bits per axis in 3D, 31 in 2D); a leaf is the
// pair (anchor key, level) and owns a contiguous range of sorted points.
// Leaves are kept sorted by (system, anchor), so "the leaf containing cell k"
// is the last leaf whose anchor is <= k (binary search).
//
// Coordinates: w = x - lo; periodic: w -= floor(w); cell = min(floor(w 2^M),
// 2^M - 1) per axis (the top face belongs to the last box).
#include <cub/cub.cuh>

#include <vector>

#include "common.cuh"

namespace dmk {
namespace {

struct LeafArrays {
  uint64_t* anchor = nullptr;
  int32_t* level = nullptr;
  int32_t* start = nullptr;
  int32_t* count = nullptr;
  int32_t* sys = nullptr;
};

// leaf arrays of one refinement step (from the plan's arena: the last step's
// arrays become the tree's)
void alloc_leaves(LeafArrays& L, int64_t n, Arena& A) {
  L.anchor = A.alloc<uint64_t>(n);
  L.level = A.alloc<int32_t>(n);
  L.start = A.alloc<int32_t>(n);
  L.count = A.alloc<int32_t>(n);
  L.sys = A.alloc<int32_t>(n);
}

template <int D>
__device__ inline double in_cell(double x, double lo, int periodic) {
  double w = x - lo;
  if (periodic) w = w - floor(w);
  return w;
}

// FP64 work runs at ~1/74 of the FP32 rate on this part, so the exact steps
// below use integer operations on the bit pattern where they can.
constexpr int64_t kOneBits = 0x3FF0000000000000LL;   // bit pattern of 1.0
// w clamped to [0, 1] (w finite): negative values (sign bit) to 0, above 1 to 1
__device__ inline double clamp01(double w) {
  const int64_t b = __double_as_longlong(w);
  return b < 0 ? 0.0 : (b > kOneBits ? 1.0 : w);
}
// floor(w 2^M) for 0 <= w <= 1, exact (w 2^M is exact in FP64)
__device__ inline int64_t cell_index(double w, int M) {
  const int64_t b = __double_as_longlong(w);
  const int e = static_cast<int>((b >> 52) & 0x7ff);   // biased exponent
  if (e == 0) return 0;                                // zero or subnormal
  const int64_t m = (b & ((int64_t(1) << 52) - 1)) | (int64_t(1) << 52);
  const int sh = 1075 - e - M;                         // 52 - (e - 1023) - M >= 52 - M for w <= 1
  return sh >= 63 ? 0 : (m >> sh);
}

template <int D>
__global__ void k_keys(int64_t N, const double* __restrict__ x, double lo0, double lo1, double lo2,
                       int periodic, int M, uint64_t* __restrict__ key, int32_t* __restrict__ idx,
                       int* __restrict__ status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double lo[3] = {lo0, lo1, lo2};
  const int64_t cmax = (int64_t(1) << M) - 1;
  int64_t c[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    double xa = x[i * D + a];
    if (!isfinite(xa)) {
      atomicOr(status, ST_NONFINITE);
      xa = lo[a];
    }
    double w = in_cell<D>(xa, lo[a], periodic);
    if (!periodic) {
      const int64_t b = __double_as_longlong(w);
      if (b < 0 || b > kOneBits) {                     // w < 0 (or -0) or w > 1
        if (b != static_cast<int64_t>(0x8000000000000000ULL)) atomicOr(status, ST_OUT_OF_RANGE);
        w = clamp01(w);
      }
    }
    const int64_t ci = cell_index(w, M);
    c[a] = ci > cmax ? cmax : ci;
  }
  key[i] = morton<D>(c);
  idx[i] = static_cast<int32_t>(i);
}

template <int D>
__global__ void k_gather_w(int64_t N, const double* __restrict__ x, const int32_t* __restrict__ perm,
                           double lo0, double lo1, double lo2, int periodic, double* __restrict__ w) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double lo[3] = {lo0, lo1, lo2};
  int64_t o = perm[i];
  for (int a = 0; a < D; ++a) {
    double xa = x[o * D + a];
    if (!isfinite(xa)) xa = lo[a];
    double v = in_cell<D>(xa, lo[a], periodic);
    if (!periodic) v = clamp01(v);
    w[a * N + i] = v;
  }
}

__global__ void k_init_roots(int n_sys, const int32_t* __restrict__ offs, LeafArrays L) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sys) return;
  L.anchor[k] = 0;
  L.level[k] = 0;
  L.start[k] = offs[k];
  L.count[k] = offs[k + 1] - offs[k];
  L.sys[k] = k;
}

template <int D>
__global__ void k_split_flags(int n, LeafArrays L, int ns, int M, const int32_t* __restrict__ flag,
                              int32_t* __restrict__ nchild) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool split = flag ? (flag[i] != 0) : (L.count[i] > ns && L.level[i] < M);
  nchild[i] = split ? (1 << D) : 1;
}

__device__ inline int32_t lower_bound_key(const uint64_t* __restrict__ keys, int32_t lo, int32_t hi,
                                          uint64_t k) {
  while (lo < hi) {
    int32_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// child j of leaf i of `in` (j = 0 only if the leaf is not split) written at
// position pos[i] + j of `out`; a child's point range is found by two
// independent binary searches in the leaf's sorted keys
template <int D>
__device__ inline void refine_child(int i, int j, const LeafArrays& in, const int32_t* __restrict__ nchild,
                                    const int32_t* __restrict__ pos, const LeafArrays& out,
                                    const uint64_t* __restrict__ skeys, int M) {
  const int32_t p = pos[i];
  if (nchild[i] == 1) {
    if (j != 0) return;
    out.anchor[p] = in.anchor[i];
    out.level[p] = in.level[i];
    out.start[p] = in.start[i];
    out.count[p] = in.count[i];
    out.sys[p] = in.sys[i];
    return;
  }
  const int lev = in.level[i];
  const int sh = D * (M - lev - 1);
  const uint64_t span = uint64_t(1) << sh;
  const int32_t s0 = in.start[i], s1 = in.start[i] + in.count[i];
  const uint64_t ca = in.anchor[i] + (uint64_t(j) << sh);
  const int32_t b = (j == 0) ? s0 : lower_bound_key(skeys, s0, s1, ca);
  const int32_t e = (j == (1 << D) - 1) ? s1 : lower_bound_key(skeys, s0, s1, ca + span);
  out.anchor[p + j] = ca;
  out.level[p + j] = lev + 1;
  out.start[p + j] = b;
  out.count[p + j] = e - b;
  out.sys[p + j] = in.sys[i];
}

// one thread per (leaf, child)
template <int D>
__global__ void k_refine(int n, LeafArrays in, const int32_t* __restrict__ nchild,
                         const int32_t* __restrict__ pos, LeafArrays out,
                         const uint64_t* __restrict__ skeys, int M) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int i = static_cast<int>(t >> D), j = static_cast<int>(t & ((1 << D) - 1));
  if (i >= n) return;
  refine_child<D>(i, j, in, nchild, pos, out, skeys, M);
}

// The same two steps with the leaf count in device memory, so that levels are
// chained without a host round trip: arrays have a capacity cap >= count,
// slots beyond the count get no children, and the last leaf writes the next
// level's count.
template <int D>
__global__ void k_split_flags_dev(int cap, const int32_t* __restrict__ d_n, LeafArrays L, int ns, int M,
                                  int32_t* __restrict__ nchild) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const int n = min(*d_n, cap);
  nchild[i] = (i < n) ? ((L.count[i] > ns && L.level[i] < M) ? (1 << D) : 1) : 0;
}

template <int D>
__global__ void k_refine_dev(int cap, int cap_out, const int32_t* __restrict__ d_n, LeafArrays in,
                             const int32_t* __restrict__ nchild, const int32_t* __restrict__ pos,
                             LeafArrays out, const uint64_t* __restrict__ skeys, int M,
                             int32_t* __restrict__ d_n_out, int* __restrict__ status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int i = static_cast<int>(t >> D), j = static_cast<int>(t & ((1 << D) - 1));
  if (i >= cap) return;
  const int n = min(*d_n, cap);
  if (i >= n) return;
  if (pos[i] + nchild[i] > cap_out) {          // cannot happen by the capacity bound; guarded anyway
    if (j == 0) atomicOr(status, ST_TREE_INCONSISTENT);
    if (i == n - 1 && j == 0) *d_n_out = min(pos[i], cap_out);
    return;
  }
  if (i == n - 1 && j == 0) *d_n_out = pos[i] + nchild[i];
  refine_child<D>(i, j, in, nchild, pos, out, skeys, M);
}

// total of an exclusive scan: out[n] = out[n - 1] + in[n - 1] (and *copy if given)
__global__ void k_scan_total(int n, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                             int32_t* __restrict__ copy) {
  const int32_t v = out[n - 1] + in[n - 1];
  out[n] = v;
  if (copy) *copy = v;
}


// first leaf of every system; also clears flag[0, n) and *any when given
__global__ void k_sys_begin(int n, int n_sys, const int32_t* __restrict__ sys, int32_t* __restrict__ begin,
                            int32_t* __restrict__ flag = nullptr, int* __restrict__ any = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i == 0 || sys[i] != sys[i - 1]) begin[sys[i]] = i;
  if (i == n - 1) begin[n_sys] = n;
  if (flag) flag[i] = 0;
  if (any && i == 0) *any = 0;
}

// last leaf in [b, e) with anchor <= key
__device__ inline int32_t find_leaf(const uint64_t* __restrict__ anchor, int32_t b, int32_t e, uint64_t key) {
  int32_t lo = b, hi = e;   // first index with anchor > key
  while (lo < hi) {
    int32_t mid = lo + ((hi - lo) >> 1);
    if (anchor[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

template <int D>
__device__ inline bool neighbour(const int64_t* c, const int* dl, int lev, int periodic, int64_t* nb, int* q) {
  const int64_t n = int64_t(1) << lev;
  for (int a = 0; a < D; ++a) {
    int64_t v = c[a] + dl[a];
    q[a] = 0;
    if (v < 0 || v >= n) {
      if (!periodic) return false;
      if (v < 0) { v += n; q[a] = 1; }        // image shifted by -1: q = +1
      else { v -= n; q[a] = -1; }
    }
    nb[a] = v;
  }
  return true;
}

// Level restriction check, one warp per leaf and one lane per neighbour
// direction: a touching leaf more than one level coarser is flagged for a split.
template <int D>
__global__ void k_balance(int n, LeafArrays L, const int32_t* __restrict__ begin, int M, int periodic,
                          int32_t* __restrict__ flag, int* __restrict__ any) {
  const int i = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int k = threadIdx.x & 31;
  const int ndir = (D == 3) ? 27 : 9;
  if (i >= n || k >= ndir) return;
  const int lev = L.level[i];
  if (lev < 2) return;
  int dl[3] = {k % 3 - 1, (k / 3) % 3 - 1, D == 3 ? (k / 9) % 3 - 1 : 0};
  if (dl[0] == 0 && dl[1] == 0 && dl[2] == 0) return;
  int64_t c[3];
  leaf_coords<D>(L.anchor[i], lev, M, c);
  int64_t nb[3];
  int q[3];
  if (!neighbour<D>(c, dl, lev, periodic, nb, q)) return;
  const int32_t b = begin[L.sys[i]], e = begin[L.sys[i] + 1];
  const int32_t X = find_leaf(L.anchor, b, e, box_anchor<D>(nb, lev, M));
  if (L.level[X] < lev - 1) {
    flag[X] = 1;
    *any = 1;
  }
}

// Near lists, one warp per leaf and one lane per neighbour direction (the
// centre direction is the leaf itself).  Each lane finds the leaves touching
// its neighbour box (one at the same or a coarser level, or the up to 4 finer
// children adjacent to the leaf); entries already found in an earlier
// direction are dropped, so the list is that of a sequential walk over the
// directions in order.  Entries go to a fixed-stride scratch (kMaxNear per
// leaf) and are compacted after the scan of the counts.
template <int D>
__global__ void __launch_bounds__(256) k_near_warp(int n, LeafArrays L, const int32_t* __restrict__ begin,
                                                   int M, int periodic, int32_t* __restrict__ sl,
                                                   int32_t* __restrict__ sq, int32_t* __restrict__ cnt_out,
                                                   int* status) {
  __shared__ int32_t s_leaf[8][32][4];
  __shared__ int32_t s_nc[8][32];
  __shared__ int32_t s_q[8][32];
  const int wid = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int i = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= n) return;                                  // whole warps leave together
  const int ndir = (D == 3) ? 27 : 9;
  const int lev = L.level[i];
  int64_t c[3];
  leaf_coords<D>(L.anchor[i], lev, M, c);
  const int32_t b = begin[L.sys[i]], e = begin[L.sys[i] + 1];
  int nc = 0;
  int32_t qp = 0;
  int32_t cand[4] = {-1, -1, -1, -1};
  if (k < ndir) {
    int dl[3] = {k % 3 - 1, (k / 3) % 3 - 1, D == 3 ? (k / 9) % 3 - 1 : 0};
    int64_t nb[3];
    int q[3];
    if (neighbour<D>(c, dl, lev, periodic, nb, q)) {
      qp = pack_q(q[0], q[1], D == 3 ? q[2] : 0);
      const int32_t X = find_leaf(L.anchor, b, e, box_anchor<D>(nb, lev, M));
      if (L.level[X] <= lev) {
        cand[nc++] = X;
      } else {
        for (int j = 0; j < (1 << D); ++j) {
          const int o[3] = {j & 1, (j >> 1) & 1, (j >> 2) & 1};
          bool ok = true;
          for (int a = 0; a < D; ++a) {
            if (dl[a] == 1 && o[a] != 0) ok = false;
            if (dl[a] == -1 && o[a] != 1) ok = false;
          }
          if (!ok) continue;
          int64_t ch[3];
          for (int a = 0; a < D; ++a) ch[a] = 2 * nb[a] + o[a];
          const uint64_t ca = box_anchor<D>(ch, lev + 1, M);
          const int32_t Y = find_leaf(L.anchor, b, e, ca);
          if (L.level[Y] != lev + 1 || L.anchor[Y] != ca) {
            atomicOr(status, ST_TREE_INCONSISTENT);
            continue;
          }
          if (nc < 4) cand[nc++] = Y;
        }
      }
    }
  }
  s_nc[wid][k] = nc;
  s_q[wid][k] = qp;
#pragma unroll
  for (int m = 0; m < 4; ++m) s_leaf[wid][k][m] = cand[m];
  __syncwarp();
  // keep the candidates not found in an earlier direction
  uint32_t keep = 0u;
  for (int m = 0; m < nc; ++m) {
    bool dup = false;
    for (int d2 = 0; d2 < k && !dup; ++d2) {
      if (s_q[wid][d2] != qp) continue;
      for (int m2 = 0; m2 < s_nc[wid][d2]; ++m2)
        if (s_leaf[wid][d2][m2] == cand[m]) dup = true;
    }
    if (!dup) keep |= 1u << m;
  }
  const int kept = __popc(keep);
  int off = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, off, o);
    if (k >= o) off += v;
  }
  const int total = __shfl_sync(0xffffffffu, off, 31);
  off -= kept;
  for (int m = 0; m < nc; ++m) {
    if (!(keep & (1u << m))) continue;
    if (off < kMaxNear) {
      sl[static_cast<int64_t>(i) * kMaxNear + off] = cand[m];
      sq[static_cast<int64_t>(i) * kMaxNear + off] = qp;
    }
    ++off;
  }
  if (k == 0) {
    if (total > kMaxNear) atomicOr(status, ST_NEAR_OVERFLOW);
    cnt_out[i] = min(total, kMaxNear);
  }
}

// scratch lists (kMaxNear stride) -> CSR, one warp per leaf
__global__ void k_near_compact(int n, const int32_t* __restrict__ cnt, const int32_t* __restrict__ off,
                               const int32_t* __restrict__ sl, const int32_t* __restrict__ sq,
                               int32_t* __restrict__ nl, int32_t* __restrict__ nq) {
  const int i = static_cast<int>((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int k = threadIdx.x & 31;
  if (i >= n) return;
  const int c = cnt[i], o = off[i];
  for (int r = k; r < c; r += 32) {
    nl[o + r] = sl[static_cast<int64_t>(i) * kMaxNear + r];
    nq[o + r] = sq[static_cast<int64_t>(i) * kMaxNear + r];
  }
}

__global__ void k_tile_count(int n, const int32_t* __restrict__ count, int32_t* __restrict__ ntile) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ntile[i] = (count[i] + kTile - 1) / kTile;
}

__global__ void k_tile_fill(int n, const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                            const int32_t* __restrict__ tile0, int32_t* __restrict__ tleaf,
                            int32_t* __restrict__ tstart, int32_t* __restrict__ tcount) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int nt = (count[i] + kTile - 1) / kTile;
  for (int k = 0; k < nt; ++k) {
    int t = tile0[i] + k;
    tleaf[t] = i;
    tstart[t] = start[i] + k * kTile;
    tcount[t] = min(kTile, count[i] - k * kTile);
  }
}

// one warp per tile (tiles below the device count *d_ntile, the grid covers a
// capacity): leaf-relative FP32 coordinates and the tile bounding box
template <int D>
__global__ void k_rel_bbox(const int32_t* __restrict__ d_ntile, int64_t N, const int32_t* __restrict__ tleaf,
                           const int32_t* __restrict__ tstart, const int32_t* __restrict__ tcount,
                           const uint64_t* __restrict__ anchor, const int32_t* __restrict__ level,
                           const double* __restrict__ w, int M, float4* __restrict__ rel,
                           float4* __restrict__ tlo, float4* __restrict__ thi) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= *d_ntile) return;
  int leaf = tleaf[warp];
  int lev = level[leaf];
  int64_t c[3] = {0, 0, 0};
  leaf_coords<D>(anchor[leaf], lev, M, c);
  float v[3] = {0.f, 0.f, 0.f};
  bool on = lane < tcount[warp];
  if (on) {
    int64_t p = tstart[warp] + lane;
    for (int a = 0; a < D; ++a) {
      // centre (c + 1/2) 2^-lev = (2c + 1) 2^-(lev+1): exact, scaled in the exponent bits
      const double centre = __longlong_as_double(__double_as_longlong(static_cast<double>(2 * c[a] + 1)) -
                                                  (static_cast<int64_t>(lev + 1) << 52));
      v[a] = __double2float_rn(w[a * N + p] - centre);
    }
    rel[p] = make_float4(v[0], v[1], v[2], 0.f);
  }
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = on ? v[a] : 3.0e38f;
    hi[a] = on ? v[a] : -3.0e38f;
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if (lane == 0) {
    tlo[warp] = make_float4(lo[0], lo[1], lo[2], 0.f);
    thi[warp] = make_float4(hi[0], hi[1], hi[2], 0.f);
  }
}

__global__ void k_set_value(int32_t* dst, int32_t v) { *dst = v; }

__global__ void k_point_sys(int n_sys, const int32_t* __restrict__ offs, int32_t* __restrict__ ps) {
  int k = blockIdx.y;
  int64_t i = offs[k] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n_sys && i < offs[k + 1]) ps[i] = k;
}

// ------------------------------------------------ point order inside leaves
// The points of a leaf are tiled 32 at a time in sorted order, and the tiles'
// bounding boxes decide which tile pairs the near field stages.  The Morton
// order jumps between distant sub-cells, so inside every leaf the sub-cells
// kHilbertLevels levels below the leaf are put in Hilbert-curve order (points
// keep their Morton order inside a sub-cell): consecutive sub-cells are then
// face neighbours and the tiles more compact (on GB300: FP32 near field 5 %
// and the 16-column kernel 6.5 % faster).  Leaves deeper than
// M - kHilbertLevels keep the Morton order.  Only plans with FP32 pair terms
// take this order: the float-float passes measured 3 % slower with it (more
// of their per-pair source-side atomics then meet on one source, the likely
// cause).
template <int D> constexpr int kHilbertLevels = (D == 3) ? 3 : 4;

// Index of cell c (b bits per axis) along the Hilbert curve, after J.
// Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707 (2004):
// the axes are turned into the transposed index (inverse undo, then Gray
// encoding) and its bits interleaved, axis 0 most significant at each level.
template <int D>
__host__ __device__ inline uint32_t hilbert_index(int b, const uint32_t* c) {
  uint32_t X[3] = {c[0], c[1], D == 3 ? c[2] : 0u};
  const uint32_t top = 1u << (b - 1);
  for (uint32_t Q = top; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    for (int i = 0; i < D; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;                                   // invert the low bits of axis 0
      } else {
        const uint32_t t = (X[0] ^ X[i]) & P;        // exchange the low bits of axes 0 and i
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < D; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = top; Q > 1; Q >>= 1)
    if (X[D - 1] & Q) t ^= Q - 1;
  for (int i = 0; i < D; ++i) X[i] ^= t;
  uint32_t h = 0;
  for (int j = b - 1; j >= 0; --j)
    for (int i = 0; i < D; ++i) h = (h << 1) | ((X[i] >> j) & 1u);
  return h;
}

// one block per leaf: Morton-ordered perm and w (in) -> leaf-local Hilbert
// order of the sub-cells (out); a stable counting sort by sub-cell rank
template <int D>
__global__ void __launch_bounds__(256) k_leaf_hilbert(int n_leaf, LeafArrays L, int M, int64_t N, int reorder,
                                                      const uint64_t* __restrict__ skeys,
                                                      const int32_t* __restrict__ perm_in,
                                                      const double* __restrict__ w_in,
                                                      int32_t* __restrict__ perm_out, double* __restrict__ w_out) {
  constexpr int HB = kHilbertLevels<D>;
  constexpr int NB = 1 << (D * HB);                  // sub-cells per leaf: 512 (3D), 256 (2D)
  __shared__ int cnt[NB], first[NB], hfirst[NB];     // counts; first slot in Morton / in Hilbert order
  __shared__ uint16_t rank[NB];                      // Hilbert rank of the sub-cell with Morton index m
  const int leaf = blockIdx.x;
  if (leaf >= n_leaf) return;
  const int s0 = L.start[leaf], c = L.count[leaf], lev = L.level[leaf];
  const int t = threadIdx.x;
  if (!reorder || lev + HB > M || c < 2) {
    for (int k = t; k < c; k += blockDim.x) {
      perm_out[s0 + k] = perm_in[s0 + k];
#pragma unroll
      for (int a = 0; a < D; ++a) w_out[a * N + s0 + k] = w_in[a * N + s0 + k];
    }
    return;
  }
  const int sh = D * (M - lev - HB);
  for (int m = t; m < NB; m += blockDim.x) {
    int64_t cm[3] = {0, 0, 0};
    demorton<D>(static_cast<uint64_t>(m), cm);
    const uint32_t cu[3] = {static_cast<uint32_t>(cm[0]), static_cast<uint32_t>(cm[1]),
                            static_cast<uint32_t>(cm[2])};
    rank[m] = static_cast<uint16_t>(hilbert_index<D>(HB, cu));
    cnt[m] = 0;
  }
  __syncthreads();
  for (int k = t; k < c; k += blockDim.x) atomicAdd(&cnt[(skeys[s0 + k] >> sh) & (NB - 1)], 1);
  __syncthreads();
  for (int m = t; m < NB; m += blockDim.x) hfirst[rank[m]] = cnt[m];
  __syncthreads();
  if (t < 32) {                                      // both exclusive scans by one warp
    constexpr int PER = NB / 32;
    int a[PER], h[PER], sa = 0, sh2 = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      a[q] = sa;
      sa += cnt[t * PER + q];
      h[q] = sh2;
      sh2 += hfirst[t * PER + q];
    }
    int xa = sa, xh = sh2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ya = __shfl_up_sync(0xffffffffu, xa, o), yh = __shfl_up_sync(0xffffffffu, xh, o);
      if (t >= o) {
        xa += ya;
        xh += yh;
      }
    }
    xa -= sa;
    xh -= sh2;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      first[t * PER + q] = xa + a[q];
      hfirst[t * PER + q] = xh + h[q];
    }
  }
  __syncthreads();
  for (int k = t; k < c; k += blockDim.x) {
    const int m = static_cast<int>((skeys[s0 + k] >> sh) & (NB - 1));
    const int dst = s0 + hfirst[rank[m]] + (k - first[m]);
    perm_out[dst] = perm_in[s0 + k];
#pragma unroll
    for (int a = 0; a < D; ++a) w_out[a * N + dst] = w_in[a * N + s0 + k];
  }
}

// Exclusive scan of n counts by one block (n <= kSmallScan): out[i] for i < n,
// the total in out[n] (and in *copy when given).  One launch where the library
// scan takes three for the small arrays of the tree build.  Each warp scans a
// contiguous segment 32 elements at a time (coalesced); a first pass forms the
// counts (kept in out[] and, if side is given, in side[]) and the warp totals,
// a second pass writes the prefix sums.  The counts come from a functor, so
// that the split flags of a refinement level are formed in the same launch.
constexpr int kSmallScan = 1024 * 64;
struct CountsIn {                                    // plain counts
  const int32_t* in;
  __device__ int32_t operator()(int i) const { return in[i]; }
};
template <int D>
struct SplitCounts {                                 // children of leaf i: 2^D if split, else 1
  LeafArrays L;
  int ns, M;
  const int32_t* flag;                               // level restriction flags, or null
  const int32_t* d_n;                                // chained level: leaf count (slots beyond get 0)
  __device__ int32_t operator()(int i) const {
    if (d_n && i >= *d_n) return 0;
    const bool split = flag ? (flag[i] != 0) : (L.count[i] > ns && L.level[i] < M);
    return split ? (1 << D) : 1;
  }
};
template <class F>
__global__ void __launch_bounds__(1024) k_scan_small(int n, F f, int32_t* __restrict__ side,
                                                     int32_t* __restrict__ out, int32_t* __restrict__ copy) {
  __shared__ int32_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int seg = (((n + 31) >> 5) + 31) & ~31;      // elements per warp, a multiple of 32
  const int b = min(w * seg, n), e = min(b + seg, n);
  int32_t sum = 0;
  for (int i = b + lane; i < e; i += 32) {
    const int32_t v = f(i);
    out[i] = v;
    if (side) side[i] = v;
    sum += v;
  }
  sum = static_cast<int32_t>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(sum)));
  if (lane == 0) wsum[w] = sum;
  __syncthreads();
  if (w == 0) {
    int32_t x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x;                                  // inclusive over warps
  }
  __syncthreads();
  int32_t run = w > 0 ? wsum[w - 1] : 0;
  for (int i0 = b; i0 < e; i0 += 32) {
    const int i = i0 + lane;
    const int32_t v = i < e ? out[i] : 0;            // this lane's own count from the first pass
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (i < e) out[i] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (t == 0) {
    out[n] = wsum[31];
    if (copy) *copy = wsum[31];
  }
}

// exclusive scan of n counts into out[0, n] (out[n] = total, also to *copy)
void scan_counts(const int32_t* in, int32_t* out, int n, cudaStream_t s, Arena& scratch, int32_t* copy,
                 int64_t& launches) {
  if (n <= kSmallScan) {
    k_scan_small<<<1, 1024, 0, s>>>(n, CountsIn{in}, nullptr, out, copy);
    ++launches;
  } else {
    size_t bytes = 0;
    DMK_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, s));
    DMK_CUDA_TRY(cub::DeviceScan::ExclusiveSum(scratch.alloc_bytes(bytes), bytes, in, out, n, s));
    k_scan_total<<<1, 1, 0, s>>>(n, in, out, copy);
    ++launches;
  }
  DMK_CUDA_TRY(cudaGetLastError());
}

// children per leaf (nchild, n entries) and their exclusive scan (pos, n + 1
// entries): one launch for the small arrays, the flags kernel and the library
// scan otherwise
template <int D>
void split_and_scan(const SplitCounts<D>& f, int n, int32_t* nchild, int32_t* pos, cudaStream_t s,
                    Arena& scratch, int64_t& launches) {
  if (n <= kSmallScan) {
    k_scan_small<<<1, 1024, 0, s>>>(n, f, nchild, pos, nullptr);
    ++launches;
    DMK_CUDA_TRY(cudaGetLastError());
    return;
  }
  if (f.d_n) k_split_flags_dev<D><<<grid_for(n, 256), 256, 0, s>>>(n, f.d_n, f.L, f.ns, f.M, nchild);
  else k_split_flags<D><<<grid_for(n, 256), 256, 0, s>>>(n, f.L, f.ns, f.M, f.flag, nchild);
  ++launches;
  DMK_CUDA_TRY(cudaGetLastError());
  scan_counts(nchild, pos, n, s, scratch, nullptr, launches);
}

template <int D>
void build_tree_t(Plan& p, const double* d_src, const int64_t* h_offsets) {
  DeviceTree& T = p.tree;
  cudaStream_t s = p.stream;
  const int M = MaxLevel<D>::value;
  T.dim = D;
  T.M = M;
  T.periodic = p.opts.periodic;
  const int64_t N = T.N;
  const int n_sys = T.n_sys;
  const int B = 256;
  const double lo0 = p.opts.box_lo[0], lo1 = p.opts.box_lo[1], lo2 = D == 3 ? p.opts.box_lo[2] : 0.0;

  int32_t* h_pin = pinned_slot();
  struct PinGuard { int32_t* q; ~PinGuard() { pinned_release(q); } } pin_guard{h_pin};
  Arena& A = p.arena;                  // the tree's arrays
  Arena scratch;                       // released when the build returns
  scratch.s = s;
  scratch.reserve(static_cast<size_t>(N) * (48 + 4 + 8 * D) + (size_t(4) << 20));

  // system offsets on the device
  std::vector<int32_t> offs32(n_sys + 1);
  for (int k = 0; k <= n_sys; ++k) offs32[k] = static_cast<int32_t>(h_offsets[k]);
  int32_t* d_offs = scratch.alloc<int32_t>(n_sys + 1);
  DMK_CUDA_TRY(cudaMemcpyAsync(d_offs, offs32.data(), (n_sys + 1) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));

  // ---- keys and sort -------------------------------------------------------
  uint64_t* key_in = scratch.alloc<uint64_t>(N);
  uint64_t* skeys = scratch.alloc<uint64_t>(N);
  int32_t* idx_in = scratch.alloc<int32_t>(N);
  int32_t* perm_m = scratch.alloc<int32_t>(N);       // Morton order; the plan keeps the leaf-Hilbert order
  double* w_m = scratch.alloc<double>(N * D);
  if (N > 0) {
    k_keys<D><<<grid_for(N, B), B, 0, s>>>(N, d_src, lo0, lo1, lo2, T.periodic, M, key_in, idx_in, p.status);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
    size_t bytes = 0;
    if (n_sys == 1) {
      DMK_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, bytes, key_in, skeys, idx_in, perm_m,
                                                   static_cast<int>(N), 0, D * M, s));
      void* tmp = scratch.alloc_bytes(bytes);
      DMK_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, bytes, key_in, skeys, idx_in, perm_m,
                                                   static_cast<int>(N), 0, D * M, s));
    } else {
      DMK_CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(
          nullptr, bytes, key_in, skeys, idx_in, perm_m, static_cast<int>(N), n_sys, d_offs, d_offs + 1,
          0, D * M, s));
      void* tmp = scratch.alloc_bytes(bytes);
      DMK_CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(
          tmp, bytes, key_in, skeys, idx_in, perm_m, static_cast<int>(N), n_sys, d_offs, d_offs + 1,
          0, D * M, s));
    }
  }
  if (N > 0) {
    k_gather_w<D><<<grid_for(N, B), B, 0, s>>>(N, d_src, perm_m, lo0, lo1, lo2, T.periodic, w_m);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
  }
  T.point_sys = A.alloc<int32_t>(N);
  if (N > 0) {
    int64_t maxn = 0;
    for (int k = 0; k < n_sys; ++k) maxn = std::max<int64_t>(maxn, h_offsets[k + 1] - h_offsets[k]);
    dim3 g(grid_for(std::max<int64_t>(maxn, 1), B), n_sys);
    k_point_sys<<<g, B, 0, s>>>(n_sys, d_offs, T.point_sys);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
  }

  // ---- (a) adaptive refinement -------------------------------------------
  // Levels are chained on the device (leaf counts in device memory, arrays
  // sized by a capacity) and the host reads the count every kChain levels.
  // Capacity: a split leaf holds more than n_s points, so at most
  // N / (n_s + 1) leaves split per level, each adding 2^D - 1 leaves.
  constexpr int kChain = 4;
  LeafArrays cur, nxt;
  alloc_leaves(cur, n_sys, A);
  k_init_roots<<<grid_for(n_sys, B), B, 0, s>>>(n_sys, d_offs, cur);
  ++p.launches;
  DMK_CUDA_TRY(cudaGetLastError());
  int32_t* begin = A.alloc<int32_t>(n_sys + 1);
  int32_t* d_cnt = scratch.alloc<int32_t>(M + 2);          // leaf count after each level
  k_set_value<<<1, 1, 0, s>>>(d_cnt, n_sys);
  ++p.launches;
  // a uniform tree (single-level Ewald split) splits every box down to its level
  const bool uniform = p.uniform_level > 0;
  const int ns_split = uniform ? -1 : p.leaf_capacity;
  const int lmax_split = uniform ? p.uniform_level : M;
  const int64_t grow = uniform ? ((int64_t(1) << D) - 1) * (int64_t(1) << (D * p.uniform_level))
                               : ((int64_t(1) << D) - 1) * (N / (int64_t(p.leaf_capacity) + 1) + 1);
  int64_t cap = n_sys;
  int64_t n_leaf = n_sys;
  for (int lev = 0; lev <= M;) {
    for (int k = 0; k < kChain && lev <= M; ++k, ++lev) {
      const int64_t cap_out = cap + grow;
      if (cap_out >= (int64_t(1) << 31)) throw Error{DMK_ERR_NOMEM, "tree too large"};
      int32_t* nch = scratch.alloc<int32_t>(cap);
      int32_t* pos = scratch.alloc<int32_t>(cap + 1);
      split_and_scan<D>(SplitCounts<D>{cur, ns_split, lmax_split, nullptr, d_cnt + lev}, static_cast<int>(cap), nch,
                        pos, s, scratch, p.launches);
      alloc_leaves(nxt, cap_out, A);
      k_refine_dev<D><<<grid_for(cap << D, B), B, 0, s>>>(static_cast<int>(cap), static_cast<int>(cap_out),
                                                     d_cnt + lev, cur, nch, pos, nxt, skeys, M, d_cnt + lev + 1,
                                                     p.status);
      ++p.launches;
      DMK_CUDA_TRY(cudaGetLastError());
      cur = nxt;
      nxt = LeafArrays();
      cap = cap_out;
    }
    // converged when the last chained level split nothing
    DMK_CUDA_TRY(cudaMemcpyAsync(h_pin, d_cnt + lev - 1, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DMK_CUDA_TRY(cudaStreamSynchronize(s));
    n_leaf = h_pin[1];
    if (h_pin[0] == h_pin[1] || lev > M) break;
  }

  // ---- (b) level restriction --------------------------------------------
  // one host round trip per round: the flags, their scan and the flag of any
  // violation are read together
  int* d_any = scratch.alloc<int>(1);
  for (int it = 0; it < 4 * M + 8; ++it) {
    int32_t* flag = scratch.alloc<int32_t>(n_leaf);
    int32_t* nch = scratch.alloc<int32_t>(n_leaf);
    int32_t* pos = scratch.alloc<int32_t>(n_leaf + 1);
    k_sys_begin<<<grid_for(n_leaf, B), B, 0, s>>>(static_cast<int>(n_leaf), n_sys, cur.sys, begin, flag, d_any);
    k_balance<D><<<grid_for(n_leaf * 32, B), B, 0, s>>>(static_cast<int>(n_leaf), cur, begin, M, T.periodic,
                                                        flag, d_any);
    split_and_scan<D>(SplitCounts<D>{cur, ns_split, lmax_split, flag, nullptr}, static_cast<int>(n_leaf), nch, pos, s,
                      scratch, p.launches);
    p.launches += 2;
    DMK_CUDA_TRY(cudaGetLastError());
    DMK_CUDA_TRY(cudaMemcpyAsync(h_pin, pos + n_leaf, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DMK_CUDA_TRY(cudaMemcpyAsync(h_pin + 2, d_any, sizeof(int), cudaMemcpyDeviceToHost, s));
    DMK_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_pin[2] == 0) break;
    const int64_t total = h_pin[0];
    if (total >= (int64_t(1) << 31)) throw Error{DMK_ERR_NOMEM, "tree too large"};
    alloc_leaves(nxt, total, A);
    k_refine<D><<<grid_for(n_leaf << D, B), B, 0, s>>>(static_cast<int>(n_leaf), cur, nch, pos, nxt, skeys, M);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
    cur = nxt;
    nxt = LeafArrays();
    n_leaf = total;
  }
  k_sys_begin<<<grid_for(n_leaf, B), B, 0, s>>>(static_cast<int>(n_leaf), n_sys, cur.sys, begin);
  ++p.launches;
  DMK_CUDA_TRY(cudaGetLastError());

  // points inside each leaf in Hilbert order of its sub-cells (FP32 pair terms)
  T.leaf_hilbert = fp32_pair_terms(p.opts) ? 1 : 0;
  T.perm = A.alloc<int32_t>(N);
  T.w = A.alloc<double>(N * D);
  if (N > 0) {
    k_leaf_hilbert<D><<<static_cast<int>(n_leaf), 256, 0, s>>>(static_cast<int>(n_leaf), cur, M, N, T.leaf_hilbert,
                                                               skeys, perm_m, w_m, T.perm, T.w);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
  }

  T.n_leaf = static_cast<int32_t>(n_leaf);
  T.leaf_anchor = cur.anchor;
  T.leaf_level = cur.level;
  T.leaf_start = cur.start;
  T.leaf_count = cur.count;
  T.leaf_sys = cur.sys;
  T.sys_leaf_begin = begin;

  // ---- near lists (at most kMaxNear entries per leaf: no host round trip) ------
  int32_t* ncount = scratch.alloc<int32_t>(n_leaf);
  int32_t* nsl = scratch.alloc<int32_t>(n_leaf * kMaxNear);
  int32_t* nsq = scratch.alloc<int32_t>(n_leaf * kMaxNear);
  T.near_off = A.alloc<int32_t>(n_leaf + 1);
  k_near_warp<D><<<grid_for(n_leaf * 32, 256), 256, 0, s>>>(static_cast<int>(n_leaf), cur, begin, M, T.periodic,
                                                            nsl, nsq, ncount, p.status);
  scan_counts(ncount, T.near_off, static_cast<int>(n_leaf), s, scratch, nullptr, p.launches);
  T.near_leaf = A.alloc<int32_t>(n_leaf * kMaxNear);
  T.near_q = A.alloc<int32_t>(n_leaf * kMaxNear);
  k_near_compact<<<grid_for(n_leaf * 32, 256), 256, 0, s>>>(static_cast<int>(n_leaf), ncount, T.near_off, nsl,
                                                           nsq, T.near_leaf, T.near_q);
  p.launches += 2;
  DMK_CUDA_TRY(cudaGetLastError());
  DMK_CUDA_TRY(cudaMemcpyAsync(h_pin + 4, T.near_off + n_leaf, sizeof(int32_t), cudaMemcpyDeviceToHost, s));

  // ---- tiles, leaf-relative FP32 coordinates, bounding boxes ---------------------
  // at most N / kTile + n_leaf tiles: allocated by that bound, counted on the device
  const int64_t tile_cap = N / kTile + n_leaf;
  T.leaf_ntile = A.alloc<int32_t>(n_leaf);
  T.leaf_tile0 = A.alloc<int32_t>(n_leaf + 1);
  int32_t* d_ntile = scratch.alloc<int32_t>(1);
  k_tile_count<<<grid_for(n_leaf, B), B, 0, s>>>(static_cast<int>(n_leaf), cur.count, T.leaf_ntile);
  scan_counts(T.leaf_ntile, T.leaf_tile0, static_cast<int>(n_leaf), s, scratch, d_ntile, p.launches);
  T.tile_leaf = A.alloc<int32_t>(tile_cap);
  T.tile_start = A.alloc<int32_t>(tile_cap);
  T.tile_count = A.alloc<int32_t>(tile_cap);
  T.tile_lo = A.alloc<float4>(tile_cap);
  T.tile_hi = A.alloc<float4>(tile_cap);
  T.rel = A.alloc<float4>(N);
  k_tile_fill<<<grid_for(n_leaf, B), B, 0, s>>>(static_cast<int>(n_leaf), cur.start, cur.count, T.leaf_tile0,
                                                T.tile_leaf, T.tile_start, T.tile_count);
  k_rel_bbox<D><<<grid_for(tile_cap * 32, 256), 256, 0, s>>>(
      d_ntile, N, T.tile_leaf, T.tile_start, T.tile_count, T.leaf_anchor, T.leaf_level, T.w, M, T.rel,
      T.tile_lo, T.tile_hi);
  p.launches += 3;
  DMK_CUDA_TRY(cudaGetLastError());
  DMK_CUDA_TRY(cudaMemcpyAsync(h_pin + 5, d_ntile, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  T.n_near = h_pin[4];
  T.n_tile = h_pin[5];
}

// ------------------------------------------------------ separate targets
// The sums of Sec. 1 are stated for target points that need not be sources.
// The tree is built from the sources (Step 1(a) counts sources); the targets
// are sorted by the Morton key of their finest cell and each goes to the leaf
// containing it: the leaves partition the box (empty leaves included) and are
// sorted by anchor, so leaf i holds the targets with keys in
// [anchor_i, anchor_{i+1}).  Per leaf they form tiles of <= 32 as the sources do.
__global__ void k_leaf_trange(int n_leaf, const uint64_t* __restrict__ anchor, int64_t NT,
                              const uint64_t* __restrict__ tkeys, int32_t* __restrict__ tstart) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_leaf) return;
  if (i == n_leaf) {
    tstart[n_leaf] = static_cast<int32_t>(NT);
    return;
  }
  int64_t lo = 0, hi = NT;                            // first target key >= anchor_i
  const uint64_t a = anchor[i];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tkeys[mid] < a) lo = mid + 1;
    else hi = mid;
  }
  tstart[i] = static_cast<int32_t>(lo);
}

__global__ void k_range_count(int n, const int32_t* __restrict__ start, int32_t* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) count[i] = start[i + 1] - start[i];
}

template <int D>
void build_targets_t(Plan& p, const double* d_trg, int64_t NT) {
  DeviceTree& T = p.tree;
  cudaStream_t s = p.stream;
  const int M = T.M;
  const int B = 256;
  const int n_leaf = T.n_leaf;
  const double lo0 = p.opts.box_lo[0], lo1 = p.opts.box_lo[1], lo2 = D == 3 ? p.opts.box_lo[2] : 0.0;
  Arena& A = p.arena;
  Arena scratch;
  scratch.s = s;
  T.sep = 1;
  T.NT = NT;
  T.tperm = A.alloc<int32_t>(NT);
  T.tw = A.alloc<double>(NT * D);
  T.trel = A.alloc<float4>(NT);
  T.leaf_tstart = A.alloc<int32_t>(n_leaf + 1);
  uint64_t* key_in = scratch.alloc<uint64_t>(NT);
  uint64_t* tkeys = scratch.alloc<uint64_t>(NT);
  int32_t* idx_in = scratch.alloc<int32_t>(NT);
  if (NT > 0) {
    k_keys<D><<<grid_for(NT, B), B, 0, s>>>(NT, d_trg, lo0, lo1, lo2, T.periodic, M, key_in, idx_in, p.status);
    ++p.launches;
    DMK_CUDA_TRY(cudaGetLastError());
    size_t bytes = 0;
    DMK_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, bytes, key_in, tkeys, idx_in, T.tperm,
                                                 static_cast<int>(NT), 0, D * M, s));
    DMK_CUDA_TRY(cub::DeviceRadixSort::SortPairs(scratch.alloc_bytes(bytes), bytes, key_in, tkeys, idx_in,
                                                 T.tperm, static_cast<int>(NT), 0, D * M, s));
    k_gather_w<D><<<grid_for(NT, B), B, 0, s>>>(NT, d_trg, T.tperm, lo0, lo1, lo2, T.periodic, T.tw);
    ++p.launches;
  }
  int32_t* tcount = scratch.alloc<int32_t>(n_leaf);
  k_leaf_trange<<<grid_for(n_leaf + 1, B), B, 0, s>>>(n_leaf, T.leaf_anchor, NT, tkeys, T.leaf_tstart);
  k_range_count<<<grid_for(n_leaf, B), B, 0, s>>>(n_leaf, T.leaf_tstart, tcount);
  p.launches += 2;
  int32_t* nttile = scratch.alloc<int32_t>(n_leaf);
  int32_t* ttile0 = scratch.alloc<int32_t>(n_leaf + 1);
  int32_t* d_ntt = scratch.alloc<int32_t>(1);
  k_tile_count<<<grid_for(n_leaf, B), B, 0, s>>>(n_leaf, tcount, nttile);
  ++p.launches;
  scan_counts(nttile, ttile0, n_leaf, s, scratch, d_ntt, p.launches);
  const int64_t cap = NT / kTile + n_leaf;
  T.ttile_leaf = A.alloc<int32_t>(cap);
  T.ttile_start = A.alloc<int32_t>(cap);
  T.ttile_count = A.alloc<int32_t>(cap);
  T.ttile_lo = A.alloc<float4>(cap);
  T.ttile_hi = A.alloc<float4>(cap);
  k_tile_fill<<<grid_for(n_leaf, B), B, 0, s>>>(n_leaf, T.leaf_tstart, tcount, ttile0, T.ttile_leaf, T.ttile_start,
                                                T.ttile_count);
  k_rel_bbox<D><<<grid_for(cap * 32, 256), 256, 0, s>>>(d_ntt, NT, T.ttile_leaf, T.ttile_start, T.ttile_count,
                                                        T.leaf_anchor, T.leaf_level, T.tw, M, T.trel, T.ttile_lo,
                                                        T.ttile_hi);
  p.launches += 2;
  DMK_CUDA_TRY(cudaGetLastError());
  int32_t* h_pin = pinned_slot();
  struct PinGuard { int32_t* q; ~PinGuard() { pinned_release(q); } } pin_guard{h_pin};
  DMK_CUDA_TRY(cudaMemcpyAsync(h_pin, d_ntt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DMK_CUDA_TRY(cudaStreamSynchronize(s));
  T.n_ttile = h_pin[0];
}

}  // namespace

void build_targets(Plan& p, const double* d_trg, int64_t n_trg) {
  if (p.opts.dim == 3) build_targets_t<3>(p, d_trg, n_trg);
  else build_targets_t<2>(p, d_trg, n_trg);
}

void build_tree(Plan& p, const double* d_src, const int64_t* h_offsets) {
  if (p.opts.dim == 3) build_tree_t<3>(p, d_src, h_offsets);
  else build_tree_t<2>(p, d_src, h_offsets);
}

void free_tree(DeviceTree& t, cudaStream_t s) {
  // the arrays live in the plan's arena, which the plan releases
  (void)s;
  t = DeviceTree();
}

}  // namespace dmk
