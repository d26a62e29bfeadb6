// Shared definitions of the DMK Stokes near-field library (device + host).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dmk_stokes.h"
#include "tables.h"

namespace dmk {

constexpr int kTile = 32;        // points per target / source tile (one warp)
constexpr int kMaxNear = 64;     // upper bound of a near list (57 in 3D)

// ----------------------------------------------------------------- errors
struct Error {
  dmk_status_t code;
  std::string msg;
};

#define DMK_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess)                                                         \
      throw ::dmk::Error{_e == cudaErrorMemoryAllocation ? DMK_ERR_NOMEM : DMK_ERR_CUDA,     \
                         std::string(#expr) + ": " + cudaGetErrorString(_e)};             \
  } while (0)

// Device status word bits (latched; read by dmk_stokes_sync_status)
enum : int {
  ST_OUT_OF_RANGE = 1,      // free-space point outside the unit box
  ST_NONFINITE = 2,         // NaN / Inf coordinate
  ST_NEAR_OVERFLOW = 4,     // near list longer than kMaxNear (tree not level-restricted)
  ST_TREE_INCONSISTENT = 8, // a fine neighbour expected to be a leaf was not
  ST_TC_TIMEOUT = 16        // a wait for tensor-core MMAs ran out (results of that evaluation invalid)
};

// ------------------------------------------------------------ Morton keys
// Bits of axis a at level-M resolution sit at positions d*b + a (axis 0 least
// significant within each group).
__host__ __device__ inline uint64_t spread3(uint64_t v) {   // 21 bits -> every 3rd
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}
__host__ __device__ inline uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}
__host__ __device__ inline uint64_t spread2(uint64_t v) {   // 32 bits -> every 2nd
  v &= 0xffffffffULL;
  v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v | (v << 2)) & 0x3333333333333333ULL;
  v = (v | (v << 1)) & 0x5555555555555555ULL;
  return v;
}
__host__ __device__ inline uint64_t compact2(uint64_t v) {
  v &= 0x5555555555555555ULL;
  v = (v ^ (v >> 1)) & 0x3333333333333333ULL;
  v = (v ^ (v >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v ^ (v >> 4)) & 0x00ff00ff00ff00ffULL;
  v = (v ^ (v >> 8)) & 0x0000ffff0000ffffULL;
  v = (v ^ (v >> 16)) & 0x00000000ffffffffULL;
  return v;
}

template <int D>
__host__ __device__ inline uint64_t morton(const int64_t* c) {
  if (D == 3) return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
  return spread2(c[0]) | (spread2(c[1]) << 1);
}
template <int D>
__host__ __device__ inline void demorton(uint64_t k, int64_t* c) {
  if (D == 3) {
    c[0] = compact3(k);
    c[1] = compact3(k >> 1);
    c[2] = compact3(k >> 2);
  } else {
    c[0] = compact2(k);
    c[1] = compact2(k >> 1);
  }
}

// integer box coordinates of a leaf at its own level
template <int D>
__host__ __device__ inline void leaf_coords(uint64_t anchor, int lev, int M, int64_t* c) {
  demorton<D>(anchor, c);
  for (int a = 0; a < D; ++a) c[a] >>= (M - lev);
}

template <int D>
__host__ __device__ inline uint64_t box_anchor(const int64_t* c, int lev, int M) {
  int64_t cc[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) cc[a] = c[a] << (M - lev);
  return morton<D>(cc);
}

template <int D> struct MaxLevel;
template <> struct MaxLevel<3> { static constexpr int value = 21; };
template <> struct MaxLevel<2> { static constexpr int value = 31; };

// q offsets of a near-list entry, packed 8 bits per axis (values -1, 0, 1)
__host__ __device__ inline int32_t pack_q(int q0, int q1, int q2) {
  return (q0 & 0xff) | ((q1 & 0xff) << 8) | ((q2 & 0xff) << 16);
}
__host__ __device__ inline int unpack_q(int32_t p, int a) {
  return static_cast<int>(static_cast<int8_t>((p >> (8 * a)) & 0xff));
}

// ----------------------------------------------------------------- plan
// MIXED precision evaluates the pair terms in FP32 from this eps up (their l2
// error is about 1e-7 to 2e-6), in float-float or FP64 below
constexpr double kFp32PairMinEps = 2e-7;
inline bool fp32_pair_terms(const dmk_stokes_opts_t& o) {
  return o.precision == DMK_PRECISION_MIXED && o.eps >= kFp32PairMinEps;
}

struct DeviceTree {
  int dim = 3;
  int M = 21;                 // key bits per axis
  int periodic = 0;
  int n_sys = 1;
  int64_t N = 0;              // points (sources == targets)
  int leaf_hilbert = 0;       // 1: points inside each leaf in Hilbert order of its sub-cells
  // points, sorted order
  int32_t* perm = nullptr;    // sorted index -> original index
  double* w = nullptr;        // in-cell coordinates, SoA [dim][N]
  float4* rel = nullptr;      // FP32 leaf-centre-relative coordinates, [N]
  int32_t* point_sys = nullptr;
  // leaves (sorted by (system, Morton anchor))
  int32_t n_leaf = 0;
  uint64_t* leaf_anchor = nullptr;
  int32_t* leaf_level = nullptr;
  int32_t* leaf_start = nullptr;
  int32_t* leaf_count = nullptr;
  int32_t* leaf_sys = nullptr;
  int32_t* sys_leaf_begin = nullptr;   // [n_sys + 1]
  // near lists (CSR)
  int32_t* near_off = nullptr;         // [n_leaf + 1]
  int32_t* near_leaf = nullptr;
  int32_t* near_q = nullptr;
  int64_t n_near = 0;
  // tiles
  int32_t n_tile = 0;
  int32_t* tile_leaf = nullptr;
  int32_t* tile_start = nullptr;
  int32_t* tile_count = nullptr;
  float4* tile_lo = nullptr;           // bounding box in the leaf-relative frame
  float4* tile_hi = nullptr;
  int32_t* leaf_tile0 = nullptr;       // first tile of each leaf
  int32_t* leaf_ntile = nullptr;
  // separate targets (single-system plans; sep == 0: the targets are the points)
  int sep = 0;
  int64_t NT = 0;
  int32_t* tperm = nullptr;            // sorted target -> caller's target index
  double* tw = nullptr;                // in-cell target coordinates, SoA [dim][NT]
  float4* trel = nullptr;              // leaf-relative FP32 target coordinates
  int32_t* leaf_tstart = nullptr;      // [n_leaf + 1] targets of each leaf (sorted)
  int32_t n_ttile = 0;
  int32_t* ttile_leaf = nullptr;
  int32_t* ttile_start = nullptr;
  int32_t* ttile_count = nullptr;
  float4* ttile_lo = nullptr;
  float4* ttile_hi = nullptr;
};

// Bump allocator over a few large stream-ordered blocks.  A plan's device
// arrays come from one arena (returned in one call per block when the plan is
// destroyed) and the tree builder's scratch from another, released when the
// build ends; a pointer from an arena is never freed on its own.
struct Arena {
  cudaStream_t s = nullptr;
  std::vector<void*> blocks;
  char* cur = nullptr;
  size_t left = 0;
  size_t next = size_t(16) << 20;       // size of the next block
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  void reserve(size_t bytes) {
    if (bytes > next) next = bytes;
  }
  void* alloc_bytes(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (bytes > left) {
      const size_t sz = std::max(bytes, next);
      void* ptr = nullptr;
      DMK_CUDA_TRY(cudaMallocAsync(&ptr, sz, s));
      blocks.push_back(ptr);
      cur = static_cast<char*>(ptr);
      left = sz;
      next = std::max(next, sz) * 2;
    }
    void* r = cur;
    cur += bytes;
    left -= bytes;
    return r;
  }
  template <typename T>
  T* alloc(size_t n) {
    return static_cast<T*>(alloc_bytes(n * sizeof(T)));
  }
  void release() {
    for (void* b : blocks) cudaFreeAsync(b, s);
    blocks.clear();
    cur = nullptr;
    left = 0;
  }
  ~Arena() { release(); }
};

// Small pinned host buffers (16 int32 each) shared by all plans of the process:
// pinned allocation costs far more than the plan build otherwise needs.
int32_t* pinned_slot();
void pinned_release(int32_t* slot);

struct EwaldState;
struct FarState;
struct Far2State;

struct Plan {
  dmk_stokes_opts_t opts{};
  int leaf_capacity = 0;
  int uniform_level = 0;       // > 0: every leaf at this level (single-level Ewald split)
  EwaldState* ewald = nullptr; // far field of components = EWALD (periodic 3D Stokeslet)
  FarState* far = nullptr;     // DMK far field of components = ALL (2D and 3D)
  cudaStream_t stream = nullptr;
  int device = 0;
  KernelTables tables;
  DeviceTree tree;
  // eval workspace (owned by the plan)
  void* fsorted = nullptr;     // sorted forces (FP32 float4 or FP64 SoA), n_rhs columns
  size_t fsorted_bytes = 0;
  double* gn_sorted = nullptr; // stresslet: sorted g (SoA) , n (SoA), g.n
  double* reduce_buf = nullptr;
  void* aux = nullptr;         // gradient / adjoint workspace, allocated on first use
  size_t aux_bytes = 0;
  int* status = nullptr;       // device status word
  int* h_status = nullptr;     // pinned host mirror (a pinned_slot)
  Arena arena;                 // device arrays of the plan
  std::string last_error;
  int64_t useful_pairs = -1;   // cached by dmk_stokes_plan_stats
  mutable int64_t launches = 0;  // kernels launched by this library for this plan
  mutable cudaEvent_t* trace = nullptr;  // set by dmk_stokes_eval_traced: events between the stages
  uint32_t magic = 0;
};

constexpr uint32_t kPlanMagic = 0xD3C5A17Bu;

// tree.cu
void build_tree(Plan& p, const double* d_src, const int64_t* h_offsets);
// separate targets of a single-system plan, located in the built tree
void build_targets(Plan& p, const double* d_trg, int64_t n_trg);
void free_tree(DeviceTree& t, cudaStream_t s);

// near.cu
void launch_near(const Plan& p, const double* d_f, const double* d_g, const double* d_n,
                 double* d_u, double* d_gradu, cudaStream_t s);
// same, with the evaluation scratch given explicitly: workspace of
// eval_workspace_bytes(opts, N) bytes, reduce_buf of 4 * n_sys doubles and,
// for a gradient, aux of aux_bytes_grad(opts, N) bytes (may be null when 0)
void launch_near_ws(const Plan& p, const double* d_f, const double* d_g, const double* d_n,
                    double* d_u, double* d_gradu, cudaStream_t s, void* workspace, double* reduce_buf,
                    void* aux);
// N points (sources), NT targets (N when the targets are the points)
size_t eval_workspace_bytes(const dmk_stokes_opts_t& o, int64_t N, int64_t NT);
size_t aux_bytes_grad(const dmk_stokes_opts_t& o, int64_t N);
size_t aux_bytes_adjoint(const dmk_stokes_opts_t& o, int64_t N);
// Gauss-Legendre nodes and weights on [-1, 1]
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// far.cu: the DMK far field (components = ALL): proxy charges, plane waves, root, interpolation
// (3D there; the 2D plans are handed to far2d.cu)
void far_setup(Plan& p);
void far_free(Plan& p);
void far_run(const Plan& p, const double* d_f, const double* d_g, const double* d_n, double* d_u, cudaStream_t s);
void far_info(const Plan& p, int32_t info[8]);
size_t far_bytes(const Plan& p);
// the tensor-core wait limit exercised on purpose (true when the wait ran out and was reported)
bool tc_wait_selftest(cudaStream_t s);
// far2d.cu: the same in 2D
Far2State* far2d_setup(Plan& p);
void far2d_free(Plan& p, Far2State* F);
void far2d_run(const Plan& p, const Far2State& F, const double* d_f, const double* d_g, const double* d_n, double* d_u,
               cudaStream_t s);
void far2d_info(const Far2State& F, int32_t info[8]);
size_t far2d_bytes(const Far2State& F);
// ewald.cu: the single-level PSWF Ewald far field (components = EWALD, periodic 3D Stokeslet)
int ewald_level(int64_t N, int ns);
void ewald_setup(Plan& p, int L);
void ewald_free(Plan& p);
void ewald_far(const Plan& p, const double* d_f, double* d_u, cudaStream_t s);
void ewald_info(const Plan& p, int32_t info[4]);

// adjoint pass of the 3D Stokeslet (v = S[w], dL/dx); aux of aux_bytes_adjoint bytes
void launch_adjoint(const Plan& p, const double* d_f, const double* d_w, double* d_v, double* d_gx,
                    cudaStream_t s, void* aux);

int64_t count_useful_pairs(const Plan& p);

// device memory helper (stream-ordered pool)
template <typename T>
T* dalloc(size_t n, cudaStream_t s) {
  void* ptr = nullptr;
  if (n == 0) n = 1;
  DMK_CUDA_TRY(cudaMallocAsync(&ptr, n * sizeof(T), s));
  return static_cast<T*>(ptr);
}
template <typename T>
void dfree(T*& ptr, cudaStream_t s) {
  if (ptr) cudaFreeAsync(ptr, s);
  ptr = nullptr;
}

// force columns the kernels are compiled for: 1, 4 or 16 (n_rhs padded up)
inline int padded_rhs(int n_rhs) { return n_rhs <= 1 ? 1 : (n_rhs <= 4 ? 4 : 16); }

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > (1 << 30)) g = (1 << 30);
  return static_cast<int>(g);
}

}  // namespace dmk

// the opaque plan handle of the C ABI
struct dmk_stokes_plan_s {
  dmk::Plan p;
  cudaStream_t last_stream = nullptr;
};

namespace dmk {
// records msg as the last error (per thread, and on the plan if not NULL); returns code
dmk_status_t record_error(dmk_stokes_plan_t plan, dmk_status_t code, const std::string& msg);
}  // namespace dmk
