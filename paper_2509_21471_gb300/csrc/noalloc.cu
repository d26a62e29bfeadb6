// Near-field evaluation that allocates no device memory.
//
// dmk_stokes_eval keeps its scratch (sorted copies of the densities and the
// per-system sums of the periodic zero mode) in a workspace owned by the plan.
// This variant takes the same inputs and outputs but puts that scratch in one
// fixed array of device memory that the library reserves statically: it never
// calls cudaMalloc, cudaMallocAsync, cudaFree or any allocating routine.  It is
// meant for code that must not allocate device memory when it evaluates, for
// example while a CUDA stream is being captured in a mode that forbids
// allocation calls, or inside an application whose device memory is owned by
// another allocator with a fixed budget.
//
// Limits and sharing (also documented in include/dmk_stokes.h):
//   * the array holds kNoAllocScratchBytes (64 MiB); a plan whose evaluation
//     needs more is rejected with DMK_ERR_INVALID_ARG before anything runs
//     (mixed precision at eps >= 2e-7: 136 bytes per point, about 493k
//     points; mixed below 2e-7: 296 bytes per point in 3D (200 in 2D),
//     about 226k points; FP64: 104 bytes per point, about 645k points; plus
//     32 bytes per system);
//   * every GPU that loads the library holds the array until the process exits;
//   * all calls on a device share the array and it keeps the last call's
//     contents; the zero-mode sums are cleared at the start of every call;
//     calls whose work overlaps on the GPU race on the array;
//   * the device address of the array is looked up once per device, with that
//     device current, by the first call on the device; make that first call
//     before any stream capture.  The address is kept for the life of the
//     process: a device reset (cudaDeviceReset) after the first call is not
//     supported.
#include <mutex>

#include "common.cuh"

namespace dmk {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (the host-side
// name g_noalloc_scratch is a stand-in, not a device address).
dmk_status_t scratch_on_current_device(void** out, std::string& msg) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return DMK_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    msg = "device index beyond the scratch table";
    return DMK_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return DMK_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return DMK_OK;
}

}  // namespace
}  // namespace dmk

extern "C" dmk_status_t dmk_stokes_eval_noalloc(dmk_stokes_plan_t plan, const double* d_f, const double* d_g,
                                                const double* d_n, double* d_u, void* stream) {
  if (!plan || plan->p.magic != dmk::kPlanMagic)
    return dmk::record_error(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  dmk::Plan& p = plan->p;
  const int64_t N = p.tree.N;
  const bool want_s = p.opts.kernels & DMK_KERNEL_STOKESLET;
  const bool want_t = p.opts.kernels & DMK_KERNEL_STRESSLET;
  if (N > 0) {
    if (want_s && !d_f) return dmk::record_error(plan, DMK_ERR_INVALID_ARG, "d_f is NULL but the Stokeslet is requested");
    if (want_t && (!d_g || !d_n))
      return dmk::record_error(plan, DMK_ERR_INVALID_ARG, "d_g / d_n NULL but the stresslet is requested");
    if (!d_u) return dmk::record_error(plan, DMK_ERR_INVALID_ARG, "d_u is NULL");
  }
  const size_t ws = (p.fsorted_bytes + 255) & ~size_t(255);
  const size_t red = 4 * sizeof(double) * static_cast<size_t>(p.tree.n_sys);
  if (ws + red > dmk::kNoAllocScratchBytes)
    return dmk::record_error(plan, DMK_ERR_INVALID_ARG,
                             "dmk_stokes_eval_noalloc: this plan needs " + std::to_string(ws + red) +
                                 " bytes of scratch; the static scratch holds " +
                                 std::to_string(dmk::kNoAllocScratchBytes) + " bytes (use dmk_stokes_eval)");
  if (p.ewald || p.far)
    return dmk::record_error(plan, DMK_ERR_UNSUPPORTED,
                             "dmk_stokes_eval_noalloc evaluates the near component only (components = NEAR)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p.device)
    return dmk::record_error(plan, DMK_ERR_INVALID_ARG, "make the plan's device current before the call");
  void* scratch = nullptr;
  std::string msg;
  dmk_status_t st = dmk::scratch_on_current_device(&scratch, msg);
  if (st != DMK_OK) return dmk::record_error(plan, st, msg);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->last_stream = s;
  try {
    dmk::launch_near_ws(p, want_s ? d_f : nullptr, want_t ? d_g : nullptr, want_t ? d_n : nullptr, d_u, nullptr,
                        s, scratch, reinterpret_cast<double*>(static_cast<char*>(scratch) + ws), nullptr);
  } catch (const dmk::Error& e) {
    return dmk::record_error(plan, e.code, e.msg);
  }
  return DMK_OK;
}
