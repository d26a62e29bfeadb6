// Explicit instantiations of the FP64 3D near-field kernels.
#include "near_kernel.cuh"

namespace dmk {
#define DMK_INST(D, KM, GR, NT, NR) template void run_near_fp64<D, KM, GR, NT, NR>(const NearParams&, cudaStream_t);
#define DMK_INST_NT(NT) DMK_FOR_EACH_VARIANT_3D_FP64(DMK_INST, NT)
DMK_NT_FP64(DMK_INST_NT)
}  // namespace dmk
