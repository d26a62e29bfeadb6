// Explicit instantiations of the mixed-precision 3D near-field kernels.
#include "near_kernel.cuh"

namespace dmk {
#define DMK_INST(D, KM, GR, NT, NR) template void run_near_mixed<D, KM, GR, NT, NR>(const NearParams&, cudaStream_t);
#define DMK_INST_NT(NT) DMK_FOR_EACH_VARIANT_3D(DMK_INST, NT)
DMK_NT_MIXED(DMK_INST_NT)
}  // namespace dmk
