// Instantiations of the adjoint kernel: float-float (per table length) and FP64.
#include "near_adj.cuh"

namespace dmk {

#define DMK_INST_A(NT) template void run_near_adj<true, NT>(const NearParams&, const AdjParams&, cudaStream_t);
DMK_NT_FP64(DMK_INST_A)
template void run_near_adj<false, 16>(const NearParams&, const AdjParams&, cudaStream_t);

}  // namespace dmk
