// Instantiations of the float-float near-field kernel (dimension x kernels x gradient x table length).
#include "near_ff.cuh"

namespace dmk {

#define DMK_INST_F(D, KM, GR, NT) \
  template void run_near_ff<D, KM, GR, NT>(const NearParams&, const FFParams&, cudaStream_t);
#define DMK_INST_F_NT(NT) DMK_FOR_EACH_FF(DMK_INST_F, NT)
DMK_NT_FP64(DMK_INST_F_NT)

}  // namespace dmk
