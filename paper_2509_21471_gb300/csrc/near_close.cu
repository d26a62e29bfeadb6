// Instantiations of the close-pair kernel (dimension x kernels x gradient x coordinates).
#include "near_close.cuh"

namespace dmk {

#define DMK_INST_C(D, KM, GR, FFC) \
  template void run_near_close<D, KM, GR, FFC>(const NearParams&, const CloseParams&, cudaStream_t);
DMK_FOR_EACH_CLOSE(DMK_INST_C)

}  // namespace dmk
