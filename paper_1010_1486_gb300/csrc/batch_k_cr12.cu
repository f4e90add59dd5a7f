// batch_k_cr12.cu -- instantiates the batched sweep kernels with the Creutz sampler for
// queue depths 1 and 2 (all three block sizes); split from the other
// launch shapes so that the library's translation units compile in parallel.
#include "batch_device.cuh"

namespace su2 {

void *batch_kernel_creutz_12(int R, int T) { return R == 1 ? batch_kernel_t<1, kBatchCreutz>(T) : batch_kernel_t<2, kBatchCreutz>(T); }

}  // namespace su2
