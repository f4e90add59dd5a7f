// batch_k_cr48.cu -- instantiates the batched sweep kernels with the Creutz sampler for
// queue depths 4 and 8 (all three block sizes); split from the other
// launch shapes so that the library's translation units compile in parallel.
#include "batch_device.cuh"

namespace su2 {

void *batch_kernel_creutz_48(int R, int T) { return R == 4 ? batch_kernel_t<4, kBatchCreutz>(T) : batch_kernel_t<8, kBatchCreutz>(T); }

}  // namespace su2
