// batch_k_kp12.cu -- instantiates the batched sweep kernels with the Kennedy-Pendleton sampler for
// queue depths 1 and 2 (all three block sizes); split from the other
// launch shapes so that the library's translation units compile in parallel.
#include "batch_kp.cuh"

namespace su2 {

void *batch_kernel_kp_12(int R, int T) { return R == 1 ? batch_kernel_t<1, kBatchKP>(T) : batch_kernel_t<2, kBatchKP>(T); }

}  // namespace su2
