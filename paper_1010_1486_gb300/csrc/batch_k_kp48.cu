// batch_k_kp48.cu -- instantiates the batched sweep kernels with the Kennedy-Pendleton sampler for
// queue depths 4 and 8 (all three block sizes); split from the other
// launch shapes so that the library's translation units compile in parallel.
#include "batch_kp.cuh"

namespace su2 {

void *batch_kernel_kp_48(int R, int T) { return R == 4 ? batch_kernel_t<4, kBatchKP>(T) : batch_kernel_t<8, kBatchKP>(T); }

}  // namespace su2
