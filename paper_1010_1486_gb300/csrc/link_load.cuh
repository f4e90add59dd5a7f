// link_load.cuh -- how kernels read links.
#pragma once

#include <cuda_runtime.h>

namespace su2 {

// A kernel whose launch never writes the links it reads uses the read-only
// path (ld.global.nc, NC = true).  The batched persistent kernel reads, in
// later phases, links that earlier phases of the same launch wrote; it uses
// ordinary cached loads (NC = false), which the fences of its grid barrier
// order after those writes, while the read-only path is defined only for data
// that no thread writes during the launch.
template <bool NC>
__device__ __forceinline__ float4 load_link(const float4 *p)
{
    return NC ? __ldg(p) : __ldca(p);
}

}  // namespace su2
