// creutz_queue.cuh -- per-warp shared-memory queues of the Creutz phase
// kernels (single lattice and batches): links whose first two trials were
// rejected wait for further Philox blocks; links with an accepted trial wait
// for their a0 (deferred_a0), direction and store, 32 at a time.
#pragma once

#include <cuda_runtime.h>

namespace su2 {

constexpr int kCrQueue = 64;  // per warp and queue: at most 31 left over + 32 pushed at once

struct CrQueues {
    // links still without an accepted trial: U~^dag, 1/(beta k) (0 on the Haar
    // branch), exp(-2 beta k), index, next Philox block
    float4 r_ut[kCrQueue];
    float r_ibk[kCrQueue], r_e[kCrQueue];
    int r_eo[kCrQueue], r_blk[kCrQueue];
    // links with an accepted trial waiting for their a0, direction and store:
    // U~^dag, x of the trial (a0 on the Haar branch), 1/(beta k), index
    float4 d_ut[kCrQueue];
    float d_val[kCrQueue], d_ibk[kCrQueue];
    int d_eo[kCrQueue];
    // when the phase measures the plaquette: the link's staple terms of the
    // directions nu < mu, for the retry and the direction queue
    float4 r_sp[kCrQueue], d_sp[kCrQueue];
};

}  // namespace su2
