// Grid-wide barrier for kernels launched cooperatively (every block resident), shared by the
// persistent kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace vga {

constexpr uint32_t kBarrierSpin = 1u << 26;  // polls (64 ns sleeps) before a barrier gives up

// Grid-wide barrier for a cooperative launch.  bar[0] counts arrivals, bar[1] is the generation
// (both start at zero).  Bounded: after `limit` polls (or on an earlier error) it sets *err and
// returns false; callers then stop.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *err, uint32_t limit = kBarrierSpin) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = bar + 1;
        volatile int32_t *verr = err;
        if (*verr) {
            ok = 0;
        } else {
            const unsigned gen = *vgen;
            __threadfence();
            const unsigned arrived = atomicAdd(bar, 1u) + 1u;
            if (arrived == gridDim.x) {
                bar[0] = 0u;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                uint32_t it = 0;
                while (*vgen == gen) {
                    if (*verr || ++it > limit) {
                        atomicExch(err, 2);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace vga
