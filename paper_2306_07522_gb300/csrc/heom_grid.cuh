// Grid-wide barrier for cooperative launches (all CTAs resident), with a bounded wait.
#pragma once

#include "heom_internal.h"

namespace heom {

// state of the grid barrier (zeroed before every launch)
struct GridBar {
    unsigned count;  // arrivals in the current generation
    unsigned gen;    // completed barriers
    int err;         // a wait ran out
    int pad;
};

// Grid barrier of the cooperative launch (every CTA resident). Generation counting: each
// CTA adds one arrival; the last arrival resets the count and publishes the next generation;
// the others wait for it with a bounded spin (about 2 s of SM clock). A wait that runs out
// raises the shared error flag; every CTA that sees the flag leaves its wait too, so no CTA
// waits for one that has gone. Returns false in every thread of a CTA that must stop.
constexpr long long kBarrierCycles = 4000000000LL;

__device__ __forceinline__ bool grid_barrier(GridBar *bar, unsigned &gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen + 1;
        __threadfence();  // this CTA's writes are visible before its arrival
        const unsigned prev = atomicAdd(&bar->count, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicExch(&bar->gen, target);
        } else {
            const long long t0 = clock64();
            for (;;) {
                unsigned g;
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(g) : "l"(&bar->gen) : "memory");
                if (g == target) break;
                if (*(volatile int *)&bar->err) { ok = 0; break; }
                if (clock64() - t0 > kBarrierCycles) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = target;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace heom
