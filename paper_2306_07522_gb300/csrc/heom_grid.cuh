// Grid-wide barrier for cooperative launches (all CTAs resident), with a bounded wait.
#pragma once

#include "heom_internal.h"

namespace heom {

// state of the grid barrier (zeroed before every launch)
struct GridBar {
    unsigned count;  // arrivals since the launch began (never reset)
    unsigned gen;    // unused
    int err;         // a wait ran out
    int pad;
};

// Grid barrier of the cooperative launch (every CTA resident). The arrival counter only grows:
// barrier number g (1, 2, ...) is complete once it holds g * gridDim.x arrivals, so the last
// arrival needs no reset and no second publication, and CTAs that run ahead into the next
// barrier only raise the count further. Each CTA's thread 0 fences the CTA's writes, adds its
// arrival, and waits with acquire loads in a bounded spin of at most `limit` SM clock
// cycles (the library's wait limit: by default 4e9, about 2 s). A wait that runs out raises
// the shared error flag; every CTA that sees the flag leaves its wait too, so no CTA waits
// for one that has gone, and the launch ends on every CTA. Returns false in every thread of
// a CTA that must stop. The counter wraps after 2^32 arrivals (28 million barriers of 152
// CTAs); the signed distance to the target stays correct across the wrap.
__device__ __forceinline__ bool grid_barrier(GridBar *bar, unsigned &gen, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (gen + 1) * gridDim.x;
        __threadfence();  // this CTA's writes are visible before its arrival
        const unsigned prev = atomicAdd(&bar->count, 1u);
        if (prev + 1u != target) {
            const long long t0 = clock64();
            for (;;) {
                unsigned c;
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(c) : "l"(&bar->count) : "memory");
                if ((int)(c - target) >= 0) break;
                if (*(volatile int *)&bar->err) { ok = 0; break; }
                if (clock64() - t0 > limit) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        gen = gen + 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace heom
