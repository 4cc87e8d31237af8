// RK4 time evolution that allocates nothing: heom_evolve_noalloc.
//
// Some callers cannot let a library call cudaMalloc or cudaFree. A process whose device
// memory is entirely held by another allocator (a framework's caching pool, a fixed
// budget) can see cudaMalloc fail, and cudaFree waits for the whole device, which stalls
// callers that keep several streams busy or run time-critical loops. heom_evolve
// allocates its three RK4 stage buffers in the hierarchy's workspace on first use; this
// variant takes them from a fixed static device array instead, so it never allocates.
//
// The array lives in this file, which holds no kernel. Host code cannot use the array's name
// as a device address (on the host it names a host-side stand-in), so the device address is
// looked up with cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device. Under the CUDA runtime's lazy module loading (the default
// since CUDA 12.2) that lookup is what loads this file's module, so the CUDA runtime reserves
// the 16 MiB on a device at the first call there, not when the library is loaded; from then
// on the device holds it until the process exits. Callers make one call with n_steps = 0 at
// start-up, before the other allocator fills the device and before any stream capture; a
// lookup that fails for want of memory returns HEOM_ENOMEM.
#include <cmath>
#include <mutex>

#include "heom_internal.h"

namespace heom {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
heom_status scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("heom_evolve_noalloc: device ordinal %d out of range", device);
        return HEOM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            set_error("heom_evolve_noalloc: the CUDA runtime could not reserve the %zu-byte "
                      "static scratch on device %d (its first call there loads it); make one "
                      "call with n_steps = 0 at start-up, before device memory fills",
                      kNoAllocScratchBytes, device);
            return HEOM_ENOMEM;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return HEOM_OK;
}

template <class R> DevView<R> view_for(const heom_hier *h);
template <> DevView<double> view_for<double>(const heom_hier *h) { return h->view64(); }
template <> DevView<float> view_for<float>(const heom_hier *h) { return h->view32(); }

template <class R>
heom_status evolve_static(heom_hier *h, cx<R> *y, int64_t B, double dt, int64_t n_steps,
                          int64_t save_every, cx<R> *traj, void *scratch, cudaStream_t s) {
    const DevView<R> v = view_for<R>(h);
    const int64_t L = h->N * h->d2 * B;
    // The three stage buffers need no clearing: stage 1 writes acc and z_a before any read,
    // and stage 2 writes z_b before stage 3 reads it.
    cx<R> *za = (cx<R> *)scratch, *zb = za + L, *acc = za + 2 * L;
    const size_t blk = (size_t)h->d2 * B * sizeof(cx<R>);
    const double u = (double)h->N * B, pass = (double)L * sizeof(cx<R>);
    int64_t saved = 0;
    if (traj) HEOM_CUDA(memcpy_counted(traj, y, blk, cudaMemcpyDeviceToDevice, s));
    for (int64_t step = 1; step <= n_steps; ++step) {
        // accounted like heom_evolve's stages: stage 1 streams 3 vector passes, 2 and 3 five,
        // 4 four
        { Prof pr(HEOM_KC_RK4, s, u, 3.0 * pass); HEOM_CUDA(launch_rk4_stage<R>(v, y, za, y, acc, B, (R)dt, 1, s)); }
        { Prof pr(HEOM_KC_RK4, s, u, 5.0 * pass); HEOM_CUDA(launch_rk4_stage<R>(v, za, zb, y, acc, B, (R)dt, 2, s)); }
        { Prof pr(HEOM_KC_RK4, s, u, 5.0 * pass); HEOM_CUDA(launch_rk4_stage<R>(v, zb, za, y, acc, B, (R)dt, 3, s)); }
        { Prof pr(HEOM_KC_RK4, s, u, 4.0 * pass); HEOM_CUDA(launch_rk4_stage<R>(v, za, zb, y, acc, B, (R)dt, 4, s)); }
        if (traj && step % save_every == 0) {
            ++saved;
            HEOM_CUDA(memcpy_counted((char *)traj + saved * blk, y, blk, cudaMemcpyDeviceToDevice, s));
        }
    }
    HEOM_CUDA(cudaStreamSynchronize(s));
    return HEOM_OK;
}

}  // namespace
}  // namespace heom

extern "C" heom_status heom_evolve_noalloc(heom_hier *h, void *ados, int64_t batch, double dt,
                                           int64_t n_steps, int64_t save_every, void *rho_traj,
                                           int prec, heom_stream s) {
    using namespace heom;
    if (!h || !ados || batch < 1 || batch % h->n_sets != 0 || !std::isfinite(dt) ||
        n_steps < 0 || (rho_traj && save_every < 1) || (prec != HEOM_FP64 && prec != HEOM_FP32) ||
        batch > 65535LL * 32) {
        set_error("heom_evolve_noalloc: need a hierarchy, ados, batch >= 1 (multiple of n_sets), "
                  "finite dt, n_steps >= 0, save_every >= 1 with a trajectory, prec FP64 or FP32");
        return HEOM_EINVAL;
    }
    const size_t elt = prec == HEOM_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
    const double need = 3.0 * (double)h->N * h->d2 * (double)batch * (double)elt;
    if (need > (double)kNoAllocScratchBytes) {
        set_error("heom_evolve_noalloc: 3 stage buffers of N*d*d*batch = %lld elements need %.0f "
                  "bytes, more than the %zu-byte static scratch; use heom_evolve",
                  (long long)(h->N * h->d2 * batch), need, kNoAllocScratchBytes);
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    void *scratch = nullptr;
    heom_status st = scratch_address(h->device, &scratch);
    if (st != HEOM_OK) return st;
    if (prec == HEOM_FP64)
        return evolve_static<double>(h, (cx<double> *)ados, batch, dt, n_steps, save_every,
                                     (cx<double> *)rho_traj, scratch, (cudaStream_t)s);
    return evolve_static<float>(h, (cx<float> *)ados, batch, dt, n_steps, save_every,
                                (cx<float> *)rho_traj, scratch, (cudaStream_t)s);
}
