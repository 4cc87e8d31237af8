// Persistent cooperative BiCGStab for one right-hand side (batch 1): the whole solve is one
// launch. Each CTA owns one ADO range (one per SM), builds that range's term programs of
// Eq. HEOM in shared memory once (from the neighbour tables, never stored elsewhere) and
// keeps them for every iteration. Vector updates touch only the CTA's own rows; the apply
// reads neighbour rows of the whole vector after a grid-wide barrier. Dot products are
// block sums written to per-block slots, added in a fixed order by every CTA after the next
// barrier, so every CTA derives the same Krylov scalars and the same convergence decision
// without any host round trip. Five grid barriers per iteration; the host reads the result
// once, at the end. In the FP64 solve the two applies of an iteration run in float-float (the
// Krylov vectors, dot products and scalars stay FP64).
#include <algorithm>
#include <cmath>

#include "heom_ff.cuh"
#include "heom_grid.cuh"
#include "heom_tile.cuh"

namespace heom {

struct PersistOut {
    int iterations;
    int status;
    double nr;   // ||r||^2 at exit
    double bn;   // ||b||^2
};

template <class R>
struct PersistArgs {
    DevView<R> v;
    const cx<R> *b;
    cx<R> *x;
    int x_zero;
    const cx<R> *shift;  // [1] or null
    R aug;
    int precond;
    cx<R> *r, *rh, *p, *vv, *ph, *sh, *t;
    float4 *phf, *shf;  // FP64 solve: float-float copies of ph and sh (the apply operands)
    double *part;  // [kSlots][G][4]
    GridBar *bar;
    long long wait_cycles;  // bound of every grid-barrier wait (SM clock cycles)
    double tol;
    int max_iter, stall_iters;
    PersistOut *out;
};

namespace {

constexpr int kPersThreads = 512;
constexpr int kSlots = 4;

// Load written earlier in this launch by another CTA: through L2 (ld.global.cg), never the
// non-coherent read-only path.
template <class R>
__device__ __forceinline__ cx<R> ld_l2(const cx<R> *p) {
    if constexpr (sizeof(R) == 8) {
        const double2 t = __ldcg(reinterpret_cast<const double2 *>(p));
        return cx<R>{t.x, t.y};
    } else {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
        return cx<R>{t.x, t.y};
    }
}

// y = (M + shift) X at one item (single column), from the item's program
template <class R>
__device__ __forceinline__ cx<R> prog_apply(const ProgSmem<R> &ps, int it, const cx<R> *X,
                                            cx<R> shift) {
    const int j0 = ps.item[it], j1 = ps.item[it + 1];
    cx<R> acc = (ps.coef[j0] + shift) * ld_l2(X + ps.src[j0]);
    for (int jj = j0 + 1; jj < j1; jj += 8) {
        cx<R> cf[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = jj + u < j1;
            const int idx = ok ? jj + u : j1 - 1;
            cf[u] = ok ? ps.coef[idx] : cx<R>{R(0), R(0)};
            xv[u] = ld_l2(X + ps.src[idx]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) fma_to(acc, cf[u], xv[u]);
    }
    return acc;
}

// The same apply in float-float for the FP64 solve: float-float coefficients (the shift
// already folded into each item's first term) and a float-float copy of X, so that the
// multiply-adds run on the FP32 pipe instead of GB300's 1/64-rate FP64 pipe; about 48
// significant bits per product and sum.
__device__ __forceinline__ cx<double> prog_apply_ff(const ProgSmem<double> &ps, int it, const float4 *X) {
    const float4 *coef = reinterpret_cast<const float4 *>(ps.coef);
    const int j0 = ps.item[it], j1 = ps.item[it + 1];
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int jj = j0; jj < j1; jj += 8) {
        float4 c[8], x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = jj + u < j1;
            const int idx = ok ? jj + u : j1 - 1;
            c[u] = ok ? coef[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[u] = __ldcg(X + ps.src[idx]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            ff_mac(rh, rl, c[u].x, c[u].z, x[u].x, x[u].z);
            ff_mac(rh, rl, -c[u].y, -c[u].w, x[u].y, x[u].w);
            ff_mac(ih, il, c[u].x, c[u].z, x[u].y, x[u].w);
            ff_mac(ih, il, c[u].y, c[u].w, x[u].x, x[u].z);
        }
    }
    return cx<double>{(double)rh + (double)rl, (double)ih + (double)il};
}

// Grid-wide sum of NV doubles: block sums to part[slot][block], grid barrier, then in every
// block warp k adds value k over all blocks (lane-strided loads through L2, then a fixed
// shuffle tree; lane 0's result is used), so every block derives bit-identical totals. Only
// the first nw warps hold values (the warps past the block's elements add nothing), so only
// they run the FP64 shuffle trees.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&val)[NV], double *part, int slot, double *s_red,
                                         double *s_tot, GridBar *bar, unsigned &gen, int nw,
                                         long long limit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < nw) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = val[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) s_red[warp * 4 + k] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < nw; ++w) x += s_red[w * 4 + threadIdx.x];
        part[((size_t)slot * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = x;
    }
    if (!grid_barrier(bar, gen, limit)) return false;
    if (warp < NV) {
        // written by the other CTAs since this CTA last read the slot: through L2, so that
        // no line of an earlier iteration cached in L1 is reused
        double x = 0.0;
        for (unsigned g = lane; g < gridDim.x; g += 32)
            x += __ldcg(part + ((size_t)slot * gridDim.x + g) * 4 + warp);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) s_tot[warp] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) val[k] = s_tot[k];
    __syncthreads();
    return true;
}

// 1/x by Newton-Raphson (r <- r (2 - x r), written r + r (1 - x r)) from the FP32 reciprocal
// as seed: the seed's relative error (<= 2^-23) squares at each step, so two steps reach FP64
// rounding. An FP64 division is a long instruction sequence on GB300's narrow FP64 pipe; this
// is six FP64-pipe instructions. Outside the seed's range (and for 0, inf, NaN) the plain
// division is used.
__device__ __forceinline__ double nr_rcp(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ cx<double> cplx_div(cx<double> a, cx<double> b) {
    const double inv = nr_rcp(b.re * b.re + b.im * b.im);
    return cx<double>{(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}
__device__ __forceinline__ bool finite_c(cx<double> a) { return isfinite(a.re) && isfinite(a.im); }

template <class R>
__global__ void __launch_bounds__(kPersThreads) k_persist_bicg(PersistArgs<R> a) {
    unsigned gen = 0;  // barriers this block has passed (the barrier starts zeroed)
    // Krylov scalars are computed once per CTA by thread 0 and broadcast (every CTA derives
    // the same values from the same grid sums); redundant FP64 divisions in all 16 warps
    // would queue on the FP64 pipe
    __shared__ double s_sc[8];
    const DevView<R> &v = a.v;
    const int d2 = v.d2;
    const int n0 = __ldg(v.pers_ado + blockIdx.x), n1 = __ldg(v.pers_ado + blockIdx.x + 1);
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_red = reinterpret_cast<double *>(smem);   // [32 warps][4]
    double *s_tot = s_red + 32 * 4;                     // [4]
    cx<R> *s_pinv = reinterpret_cast<cx<R> *>(s_tot + 4);
    ProgSmem<R> ps = prog_layout<R>(v.pers_terms, v.pers_slots, v.pers_ados, d2,
                                    reinterpret_cast<unsigned char *>(s_pinv + (size_t)v.pers_ados * d2));
    build_programs<R>(v, ps, n0, n1, a.aug, 0);
    const cx<R> shift = a.shift ? a.shift[0] : cx<R>{R(0), R(0)};
    const int items = (n1 - n0) * d2;
    const int64_t row0 = (int64_t)n0 * d2;
    // warps that hold elements (thread t takes items t, t + blockDim.x, ...)
    const int nw_act = max(1, min((int)(blockDim.x >> 5), (items + 31) >> 5));
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int pp = it / d2, e = it - pp * d2;
        const int64_t n = n0 + pp;
        s_pinv[it] = a.precond ? precond_inv(v, n, e, 0, damping_of(v, n, 0), shift)
                               : cx<R>{R(1), R(0)};
    }
    __syncthreads();

    // ---- r = b - A x, rh = r, p = v = 0
    double val2[2] = {0.0, 0.0};
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int64_t i = row0 + it;
        cx<R> ax{R(0), R(0)};
        if (!a.x_zero) ax = prog_apply(ps, it, a.x, shift);
        const cx<R> bi = a.b[i];
        const cx<R> ri = bi - ax;
        a.r[i] = ri;
        a.rh[i] = ri;
        a.p[i] = cx<R>{R(0), R(0)};
        a.vv[i] = cx<R>{R(0), R(0)};
        val2[0] += (double)norm2(ri);
        val2[1] += (double)norm2(bi);
    }
    if constexpr (sizeof(R) == 8) {
        // float-float programs for the iteration: fold the shift into every item's first
        // (damping) term, then split the coefficients in place (16 bytes either way)
        __syncthreads();
        if (a.shift)
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                cx<R> &c0 = ps.coef[ps.item[it]];
                c0 = c0 + shift;
            }
        __syncthreads();
        float4 *cf = reinterpret_cast<float4 *>(ps.coef);
        for (int t = threadIdx.x; t < ps.item[items]; t += blockDim.x) cf[t] = ff_split(ps.coef[t]);
        __syncthreads();
    }
    const bool started = grid_sum<2>(val2, a.part, 0, s_red, s_tot, a.bar, gen, nw_act, a.wait_cycles);
    double nr = val2[0];
    const double bn = val2[1], tol2 = a.tol * a.tol;
    cx<double> rho{nr, 0.0}, rho_old{1.0, 0.0}, alpha{1.0, 0.0}, omega{1.0, 0.0};
    int status = !started ? HEOM_ETIMEOUT : (nr <= tol2 * bn) ? 0 : -1, it_done = 0;
    double best = nr, rhn = nr;  // rhn = ||rh||^2
    int best_it = 0;
    for (int iter = 1; status < 0 && iter <= a.max_iter; ++iter) {
        // ---- restart when rh has become nearly orthogonal to r: rh = r, p = r;
        // beta = (rho / rho_old)(alpha / omega)
        if (threadIdx.x == 0) {
            const bool rs = iter > 1 && norm2(rho) < kRestartTau2 * rhn * nr;
            const cx<double> rr = rs ? cx<double>{nr, 0.0} : rho;
            const cx<double> bb = cplx_div(rr, rho_old) * cplx_div(alpha, omega);
            s_sc[0] = rs ? 1.0 : 0.0;
            s_sc[1] = bb.re;
            s_sc[2] = bb.im;
        }
        __syncthreads();
        const bool restart = s_sc[0] != 0.0;
        const cx<double> beta{s_sc[1], s_sc[2]};
        if (restart) {
            rho = cx<double>{nr, 0.0};
            rhn = nr;
        }
        // ---- p = r + beta (p - omega v), ph = P^-1 p
        const cx<R> bt = cast<R>(beta), om = cast<R>(omega);
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int64_t i = row0 + it;
            const cx<R> ri = a.r[i];
            const cx<R> pi = restart ? ri : ri + bt * (a.p[i] - om * a.vv[i]);
            if (restart) a.rh[i] = ri;
            a.p[i] = pi;
            const cx<R> phi = pi * s_pinv[it];
            a.ph[i] = phi;
            if constexpr (sizeof(R) == 8) a.phf[i] = ff_split(phi);
        }
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = HEOM_ETIMEOUT; break; }
        // ---- v = A ph, (rh, v)
        double d1[2] = {0.0, 0.0};
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int64_t i = row0 + it;
            cx<R> y;
            if constexpr (sizeof(R) == 8) y = prog_apply_ff(ps, it, a.phf);
            else y = prog_apply(ps, it, a.ph, shift);
            a.vv[i] = y;
            const cx<double> yd = cast<double>(y), wd = cast<double>(a.rh[i]);
            d1[0] += wd.re * yd.re + wd.im * yd.im;
            d1[1] += wd.re * yd.im - wd.im * yd.re;
        }
        if (!grid_sum<2>(d1, a.part, 1, s_red, s_tot, a.bar, gen, nw_act, a.wait_cycles)) { status = HEOM_ETIMEOUT; break; }
        const cx<double> rv{d1[0], d1[1]};
        if (norm2(rv) == 0.0) { status = HEOM_EBREAKDOWN; it_done = iter; break; }
        if (threadIdx.x == 0) {
            const cx<double> al0 = cplx_div(rho, rv);
            s_sc[3] = al0.re;
            s_sc[4] = al0.im;
        }
        __syncthreads();
        alpha = cx<double>{s_sc[3], s_sc[4]};
        // ---- s = r - alpha v (in r), sh = P^-1 s
        const cx<R> al = cast<R>(alpha);
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int64_t i = row0 + it;
            const cx<R> si = a.r[i] - al * a.vv[i];
            a.r[i] = si;
            const cx<R> shi = si * s_pinv[it];
            a.sh[i] = shi;
            if constexpr (sizeof(R) == 8) a.shf[i] = ff_split(shi);
        }
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = HEOM_ETIMEOUT; break; }
        // ---- t = A sh, (t, s), (t, t)
        double d2v[3] = {0.0, 0.0, 0.0};
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int64_t i = row0 + it;
            cx<R> y;
            if constexpr (sizeof(R) == 8) y = prog_apply_ff(ps, it, a.shf);
            else y = prog_apply(ps, it, a.sh, shift);
            a.t[i] = y;
            const cx<double> yd = cast<double>(y), wd = cast<double>(a.r[i]);
            d2v[0] += yd.re * wd.re + yd.im * wd.im;
            d2v[1] += yd.re * wd.im - yd.im * wd.re;
            d2v[2] += yd.re * yd.re + yd.im * yd.im;
        }
        if (!grid_sum<3>(d2v, a.part, 2, s_red, s_tot, a.bar, gen, nw_act, a.wait_cycles)) { status = HEOM_ETIMEOUT; break; }
        if (threadIdx.x == 0) {
            const double it2 = d2v[2] == 0.0 ? 0.0 : nr_rcp(d2v[2]);
            s_sc[5] = d2v[0] * it2;
            s_sc[6] = d2v[1] * it2;
        }
        __syncthreads();
        omega = cx<double>{s_sc[5], s_sc[6]};
        if (!finite_c(omega) || !finite_c(alpha)) { status = HEOM_EBREAKDOWN; it_done = iter; break; }
        // ---- x += alpha ph + omega sh, r = s - omega t, (rh, r), ||r||^2
        const cx<R> omr = cast<R>(omega);
        double d3[3] = {0.0, 0.0, 0.0};
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int64_t i = row0 + it;
            a.x[i] = a.x[i] + al * a.ph[i] + omr * a.sh[i];
            const cx<R> ri = a.r[i] - omr * a.t[i];
            a.r[i] = ri;
            const cx<double> rd = cast<double>(ri), hd = cast<double>(a.rh[i]);
            d3[0] += hd.re * rd.re + hd.im * rd.im;
            d3[1] += hd.re * rd.im - hd.im * rd.re;
            d3[2] += rd.re * rd.re + rd.im * rd.im;
        }
        if (!grid_sum<3>(d3, a.part, 3, s_red, s_tot, a.bar, gen, nw_act, a.wait_cycles)) { status = HEOM_ETIMEOUT; break; }
        rho_old = rho;
        rho = cx<double>{d3[0], d3[1]};
        nr = d3[2];
        it_done = iter;
        if (!isfinite(nr)) { status = HEOM_EBREAKDOWN; break; }
        if (nr <= tol2 * bn) { status = 0; break; }
        // no new minimum for stall_iters iterations: stalled (or diverging); the result is
        // usable if it still improved on the start. Single large transients (a near
        // breakdown just after a restart) are allowed: the recursion often recovers.
        if (nr < best) { best = nr; best_it = iter; }
        else if (iter - best_it >= a.stall_iters) {
            status = nr < bn ? HEOM_ENOCONV : HEOM_EBREAKDOWN;
            break;
        }
    }
    if (status < 0) status = HEOM_ENOCONV;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.out = PersistOut{it_done, status, nr, bn};
}

template <class R> DevView<R> view_of_p(const heom_hier *h);
template <> DevView<double> view_of_p<double>(const heom_hier *h) { return h->view64(); }
template <> DevView<float> view_of_p<float>(const heom_hier *h) { return h->view32(); }

template <class R>
size_t persist_smem(const DevView<R> &v) {
    return 32 * 4 * sizeof(double) + 4 * sizeof(double) + (size_t)v.pers_ados * v.d2 * sizeof(cx<R>) +
           prog_smem_bytes<R>(v.pers_terms, v.pers_slots, v.pers_ados, v.d2) + 64;
}

}  // namespace

template <class R>
bool persist_ok(const heom_hier *h) {
    if (h->pers_ranges < 1 || h->n_sets != 1 || h->has_caps) return false;
    const DevView<R> v = view_of_p<R>(h);
    return persist_smem(v) <= 200 * 1024;
}
template bool persist_ok<double>(const heom_hier *);
template bool persist_ok<float>(const heom_hier *);

// One persistent BiCGStab solve of (M + shift + aug e00 tr) x = b for a single column.
template <class R>
heom_status bicgstab_persistent(heom_hier *h, const cx<R> *b, cx<R> *x, bool x_zero,
                                const cx<R> *shift, R aug, double tol, int max_iter,
                                int stall_iters, int *iters, int *status, double *rel_res,
                                cudaStream_t s) {
    const DevView<R> v = view_of_p<R>(h);
    const int64_t rows = h->N * h->d2;
    const int G = h->pers_ranges;
    const size_t vec = ((size_t)rows * sizeof(cx<R>) + 255) & ~size_t(255);
    const size_t fvec = sizeof(R) == 8 ? (((size_t)rows * sizeof(float4) + 255) & ~size_t(255)) : 0;
    const size_t bytes = 7 * vec + 2 * fvec + (size_t)kSlots * G * 4 * sizeof(double) + 512;
    heom_status st = ensure_ws(h->ws_pers, bytes);
    if (st != HEOM_OK) return st;
    char *base = (char *)h->ws_pers.p;
    PersistArgs<R> a{};
    a.v = v;
    a.b = b;
    a.x = x;
    a.x_zero = x_zero ? 1 : 0;
    a.shift = shift;
    a.aug = aug;
    a.precond = 1;
    cx<R> **vecs[7] = {&a.r, &a.rh, &a.p, &a.vv, &a.ph, &a.sh, &a.t};
    for (int i = 0; i < 7; ++i) *vecs[i] = (cx<R> *)(base + i * vec);
    if (fvec) {
        a.phf = (float4 *)(base + 7 * vec);
        a.shf = (float4 *)(base + 7 * vec + fvec);
    }
    a.part = (double *)(base + 7 * vec + 2 * fvec);
    a.out = (PersistOut *)((char *)a.part + (size_t)kSlots * G * 4 * sizeof(double));
    a.bar = (GridBar *)((char *)a.out + 128);
    HEOM_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(GridBar), s));
    a.tol = tol;
    a.max_iter = max_iter;
    a.stall_iters = stall_iters;
    a.wait_cycles = wait_limit_cycles();
    if (x_zero) HEOM_CUDA(cudaMemsetAsync(x, 0, rows * sizeof(cx<R>), s));
    const size_t sm = persist_smem(v);
    HEOM_CUDA(cudaFuncSetAttribute(k_persist_bicg<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    void *args[] = {&a};
    {
        Prof pr(sizeof(R) == 4 ? HEOM_KC_KRYLOV_APPLY32 : HEOM_KC_KRYLOV_APPLY64, s, 0.0, 0.0);
        HEOM_CUDA(cudaLaunchCooperativeKernel((const void *)k_persist_bicg<R>, dim3(G), dim3(kPersThreads),
                                              args, sm, s));
    }
    PersistOut o{};
    HEOM_CUDA(memcpy_counted(&o, a.out, sizeof(o), cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    *iters = o.iterations;
    *status = o.status;
    *rel_res = o.bn > 0 ? std::sqrt(o.nr / o.bn) : 0.0;
    if (o.status == HEOM_ETIMEOUT)  // every CTA has left; the caller reports the column
        set_error("persistent BiCGStab: a grid-barrier wait ran out after %lld cycles",
                  (long long)a.wait_cycles);
    // launch accounting: two applies per iteration, ADO-applies as units
    prof_add(sizeof(R) == 4 ? HEOM_KC_KRYLOV_APPLY32 : HEOM_KC_KRYLOV_APPLY64,
             2.0 * o.iterations * (double)h->N, 2.0 * o.iterations * 3.0 * (double)rows * sizeof(cx<R>));
    return HEOM_OK;
}

template heom_status bicgstab_persistent<double>(heom_hier *, const cx<double> *, cx<double> *, bool,
                                                 const cx<double> *, double, double, int, int, int *,
                                                 int *, double *, cudaStream_t);
template heom_status bicgstab_persistent<float>(heom_hier *, const cx<float> *, cx<float> *, bool,
                                                const cx<float> *, float, double, int, int, int *,
                                                int *, double *, cudaStream_t);

}  // namespace heom
