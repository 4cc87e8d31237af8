// The hot path: y = M x over all ADOs and batch columns (Eq. HEOM), matrix-free.
//
// Mapping: one thread per output element (ADO n, element e = r*d + c, column b). A block is
// (bx, by) threads with bx consecutive batch columns and by consecutive (n, e) rows, so a
// warp reads 32 consecutive columns of one row (batched solves, coalesced 256/512-byte
// segments) or 32 consecutive elements of neighbouring ADOs (batch 1). Every operand of an
// output element -- its own block, the blocks of its raised and lowered neighbours -- is
// read straight from global memory; re-reads of a block by its neighbours are served by L1
// and L2. Operators are applied through their sparse row/column lists, so the d_sigma of
// the fermionic baths cost one multiply-add per neighbour and side.
#include <algorithm>
#include <cstdint>

#include "heom_tile.cuh"

namespace heom {

Geom make_geom(int64_t rows, int64_t B, int max_blocks_x) {
    Geom g;
    int bx = 1;
    while (bx < B && bx < 32) bx <<= 1;
    int by = 256 / bx;
    g.block = dim3(bx, by, 1);
    int64_t gy = (B + bx - 1) / bx;
    int64_t gx = (rows + by - 1) / by;
    if (max_blocks_x > 0 && gx > max_blocks_x) gx = max_blocks_x;
    if (gx < 1) gx = 1;
    g.grid = dim3((unsigned)gx, (unsigned)gy, 1);
    g.rows = rows;
    g.B = B;
    return g;
}

template <class R>
__global__ void __launch_bounds__(256) k_apply(DevView<R> v, const cx<R> *__restrict__ x,
                                               cx<R> *__restrict__ y, int64_t B,
                                               int64_t cols_per_set, ApplyMods<R> mods) {
    const int64_t b = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t rows = v.N * v.d2;
    if (b >= B) return;
    const int set = (int)(b / cols_per_set);
    for (int64_t row = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; row < rows;
         row += (int64_t)gridDim.x * blockDim.y) {
        const int64_t n = row / v.d2;
        const int e = (int)(row - n * v.d2);
        const cx<R> damp = damping_of(v, n, set);
        cx<R> acc = apply_point(v, x, n, e, b, B, set, damp);
        if (mods.shift) fma_to(acc, mods.shift[b], x[row * B + b]);
        if (mods.aug != R(0) && row == 0) {
            cx<R> tr{R(0), R(0)};
            for (int i = 0; i < v.d; ++i) tr = tr + x[(int64_t)(i * v.d + i) * B + b];
            acc = acc + mods.aug * tr;
        }
        y[row * B + b] = acc;
    }
}

template <class R>
cudaError_t launch_apply(const DevView<R> &v, const cx<R> *x, cx<R> *y, int64_t B,
                         const ApplyMods<R> &mods, cudaStream_t s) {
    // the tiled kernel reads and writes 16-byte vectors: both buffers must be 16-byte aligned
    if (tile_ok(v, B) && (((uintptr_t)x | (uintptr_t)y) & 15) == 0) {
        TileArgs<R> a{};
        a.v = v;
        a.x = x;
        a.out = y;
        a.shift = mods.shift;
        a.aug = mods.aug;
        a.B = B;
        return launch_tile<R, TM_STORE>(a, s);
    }
    Geom g = make_geom(v.N * v.d2, B, 1 << 30);
    k_apply<R><<<g.grid, g.block, 0, s>>>(v, x, y, B, B / v.n_sets, mods);
    return cudaGetLastError();
}

template cudaError_t launch_apply<double>(const DevView<double> &, const cx<double> *,
                                          cx<double> *, int64_t, const ApplyMods<double> &,
                                          cudaStream_t);
template cudaError_t launch_apply<float>(const DevView<float> &, const cx<float> *, cx<float> *,
                                         int64_t, const ApplyMods<float> &, cudaStream_t);

}  // namespace heom

extern "C" heom_status heom_apply(const heom_hier *h, const void *x, void *y, int64_t batch,
                                  int prec, heom_stream s) {
    if (!h || !x || !y || batch < 1 || batch % h->n_sets != 0 ||
        (prec != HEOM_FP64 && prec != HEOM_FP32)) {
        heom::set_error("heom_apply: need a hierarchy, x, y, batch >= 1 (multiple of n_sets) and "
                        "prec FP64 or FP32");
        return HEOM_EINVAL;
    }
    if (batch > 65535LL * 32) {
        heom::set_error("heom_apply: batch larger than 2097120");
        return HEOM_EINVAL;
    }
    const size_t elt = prec == HEOM_FP64 ? 16 : 8;
    const size_t bytes = (size_t)h->N * h->d2 * batch * elt;
    const char *xs = (const char *)x, *ys = (const char *)y;
    if (xs < ys + bytes && ys < xs + bytes) {
        heom::set_error("heom_apply: x and y overlap");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    cudaError_t e;
    // accounted here, not in launch_apply: the solvers that call launch_apply account the
    // launch under their own kernel class
    heom::Prof pr(HEOM_KC_APPLY, (cudaStream_t)s, (double)h->N * batch, 2.0 * bytes);
    if (prec == HEOM_FP64) {
        heom::ApplyMods<double> m{nullptr, 0.0};
        e = heom::launch_apply(h->view64(), (const heom::cx<double> *)x, (heom::cx<double> *)y,
                               batch, m, (cudaStream_t)s);
    } else {
        heom::ApplyMods<float> m{nullptr, 0.0f};
        e = heom::launch_apply(h->view32(), (const heom::cx<float> *)x, (heom::cx<float> *)y,
                               batch, m, (cudaStream_t)s);
    }
    if (e != cudaSuccess) return heom::cuda_fail(e, "heom_apply launch");
    return HEOM_OK;
}

// ------------------------------------------------------------------ autotuner
namespace heom {
namespace {

// deterministic bounded input: re, im of x[i] from a 64-bit mix of i, in [-1, 1)
template <class R>
__global__ void k_tune_fill(int64_t total, cx<R> *x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9e3779b97f4a7c15ULL;
        z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ULL;
        z ^= z >> 29;
        const double a = (double)(z >> 40) * (1.0 / 8388608.0) - 1.0;
        const double b = (double)((z >> 16) & 0xffffffULL) * (1.0 / 8388608.0) - 1.0;
        x[i] = cx<R>{R(a), R(b)};
    }
}

// average device time of `reps` applies of the hierarchy's current configuration
template <class R>
heom_status tune_time(heom_hier *h, const cx<R> *x, cx<R> *y, int64_t B, cudaStream_t s, double *us) {
    const ApplyMods<R> m{nullptr, R(0)};
    auto view = [&]() {
        if constexpr (sizeof(R) == 8) return h->view64();
        else return h->view32();
    };
    const DevView<R> cur = view();
    cudaEvent_t e0, e1;
    HEOM_CUDA(cudaEventCreate(&e0));
    HEOM_CUDA(cudaEventCreate(&e1));
    const int reps = 5;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_apply(cur, x, y, B, m, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch_apply(cur, x, y, B, m, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "heom_autotune");
    *us = 1e3 * ms / reps;
    return HEOM_OK;
}

template <class R>
heom_status autotune(heom_hier *h, int64_t B, double *cand, int *tiled, int *per_sm, int *variant,
                     double *best, cudaStream_t s) {
    const int64_t total = h->N * h->d2 * B;
    DBuf buf;
    heom_status st = dalloc(buf, 2 * total * sizeof(cx<R>));
    if (st != HEOM_OK) return st;
    cx<R> *x = (cx<R> *)buf.p, *y = x + total;
    k_tune_fill<R><<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(total, x);
    const int per_sm0 = h->tile_per_sm, var0 = h->tile_var;
    const int64_t min_b0 = h->tile_min_b;
    // candidate 0: the per-element kernel (tiled kernel switched off)
    h->tile_min_b = INT64_MAX;
    double t0 = 0.0;
    st = tune_time<R>(h, x, y, B, s, &t0);
    cand[0] = t0;
    int best_p = 0, best_v = var0;
    double best_t = t0;
    // candidates 1..5: the tiled kernel with 1..5 ADO ranges per SM, each with every FP32
    // variant (FP64 has one); cand[p] keeps the fastest variant at p ranges per SM
    const bool tile_possible = B >= 16 && h->n_sets == 1 && !(sizeof(R) == 4 && (B & 1));
    const int n_var = sizeof(R) == 4 ? kTileVariants : 1;
    for (int p = 1; p <= 5 && st == HEOM_OK; ++p) {
        cand[p] = -1.0;
        if (!tile_possible) continue;
        if ((st = set_tile_partition(h, p)) != HEOM_OK) break;
        h->tile_min_b = 16;
        for (int var = 0; var < n_var && st == HEOM_OK; ++var) {
            h->tile_var = var;
            bool ok;
            if constexpr (sizeof(R) == 8) ok = tile_ok(h->view64(), B);
            else ok = tile_ok(h->view32(), B) && tile_var_of(h->view32(), B) == var;
            if (!ok) continue;  // ranges exceed the shared-memory budget, or B too narrow
            double t = 0.0;
            if ((st = tune_time<R>(h, x, y, B, s, &t)) != HEOM_OK) break;
            if (cand[p] < 0 || t < cand[p]) cand[p] = t;
            if (t < best_t) { best_t = t; best_p = p; best_v = var; }
        }
    }
    dfree(buf);
    if (st != HEOM_OK) {  // leave the configuration as it was
        set_tile_partition(h, per_sm0);
        h->tile_min_b = min_b0;
        h->tile_var = var0;
        return st;
    }
    // keep the winner: tiled with best_p ranges per SM and variant best_v, or the per-element
    // kernel for batches up to this width (wider batches keep the tiled kernel at its default
    // granularity)
    if (best_p > 0) {
        st = set_tile_partition(h, best_p);
        h->tile_min_b = 16;
        if (sizeof(R) == 4) h->tile_var = best_v;
    } else {
        st = set_tile_partition(h, per_sm0 > 0 ? per_sm0 : 2);
        h->tile_min_b = B + 1;
        h->tile_var = var0;
    }
    *tiled = best_p > 0;
    *per_sm = best_p;
    *variant = best_p > 0 ? (sizeof(R) == 4 ? best_v : 0) : -1;
    *best = best_t;
    return st;
}

}  // namespace
}  // namespace heom

extern "C" heom_status heom_autotune(heom_hier *h, int64_t batch, int prec, double *candidates_us,
                                     int *tiled, int *ctas_per_sm, double *best_us, int *variant,
                                     heom_stream s) {
    if (!h || batch < 1 || batch > 65535LL * 32 || (prec != HEOM_FP64 && prec != HEOM_FP32)) {
        heom::set_error("heom_autotune: need a hierarchy, 1 <= batch <= 2097120, prec FP64 or FP32");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    double cand[6], best = 0.0;
    int t = 0, p = 0, var = -1;
    const heom_status st = prec == HEOM_FP64
                               ? heom::autotune<double>(h, batch, cand, &t, &p, &var, &best, (cudaStream_t)s)
                               : heom::autotune<float>(h, batch, cand, &t, &p, &var, &best, (cudaStream_t)s);
    if (st != HEOM_OK) return st;
    if (candidates_us) for (int i = 0; i < 6; ++i) candidates_us[i] = cand[i];
    if (tiled) *tiled = t;
    if (ctas_per_sm) *ctas_per_sm = p;
    if (best_us) *best_us = best;
    if (variant) *variant = var;
    return HEOM_OK;
}

extern "C" heom_status heom_set_tile_config(heom_hier *h, int ctas_per_sm, int variant) {
    if (!h || ctas_per_sm < 1 || ctas_per_sm > 5 || variant < 0 ||
        variant >= heom::kTileVariants) {
        heom::set_error("heom_set_tile_config: need a hierarchy, 1 <= ctas_per_sm <= 5 and "
                        "0 <= variant < %d", heom::kTileVariants);
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    const heom_status st = heom::set_tile_partition(h, ctas_per_sm);
    if (st != HEOM_OK) return st;
    h->tile_var = variant;
    h->tile_min_b = 16;
    return HEOM_OK;
}
