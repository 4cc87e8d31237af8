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
    if (tile_ok(v, B)) {
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
    HEOM_CUDA(cudaSetDevice(h->device));
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
