// Shift-invariant Krylov solves for spectra (Methods, numerical computation of the
// spectrum): every frequency w of a density of states solves (M -+ i w) x = b with the same
// M and the same b, so all of them live in one Krylov space K_m(M, b). One FP64 Arnoldi
// process (classical Gram-Schmidt, reorthogonalised once) builds an orthonormal basis V and
// the Hessenberg matrix Hb with M V_m = V_{m+1} Hb_m; for each shift s the least-squares
// problem min || beta e_1 - (Hb_m + s I~) y || gives x_s = V_m y_s and its residual norm
// (GMRES on the shifted system; the shift leaves the basis unchanged). Only the tier-0 block
// of every x_s is formed, because the spectrum is a trace over it.
//
// Batch columns are independent Arnoldi processes (different right-hand sides, and
// different parameter sets when the hierarchy holds several); each has its own list of
// shifts. Everything per shift runs on the device: Givens rotations are applied one new
// Hessenberg column at a time (residual estimates every step) and the final triangular
// solve regenerates the columns of R from the rotations, so memory per shift is O(m).
#include <algorithm>
#include <cmath>
#include <vector>

#include "heom_tile.cuh"

namespace heom {
namespace {

constexpr int kDotThreads = 256;

// Partial dot products over a chunk of rows: part[c][i][b] = sum_{rows of chunk c}
// conj(V_i[row][b]) w[row][b]; grid (i, chunk). Deterministic (no atomics).
__global__ void __launch_bounds__(kDotThreads) k_multidot(int64_t rows, int64_t B, int nv,
                                                          const cx<double> *__restrict__ V,
                                                          int64_t vstride,
                                                          const cx<double> *__restrict__ w,
                                                          cx<double> *__restrict__ part) {
    const int i = blockIdx.x, c = blockIdx.y, nc = gridDim.y;
    const int64_t L = rows * B;
    const int64_t t0 = L * c / nc, t1 = L * (c + 1) / nc;
    const cx<double> *Vi = V + (int64_t)i * vstride;
    __shared__ double sre[kDotThreads], sim[kDotThreads];
    for (int64_t b = 0; b < B; ++b) {
        double re = 0.0, im = 0.0;
        // elements t of column b inside [t0, t1): t = row * B + b
        int64_t tb = t0 + ((b - t0 % B) + B) % B;
        for (int64_t t = tb + (int64_t)threadIdx.x * B; t < t1; t += (int64_t)blockDim.x * B) {
            const cx<double> a = Vi[t], x = w[t];
            re += a.re * x.re + a.im * x.im;
            im += a.re * x.im - a.im * x.re;
        }
        sre[threadIdx.x] = re;
        sim[threadIdx.x] = im;
        __syncthreads();
        for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                sre[threadIdx.x] += sre[threadIdx.x + s];
                sim[threadIdx.x] += sim[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) part[((int64_t)c * nv + i) * B + b] = cx<double>{sre[0], sim[0]};
        __syncthreads();
    }
}

// h[i][b] = sum_c part[c][i][b]; Hb[i][j][b] += h[i][b] (column j of the Hessenberg matrix
// accumulates both Gram-Schmidt passes)
__global__ void k_reduce_h(int nc, int nv, int64_t B, const cx<double> *__restrict__ part,
                           cx<double> *__restrict__ h, cx<double> *__restrict__ Hb, int j, int mmax) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nv * B;
         t += (int64_t)gridDim.x * blockDim.x) {
        cx<double> acc{0.0, 0.0};
        for (int c = 0; c < nc; ++c) acc = acc + part[(int64_t)c * nv * B + t];
        h[t] = acc;
        const int64_t i = t / B, b = t - i * B;
        cx<double> &e = Hb[(i * mmax + j) * B + b];
        e = e + acc;
    }
}

// w[row][b] -= sum_i V_i[row][b] h[i][b]
__global__ void k_gs_update(int64_t rows, int64_t B, int nv, const cx<double> *__restrict__ V,
                            int64_t vstride, const cx<double> *__restrict__ h,
                            cx<double> *__restrict__ w) {
    const int64_t total = rows * B;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t % B;
        cx<double> acc = w[t];
        for (int i = 0; i < nv; ++i) {
            const cx<double> hi = h[(int64_t)i * B + b];
            const cx<double> vi = V[(int64_t)i * vstride + t];
            acc.re -= vi.re * hi.re - vi.im * hi.im;
            acc.im -= vi.re * hi.im + vi.im * hi.re;
        }
        w[t] = acc;
    }
}

// Hb[j+1][j][b] = nrm[b]
__global__ void k_set_sub(cx<double> *__restrict__ Hb, int j, int mmax, int64_t B,
                          const double *__restrict__ nrm) {
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x)
        Hb[((int64_t)(j + 1) * mmax + j) * B + b] = cx<double>{nrm[b], 0.0};
}

// nrm[b] = ||w[:, b]|| (one block per column)
__global__ void __launch_bounds__(kDotThreads) k_colnorm(int64_t rows, int64_t B,
                                                         const cx<double> *__restrict__ w,
                                                         double *__restrict__ nrm) {
    const int64_t b = blockIdx.x;
    __shared__ double s[kDotThreads];
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += norm2(w[r * B + b]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) nrm[b] = std::sqrt(s[0]);
}

// out[row][b] = w[row][b] / nrm[b] (nrm = 0 leaves zeros: exact invariant subspace)
__global__ void k_scale_by(int64_t total, int64_t B, const cx<double> *__restrict__ w,
                           const double *__restrict__ nrm, cx<double> *__restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double n = nrm[t % B];
        out[t] = n > 0.0 ? (1.0 / n) * w[t] : cx<double>{0.0, 0.0};
    }
}

// Complex Givens rotation zeroing b in (a, b): [c s; -conj(s) c] with c real.
__device__ inline void givens(cx<double> a, cx<double> b, double &c, cx<double> &s, cx<double> &r) {
    const double na = std::sqrt(norm2(a)), nb = std::sqrt(norm2(b));
    if (nb == 0.0) { c = 1.0; s = {0.0, 0.0}; r = a; return; }
    if (na == 0.0) { c = 0.0; s = (1.0 / nb) * conj(b); r = cx<double>{nb, 0.0}; return; }
    const double nr = std::sqrt(na * na + nb * nb);
    const cx<double> ph = (1.0 / na) * a;  // a / |a|
    c = na / nr;
    s = (1.0 / nr) * (ph * conj(b));
    r = ph * cx<double>{nr, 0.0};
}

// Per (column b, shift k): apply the stored rotations to Hessenberg column j of the shifted
// matrix, make the new rotation, update g and the residual estimate |g_{j+1}| / beta.
// Hb: [mmax+1][mmax][B] (row i, column j, batch b). rot_c [S][mmax], rot_s [S][mmax],
// g [S][mmax+1], shift [S], col_of [S] (the batch column of shift k), res [S].
__global__ void k_shift_step(int j, int mmax, int64_t B, int64_t S, const cx<double> *__restrict__ Hb,
                             const cx<double> *__restrict__ shift, const int *__restrict__ col_of,
                             double *__restrict__ rot_c, cx<double> *__restrict__ rot_s,
                             cx<double> *__restrict__ g, const double *__restrict__ beta,
                             double *__restrict__ res) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const int64_t b = col_of[k];
    double *rc = rot_c + k * mmax;
    cx<double> *rs = rot_s + k * mmax;
    cx<double> *gk = g + k * (mmax + 1);
    // column j of Hb + shift * I~ ; apply rotations 0..j-1 on the fly
    cx<double> hj = Hb[((int64_t)0 * mmax + j) * B + b];
    if (j == 0) hj = hj + shift[k];
    for (int i = 0; i < j; ++i) {
        cx<double> hi1 = Hb[((int64_t)(i + 1) * mmax + j) * B + b];
        if (i + 1 == j) hi1 = hi1 + shift[k];
        const double c = rc[i];
        const cx<double> s = rs[i];
        // (hj, hi1) <- (c hj + s hi1, -conj(s) hj + c hi1): row i is final, row i+1 carries on
        hj = c * hi1 - conj(s) * hj;
    }
    const cx<double> hsub = Hb[((int64_t)(j + 1) * mmax + j) * B + b];
    double c;
    cx<double> s, r;
    givens(hj, hsub, c, s, r);
    rc[j] = c;
    rs[j] = s;
    const cx<double> gj = gk[j];
    gk[j] = c * gj;
    gk[j + 1] = cx<double>{0.0, 0.0} - conj(s) * gj;
    res[k] = std::sqrt(norm2(gk[j + 1])) / beta[b];
}

// Per shift: solve R y = g (column-oriented back substitution, columns of R regenerated
// from the rotations) for the first m Hessenberg columns and form the tier-0 block
// x0[e] = sum_l V_l[e][b] y_l, e < d2. Work arrays y [S][mmax] (scratch), x0 [S][d2].
__global__ void k_shift_solve(int m, int mmax, int64_t B, int64_t S, int d2,
                              const cx<double> *__restrict__ Hb, const cx<double> *__restrict__ shift,
                              const int *__restrict__ col_of, const double *__restrict__ rot_c,
                              const cx<double> *__restrict__ rot_s, const cx<double> *__restrict__ g,
                              cx<double> *__restrict__ gw, cx<double> *__restrict__ y,
                              cx<double> *__restrict__ colbuf, const cx<double> *__restrict__ V,
                              int64_t vstride, cx<double> *__restrict__ x0) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const int64_t b = col_of[k];
    const double *rc = rot_c + k * mmax;
    const cx<double> *rs = rot_s + k * mmax;
    cx<double> *gk = gw + k * (mmax + 1);
    cx<double> *yk = y + k * mmax;
    cx<double> *col = colbuf + k * (mmax + 1);
    for (int i = 0; i <= m; ++i) gk[i] = g[k * (mmax + 1) + i];
    for (int l = m - 1; l >= 0; --l) {
        // column l of R: rotations 0..l-1 applied to column l of Hb + shift I~
        for (int i = 0; i <= l + 1; ++i) {
            cx<double> v = Hb[((int64_t)i * mmax + l) * B + b];
            if (i == l) v = v + shift[k];
            col[i] = v;
        }
        for (int i = 0; i < l; ++i) {
            const double c = rc[i];
            const cx<double> s = rs[i];
            const cx<double> a0 = col[i], a1 = col[i + 1];
            col[i] = c * a0 + s * a1;
            col[i + 1] = c * a1 - conj(s) * a0;
        }
        {   // the diagonal entry after rotation l
            const double c = rc[l];
            const cx<double> s = rs[l];
            col[l] = c * col[l] + s * col[l + 1];
        }
        const cx<double> yl = cdiv(gk[l], col[l]);
        yk[l] = yl;
        for (int i = 0; i < l; ++i) gk[i] = gk[i] - col[i] * yl;
    }
    for (int e = 0; e < d2; ++e) {
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < m; ++l) fma_to(acc, V[(int64_t)l * vstride + (int64_t)e * B + b], yk[l]);
        x0[k * d2 + e] = acc;
    }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16); }

}  // namespace

// Shift-invariant GMRES for B right-hand sides (columns of bvec, [rows][B], FP64) with S
// shifts in total: shift k (value shift[k], host) belongs to column col_of[k]. Returns the
// tier-0 blocks x0 [S][d2] (host) and the residual estimates res [S] (host); the number of
// Arnoldi steps taken in *steps. Converged when every residual <= tol, else at mmax steps.
heom_status shifted_gmres(heom_hier *h, const cx<double> *bvec, int64_t B,
                          const std::vector<cx<double>> &shift, const std::vector<int> &col_of,
                          double tol, int mmax, std::vector<cx<double>> &x0,
                          std::vector<double> &res, int *steps, cudaStream_t s) {
    const int64_t rows = h->N * h->d2, L = rows * B, S = (int64_t)shift.size();
    const int d2 = h->d2;
    // device memory: basis V [mmax+1][L], w [L], Hb [mmax+1][mmax][B], h tmp [mmax+1][B],
    // norms [B], beta [B], per shift: rot_c, rot_s, g, gw, y, colbuf, x0, res, shift, col_of
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t oV = take((size_t)(mmax + 1) * L * 16), ow = take((size_t)L * 16),
                 oH = take((size_t)(mmax + 1) * mmax * B * 16), oh = take((size_t)(mmax + 1) * B * 16),
                 on = take((size_t)B * 8), obeta = take((size_t)B * 8),
                 orc = take((size_t)S * mmax * 8), ors = take((size_t)S * mmax * 16),
                 og = take((size_t)S * (mmax + 1) * 16), ogw = take((size_t)S * (mmax + 1) * 16),
                 oy = take((size_t)S * mmax * 16), ocb = take((size_t)S * (mmax + 1) * 16),
                 ox0 = take((size_t)S * d2 * 16), ores = take((size_t)S * 8),
                 osh = take((size_t)S * 16), oco = take((size_t)S * 4);
    // row chunks of the partial dot products: enough blocks to fill the GPU at small j
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, L / 4096));
    const size_t opart = take((size_t)nchunk * (mmax + 1) * B * 16);
    heom_status st = ensure_ws(h->ws, off);
    if (st != HEOM_OK) return st;
    char *base = (char *)h->ws.p;
    cx<double> *V = (cx<double> *)(base + oV), *w = (cx<double> *)(base + ow),
               *Hb = (cx<double> *)(base + oH), *ht = (cx<double> *)(base + oh);
    double *nrm = (double *)(base + on), *beta = (double *)(base + obeta);
    double *rot_c = (double *)(base + orc);
    cx<double> *rot_s = (cx<double> *)(base + ors), *g = (cx<double> *)(base + og),
               *gw = (cx<double> *)(base + ogw), *y = (cx<double> *)(base + oy),
               *cb = (cx<double> *)(base + ocb), *dx0 = (cx<double> *)(base + ox0),
               *dsh = (cx<double> *)(base + osh);
    double *dres = (double *)(base + ores);
    int *dco = (int *)(base + oco);
    cx<double> *part = (cx<double> *)(base + opart);
    HEOM_CUDA(memcpy_counted(dsh, shift.data(), S * 16, cudaMemcpyHostToDevice, s));
    HEOM_CUDA(memcpy_counted(dco, col_of.data(), S * 4, cudaMemcpyHostToDevice, s));
    HEOM_CUDA(cudaMemsetAsync(Hb, 0, (size_t)(mmax + 1) * mmax * B * 16, s));
    // v_0 = b / ||b||, g = (beta, 0, ...)
    {
        Prof pr(HEOM_KC_OTHER, s, (double)L, 2.0 * L * 16);
        k_colnorm<<<(unsigned)B, kDotThreads, 0, s>>>(rows, B, bvec, beta);
        k_scale_by<<<blocks_for(L), 256, 0, s>>>(L, B, bvec, beta, V);
    }
    std::vector<double> hbeta(B);
    HEOM_CUDA(memcpy_counted(hbeta.data(), beta, B * 8, cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    {
        std::vector<cx<double>> g0((size_t)S * (mmax + 1), cx<double>{0.0, 0.0});
        for (int64_t k = 0; k < S; ++k) g0[(size_t)k * (mmax + 1)] = cx<double>{hbeta[col_of[k]], 0.0};
        HEOM_CUDA(memcpy_counted(g, g0.data(), g0.size() * 16, cudaMemcpyHostToDevice, s));
    }
    const DevView<double> v = h->view64();
    const bool tiled = tile_ok(v, B);
    TileArgs<double> ta{};
    ta.v = v;
    ta.B = B;
    const Geom gapply = make_geom(rows, B, 1 << 30);
    std::vector<double> hres(S, 1.0);
    int m = 0, check = 5;
    for (int j = 0; j < mmax; ++j) {
        const cx<double> *vj = V + (int64_t)j * L;
        {   // w = M v_j
            Prof pr(HEOM_KC_KRYLOV_APPLY64, s, (double)h->N * B, 2.0 * L * 16);
            if (tiled) {
                ta.x = vj;
                ta.out = w;
                HEOM_CUDA((launch_tile<double, TM_STORE>(ta, s)));
            } else {
                ApplyMods<double> mods{nullptr, 0.0};
                HEOM_CUDA(launch_apply(v, vj, w, B, mods, s));
            }
        }
        {   // classical Gram-Schmidt, twice; Hb[:, j] accumulates both passes
            Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)(j + 1) * L, 2.0 * (2.0 * (j + 1) + 2.0) * L * 16);
            for (int pass = 0; pass < 2; ++pass) {
                k_multidot<<<dim3((unsigned)(j + 1), (unsigned)nchunk), kDotThreads, 0, s>>>(
                    rows, B, j + 1, V, L, w, part);
                k_reduce_h<<<blocks_for((int64_t)(j + 1) * B), 256, 0, s>>>(nchunk, j + 1, B, part, ht, Hb, j, mmax);
                k_gs_update<<<blocks_for(L), 256, 0, s>>>(rows, B, j + 1, V, L, ht, w);
            }
        }
        {   // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)L, 3.0 * L * 16);
            k_colnorm<<<(unsigned)B, kDotThreads, 0, s>>>(rows, B, w, nrm);
            k_scale_by<<<blocks_for(L), 256, 0, s>>>(L, B, w, nrm, V + (int64_t)(j + 1) * L);
            k_set_sub<<<1, 32, 0, s>>>(Hb, j, mmax, B, nrm);
            k_shift_step<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(j, mmax, B, S, Hb, dsh, dco, rot_c,
                                                                   rot_s, g, beta, dres);
        }
        HEOM_CUDA(cudaGetLastError());
        m = j + 1;
        if (m % check == 0 || m == mmax) {
            HEOM_CUDA(memcpy_counted(hres.data(), dres, S * 8, cudaMemcpyDeviceToHost, s));
            HEOM_CUDA(cudaStreamSynchronize(s));
            double worst = 0.0;
            for (double r : hres) worst = std::max(worst, std::isfinite(r) ? r : 1e300);
            if (worst <= tol) break;
            check = std::min(check + 5, 20);
        }
    }
    {
        Prof pr(HEOM_KC_OTHER, s, (double)S, (double)S * m * 16);
        k_shift_solve<<<(unsigned)((S + 63) / 64), 64, 0, s>>>(m, mmax, B, S, d2, Hb, dsh, dco, rot_c, rot_s,
                                                               g, gw, y, cb, V, L, dx0);
    }
    HEOM_CUDA(cudaGetLastError());
    x0.resize((size_t)S * d2);
    res.resize(S);
    HEOM_CUDA(memcpy_counted(x0.data(), dx0, (size_t)S * d2 * 16, cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(memcpy_counted(res.data(), dres, S * 8, cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    *steps = m;
    return HEOM_OK;
}

}  // namespace heom
