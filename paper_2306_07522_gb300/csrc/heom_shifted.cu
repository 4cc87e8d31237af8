// Shift-invariant Krylov solves for spectra (Methods, numerical computation of the
// spectrum): every frequency w of a density of states solves (M -+ i w) x = b with the same
// M and the same b, so all of them live in one Krylov space K_m(M, b). One FP64 Arnoldi
// process (classical Gram-Schmidt, reorthogonalised when one pass loses too much) builds an
// orthonormal basis V and the Hessenberg matrix Hb with M V_m = V_{m+1} Hb_m; for each shift s the least-squares
// problem min || beta e_1 - (Hb_m + s I~) y || gives x_s = V_m y_s and its residual norm
// (GMRES on the shifted system; the shift leaves the basis unchanged). Only the tier-0 block
// of every x_s is formed, because the spectrum is a trace over it.
//
// Batch columns are independent Arnoldi processes (different right-hand sides, and
// different parameter sets when the hierarchy holds several); each has its own list of
// shifts. Everything per shift runs on the device: at every convergence check each shift's
// Givens QR takes in the Hessenberg columns added since the last one (residual estimates at
// the check), and the final triangular solve regenerates the columns of R from the
// rotations, so memory per shift is O(m).
#include <algorithm>
#include <cmath>
#include <vector>

#include "heom_ff.cuh"
#include "heom_tile.cuh"

namespace heom {
namespace {

constexpr int kDotThreads = 256;

// Work chunks of the float-float Gram-Schmidt kernels: rows row0 .. row1-1 of the [rows][B]
// vectors, whose columns 0 .. acols-1 can be nonzero (acols < B where parameter sets are
// truncated below the rows' ADOs, sets ordered deepest first; the other entries of every
// Krylov vector are zero and no Gram-Schmidt kernel reads or writes them). In a chunk the
// first T = (256 / acols) acols threads of a block each own one column, col = tid % acols,
// and rows row0 + tid / acols, stepping by 256 / acols: only active entries get threads.
struct GsChunk {
    int32_t row0, row1, acols, pad;
};

__device__ __forceinline__ bool chunk_lane(const GsChunk &ch, int &col, int &rstep, int64_t &row) {
    rstep = kDotThreads / ch.acols;
    col = threadIdx.x % ch.acols;
    row = ch.row0 + threadIdx.x / ch.acols;
    return (int)threadIdx.x < rstep * ch.acols;
}

// Hessenberg matrices of all columns, column-major: entry (i, j) of column b's matrix at
// Hb[(j (mmax + 1) + i) B + b], so that one Hessenberg column is contiguous.
__device__ __forceinline__ int64_t hb_at(int i, int j, int mmax, int64_t B, int64_t b) {
    return ((int64_t)j * (mmax + 1) + i) * B + b;
}

// Partial dot products over a chunk of rows: part[c][i][b] = sum_{rows of chunk c}
// conj(V_i[row][b]) w[row][b]; grid (i, chunk). Deterministic (no atomics). When B is a
// power of two dividing the block size every thread keeps one column and the chunk is read
// once for all columns; otherwise one sweep per column.
__global__ void __launch_bounds__(kDotThreads) k_multidot(int64_t rows, int64_t B, int nv,
                                                          const cx<double> *__restrict__ V,
                                                          int64_t vstride,
                                                          const cx<double> *__restrict__ w,
                                                          cx<double> *__restrict__ part,
                                                          const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x, c = blockIdx.y, nc = gridDim.y;
    const int64_t L = rows * B;
    const int64_t t0 = L * c / nc, t1 = L * (c + 1) / nc;
    const cx<double> *Vi = V + (int64_t)i * vstride;
    __shared__ double sre[kDotThreads], sim[kDotThreads];
    if (B <= kDotThreads && (kDotThreads % B) == 0) {
        // t0 rounded down to a multiple of B keeps column b = threadIdx.x % B for every t
        const int64_t tb = t0 - t0 % B;
        double re = 0.0, im = 0.0;
        for (int64_t t = tb + threadIdx.x; t < t1; t += kDotThreads) {
            if (t < t0) continue;
            const cx<double> a = Vi[t], x = w[t];
            re += a.re * x.re + a.im * x.im;
            im += a.re * x.im - a.im * x.re;
        }
        sre[threadIdx.x] = re;
        sim[threadIdx.x] = im;
        __syncthreads();
        for (int s = kDotThreads >> 1; s >= B; s >>= 1) {
            if (threadIdx.x < s) {
                sre[threadIdx.x] += sre[threadIdx.x + s];
                sim[threadIdx.x] += sim[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x < B) part[((int64_t)c * nv + i) * B + threadIdx.x] = cx<double>{sre[threadIdx.x], sim[threadIdx.x]};
        return;
    }
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

// wf[t] = split(w[t])
__global__ void k_split(int64_t total, const cx<double> *__restrict__ w, float4 *__restrict__ wf) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        wf[t] = ff_split(w[t]);
}

// wf = split(w) on the active entries of the chunks (blocks stride over the chunks)
__global__ void __launch_bounds__(kDotThreads) k_split_chunks(int64_t B, const cx<double> *__restrict__ w,
                                                              float4 *__restrict__ wf,
                                                              const GsChunk *__restrict__ chunks, int nch) {
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const GsChunk ch = chunks[c];
        int col, rstep;
        int64_t row;
        if (!chunk_lane(ch, col, rstep, row)) continue;
        for (; row < ch.row1; row += rstep) {
            const int64_t t = row * B + col;
            wf[t] = ff_split(w[t]);
        }
    }
}

// Float-float partial dot products over a chunk: part[c][i][b] = sum_{rows of chunk c}
// conj(V_i[row][b]) w[row][b] (FP64 result; zero for the chunk's inactive columns), the basis
// vectors taken kMdTile at a time: block (tile, chunk) reads its chunk of w once for the
// tile's basis vectors, with one float-float accumulator pair per basis vector; the tile's
// loads of an element are independent, so they are in flight together. Every thread sums its
// own column's entries in a fixed order, and the per-column sum over the threads runs in a
// fixed order too: the result is deterministic.
constexpr int kMdTile = 8;
__global__ void __launch_bounds__(kDotThreads) k_multidot_ff_tiled(int64_t B, int nv,
                                                                   const float4 *__restrict__ Vf,
                                                                   int64_t vstride,
                                                                   const float4 *__restrict__ wf,
                                                                   cx<double> *__restrict__ part,
                                                                   const int *__restrict__ skip,
                                                                   const GsChunk *__restrict__ chunks) {
    if (skip && *skip) return;
    const int i0 = blockIdx.x * kMdTile, c = blockIdx.y;
    const int nt = min(kMdTile, nv - i0);
    const GsChunk ch = chunks[c];
    __shared__ double sre[kMdTile][kDotThreads], sim[kMdTile][kDotThreads];
    float rh[kMdTile], rl[kMdTile], ih[kMdTile], il[kMdTile];
#pragma unroll
    for (int k = 0; k < kMdTile; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.f;
    const float4 *V0 = Vf + (int64_t)i0 * vstride;
    int col, rstep;
    int64_t row;
    if (chunk_lane(ch, col, rstep, row)) {
        for (; row < ch.row1; row += rstep) {
            const int64_t t = row * B + col;
            const float4 x = wf[t];
            float4 a[kMdTile];
#pragma unroll
            for (int k = 0; k < kMdTile; ++k)
                if (k < nt) a[k] = V0[(int64_t)k * vstride + t];
#pragma unroll
            for (int k = 0; k < kMdTile; ++k) {
                if (k < nt) {  // conj(a) x
                    ff_mac(rh[k], rl[k], a[k].x, a[k].z, x.x, x.z);
                    ff_mac(rh[k], rl[k], a[k].y, a[k].w, x.y, x.w);
                    ff_mac(ih[k], il[k], a[k].x, a[k].z, x.y, x.w);
                    ff_mac(ih[k], il[k], -a[k].y, -a[k].w, x.x, x.z);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kMdTile; ++k) {
        sre[k][threadIdx.x] = (double)rh[k] + (double)rl[k];
        sim[k][threadIdx.x] = (double)ih[k] + (double)il[k];
    }
    __syncthreads();
    if (threadIdx.x < B) {
        const int per = kDotThreads / ch.acols;
        for (int k = 0; k < nt; ++k) {
            double re = 0.0, im = 0.0;
            if ((int)threadIdx.x < ch.acols)
                for (int q = 0; q < per; ++q) {
                    re += sre[k][threadIdx.x + q * ch.acols];
                    im += sim[k][threadIdx.x + q * ch.acols];
                }
            part[((int64_t)c * nv + i0 + k) * B + threadIdx.x] = cx<double>{re, im};
        }
    }
}

// wf[row][b] -= sum_i V_i[row][b] h_i[b] in float-float (hf = split h), on the active
// entries of the chunks (blocks stride over the chunks)
__global__ void __launch_bounds__(kDotThreads) k_gs_update_ff(int64_t B, int nv, const float4 *__restrict__ Vf,
                                                              int64_t vstride, const float4 *__restrict__ hf,
                                                              float4 *__restrict__ wf, const int *__restrict__ skip,
                                                              const GsChunk *__restrict__ chunks, int nch) {
    if (skip && *skip) return;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const GsChunk ch = chunks[c];
        int col, rstep;
        int64_t row;
        if (!chunk_lane(ch, col, rstep, row)) continue;
        for (; row < ch.row1; row += rstep) {
            const int64_t t = row * B + col;
            const float4 w0 = wf[t];
            float rh = w0.x, rl = w0.z, ih = w0.y, il = w0.w;
            for (int i = 0; i < nv; ++i) {
                const float4 h = hf[(int64_t)i * B + col];
                const float4 v = Vf[(int64_t)i * vstride + t];
                // -= v h: re -= v.re h.re - v.im h.im, im -= v.re h.im + v.im h.re
                ff_mac(rh, rl, -v.x, -v.z, h.x, h.z);
                ff_mac(rh, rl, v.y, v.w, h.y, h.w);
                ff_mac(ih, il, -v.x, -v.z, h.y, h.w);
                ff_mac(ih, il, -v.y, -v.w, h.x, h.z);
            }
            ff_norm(rh, rl);
            ff_norm(ih, il);
            wf[t] = make_float4(rh, ih, rl, il);
        }
    }
}

// Partial squared column norms (FP64) of a float-float vector over a chunk: part[c][b];
// grid (chunk, b); zero for the chunk's inactive columns.
__global__ void __launch_bounds__(kDotThreads) k_colnorm_part_ff(int64_t B, const float4 *__restrict__ wf,
                                                                 double *__restrict__ part,
                                                                 const GsChunk *__restrict__ chunks) {
    const int c = blockIdx.x;
    const int64_t b = blockIdx.y;
    const GsChunk ch = chunks[c];
    __shared__ double sh[kDotThreads];
    double acc = 0.0;
    if (b < ch.acols)
        for (int64_t r = ch.row0 + threadIdx.x; r < ch.row1; r += blockDim.x) acc += norm2(ff_join(wf[r * B + b]));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)c * B + b] = sh[0];
}

// v = w / nrm[b] in FP64 (for the FP64 apply; skipped when v is null) and its float-float
// split (for Gram-Schmidt and the float-float apply); in place on wf, on the active entries of the chunks (the others stay zero in v). nrm = 0
// leaves zeros (exact invariant subspace).
__global__ void __launch_bounds__(kDotThreads) k_scale_ff(int64_t B, float4 *__restrict__ wf,
                                                          const double *__restrict__ nrm,
                                                          cx<double> *__restrict__ v,
                                                          const GsChunk *__restrict__ chunks, int nch) {
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const GsChunk ch = chunks[c];
        int col, rstep;
        int64_t row;
        if (!chunk_lane(ch, col, rstep, row)) continue;
        const double n = nrm[col];
        for (; row < ch.row1; row += rstep) {
            const int64_t t = row * B + col;
            const cx<double> x = n > 0.0 ? (1.0 / n) * ff_join(wf[t]) : cx<double>{0.0, 0.0};
            if (v) v[t] = x;
            wf[t] = ff_split(x);
        }
    }
}

// ---------------------------------------------------------------- float-float apply
// (H, L) += c x for float-float complex c, x ({hi.re, hi.im, lo.re, lo.im}):
// (re, im) += (c.re, c.re) (x.re, x.im) + (c.im, c.im) (-x.im, x.re) in packed pairs.
__device__ __forceinline__ void cmac_ff(float2 &H, float2 &L, float4 c, float4 x) {
    ff2_mac(H, L, make_float2(c.x, c.x), make_float2(c.z, c.z), make_float2(x.x, x.y), make_float2(x.z, x.w),
            make_float2(-x.x, -x.y));
    ff2_mac(H, L, make_float2(c.y, c.y), make_float2(c.w, c.w), make_float2(-x.y, x.x), make_float2(-x.w, x.z),
            make_float2(x.y, -x.x));
}
__device__ __forceinline__ float4 ff_pack(float2 H, float2 L) {
    float rh = H.x, rl = L.x, ih = H.y, il = L.y;
    ff_norm(rh, rl);
    ff_norm(ih, il);
    return make_float4(rh, ih, rl, il);
}
// c x for float-float complex values
__device__ __forceinline__ float4 cmul_ff(float4 c, float4 x) {
    float2 H = make_float2(0.f, 0.f), L = H;
    cmac_ff(H, L, c, x);
    return ff_pack(H, L);
}
// -i m a for a float-float complex a and a small integer m: (m a.im, -m a.re)
__device__ __forceinline__ float4 mul_mi_ff(float m, float4 a) {
    float rh = a.y, rl = a.w, ih = -a.x, il = -a.z;
    ff_scale(rh, rl, m, 0.f);
    ff_scale(ih, il, m, 0.f);
    return make_float4(rh, ih, rl, il);
}

// Y = M X in float-float for batched columns of several parameter sets (column b belongs to
// set set_of[b]): Eq. HEOM at every (ADO n, element e, column b), the terms in the order of the
// per-element FP64 apply, every product a float-float one (unit roundoff 2^-48 instead of
// FP64's 2^-53, at FP32 issue rates). An ADO beyond its column's set truncation is written
// as zero, and neighbours beyond it are skipped (their entries are zero). A thread takes CPT
// adjacent columns of one parameter set (set_of equal on each aligned CPT columns), so the decoding of the
// neighbour entries and every coefficient product serve all of them; operator values of +-1
// (fermionic annihilators with their Jordan-Wigner signs) skip the coefficient product.
template <int CPT>
__global__ void __launch_bounds__(256, 3) k_apply_ff(DevView<double> v, const float4 *__restrict__ X,
                                                     float4 *__restrict__ Y, int64_t B,
                                                     const int *__restrict__ set_of) {
    const int d = v.d, d2 = v.d2;
    const int64_t BT = B / CPT, total = v.N * d2 * BT;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / BT, b = (t - row * BT) * CPT, n = row / d2;
        const int e = (int)(row - n * d2), set = set_of[b];
        float4 *Yo = Y + row * B + b;
        if (beyond_cap(v, n, set)) {
#pragma unroll
            for (int u = 0; u < CPT; ++u) Yo[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const int cap = v.set_cap ? v.set_cap[set] : 0x7fffffff;
        const int r = e / d, c = e - r * d;
        const float4 *Xn = X + n * d2 * B + b;
        float2 H[CPT], L[CPT];
#pragma unroll
        for (int u = 0; u < CPT; ++u) H[u] = L[u] = make_float2(0.f, 0.f);
        {   // damping: -sum_k count_k rate_k x
            float2 DH = make_float2(0.f, 0.f), DL = DH;
            const int o1 = __ldg(v.occ_ptr + n + 1);
            for (int o = __ldg(v.occ_ptr + n); o < o1; ++o) {
                const int packed = __ldg(reinterpret_cast<const int *>(v.occ) + o);
                const int k = (int)(int16_t)(packed & 0xffff);
                const float cnt = (float)(int16_t)(packed >> 16);
                const float4 rt = v.ratef[(int64_t)set * v.K + k];
                ff2_mac(DH, DL, make_float2(cnt, cnt), make_float2(0.f, 0.f), make_float2(rt.x, rt.y),
                        make_float2(rt.z, rt.w), make_float2(-rt.x, -rt.y));
            }
            const float4 dm = ff_pack(DH, DL), ndm = make_float4(-dm.x, -dm.y, -dm.z, -dm.w);
#pragma unroll
            for (int u = 0; u < CPT; ++u) cmac_ff(H[u], L[u], ndm, Xn[(int64_t)e * B + u]);
        }
        const float4 *sv = v.s_valf + (int64_t)set * v.nS;
        for (int j = __ldg(v.s_ptr + e), j1 = __ldg(v.s_ptr + e + 1); j < j1; ++j) {
            const float4 cv = sv[j];
            const float4 *xs = Xn + (int64_t)__ldg(v.s_src + j) * B;
#pragma unroll
            for (int u = 0; u < CPT; ++u) cmac_ff(H[u], L[u], cv, xs[u]);
        }
        const int t1 = __ldg(v.row_ptr + n + 1);
        for (int q = __ldg(v.row_ptr + n); q < t1; ++q) {
            const int4 raw = __ldg(reinterpret_cast<const int4 *>(v.ent) + q);
            const int nb = raw.x;
            if (v.set_cap) {  // neighbours beyond the set's tiers are not in its hierarchy
                const int tn = __ldg(v.ado_tier + nb);
                if ((tn & 0xffff) > (cap & 0xffff) || (tn >> 16) > (cap >> 16)) continue;
            }
            const int op = (int)(int16_t)(raw.y & 0xffff);
            const int k = (int)(int16_t)(raw.y >> 16);
            const int dir = (int)(int16_t)(raw.z & 0xffff);
            const float ml = (float)(int16_t)(raw.z >> 16);
            const float mr = (float)(int16_t)(raw.w & 0xffff);
            float4 cl, cr;  // -i * mult * (a | b)
            if (dir > 0) {
                cl = make_float4(0.f, -ml, 0.f, 0.f);
                cr = make_float4(0.f, -mr, 0.f, 0.f);
            } else {
                const int64_t pk = (int64_t)set * v.K + k;
                cl = mul_mi_ff(ml, v.coefLf[pk]);
                cr = mul_mi_ff(mr, v.coefRf[pk]);
            }
            const float4 *Xb = X + (int64_t)nb * d2 * B + b;
            const int base = op * (d + 1);
            for (int j = __ldg(v.op_rptr + base + r), j1 = __ldg(v.op_rptr + base + r + 1); j < j1; ++j) {
                const float4 ov = v.op_rvalf[j];
                const float4 cf = ov.y == 0.f && ov.z == 0.f && ov.w == 0.f && (ov.x == 1.f || ov.x == -1.f)
                                      ? make_float4(ov.x * cl.x, ov.x * cl.y, ov.x * cl.z, ov.x * cl.w)
                                      : cmul_ff(cl, ov);
                const float4 *xs = Xb + (int64_t)(__ldg(v.op_rcol + j) * d + c) * B;
#pragma unroll
                for (int u = 0; u < CPT; ++u) cmac_ff(H[u], L[u], cf, xs[u]);
            }
            for (int j = __ldg(v.op_cptr + base + c), j1 = __ldg(v.op_cptr + base + c + 1); j < j1; ++j) {
                const float4 ov = v.op_cvalf[j];
                const float4 cf = ov.y == 0.f && ov.z == 0.f && ov.w == 0.f && (ov.x == 1.f || ov.x == -1.f)
                                      ? make_float4(ov.x * cr.x, ov.x * cr.y, ov.x * cr.z, ov.x * cr.w)
                                      : cmul_ff(cr, ov);
                const float4 *xs = Xb + (int64_t)(r * d + __ldg(v.op_crow + j)) * B;
#pragma unroll
                for (int u = 0; u < CPT; ++u) cmac_ff(H[u], L[u], cf, xs[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < CPT; ++u) Yo[u] = ff_pack(H[u], L[u]);
    }
}

// ---------------------------------------------------------------- delayed reorthogonalisation
// Arnoldi with classical Gram-Schmidt reorthogonalised one step late (DCGS2: Swirydowicz,
// Langou, Thomas, Yamazaki, "Low synchronization Gram-Schmidt and GMRES algorithms", 2020),
// per batch column. After step j-1 the slots hold q_0 .. q_{j-1} (final, orthonormal) and
// p_j, the new vector after one projection and not normalised: M q_{j-1} = Q_j h' + p_j with
// h' = Hb(0..j-1, j-1) provisional. Step j applies M to p_j (z = M p_j) and then, with ONE
// read of the basis for the dot products and one for the update:
//   a = Q_j^H p_j, c = Q_j^H z, e = p_j^H z, f = p_j^H p_j         (k_dots2_ff_tiled)
//   sigma = sqrt(f - |a|^2), q_j = (p_j - Q_j a) / sigma            (p_j = Q_j a + sigma q_j)
//   Hb(0..j-1, j-1) += a, Hb(j, j-1) = sigma                        (column j-1 final)
//   t = Q_{j+1}^H z = (c, (e - a^H c) / sigma)
//   Hb(0..j, j) = (t - Hb(0..j, 0..j-1) a) / sigma                   (M q_j = (z - M Q_j a) / sigma)
//   p_{j+1} = (z - Q_{j+1} t) / sigma                               (k_update2_ff)
// so every vector is projected out twice, as in two-pass classical Gram-Schmidt, at the
// memory traffic of one pass, and no separate normalisation pass is needed (sigma of the next
// step is the subdiagonal entry); column j of Hb becomes final one step later. q_0 = p_0 =
// b / beta exactly (step 0 takes sigma = 1).

// part[c][i][r][b] = sum over chunk c of conj(V_i) x_r for x_0 = p (= slot nv - 1 of the
// basis) and x_1 = z: the two dot-product sets of one step in one read of the basis, tiled
// kD2Tile basis vectors per block as in k_multidot_ff_tiled (deterministic, per-column fixed
// order, zero for the chunk's inactive columns).
constexpr int kD2Tile = 6;
__global__ void __launch_bounds__(kDotThreads, 2) k_dots2_ff_tiled(int64_t B, int nv, const float4 *__restrict__ Vf,
                                                                int64_t vstride, const float4 *__restrict__ zf,
                                                                cx<double> *__restrict__ part,
                                                                const GsChunk *__restrict__ chunks) {
    const int i0 = blockIdx.x * kD2Tile, c = blockIdx.y;
    const int nt = min(kD2Tile, nv - i0);
    const GsChunk ch = chunks[c];
    const float4 *pf = Vf + (int64_t)(nv - 1) * vstride;
    __shared__ double sre[kD2Tile][kDotThreads], sim[kD2Tile][kDotThreads];
    // accumulators of <V_k, x_r> as packed (re, im) pairs: high and low words
    float2 H[kD2Tile][2], L[kD2Tile][2];
#pragma unroll
    for (int k = 0; k < kD2Tile; ++k)
#pragma unroll
        for (int r = 0; r < 2; ++r) H[k][r] = L[k][r] = make_float2(0.f, 0.f);
    const float4 *V0 = Vf + (int64_t)i0 * vstride;
    int col, rstep;
    int64_t row;
    if (chunk_lane(ch, col, rstep, row)) {
        for (; row < ch.row1; row += rstep) {
            const int64_t t = row * B + col;
            // conj(a) x = a.re (x.re, x.im) + a.im (x.im, -x.re): the two packed products
            float2 XH[2], XL[2], nXH[2], YH[2], YL[2], nYH[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float4 x = r ? zf[t] : pf[t];
                XH[r] = make_float2(x.x, x.y);
                XL[r] = make_float2(x.z, x.w);
                nXH[r] = make_float2(-x.x, -x.y);
                YH[r] = make_float2(x.y, -x.x);
                YL[r] = make_float2(x.w, -x.z);
                nYH[r] = make_float2(-x.y, x.x);
            }
            float4 a[kD2Tile];
#pragma unroll
            for (int k = 0; k < kD2Tile; ++k)
                if (k < nt) a[k] = V0[(int64_t)k * vstride + t];
#pragma unroll
            for (int k = 0; k < kD2Tile; ++k) {
                if (k < nt) {
                    const float2 ARh = make_float2(a[k].x, a[k].x), ARl = make_float2(a[k].z, a[k].z);
                    const float2 AIh = make_float2(a[k].y, a[k].y), AIl = make_float2(a[k].w, a[k].w);
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        ff2_mac(H[k][r], L[k][r], ARh, ARl, XH[r], XL[r], nXH[r]);
                        ff2_mac(H[k][r], L[k][r], AIh, AIl, YH[r], YL[r], nYH[r]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r) __syncthreads();
#pragma unroll
        for (int k = 0; k < kD2Tile; ++k) {
            sre[k][threadIdx.x] = (double)H[k][r].x + (double)L[k][r].x;
            sim[k][threadIdx.x] = (double)H[k][r].y + (double)L[k][r].y;
        }
        __syncthreads();
        if (threadIdx.x < B) {
            const int per = kDotThreads / ch.acols;
            for (int k = 0; k < nt; ++k) {
                double re = 0.0, im = 0.0;
                if ((int)threadIdx.x < ch.acols)
                    for (int q = 0; q < per; ++q) {
                        re += sre[k][threadIdx.x + q * ch.acols];
                        im += sim[k][threadIdx.x + q * ch.acols];
                    }
                part[(((int64_t)c * nv + i0 + k) * 2 + r) * B + threadIdx.x] = cx<double>{re, im};
            }
        }
    }
}

// D[i][r][b] = sum_c part[c][i][r][b]
__global__ void k_reduce_dots2(int nc, int nv, int64_t B, const cx<double> *__restrict__ part,
                               cx<double> *__restrict__ D) {
    const int64_t n = (int64_t)nv * 2 * B;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        cx<double> acc{0.0, 0.0};
        for (int c = 0; c < nc; ++c) acc = acc + part[(int64_t)c * n + t];
        D[t] = acc;
    }
}

// The scalars of step j for column b = blockIdx.x (see the comment above): sigma, the final
// column j-1 and the provisional column j of Hb, and the update's coefficients: cfa[i][b] =
// a_i (FP32: the correction Q_j a is at the level of the lost orthogonality, so its FP32
// error is far below float-float rounding; as two packed pairs), cft[i][b] = t_i (float-float,
// i <= j; three float4 in the form the packed update takes), rsig[b] = 1 / sigma (float-float;
// 0 when p_j lies in span(Q_j): the columns from there on are zero).
__global__ void __launch_bounds__(256) k_dcgs_coef(int j, int mmax, int64_t B, const cx<double> *__restrict__ D,
                                                   cx<double> *__restrict__ Hb, float4 *__restrict__ cfa,
                                                   float4 *__restrict__ cft, float2 *__restrict__ rsig) {
    const int64_t b = blockIdx.x;
    __shared__ double s_aa[256], s_re[256], s_im[256];
    __shared__ double s_sig, s_inv, s_nu;
    __shared__ cx<double> s_tj;
    auto Da = [&](int i) { return D[((int64_t)i * 2 + 0) * B + b]; };
    auto Dc = [&](int i) { return D[((int64_t)i * 2 + 1) * B + b]; };
    double aa = 0.0, re = 0.0, im = 0.0;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const cx<double> a = Da(i), c = Dc(i);
        aa += norm2(a);
        re += a.re * c.re + a.im * c.im;  // conj(a) c
        im += a.re * c.im - a.im * c.re;
    }
    s_aa[threadIdx.x] = aa;
    s_re[threadIdx.x] = re;
    s_im[threadIdx.x] = im;
    __syncthreads();
    for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            s_aa[threadIdx.x] += s_aa[threadIdx.x + k];
            s_re[threadIdx.x] += s_re[threadIdx.x + k];
            s_im[threadIdx.x] += s_im[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double sig = 1.0;
        if (j > 0) {
            const double s2 = Da(j).re - s_aa[0];
            sig = s2 > 0.0 ? std::sqrt(s2) : 0.0;
        }
        const double inv = sig > 0.0 ? 1.0 / sig : 0.0;
        const cx<double> e = Dc(j);
        s_sig = sig;
        s_inv = inv;
        s_nu = j > 0 ? 1.0 : 0.0;  // p_j is the previous step's w itself, not normalised
        s_tj = inv * cx<double>{e.re - s_re[0], e.im - s_im[0]};
        const float h = (float)inv;
        rsig[b] = make_float2(h, (float)(inv - (double)h));
    }
    __syncthreads();
    const double sig = s_sig, inv = s_inv, nu = s_nu;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        // row i of Hb(0..j, 0..j-1) a, with column j-1 corrected first
        cx<double> acc{0.0, 0.0};
        for (int k = i > 0 ? i - 1 : 0; k < j - 1; ++k) acc = acc + Hb[hb_at(i, k, mmax, B, b)] * Da(k);
        if (j > 0) {
            cx<double> hc;
            if (i < j) {
                hc = Hb[hb_at(i, j - 1, mmax, B, b)] + nu * Da(i);
            } else {
                hc = cx<double>{nu * sig, 0.0};
            }
            Hb[hb_at(i, j - 1, mmax, B, b)] = hc;
            acc = acc + hc * Da(j - 1);
        }
        const cx<double> ti = i < j ? Dc(i) : s_tj;
        Hb[hb_at(i, j, mmax, B, b)] = inv * (ti - acc);
        // w -= v t as w += (v.re, v.re) * B1 + (v.im, v.im) * B2 with B1 = -t and
        // B2 = (t.im, -t.re), high and low words, and the negated high words
        const float4 f = ff_split(ti);
        float4 *rec = cft + ((int64_t)i * B + b) * 3;
        rec[0] = make_float4(-f.x, -f.y, -f.z, -f.w);
        rec[1] = make_float4(f.y, -f.x, f.w, -f.z);
        rec[2] = make_float4(f.x, f.y, -f.y, f.x);
        if (i < j) {  // Q a as (v.re, v.re) * (a.re, a.im) + (v.im, v.im) * (-a.im, a.re)
            const cx<double> a = Da(i);
            cfa[(int64_t)i * B + b] = make_float4((float)a.re, (float)a.im, -(float)a.im, (float)a.re);
        }
    }
}

// 16-byte asynchronous global -> shared copies (each thread copies and later reads only its
// own slots, so completion of its own groups is all the ordering it needs)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The update of step j on the active entries (blocks stride over the chunks): slot j of the
// basis turns from p_j into q_j = (p_j - Q_j a) / sigma (float-float; FP64 in its first
// q64_rows rows, the rows the solution is formed from), slot j + 1 from z into
// w = (z - Q_j t - q_j t_j) / sigma (float-float), which is p_{j+1} as it stands: it is not
// normalised (the next step's sigma is the exact subdiagonal entry). A thread takes kUpRows of its
// rows at a time, so each coefficient record it loads serves them all, and streams their
// basis entries through a per-thread ring of kUpDepth stages in shared memory filled by
// asynchronous copies, so kUpDepth x kUpRows loads are in flight while it computes; the
// multiply-adds run on packed (re, im) pairs.
constexpr int kUpRows = 4, kUpDepth = 4;
constexpr size_t kUpSmem = (size_t)kUpDepth * kUpRows * kDotThreads * sizeof(float4);
__global__ void __launch_bounds__(kDotThreads, 2) k_update2_ff(int64_t B, int j, float4 *__restrict__ Vf,
                                                            int64_t vstride, cx<double> *__restrict__ q64,
                                                            int64_t q64_rows,
                                                            const float4 *__restrict__ cfa,
                                                            const float4 *__restrict__ cft,
                                                            const float2 *__restrict__ rsig,
                                                            const GsChunk *__restrict__ chunks, int nch) {
    extern __shared__ float4 ring[];  // [kUpDepth][kUpRows][kDotThreads]
    float4 *pf = Vf + (int64_t)j * vstride, *zf = Vf + (int64_t)(j + 1) * vstride;
    auto slot = [&](int i, int g) { return ring + ((size_t)((i % kUpDepth) * kUpRows + g) * kDotThreads + threadIdx.x); };
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const GsChunk ch = chunks[c];
        int col, rstep;
        int64_t row;
        if (chunk_lane(ch, col, rstep, row)) {
            const float2 rs = rsig[col];
            const float4 *tjr = cft + ((int64_t)j * B + col) * 3;
            const float4 tj = make_float4(-tjr[0].x, -tjr[0].y, -tjr[0].z, -tjr[0].w);  // t_j
            for (; row < ch.row1; row += (int64_t)kUpRows * rstep) {
                int64_t tt[kUpRows];
                bool ok[kUpRows];
                float2 WH[kUpRows], WL[kUpRows], CA[kUpRows];
#pragma unroll
                for (int g = 0; g < kUpRows; ++g) {
                    const int64_t r = row + (int64_t)g * rstep;
                    ok[g] = r < ch.row1;
                    tt[g] = (ok[g] ? r : row) * B + col;  // a valid address for the idle rows
                    const float4 z = zf[tt[g]];
                    WH[g] = make_float2(z.x, z.y);
                    WL[g] = make_float2(z.z, z.w);
                    CA[g] = make_float2(0.f, 0.f);
                }
                auto issue = [&](int i) {
                    const float4 *Vi = Vf + (int64_t)i * vstride;
#pragma unroll
                    for (int g = 0; g < kUpRows; ++g) cp_async16(slot(i, g), Vi + tt[g]);
                };
#pragma unroll
                for (int q = 0; q < kUpDepth - 1; ++q) {
                    if (q < j) issue(q);
                    cp_async_commit();
                }
                for (int i = 0; i < j; ++i) {
                    if (i + kUpDepth - 1 < j) issue(i + kUpDepth - 1);
                    cp_async_commit();
                    cp_async_wait<kUpDepth - 1>();  // the group of basis vector i has landed
                    const float4 *rec = cft + ((int64_t)i * B + col) * 3;
                    const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], a = cfa[(int64_t)i * B + col];
                    const float2 B1h = make_float2(r0.x, r0.y), B1l = make_float2(r0.z, r0.w);
                    const float2 B2h = make_float2(r1.x, r1.y), B2l = make_float2(r1.z, r1.w);
                    const float2 nB1h = make_float2(r2.x, r2.y), nB2h = make_float2(r2.z, r2.w);
                    const float2 A1 = make_float2(a.x, a.y), A2 = make_float2(a.z, a.w);
#pragma unroll
                    for (int g = 0; g < kUpRows; ++g) {
                        const float4 v = *slot(i, g);
                        const float2 VRh = make_float2(v.x, v.x), VRl = make_float2(v.z, v.z);
                        const float2 VIh = make_float2(v.y, v.y), VIl = make_float2(v.w, v.w);
                        ff2_mac(WH[g], WL[g], VRh, VRl, B1h, B1l, nB1h);
                        ff2_mac(WH[g], WL[g], VIh, VIl, B2h, B2l, nB2h);
                        CA[g] = f2_fma(VRh, A1, CA[g]);
                        CA[g] = f2_fma(VIh, A2, CA[g]);
                    }
                }
                cp_async_wait<0>();
#pragma unroll
                for (int g = 0; g < kUpRows; ++g) {
                    if (!ok[g]) continue;
                    const int64_t t = tt[g];
                    const float4 p = pf[t];
                    // q = (p - Q a) / sigma
                    float qrh, qrl, qih, qil, er, ei;
                    two_sum(p.x, -CA[g].x, qrh, er);
                    two_sum(p.y, -CA[g].y, qih, ei);
                    qrl = p.z + er;
                    qil = p.w + ei;
                    ff_norm(qrh, qrl);
                    ff_norm(qih, qil);
                    ff_scale(qrh, qrl, rs.x, rs.y);
                    ff_scale(qih, qil, rs.x, rs.y);
                    // w = (z - Q t - q t_j) / sigma
                    float rh = WH[g].x, rl = WL[g].x, ih = WH[g].y, il = WL[g].y;
                    ff_mac(rh, rl, -qrh, -qrl, tj.x, tj.z);
                    ff_mac(rh, rl, qih, qil, tj.y, tj.w);
                    ff_mac(ih, il, -qrh, -qrl, tj.y, tj.w);
                    ff_mac(ih, il, -qih, -qil, tj.x, tj.z);
                    ff_norm(rh, rl);
                    ff_norm(ih, il);
                    ff_scale(rh, rl, rs.x, rs.y);
                    ff_scale(ih, il, rs.x, rs.y);
                    pf[t] = make_float4(qrh, qih, qrl, qil);
                    if (t < q64_rows * B) q64[t] = cx<double>{(double)qrh + (double)qrl, (double)qih + (double)qil};
                    zf[t] = make_float4(rh, ih, rl, il);
                }
            }
        }
    }
}

// h[i][b] = sum_c part[c][i][b] for i < nv (and its float-float split hf when hf is not
// null); Hb(i, j)[b] += h[i][b] for i < nh (column j of
// the Hessenberg matrix accumulates both Gram-Schmidt passes; entry nh, when nv > nh, is the
// squared norm of the vector itself). With a non-null skip flag the kernel does nothing when
// the flag is set.
__global__ void k_reduce_h(int nc, int nv, int nh, int64_t B, const cx<double> *__restrict__ part,
                           cx<double> *__restrict__ h, float4 *__restrict__ hf, cx<double> *__restrict__ Hb,
                           int j, int mmax, const int *__restrict__ skip) {
    if (skip && *skip) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nv * B;
         t += (int64_t)gridDim.x * blockDim.x) {
        cx<double> acc{0.0, 0.0};
        for (int c = 0; c < nc; ++c) acc = acc + part[(int64_t)c * nv * B + t];
        h[t] = acc;
        if (hf) hf[t] = ff_split(acc);
        const int64_t i = t / B, b = t - i * B;
        if (i < nh) {
            cx<double> &e = Hb[hb_at((int)i, j, mmax, B, b)];
            e = e + acc;
        }
    }
}

// Whether the second Gram-Schmidt pass can be skipped: after one classical pass the vector
// keeps norm^2 = |w|^2 - sum_i |h_i|^2 (V orthonormal); when that is at least kKeep^2 |w|^2
// for every column, the orthogonality lost in the pass is at most about eps / kKeep per step
// and a second pass would change nothing measurable. skip = 1 in that case; ran[j] records
// whether pass 2 of step j runs (the work accounting reads it back).
constexpr double kKeep2 = 0.05 * 0.05;
__global__ void k_reorth_flag(int nh, int64_t B, const cx<double> *__restrict__ h, int *__restrict__ skip,
                              int *__restrict__ ran, int j) {
    __shared__ int need;
    if (threadIdx.x == 0) need = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t b = warp; b < B; b += nw) {  // one warp per column
        double sacc = 0.0;
        for (int i = lane; i < nh; i += 32) sacc += norm2(h[(int64_t)i * B + b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        const double w2 = h[(int64_t)nh * B + b].re;
        if (lane == 0 && !(w2 - sacc >= kKeep2 * w2)) need = 1;  // also when not finite
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *skip = need ? 0 : 1;
        ran[j] = need;
    }
}

// w[row][b] -= sum_i V_i[row][b] h[i][b]
__global__ void k_gs_update(int64_t rows, int64_t B, int nv, const cx<double> *__restrict__ V,
                            int64_t vstride, const cx<double> *__restrict__ h,
                            cx<double> *__restrict__ w, const int *__restrict__ skip) {
    if (skip && *skip) return;
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


// Partial squared column norms over a chunk of rows: part[c][b]; grid (chunk, b).
__global__ void __launch_bounds__(kDotThreads) k_colnorm_part(int64_t rows, int64_t B,
                                                              const cx<double> *__restrict__ w,
                                                              double *__restrict__ part) {
    const int c = blockIdx.x, nc = gridDim.x;
    const int64_t b = blockIdx.y;
    const int64_t r0 = rows * c / nc, r1 = rows * (c + 1) / nc;
    __shared__ double sh[kDotThreads];
    double acc = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc += norm2(w[r * B + b]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)c * B + b] = sh[0];
}

// nrm[b] = sqrt(sum_c part[c][b]); with Hb, also Hb(j+1, j)[b] = nrm[b]
__global__ void k_colnorm_fin(int nc, int64_t B, const double *__restrict__ part,
                              double *__restrict__ nrm, cx<double> *__restrict__ Hb, int j, int mmax) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nc; ++c) acc += part[(int64_t)c * B + b];
        const double n = std::sqrt(acc);
        nrm[b] = n;
        if (Hb) Hb[hb_at(j + 1, j, mmax, B, b)] = cx<double>{n, 0.0};
    }
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

// ---------------------------------------------------------------- per-shift Givens QR
// One thread per shift. Applying the stored rotations to a Hessenberg column is a chain:
// with carry = H(0, l) and a_i = H(i+1, l) (+ shift on the diagonal), rotation i fixes row i
// as R(i, l) = c_i carry + s_i a_i and carries carry <- -conj(s_i) carry + c_i a_i on. GB300
// issues FP64 at 1/64 of its FP32 rate, so the chains are walked once, serially, by their
// own thread (a warp-parallel scan of the chain would repeat each complex product on every
// lane); the many shifts supply the parallelism.

// Shifts' Givens QR of the new Hessenberg columns j0 .. j1-1 of (Hb + shift I~): apply the
// stored rotations, make rotation j, update g; then the residual estimate |g_{j1}| / beta.
// Per-shift arrays are [S][mmax] (rot_c, rot_s, rdiag: the diagonal R(j, j) for the back
// substitution) and [S][mmax+1] (g); shift [S], col_of [S] (the batch column of shift k),
// res [S].
// With klist, the S shifts taken are klist[0 .. S-1]. With Hbf (the float-float split of Hb's
// columns j0 .. j1-1) the chain runs in float-float
// from the split rotations rcf, rsf, which the kernel also writes (FP32 pipe: GB300 issues
// FP64 at 1/64 of the FP32 rate); the new rotation itself and g stay FP64.
__global__ void __launch_bounds__(64) k_shift_steps(int j0, int j1, int mmax, int64_t B, int64_t S,
                                                    const cx<double> *__restrict__ Hb,
                                                    const cx<double> *__restrict__ shift,
                                                    const int *__restrict__ col_of,
                                                    double *__restrict__ rot_c, cx<double> *__restrict__ rot_s,
                                                    cx<double> *__restrict__ rdiag, cx<double> *__restrict__ g,
                                                    const double *__restrict__ beta, double *__restrict__ res,
                                                    const float4 *__restrict__ Hbf, float2 *__restrict__ rot_cf,
                                                    float4 *__restrict__ rot_sf, const int *__restrict__ klist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    const int64_t k = klist ? klist[t] : t;
    const int64_t b = col_of[k];
    const cx<double> shk = shift[k];
    double *rc = rot_c + k * mmax;
    cx<double> *rs = rot_s + k * mmax;
    cx<double> *gk = g + k * (mmax + 1);
    float2 *rcf = Hbf ? rot_cf + k * mmax : nullptr;
    float4 *rsf = Hbf ? rot_sf + k * mmax : nullptr;
    const float4 shf = ff_split(shk);
    for (int j = j0; j < j1; ++j) {
        // (the chain is walked from the stored rotations; see the comment above)
        cx<double> hj;
        if (Hbf) {
            float4 h = Hbf[hb_at(0, j, mmax, B, b)];
            if (j == 0) {
                ff_add(h.x, h.z, shf.x, shf.z);
                ff_add(h.y, h.w, shf.y, shf.w);
            }
            for (int i = 0; i < j; ++i) {
                float4 hi1 = Hbf[hb_at(i + 1, j, mmax, B, b)];
                if (i + 1 == j) {
                    ff_add(hi1.x, hi1.z, shf.x, shf.z);
                    ff_add(hi1.y, hi1.w, shf.y, shf.w);
                }
                h = ff_rot_step(rcf[i], rsf[i], hi1, h);
            }
            hj = ff_join(h);
        } else {
            hj = Hb[hb_at(0, j, mmax, B, b)];
            if (j == 0) hj = hj + shk;
            for (int i = 0; i < j; ++i) {
                cx<double> hi1 = Hb[hb_at(i + 1, j, mmax, B, b)];
                if (i + 1 == j) hi1 = hi1 + shk;
                hj = rc[i] * hi1 - conj(rs[i]) * hj;
            }
        }
        double c;
        cx<double> sn, r;
        givens_rot(hj, Hb[hb_at(j + 1, j, mmax, B, b)], c, sn, r);
        rc[j] = c;
        rs[j] = sn;
        if (Hbf) {
            const float ch = __double2float_rn(c);
            rcf[j] = make_float2(ch, __double2float_rn(c - (double)ch));
            rsf[j] = ff_split(sn);
        }
        rdiag[k * mmax + j] = r;
        const cx<double> gj = gk[j];
        gk[j] = c * gj;
        gk[j + 1] = cx<double>{0.0, 0.0} - conj(sn) * gj;
    }
    res[k] = std::sqrt(norm2(gk[j1])) / beta[b];
}

// Solve R y = g for the first m Hessenberg columns of every shift (column-oriented back
// substitution: y_l = g_l / R(l, l), then g_i -= R(i, l) y_l for i < l, the entries R(i, l)
// regenerated from Hb and the stored rotations) and form the tier-0 block
// x0[e] = sum_l V_l[e][b] y_l, e < d2. The block's rotations, g and y are staged in shared
// memory, interleaved by thread ([i][thread]) so that a warp's accesses fall in distinct
// banks: the chains then read on-chip memory instead of 32 scattered L2 sectors per step.
constexpr int kSolveThreads = 32;
__global__ void __launch_bounds__(kSolveThreads) k_shift_solve(int m, int mmax, int64_t B, int64_t S, int d2,
                                                               const cx<double> *__restrict__ Hb,
                                                               const cx<double> *__restrict__ shift,
                                                               const int *__restrict__ col_of,
                                                               const double *__restrict__ rot_c,
                                                               const cx<double> *__restrict__ rot_s,
                                                               const cx<double> *__restrict__ rdiag,
                                                               const cx<double> *__restrict__ g,
                                                               const cx<double> *__restrict__ V, int64_t vstride,
                                                               cx<double> *__restrict__ x0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x, bd = blockDim.x;
    cx<double> *sm = reinterpret_cast<cx<double> *>(smem_raw);
    cx<double> *gw = sm + t, *y = sm + (int64_t)m * bd + t, *ss = sm + 2 * (int64_t)m * bd + t;
    double *sc = reinterpret_cast<double *>(sm + 3 * (int64_t)m * bd) + t;  // element i at [i * bd]
    const int64_t k = (int64_t)blockIdx.x * bd + t;
    if (k >= S) return;
    const int64_t b = col_of[k];
    const cx<double> shk = shift[k];
    for (int i = 0; i < m; ++i) {
        gw[(int64_t)i * bd] = g[k * (mmax + 1) + i];
        sc[(int64_t)i * bd] = rot_c[k * mmax + i];
        ss[(int64_t)i * bd] = rot_s[k * mmax + i];
    }
    for (int l = m - 1; l >= 0; --l) {
        const cx<double> yl = cdiv(gw[(int64_t)l * bd], rdiag[k * mmax + l]);
        y[(int64_t)l * bd] = yl;
        cx<double> carry = Hb[hb_at(0, l, mmax, B, b)];
        if (l == 0) carry = carry + shk;
        for (int i = 0; i < l; ++i) {
            cx<double> a1 = Hb[hb_at(i + 1, l, mmax, B, b)];
            if (i + 1 == l) a1 = a1 + shk;
            const double c = sc[(int64_t)i * bd];
            const cx<double> sn = ss[(int64_t)i * bd];
            const cx<double> ril = c * carry + sn * a1;
            carry = c * a1 - conj(sn) * carry;
            cx<double> &gi = gw[(int64_t)i * bd];
            gi = gi - ril * yl;
        }
    }
    for (int e0 = 0; e0 < d2; e0 += 4) {  // four independent accumulations
        cx<double> acc[4] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int l = 0; l < m; ++l) {
            const cx<double> yl = y[(int64_t)l * bd];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + u < d2) fma_to(acc[u], V[(int64_t)l * vstride + (int64_t)(e0 + u) * B + b], yl);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e0 + u < d2) x0[k * d2 + e0 + u] = acc[u];
    }
}
constexpr int kSolveSmemMax = 200 * 1024;

// Strict upper part of every shift's triangular factor R = Q^H (H - s I), one thread per
// (shift, column l): the thread applies the shift's stored rotations 0 .. l-1 to column l of
// the shifted Hessenberg matrix and writes R[i][l], i < l, to R + k * rtri + l (l - 1) / 2 + i.
// Columns are independent, so the m chains of a shift run in parallel (grid y = column); a
// block holds 64 shifts of one column, which read the same Hessenberg column.
__global__ void __launch_bounds__(64) k_shift_rform(int m, int mmax, int64_t rtri, int64_t B, int64_t S,
                                                    const cx<double> *__restrict__ Hb,
                                                    const cx<double> *__restrict__ shift,
                                                    const int *__restrict__ col_of,
                                                    const double *__restrict__ rot_c,
                                                    const cx<double> *__restrict__ rot_s,
                                                    cx<double> *__restrict__ R) {
    const int l = (int)blockIdx.y + 1;  // column 0 has no entries above the diagonal
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= m || k >= S) return;
    const int64_t b = col_of[k];
    const cx<double> shk = shift[k];
    const double *rc = rot_c + k * mmax;
    const cx<double> *rs = rot_s + k * mmax;
    cx<double> *Rl = R + k * rtri + (int64_t)l * (l - 1) / 2;
    cx<double> carry = Hb[hb_at(0, l, mmax, B, b)];
    for (int i = 0; i < l; ++i) {
        cx<double> a1 = Hb[hb_at(i + 1, l, mmax, B, b)];
        if (i + 1 == l) a1 = a1 + shk;
        const double c = rc[i];
        const cx<double> sn = rs[i];
        Rl[i] = c * carry + sn * a1;
        carry = c * a1 - conj(sn) * carry;
    }
}

// Back substitution from the stored triangular factor (no rotation chain is walked here):
// y = R^{-1} g column by column (l = m-1 .. 0: y_l = g_l / R_ll, then g_i -= R_il y_l for
// i < l), then x0 = V_0 y on the tier-0 elements. Four lanes per shift, eight shifts per
// 32-thread block (enough blocks to reach every SM); lane q of a quad updates the rows
// i = q mod 4 and sums the elements e = q mod 4. The reciprocals 1 / R_ll are formed before
// the column loop (independent divisions that overlap), so the loop's serial chain holds one
// complex product per column instead of a division. g, y and the reciprocals of the block's
// shifts sit in shared memory: 3 * 8 * m complex values.
constexpr int kBsShifts = 8;
__global__ void __launch_bounds__(32) k_shift_backsub(int m, int mmax, int64_t rtri, int64_t B, int64_t S,
                                                      int d2, const int *__restrict__ col_of,
                                                      const cx<double> *__restrict__ R,
                                                      const cx<double> *__restrict__ rdiag,
                                                      const cx<double> *__restrict__ g,
                                                      const cx<double> *__restrict__ V, int64_t vstride,
                                                      cx<double> *__restrict__ x0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x, q = lane & 3, slot = lane >> 2;
    cx<double> *sg = reinterpret_cast<cx<double> *>(smem_raw) + (int64_t)slot * m;
    cx<double> *sy = reinterpret_cast<cx<double> *>(smem_raw) + (int64_t)(kBsShifts + slot) * m;
    cx<double> *sinv = reinterpret_cast<cx<double> *>(smem_raw) + (int64_t)(2 * kBsShifts + slot) * m;
    const int64_t k_raw = (int64_t)blockIdx.x * kBsShifts + slot;
    const bool valid = k_raw < S;
    const int64_t k = valid ? k_raw : S - 1;  // idle quads repeat the last shift, store nothing
    const int64_t b = col_of[k];
    for (int i = q; i < m; i += 4) {
        sg[i] = g[k * (mmax + 1) + i];
        const cx<double> d = rdiag[k * mmax + i];
        sinv[i] = (1.0 / norm2(d)) * conj(d);
    }
    __syncwarp();
    const cx<double> *Rk = R + k * rtri;
    for (int l = m - 1; l >= 0; --l) {
        cx<double> yl{0.0, 0.0};
        if (q == (l & 3)) {
            yl = sg[l] * sinv[l];
            sy[l] = yl;
        }
        const int src = (lane & ~3) | (l & 3);
        yl.re = __shfl_sync(0xffffffffu, yl.re, src);
        yl.im = __shfl_sync(0xffffffffu, yl.im, src);
        const cx<double> *Rl = Rk + (int64_t)l * (l - 1) / 2;
        for (int i = q; i < l; i += 4) sg[i] = sg[i] - Rl[i] * yl;
        __syncwarp();
    }
    for (int e = q; e < d2; e += 4) {
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < m; ++l) fma_to(acc, V[(int64_t)l * vstride + (int64_t)e * B + b], sy[l]);
        if (valid) x0[k * d2 + e] = acc;
    }
}

// The same solve for any m, one thread per shift walking the rotation chains (used when m
// exceeds the register budget of k_shift_solve). Work arrays gw [S][mmax+1], y [S][mmax].
__global__ void k_shift_solve_long(int m, int mmax, int64_t B, int64_t S, int d2,
                                   const cx<double> *__restrict__ Hb, const cx<double> *__restrict__ shift,
                                   const int *__restrict__ col_of, const double *__restrict__ rot_c,
                                   const cx<double> *__restrict__ rot_s, const cx<double> *__restrict__ rdiag,
                                   const cx<double> *__restrict__ g, cx<double> *__restrict__ gw,
                                   cx<double> *__restrict__ y, const cx<double> *__restrict__ V,
                                   int64_t vstride, cx<double> *__restrict__ x0) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const int64_t b = col_of[k];
    const cx<double> shk = shift[k];
    cx<double> *gk = gw + k * (mmax + 1);
    cx<double> *yk = y + k * mmax;
    for (int i = 0; i < m; ++i) gk[i] = g[k * (mmax + 1) + i];
    for (int l = m - 1; l >= 0; --l) {
        const cx<double> yl = cdiv(gk[l], rdiag[k * mmax + l]);
        yk[l] = yl;
        cx<double> carry = Hb[hb_at(0, l, mmax, B, b)];
        if (l == 0) carry = carry + shk;
        for (int i = 0; i < l; ++i) {
            cx<double> a1 = Hb[hb_at(i + 1, l, mmax, B, b)];
            if (i + 1 == l) a1 = a1 + shk;
            const double c = rot_c[k * mmax + i];
            const cx<double> s = rot_s[k * mmax + i];
            const cx<double> ril = c * carry + s * a1;
            carry = c * a1 - conj(s) * carry;
            gk[i] = gk[i] - ril * yl;
        }
    }
    for (int e = 0; e < d2; ++e) {
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < m; ++l) fma_to(acc, V[(int64_t)l * vstride + (int64_t)e * B + b], yk[l]);
        x0[k * d2 + e] = acc;
    }
}

// The same solve in float-float (any m): R(i, l) regenerated by the float-float chains from
// Hbf and the split rotations, y_l = g_l / R(l, l) in FP64 (one division per column), the
// back substitution's updates of g and x0 = V_0 y from the float-float tier-0 rows of the
// basis (Vf), for the S shifts klist[0 .. S-1]. Work arrays gw [S][mmax+1] and y [S][mmax]
// (indexed by shift) hold float-float values.
__global__ void __launch_bounds__(64) k_shift_solve_ff(int m, int mmax, int64_t B, int64_t S, int d2,
                                                       const float4 *__restrict__ Hbf,
                                                       const cx<double> *__restrict__ shift,
                                                       const int *__restrict__ col_of,
                                                       const float2 *__restrict__ rot_cf,
                                                       const float4 *__restrict__ rot_sf,
                                                       const cx<double> *__restrict__ rdiag,
                                                       const cx<double> *__restrict__ g, float4 *__restrict__ gw,
                                                       float4 *__restrict__ y, const float4 *__restrict__ Vf,
                                                       int64_t vstride, cx<double> *__restrict__ x0,
                                                       const int *__restrict__ klist) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    const int64_t k = klist[t];
    const int64_t b = col_of[k];
    const float4 shf = ff_split(shift[k]);
    const float2 *rcf = rot_cf + k * mmax;
    const float4 *rsf = rot_sf + k * mmax;
    float4 *gk = gw + k * (mmax + 1);
    float4 *yk = y + k * mmax;
    for (int i = 0; i < m; ++i) gk[i] = ff_split(g[k * (mmax + 1) + i]);
    for (int l = m - 1; l >= 0; --l) {
        const cx<double> yl = cdiv(ff_join(gk[l]), rdiag[k * mmax + l]);
        const float4 yf = ff_split(yl);
        yk[l] = yf;
        const float4 nyf = make_float4(-yf.x, -yf.y, -yf.z, -yf.w);
        float4 carry = Hbf[hb_at(0, l, mmax, B, b)];
        if (l == 0) {
            ff_add(carry.x, carry.z, shf.x, shf.z);
            ff_add(carry.y, carry.w, shf.y, shf.w);
        }
        for (int i = 0; i < l; ++i) {
            float4 a1 = Hbf[hb_at(i + 1, l, mmax, B, b)];
            if (i + 1 == l) {
                ff_add(a1.x, a1.z, shf.x, shf.z);
                ff_add(a1.y, a1.w, shf.y, shf.w);
            }
            const float2 c = rcf[i];
            const float4 sn = rsf[i];
            // R(i, l) = c carry + s a1; carry <- c a1 - conj(s) carry
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            ff_mac(rh, rl, c.x, c.y, carry.x, carry.z);
            ff_mac(ih, il, c.x, c.y, carry.y, carry.w);
            ff_cmac(rh, rl, ih, il, sn, a1);
            ff_norm(rh, rl);
            ff_norm(ih, il);
            carry = ff_rot_step(c, sn, a1, carry);
            // g_i -= R(i, l) y_l
            float4 gi = gk[i];
            float gr = gi.x, grl = gi.z, gim = gi.y, gil = gi.w;
            ff_cmac(gr, grl, gim, gil, make_float4(rh, ih, rl, il), nyf);
            ff_norm(gr, grl);
            ff_norm(gim, gil);
            gk[i] = make_float4(gr, gim, grl, gil);
        }
    }
    for (int e = 0; e < d2; ++e) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int l = 0; l < m; ++l) ff_cmac(rh, rl, ih, il, Vf[(int64_t)l * vstride + (int64_t)e * B + b], yk[l]);
        x0[k * d2 + e] = cx<double>{(double)rh + (double)rl, (double)ih + (double)il};
    }
}

// Hbf = float-float split of Hessenberg columns j0 .. j1-1 (rows 0 .. mmax)
__global__ void k_split_hb(int j0, int j1, int mmax, int64_t B, const cx<double> *__restrict__ Hb,
                           float4 *__restrict__ Hbf) {
    const int64_t n = (int64_t)(j1 - j0) * (mmax + 1) * B, off = (int64_t)j0 * (mmax + 1) * B;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        Hbf[off + t] = ff_split(Hb[off + t]);
}

// Column compaction of the Krylov state when parameter sets leave the shift-invariant process
// (all their shifts converged): column c of the new layout is column map[c] of the old one.
// The basis (nslots slots of rows x Bo entries into rows x Bn), the Hessenberg matrices (ne
// entries (i, j) per column) and beta move; nothing else is per column.
__global__ void k_compact_basis(int64_t nslots, int64_t rows, int64_t Bo, int64_t Bn, const int *__restrict__ map,
                                const float4 *__restrict__ src, float4 *__restrict__ dst) {
    const int64_t total = nslots * rows * Bn;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sr = t / Bn, c = t - sr * Bn;  // sr = slot * rows + row
        dst[t] = src[sr * Bo + map[c]];
    }
}
__global__ void k_compact_hb(int64_t ne, int64_t Bo, int64_t Bn, const int *__restrict__ map,
                             const cx<double> *__restrict__ src, cx<double> *__restrict__ dst,
                             const double *__restrict__ beta, double *__restrict__ beta_out) {
    const int64_t total = ne * Bn;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / Bn, c = t - e * Bn;
        dst[t] = src[e * Bo + map[c]];
        if (e == 0) beta_out[c] = beta[map[c]];
    }
}

// g[k][0] = beta of shift k's column
__global__ void k_init_g(int64_t S, int mmax, const int *__restrict__ col_of,
                         const double *__restrict__ beta, cx<double> *__restrict__ g) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S;
         k += (int64_t)gridDim.x * blockDim.x)
        g[k * (mmax + 1)] = cx<double>{beta[col_of[k]], 0.0};
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16); }

}  // namespace

// Work chunks of the float-float Gram-Schmidt kernels for a column layout in which ADO n has
// acols[n] active (leading) columns: runs of ADOs with equal counts, cut into pieces of about
// 1/456 of the active entries (at least 4096) so that one tile of basis vectors fills the GPU,
// and the update's pieces, the same cut about 8x finer (its blocks stride over them in one
// wave of resident blocks, so that the last pieces balance across the SMs). Returns the
// active entries; *runs = the number of runs.
static int64_t make_chunks(const std::vector<int> &acols, int d2, std::vector<GsChunk> &ch, std::vector<GsChunk> &uch,
                    int *runs) {
    ch.clear();
    uch.clear();
    const int64_t N = (int64_t)acols.size();
    int64_t act = 0;
    for (int64_t n = 0; n < N; ++n) act += (int64_t)d2 * acols[(size_t)n];
    const int64_t target = std::max<int64_t>(4096, act / 456);
    int nr = 0;
    for (int64_t n = 0; n < N;) {
        const int a = acols[(size_t)n];
        int64_t n1 = n;
        while (n1 < N && acols[(size_t)n1] == a) ++n1;
        ++nr;
        if (a > 0) {
            const int64_t r0 = n * d2, r1 = n1 * d2, step = std::max<int64_t>(1, target / a);
            for (int64_t r = r0; r < r1; r += step)
                ch.push_back(GsChunk{(int32_t)r, (int32_t)std::min(r1, r + step), a, 0});
        }
        n = n1;
    }
    for (const GsChunk &c0 : ch) {
        const int64_t rows_c = c0.row1 - c0.row0, ustep = std::max<int64_t>(1, (rows_c + 7) / 8);
        for (int64_t r = c0.row0; r < c0.row1; r += ustep)
            uch.push_back(GsChunk{(int32_t)r, (int32_t)std::min<int64_t>(c0.row1, r + ustep), c0.acols, 0});
    }
    if (runs) *runs = nr;
    return act;
}

// Device buffers of the delayed-reorthogonalisation process (see shifted_gmres).
struct DcgsBufs {
    float4 *VA, *VB;             // two float-float bases of (mmax + 1) x rows x B entries
    cx<double> *Hb, *Hb2;        // Hessenberg matrices and their compaction target
    float4 *Hbf;                 // float-float split of the final Hessenberg columns
    double *beta, *beta2;        // ||b|| per column and its compaction target
    cx<double> *part, *D;        // partial and reduced dot products
    float4 *cfa, *cft;           // update coefficients
    float2 *rsig;                // 1 / sigma per column
    const cx<double> *shift;     // [S]
    int *col_of;                 // [S] current column of each shift
    double *rot_c;
    cx<double> *rot_s, *rdiag, *g;
    double *res;                 // [S] residual estimates
    float2 *rot_cf;
    float4 *rot_sf, *gw, *y;
    cx<double> *x0;              // [S][d2]
    GsChunk *ch, *uch;           // chunk tables (capacities ch_cap, uch_cap)
    int ch_cap, uch_cap;
    int *klist, *kfroz, *set_of, *map;
};

// The shift-invariant Arnoldi process with delayed reorthogonalisation for B columns, from
// v_0 = b / beta in VA slot 0 (g and beta set), with every shift's Givens QR advanced at the
// convergence checks (every 10 steps). A parameter set all of whose shifts have converged
// leaves the process: its shifts' tier-0 blocks are solved at once from the columns so far,
// and when enough columns have left (at least 1/16 of them) the remaining columns are
// compacted into a narrower layout (basis, Hessenberg matrices, beta; the shifts' own arrays
// stay), so the later steps stream only the columns still running. Ends with the final solve
// of the shifts still running; *steps = the Arnoldi steps taken (applies).
static heom_status dcgs_process(heom_hier *h, int64_t B, int64_t S, int mmax, double tol, std::vector<int> col_of,
                         DcgsBufs &bf, int *steps, cudaStream_t s) {
    const int64_t rows = h->N * h->d2;
    const int d2 = h->d2;
    const int64_t cps = B / h->n_sets;
    const DevView<double> v = h->view64();
    int dev = 0, sms = 0, occ = 0;
    HEOM_CUDA(cudaGetDevice(&dev));
    HEOM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HEOM_CUDA(cudaFuncSetAttribute(k_update2_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpSmem));
    HEOM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update2_ff, kDotThreads, kUpSmem));
    std::vector<int> cur((size_t)B);  // original column of each current column
    for (int64_t c = 0; c < B; ++c) cur[(size_t)c] = (int)c;
    std::vector<int> act((size_t)S);  // shifts still running
    for (int64_t k = 0; k < S; ++k) act[(size_t)k] = (int)k;
    int64_t Bc = B, Lc = rows * B;
    float4 *Vc = bf.VA, *Vo = bf.VB;
    cx<double> *Hc = bf.Hb, *Ho = bf.Hb2;
    double *bc = bf.beta, *bo = bf.beta2;
    std::vector<GsChunk> ch, uch;
    int nch = 0, nuch = 0, gsu = 1;
    double Lg = 0.0;
    // chunk tables and sets of the current layout: ADO n keeps the current columns whose set is
    // below act_ado[n] (a leading block: columns stay in set order)
    auto relayout = [&]() -> heom_status {
        std::vector<int> set_c((size_t)Bc), acols((size_t)h->N);
        for (int64_t c = 0; c < Bc; ++c) set_c[(size_t)c] = (int)(cur[(size_t)c] / cps);
        for (int64_t n = 0; n < h->N; ++n)
            acols[(size_t)n] = h->has_act ? (int)(std::lower_bound(set_c.begin(), set_c.end(), h->act_ado[n]) -
                                                  set_c.begin())
                                          : (int)Bc;
        Lg = (double)make_chunks(acols, d2, ch, uch, nullptr);
        nch = (int)ch.size();
        nuch = (int)uch.size();
        if (nch > bf.ch_cap || nuch > bf.uch_cap) {
            set_error("shift-invariant solver: chunk table overflow");
            return HEOM_EINVAL;
        }
        if (nch) HEOM_CUDA(memcpy_counted(bf.ch, ch.data(), nch * sizeof(GsChunk), cudaMemcpyHostToDevice, s));
        if (nuch) HEOM_CUDA(memcpy_counted(bf.uch, uch.data(), nuch * sizeof(GsChunk), cudaMemcpyHostToDevice, s));
        HEOM_CUDA(memcpy_counted(bf.set_of, set_c.data(), Bc * sizeof(int), cudaMemcpyHostToDevice, s));
        gsu = std::max(1, std::min(nuch, std::max(occ, 1) * sms));
        return HEOM_OK;
    };
    auto upload_shifts = [&]() -> heom_status {
        HEOM_CUDA(memcpy_counted(bf.klist, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        HEOM_CUDA(memcpy_counted(bf.col_of, col_of.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
        return HEOM_OK;
    };
    // final solve of the listed shifts from the first mf Hessenberg columns
    auto solve_shifts = [&](const int *klist, int64_t nk, int mf) -> heom_status {
        if (nk == 0 || mf == 0) return HEOM_OK;
        Prof pr(HEOM_KC_OTHER, s, (double)nk, (double)nk * mf * 16);
        k_shift_solve_ff<<<(unsigned)((nk + 63) / 64), 64, 0, s>>>(mf, mmax, Bc, nk, d2, bf.Hbf, bf.shift, bf.col_of,
                                                                   bf.rot_cf, bf.rot_sf, bf.rdiag, bf.g, bf.gw, bf.y,
                                                                   Vc, Lc, bf.x0, klist);
        HEOM_CUDA(cudaGetLastError());
        return HEOM_OK;
    };
    heom_status st = relayout();
    if (st != HEOM_OK) return st;
    st = upload_shifts();
    if (st != HEOM_OK) return st;
    std::vector<double> hres((size_t)S, 1.0);
    int m = 0, j_done = 0;
    for (int j = 0; j < mmax; ++j) {
        float4 *zf = Vc + (int64_t)(j + 1) * Lc;
        {   // z = M p_j, float-float from and into the basis
            Prof pr(HEOM_KC_KRYLOV_APPLY64, s, Lg / d2, 2.0 * Lg * 16);
            const int64_t grid = std::min<int64_t>((Lc + 255) / 256, 152 * 16);
            if (cps % 2 == 0)
                k_apply_ff<2><<<(unsigned)grid, 256, 0, s>>>(v, Vc + (int64_t)j * Lc, zf, Bc, bf.set_of);
            else
                k_apply_ff<1><<<(unsigned)grid, 256, 0, s>>>(v, Vc + (int64_t)j * Lc, zf, Bc, bf.set_of);
        }
        {   // one read of the basis for the dots, one for the update
            Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)(j + 1) * Lg, (2.0 * j + 6.0) * Lg * 16);
            pr.kernels = 4;
            k_dots2_ff_tiled<<<dim3((unsigned)((j + 1 + kD2Tile - 1) / kD2Tile), (unsigned)nch), kDotThreads, 0, s>>>(
                Bc, j + 1, Vc, Lc, zf, bf.part, bf.ch);
            k_reduce_dots2<<<blocks_for((int64_t)(j + 1) * 2 * Bc), 256, 0, s>>>(nch, j + 1, Bc, bf.part, bf.D);
            k_dcgs_coef<<<(unsigned)Bc, 256, 0, s>>>(j, mmax, Bc, bf.D, Hc, bf.cfa, bf.cft, bf.rsig);
            k_update2_ff<<<gsu, kDotThreads, kUpSmem, s>>>(Bc, j, Vc, Lc, nullptr, 0, bf.cfa, bf.cft, bf.rsig, bf.uch,
                                                           nuch);
        }
        HEOM_CUDA(cudaGetLastError());
        m = j + 1;
        if ((m % 10 != 0 && m != mmax) || m - 1 <= j_done) continue;
        const int mf = m - 1;  // column m - 1 of Hb becomes final only at the next step
        {   // the running shifts' Givens QR catches up with the new final columns
            Prof pr(HEOM_KC_OTHER, s, (double)act.size() * (mf - j_done), 0.0);
            pr.kernels = 2;
            k_split_hb<<<blocks_for((int64_t)(mf - j_done) * (mmax + 1) * Bc), 256, 0, s>>>(j_done, mf, mmax, Bc, Hc,
                                                                                          bf.Hbf);
            k_shift_steps<<<(unsigned)((act.size() + 63) / 64), 64, 0, s>>>(
                j_done, mf, mmax, Bc, (int64_t)act.size(), Hc, bf.shift, bf.col_of, bf.rot_c, bf.rot_s, bf.rdiag, bf.g,
                bc, bf.res, bf.Hbf, bf.rot_cf, bf.rot_sf, bf.klist);
        }
        j_done = mf;
        HEOM_CUDA(memcpy_counted(hres.data(), bf.res, S * 8, cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(cudaStreamSynchronize(s));
        // a column is done when all its running shifts are; a parameter set when all its columns are
        std::vector<char> done_c((size_t)Bc, 1);
        bool all = true;
        for (int k : act)
            if (!(hres[(size_t)k] <= tol)) {
                done_c[(size_t)col_of[(size_t)k]] = 0;
                all = false;
            }
        if (all || m == mmax) break;
        std::vector<char> leave((size_t)Bc, 0);
        int64_t n_leave = 0;
        for (int64_t c0 = 0; c0 < Bc;) {  // runs of one set
            int64_t c1 = c0;
            bool d = true;
            while (c1 < Bc && cur[(size_t)c1] / cps == cur[(size_t)c0] / cps) {
                d = d && done_c[(size_t)c1];
                ++c1;
            }
            if (d) {
                for (int64_t c = c0; c < c1; ++c) leave[(size_t)c] = 1;
                n_leave += c1 - c0;
            }
            c0 = c1;
        }
        if (n_leave == 0 || n_leave < Bc / 16) continue;
        // the leaving shifts: tier-0 blocks from the mf final columns, in the current layout
        std::vector<int> kf, keep;
        for (int k : act) (leave[(size_t)col_of[(size_t)k]] ? kf : keep).push_back(k);
        HEOM_CUDA(memcpy_counted(bf.kfroz, kf.data(), kf.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        st = solve_shifts(bf.kfroz, (int64_t)kf.size(), mf);
        if (st != HEOM_OK) return st;
        // compact the running columns (slots 0 .. m: q_0 .. q_{m-1} and p_m)
        std::vector<int> map, inv((size_t)Bc, -1);
        for (int64_t c = 0; c < Bc; ++c)
            if (!leave[(size_t)c]) {
                inv[(size_t)c] = (int)map.size();
                map.push_back((int)c);
            }
        const int64_t Bn = (int64_t)map.size(), Ln = rows * Bn;
        HEOM_CUDA(memcpy_counted(bf.map, map.data(), Bn * sizeof(int), cudaMemcpyHostToDevice, s));
        {
            Prof pr(HEOM_KC_OTHER, s, (double)(m + 1) * Ln, 2.0 * (m + 1) * Ln * 16);
            pr.kernels = 3;
            k_compact_basis<<<blocks_for((int64_t)(m + 1) * Ln), 256, 0, s>>>(m + 1, rows, Bc, Bn, bf.map, Vc, Vo);
            const int64_t ne = (int64_t)(mmax + 1) * mmax;
            k_compact_hb<<<blocks_for(ne * Bn), 256, 0, s>>>(ne, Bc, Bn, bf.map, Hc, Ho, bc, bo);
            k_split_hb<<<blocks_for((int64_t)j_done * (mmax + 1) * Bn), 256, 0, s>>>(0, j_done, mmax, Bn, Ho, bf.Hbf);
        }
        HEOM_CUDA(cudaGetLastError());
        std::swap(Vc, Vo);
        std::swap(Hc, Ho);
        std::swap(bc, bo);
        std::vector<int> cur_n((size_t)Bn);
        for (int64_t c = 0; c < Bn; ++c) cur_n[(size_t)c] = cur[(size_t)map[(size_t)c]];
        cur.swap(cur_n);
        for (int k : keep) col_of[(size_t)k] = inv[(size_t)col_of[(size_t)k]];
        for (int k : kf) col_of[(size_t)k] = 0;  // no longer read
        act.swap(keep);
        Bc = Bn;
        Lc = Ln;
        st = relayout();
        if (st != HEOM_OK) return st;
        st = upload_shifts();
        if (st != HEOM_OK) return st;
    }
    st = solve_shifts(bf.klist, (int64_t)act.size(), j_done);
    if (st != HEOM_OK) return st;
    *steps = m;
    return HEOM_OK;
}

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
    {   // the basis (FP64 + float-float split) and the per-shift arrays grow with mmax: keep
        // them within 60 % of the free device memory
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            // the hierarchy's own workspace is reused (or grown), and the workspaces the library
            // keeps cached on this device are freed when an allocation needs their memory
            free_b += h->ws.bytes + ws_cached_total(h->device);
            const double per_step = 32.0 * (double)L + 112.0 * (double)S + (64.0 + 32.0 * 456) * (double)B;
            const double fixed = 64.0 * (double)L + 48.0 * (double)S + (double)(64 * 2 + 2) * B * 16.0;
            const double avail = 0.6 * (double)free_b - fixed;
            const int fit = avail > per_step ? (int)std::min(2.0e9, avail / per_step) - 1 : 0;
            if (fit < 1) {
                set_error("shift-invariant solver: not enough device memory for %lld columns and %lld shifts",
                          (long long)B, (long long)S);
                return HEOM_ENOMEM;
            }
            mmax = std::min(mmax, fit);
            // the Hessenberg matrices (FP64, its compaction target and the float-float split)
            // grow as mmax^2: within a tenth of the free memory
            while (mmax > 8 && 48.0 * (double)B * (mmax + 1.0) * mmax > 0.1 * (double)free_b) mmax -= 8;
        }
    }
    // device memory: basis V [mmax+1][L] (the new vector is formed in its slot), Hb
    // (column-major, see hb_at), h tmp [mmax+2][B], norms [B], beta [B], per shift: rot_c,
    // rot_s, g, gw, y, rdiag, x0, res, shift, col_of
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t oV = take((size_t)(mmax + 1) * L * 16),
                 oH = take((size_t)(mmax + 1) * mmax * B * 16), oh = take((size_t)(mmax + 2) * B * 16),
                 on = take((size_t)B * 8), obeta = take((size_t)B * 8),
                 orc = take((size_t)S * mmax * 8), ors = take((size_t)S * mmax * 16),
                 og = take((size_t)S * (mmax + 1) * 16), ogw = take((size_t)S * (mmax + 1) * 16),
                 oy = take((size_t)S * mmax * 16), ocb = take((size_t)S * mmax * 16),
                 ox0 = take((size_t)S * d2 * 16), ores = take((size_t)S * 8),
                 osh = take((size_t)S * 16), oco = take((size_t)S * 4);
    // row chunks of the FP64 partial dot products
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(456, L / 4096));
    // float-float Gram-Schmidt (B up to the block size): a split copy of the basis and of h,
    // and its work chunks -- runs of ADOs whose rows have the same active columns (all B
    // unless parameter sets are truncated deepest first), cut into pieces of about
    // 1/456 of the active entries so that one tile of basis vectors fills the GPU
    const bool ffgs = B <= kDotThreads;
    std::vector<GsChunk> chunks, uchunks;
    int64_t act_total = 0;
    int runs = 0;
    if (ffgs) {
        const int64_t cps = B / h->n_sets;
        std::vector<int> acols((size_t)h->N);
        for (int64_t n = 0; n < h->N; ++n) acols[(size_t)n] = h->has_act ? (int)(h->act_ado[n] * cps) : (int)B;
        act_total = make_chunks(acols, d2, chunks, uchunks, &runs);
    }
    const int nch = (int)chunks.size();
    const int nuch = (int)uchunks.size();
    // chunk-table capacity for every later column layout (compaction only merges runs)
    const int ch_cap = std::max(nch, 456 + runs + 1), uch_cap = 8 * ch_cap;
    const int npc = std::max(nchunk, ch_cap);  // partial-dot chunks
    const size_t opart = take((size_t)npc * (mmax + 2) * 2 * B * 16), oskip = take(sizeof(int)),
                 oran = take((size_t)mmax * sizeof(int));
    const size_t onp = take((size_t)std::max(npc, nuch) * B * 8);
    const size_t och = take((size_t)ch_cap * sizeof(GsChunk)), ouch = take((size_t)uch_cap * sizeof(GsChunk));
    // column compaction (delayed-reorthogonalisation process): second Hessenberg and beta
    // arrays, shift lists, the set of each column, the column map
    const size_t oHb2 = ffgs ? take((size_t)(mmax + 1) * mmax * B * 16) : 0,
                 obeta2 = take((size_t)B * 8), okl = take((size_t)S * 4), okf = take((size_t)S * 4),
                 oset = take((size_t)B * 4), omap = take((size_t)B * 4);
    const size_t oVf = ffgs ? take((size_t)(mmax + 1) * L * 16) : 0,
                 ohf = ffgs ? take((size_t)(mmax + 2) * B * 16) : 0;
    // the delayed-reorthogonalisation scalars: dots D [mmax+1][2][B], coefficients
    const size_t oD = ffgs ? take((size_t)(mmax + 1) * 2 * B * 16) : 0,
                 ocfa = ffgs ? take((size_t)(mmax + 1) * B * 16) : 0,
                 ocft = ffgs ? take((size_t)(mmax + 1) * B * 48) : 0, orsig = ffgs ? take((size_t)B * 8) : 0;
    // every shift's triangular factor (strict upper part) for the final solve, for up to mp
    // steps when that fits 1 GiB (more steps solve by walking the rotation chains instead)
    const bool pers = ffgs && arnoldi_persistent_ok(h, B, mmax);
    const int mp = std::min(mmax, arnoldi_max_steps());
    const int64_t rtri = (int64_t)mp * (mp - 1) / 2;
    const bool keepR = (double)S * (double)rtri * 16.0 <= (double)(1ull << 30);
    const size_t oR = keepR ? take((size_t)S * std::max<int64_t>(rtri, 1) * 16) : 0;
    // the persistent Arnoldi's float-float copies of the rotations
    const size_t orcf = ffgs ? take((size_t)S * mmax * 8) : 0, orsf = ffgs ? take((size_t)S * mmax * 16) : 0;
    const size_t ohbf = ffgs ? take((size_t)(mmax + 1) * mmax * B * 16) : 0;
    heom_status st = ensure_ws(h->ws, off);
    if (st != HEOM_OK) return st;
    char *base = (char *)h->ws.p;
    cx<double> *V = (cx<double> *)(base + oV), *Hb = (cx<double> *)(base + oH),
               *ht = (cx<double> *)(base + oh);
    double *nrm = (double *)(base + on), *beta = (double *)(base + obeta);
    double *rot_c = (double *)(base + orc);
    cx<double> *rot_s = (cx<double> *)(base + ors), *g = (cx<double> *)(base + og),
               *gw = (cx<double> *)(base + ogw), *y = (cx<double> *)(base + oy),
               *rdiag = (cx<double> *)(base + ocb), *dx0 = (cx<double> *)(base + ox0),
               *dsh = (cx<double> *)(base + osh);
    double *dres = (double *)(base + ores);
    int *dco = (int *)(base + oco);
    cx<double> *part = (cx<double> *)(base + opart);
    double *npart = (double *)(base + onp);
    int *dskip = (int *)(base + oskip), *dran = (int *)(base + oran);
    float4 *Vf = ffgs ? (float4 *)(base + oVf) : nullptr;
    float4 *hft = ffgs ? (float4 *)(base + ohf) : nullptr;
    cx<double> *dD = ffgs ? (cx<double> *)(base + oD) : nullptr;
    float2 *rsig = ffgs ? (float2 *)(base + orsig) : nullptr;
    float4 *cfa = ffgs ? (float4 *)(base + ocfa) : nullptr, *cft = ffgs ? (float4 *)(base + ocft) : nullptr;
    cx<double> *Rst = keepR ? (cx<double> *)(base + oR) : nullptr;
    float2 *rot_cf = ffgs ? (float2 *)(base + orcf) : nullptr;
    float4 *rot_sf = ffgs ? (float4 *)(base + orsf) : nullptr;
    float4 *Hbf = ffgs ? (float4 *)(base + ohbf) : nullptr;
    HEOM_CUDA(memcpy_counted(dsh, shift.data(), S * 16, cudaMemcpyHostToDevice, s));
    HEOM_CUDA(memcpy_counted(dco, col_of.data(), S * 4, cudaMemcpyHostToDevice, s));
    HEOM_CUDA(cudaMemsetAsync(Hb, 0, (size_t)(mmax + 1) * mmax * B * 16, s));
    // v_0 = b / ||b||, g = (beta, 0, ...)
    {
        Prof pr(HEOM_KC_OTHER, s, (double)L, 2.0 * L * 16);
        k_colnorm_part<<<dim3((unsigned)nchunk, (unsigned)B), kDotThreads, 0, s>>>(rows, B, bvec, npart);
        k_colnorm_fin<<<blocks_for(B), 256, 0, s>>>(nchunk, B, npart, beta, nullptr, 0, mmax);
        k_scale_by<<<blocks_for(L), 256, 0, s>>>(L, B, bvec, beta, V);
        if (ffgs) k_split<<<blocks_for(L), 256, 0, s>>>(L, V, Vf);
        pr.kernels = ffgs ? 4 : 3;
    }
    // g = (beta_b, 0, ...) per shift
    HEOM_CUDA(cudaMemsetAsync(g, 0, (size_t)S * (mmax + 1) * 16, s));
    {
        Prof pr(HEOM_KC_OTHER, s, (double)S, (double)S * 16);
        k_init_g<<<blocks_for(S), 256, 0, s>>>(S, mmax, dco, beta, g);
    }
    const DevView<double> v = h->view64();
    const bool tiled = tile_ok(v, B);
    const GsChunk *dch = (const GsChunk *)(base + och);
    if (nch > 0) HEOM_CUDA(memcpy_counted((void *)dch, chunks.data(), nch * sizeof(GsChunk), cudaMemcpyHostToDevice, s));
    const GsChunk *duch = (const GsChunk *)(base + ouch);  // filled by the process's layout
    const int gsb = std::max(1, std::min(nch, 152 * 8));  // blocks of the chunk-striding kernels

    // elements of one vector that can be nonzero (truncated sets: the kept rows of each
    // column), and the ADO-applies of one apply: the work and the algorithmic bytes counted
    const int64_t cps = B / h->n_sets;
    const double Lk = h->has_caps ? (double)h->kept_rowsets * cps : (double)L;
    const double Lg = ffgs ? (double)act_total : (double)L;  // what the Gram-Schmidt kernels stream
    TileArgs<double> ta{};
    ta.v = v;
    ta.B = B;
    std::vector<double> hres(S, 1.0);
    int m = 0, check = 5, j_done = 0;
    bool done = false;
    if (pers) {
        // the whole solve (up to its shared-memory limit of steps) in one cooperative launch
        int psteps = 0;
        heom_status pst = arnoldi_persistent(h, B, mmax, mp, Vf, V, Hb, S, dsh, dco, rot_c, rot_s, rdiag, g,
                                             rot_cf, rot_sf, beta, dres, tol, &psteps, &done, s);
        if (pst != HEOM_OK) {
            *steps = psteps;
            return pst;
        }
        m = j_done = psteps;
    }
    const int j_pers = m;  // steps taken by the persistent kernel (accounted there)
    // delayed reorthogonalisation from the first step (after the persistent kernel's steps
    // the basis is already final: the two-pass step continues it); Hessenberg column j is
    // final only after step j + 1, so the shifts' QR and the solution stay one column behind
    const bool dcgs = ffgs && m == 0 && mmax >= 3;
    if (dcgs) {
        DcgsBufs bf{};
        bf.VA = Vf;
        bf.VB = reinterpret_cast<float4 *>(V);  // the FP64 basis is not needed past v_0
        bf.Hb = Hb;
        bf.Hb2 = (cx<double> *)(base + oHb2);
        bf.Hbf = Hbf;
        bf.beta = beta;
        bf.beta2 = (double *)(base + obeta2);
        bf.part = part;
        bf.D = dD;
        bf.cfa = cfa;
        bf.cft = cft;
        bf.rsig = rsig;
        bf.shift = dsh;
        bf.col_of = dco;
        bf.rot_c = rot_c;
        bf.rot_s = rot_s;
        bf.rdiag = rdiag;
        bf.g = g;
        bf.res = dres;
        bf.rot_cf = rot_cf;
        bf.rot_sf = rot_sf;
        bf.gw = (float4 *)gw;
        bf.y = (float4 *)y;
        bf.x0 = dx0;
        bf.ch = const_cast<GsChunk *>(dch);
        bf.uch = const_cast<GsChunk *>(duch);
        bf.ch_cap = ch_cap;
        bf.uch_cap = uch_cap;
        bf.klist = (int *)(base + okl);
        bf.kfroz = (int *)(base + okf);
        bf.set_of = (int *)(base + oset);
        bf.map = (int *)(base + omap);
        st = dcgs_process(h, B, S, mmax, tol, col_of, bf, steps, s);
        if (st != HEOM_OK) return st;
        x0.resize((size_t)S * d2);
        res.resize(S);
        HEOM_CUDA(memcpy_counted(x0.data(), dx0, (size_t)S * d2 * 16, cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(memcpy_counted(res.data(), dres, S * 8, cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(cudaStreamSynchronize(s));
        return HEOM_OK;
    }
    for (int j = m; j < mmax && !done; ++j) {
        const cx<double> *vj = V + (int64_t)j * L;
        cx<double> *w = V + (int64_t)(j + 1) * L;  // the new vector is built in place
        {   // w = M v_j
            Prof pr(HEOM_KC_KRYLOV_APPLY64, s, Lk / h->d2, 2.0 * Lk * 16);
            if (tiled) {
                ta.x = vj;
                ta.out = w;
                HEOM_CUDA((launch_tile<double, TM_STORE>(ta, s)));
            } else {
                ApplyMods<double> mods{nullptr, 0.0};
                HEOM_CUDA(launch_apply(v, vj, w, B, mods, s));
            }
        }
        if (ffgs) {
            float4 *wf = Vf + (int64_t)(j + 1) * L;
            {   // classical Gram-Schmidt in float-float; pass 1 also yields |w|^2 (w's dot with
                // itself), from which k_reorth_flag decides on the device whether pass 2 runs
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)(j + 1) * Lg, (2.0 * (j + 1) + 5.0) * Lg * 16);
                pr.kernels = 5;
                k_split_chunks<<<gsb, kDotThreads, 0, s>>>(B, w, wf, dch, nch);
                k_multidot_ff_tiled<<<dim3((unsigned)((j + 2 + kMdTile - 1) / kMdTile), (unsigned)nch),
                                      kDotThreads, 0, s>>>(B, j + 2, Vf, L, wf, part, nullptr, dch);
                k_reduce_h<<<blocks_for((int64_t)(j + 2) * B), 256, 0, s>>>(nch, j + 2, j + 1, B, part, ht,
                                                                           hft, Hb, j, mmax, nullptr);
                k_reorth_flag<<<1, 128, 0, s>>>(j + 1, B, ht, dskip, dran, j);
                k_gs_update_ff<<<gsb, kDotThreads, 0, s>>>(B, j + 1, Vf, L, hft, wf, nullptr, dch, nch);
            }
            {   // pass 2 (skipped on the device when pass 1 kept enough of w; its work is
                // added to the accounting from the device's record after the solve)
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, 0.0, 0.0);
                pr.kernels = 3;
                k_multidot_ff_tiled<<<dim3((unsigned)((j + 1 + kMdTile - 1) / kMdTile), (unsigned)nch),
                                      kDotThreads, 0, s>>>(B, j + 1, Vf, L, wf, part, dskip, dch);
                k_reduce_h<<<blocks_for((int64_t)(j + 1) * B), 256, 0, s>>>(nch, j + 1, j + 1, B, part, ht,
                                                                           hft, Hb, j, mmax, dskip);
                k_gs_update_ff<<<gsb, kDotThreads, 0, s>>>(B, j + 1, Vf, L, hft, wf, dskip, dch, nch);
            }
            {   // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j} (FP64 and split)
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, Lg, 4.0 * Lg * 16);
                pr.kernels = 3;
                k_colnorm_part_ff<<<dim3((unsigned)nch, (unsigned)B), kDotThreads, 0, s>>>(B, wf, npart, dch);
                k_colnorm_fin<<<blocks_for(B), 256, 0, s>>>(nch, B, npart, nrm, Hb, j, mmax);
                k_scale_ff<<<gsb, kDotThreads, 0, s>>>(B, wf, nrm, w, dch, nch);
            }
        } else {
            {   // classical Gram-Schmidt in FP64, as above
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)(j + 1) * L, (2.0 * (j + 1) + 3.0) * L * 16);
                pr.kernels = 4;
                k_multidot<<<dim3((unsigned)(j + 2), (unsigned)nchunk), kDotThreads, 0, s>>>(
                    rows, B, j + 2, V, L, w, part, nullptr);
                k_reduce_h<<<blocks_for((int64_t)(j + 2) * B), 256, 0, s>>>(nchunk, j + 2, j + 1, B, part, ht,
                                                                           nullptr, Hb, j, mmax, nullptr);
                k_reorth_flag<<<1, 128, 0, s>>>(j + 1, B, ht, dskip, dran, j);
                k_gs_update<<<blocks_for(L), 256, 0, s>>>(rows, B, j + 1, V, L, ht, w, nullptr);
            }
            {
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, 0.0, 0.0);
                pr.kernels = 3;
                k_multidot<<<dim3((unsigned)(j + 1), (unsigned)nchunk), kDotThreads, 0, s>>>(
                    rows, B, j + 1, V, L, w, part, dskip);
                k_reduce_h<<<blocks_for((int64_t)(j + 1) * B), 256, 0, s>>>(nchunk, j + 1, j + 1, B, part, ht,
                                                                           nullptr, Hb, j, mmax, dskip);
                k_gs_update<<<blocks_for(L), 256, 0, s>>>(rows, B, j + 1, V, L, ht, w, dskip);
            }
            {
                Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)L, 3.0 * L * 16);
                pr.kernels = 3;
                k_colnorm_part<<<dim3((unsigned)nchunk, (unsigned)B), kDotThreads, 0, s>>>(rows, B, w, npart);
                k_colnorm_fin<<<blocks_for(B), 256, 0, s>>>(nchunk, B, npart, nrm, Hb, j, mmax);
                k_scale_by<<<blocks_for(L), 256, 0, s>>>(L, B, w, nrm, w);
            }
        }
        HEOM_CUDA(cudaGetLastError());
        m = j + 1;
        if ((m % check == 0 || m == mmax) && m > j_done) {
            const int mf = m;
            {   // every shift's Givens QR catches up with the new Hessenberg columns
                Prof pr(HEOM_KC_OTHER, s, (double)S * (mf - j_done), 0.0);
                k_shift_steps<<<(unsigned)((S + 63) / 64), 64, 0, s>>>(j_done, mf, mmax, B, S, Hb, dsh, dco, rot_c,
                                                                      rot_s, rdiag, g, beta, dres, nullptr, nullptr,
                                                                      nullptr, nullptr);
            }
            j_done = mf;
            HEOM_CUDA(memcpy_counted(hres.data(), dres, S * 8, cudaMemcpyDeviceToHost, s));
            HEOM_CUDA(cudaStreamSynchronize(s));
            double worst = 0.0;
            for (double r : hres) worst = std::max(worst, std::isfinite(r) ? r : 1e300);
            if (worst <= tol) break;
            check = std::min(check + 5, 20);
        }
    }
    const int mf = j_done;  // the Hessenberg columns the shifts' QR has taken in
    if (keepR && mf <= mp && mf > 0) {
        // R from the stored rotations (all columns at once), then back substitution
        Prof pr(HEOM_KC_OTHER, s, (double)S, (double)S * mf * 16);
        pr.kernels = mf > 1 ? 2 : 1;
        if (mf > 1)
            k_shift_rform<<<dim3((unsigned)((S + 63) / 64), (unsigned)(mf - 1)), 64, 0, s>>>(
                mf, mmax, rtri, B, S, Hb, dsh, dco, rot_c, rot_s, Rst);
        const size_t smb = (size_t)3 * kBsShifts * mf * sizeof(cx<double>);
        if (smb > 48 * 1024)
            HEOM_CUDA(cudaFuncSetAttribute(k_shift_backsub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
        k_shift_backsub<<<(unsigned)((S + kBsShifts - 1) / kBsShifts), 32, smb, s>>>(
            mf, mmax, rtri, B, S, d2, dco, Rst, rdiag, g, V, L, dx0);
    } else {
        Prof pr(HEOM_KC_OTHER, s, (double)S, (double)S * mf * 16);
        const size_t smb = (size_t)mf * kSolveThreads * (3 * sizeof(cx<double>) + sizeof(double));
        if (smb <= (size_t)kSolveSmemMax) {
            if (smb > 48 * 1024)
                HEOM_CUDA(cudaFuncSetAttribute(k_shift_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
            k_shift_solve<<<(unsigned)((S + kSolveThreads - 1) / kSolveThreads), kSolveThreads, smb, s>>>(
                mf, mmax, B, S, d2, Hb, dsh, dco, rot_c, rot_s, rdiag, g, V, L, dx0);
        } else {
            k_shift_solve_long<<<(unsigned)((S + 63) / 64), 64, 0, s>>>(mf, mmax, B, S, d2, Hb, dsh, dco, rot_c,
                                                                        rot_s, rdiag, g, gw, y, V, L, dx0);
        }
    }
    HEOM_CUDA(cudaGetLastError());
    if (prof_on() && m > j_pers) {
        // the second Gram-Schmidt passes that ran: j + 1 basis vectors read by the dots and
        // by the update, w read twice and written once
        std::vector<int> ran((size_t)m);
        HEOM_CUDA(cudaMemcpyAsync(ran.data(), dran, (size_t)m * sizeof(int), cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(cudaStreamSynchronize(s));
        for (int j = j_pers; j < m; ++j)
            if (ran[j]) prof_add(HEOM_KC_KRYLOV_VECTOR, (double)(j + 1) * Lg, (2.0 * (j + 1) + 3.0) * Lg * 16);
    }
    x0.resize((size_t)S * d2);
    res.resize(S);
    HEOM_CUDA(memcpy_counted(x0.data(), dx0, (size_t)S * d2 * 16, cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(memcpy_counted(res.data(), dres, S * 8, cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    *steps = m;
    return HEOM_OK;
}

}  // namespace heom
