// Tiled HEOM apply for batched columns (B >= 16): one CTA per range of ADOs, persistent over
// the batch; one warp per 32 x VC-column slice of a column chunk.
//
// For each ADO n the CTA first writes the ADO's whole term program into shared memory:
// for every output element e of the d x d block the list of (source element, complex
// coefficient) pairs of Eq. HEOM -- the damping term, the system superoperator (commutator
// with H plus any Lindblad terms), and the left and right products of every raising /
// lowering neighbour with its coupling operator, coefficients already multiplied by the
// exponent factors and signs. Every warp then streams its columns through that program. Per
// term and lane: one broadcast shared-memory read of the term's record (coefficient and row
// offset: FP32) or two (FP64), VC/2 16-byte coalesced loads (FP32, VC = 4 or 2 columns) or one
// (FP64), and two packed f32x2 FMAs per column (FP32) or one complex FMA (FP64). The warp-uniform
// work (decoding neighbour entries, operator structure, coefficients, row offsets) is done
// once per ADO per CTA instead of once per lane and term.
//
// Program order per element: damping, system superoperator, then every neighbour entry (left
// products before right products), then the trace row -- the order in which the
// per-element kernel (apply_point) adds the same terms. The FP32 sweep accumulates the real
// and imaginary parts of the coefficients in separate sums, so its rounding differs from the
// per-element kernel's (both within FP32 accuracy of the exact apply).
#pragma once

#include <algorithm>

#include "heom_kernels.cuh"

namespace heom {

constexpr int kTileWarps = 8;

// Epilogue modes of the tiled kernel
enum TileMode {
    TM_STORE = 0,    // y = M x
    TM_BICG_V = 1,   // v = A ph;   acc_rv += (rh, v)
    TM_BICG_T = 2,   // t = A sh;   acc_ts += (t, s), acc_tt += (t, t)
    TM_RESID = 3,    // r = b - A x; acc_nr += |r|^2, bnorm2 += |b|^2
    TM_RK4 = 4,      // fused RK4 stage (stage number in args)
    TM_NORMS = 5     // |M x|^2, |x|^2 per column
};

template <class R>
struct TileArgs {
    DevView<R> v;
    const cx<R> *x;      // input vector of the apply
    cx<R> *out;          // output (y, v, t, r, z_out)
    const cx<R> *w;      // dot operand (rh, s), right-hand side b (TM_RESID)
    cx<R> *y;            // RK4 state
    cx<R> *acc;          // RK4 accumulator
    const cx<R> *shift;  // [B] or null
    R aug;               // trace augmentation of the (0,(0,0)) equation
    R dt;
    int stage;
    ColState *st;        // per-column solver state (dot modes)
    double *norms;       // TM_NORMS output [2B]
    int64_t B;
    int set;             // parameter set (every column of this launch uses it)
};

// Shared-memory layout of the term programs of one ADO range (see build_programs).
template <class R>
struct ProgSmem {
    cx<R> *coef, *cl, *cr;
    int32_t *src, *off, *item, *nb, *op, *pb, *scan;
};

template <class R>
__host__ __device__ inline size_t prog_smem_bytes(int terms, int slots, int ados, int d2) {
    const size_t pairs = (size_t)slots / (size_t)d2 + 1, items = (size_t)ados * d2 + 1;
    return ((size_t)terms + 2 * pairs) * sizeof(cx<R>) +
           ((size_t)terms + (size_t)slots + items + 2 * pairs + (size_t)ados + 2 + 1024) *
               sizeof(int32_t) + 32;
}

template <class R>
__device__ inline ProgSmem<R> prog_layout(int terms, int slots, int ados, int d2,
                                          unsigned char *base) {
    ProgSmem<R> s;
    const int pairs = slots / d2 + 1, items = ados * d2 + 1;
    s.coef = reinterpret_cast<cx<R> *>(base);  // [terms]
    s.cl = s.coef + terms;                       // [pairs]
    s.cr = s.cl + pairs;                         // [pairs]
    s.src = reinterpret_cast<int32_t *>(s.cr + pairs);  // [terms]
    s.off = s.src + terms;                       // [triples]
    s.item = s.off + slots;                      // [items] program start of (p, e)
    s.nb = s.item + items;                       // [pairs]
    s.op = s.nb + pairs;                         // [pairs] op slot / -1 H / -2 trace / -3 damping
    s.pb = s.op + pairs;                         // [ados + 2] first pair of ADO p
    s.scan = s.pb + ados + 2;                    // [<= 1024 threads] scan scratch
    return s;
}

// Build, in shared memory, the term programs of ADOs n0 .. n1-1 (all threads of the block
// take part; blockDim.x a multiple of 32, at most 1024). Program layout: triples (ADO p,
// element e, entry t) in that order, entry t = 0 damping, t = 1 system commutator,
// t = 2 .. E_p + 1 neighbour entries, t = E_p + 2 trace row (ADO 0 of the steady-state
// system only); an exclusive scan of their term counts gives every term's slot, so each
// (p, e) item's terms are contiguous and in the apply_point order. Item i = p * d2 + e
// holds terms item[i] .. item[i+1]-1 as (source element src, coefficient coef).
template <class R>
__device__ void build_programs(const DevView<R> &v, ProgSmem<R> &ps, int n0, int n1, R aug,
                               int set) {
    const int d = v.d, d2 = v.d2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    const int P = n1 - n0;
    cx<R> *s_coef = ps.coef, *s_cl = ps.cl, *s_cr = ps.cr;
    int32_t *s_src = ps.src, *s_off = ps.off, *s_item = ps.item, *s_nb = ps.nb, *s_op = ps.op,
            *s_pb = ps.pb, *s_scan = ps.scan;
    // ---------------- pair bases (entries + 3 per ADO): warp 0 scans the ranges' ADOs
    if (warp == 0) {
        int carry = 0;
        for (int p0 = 0; p0 < P; p0 += 32) {
            const int p = p0 + lane;
            const int cnt = p < P ? __ldg(v.row_ptr + n0 + p + 1) - __ldg(v.row_ptr + n0 + p) + 3 : 0;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int nbv = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += nbv;
            }
            if (p < P) s_pb[p] = carry + incl - cnt;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) s_pb[P] = carry;
    }
    __syncthreads();
    const int n_pairs = s_pb[P];
    const int n_triples = n_pairs * d2;
    auto ado_of_pair = [&](int q) {  // largest p with s_pb[p] <= q
        int lo = 0, hi = P - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pb[mid] <= q) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    // ---------------- per pair: source block and left/right factors
    for (int q = tid; q < n_pairs; q += blockDim.x) {
        const int p = ado_of_pair(q), t = q - s_pb[p];
        const int n = n0 + p;
        const int e0 = __ldg(v.row_ptr + n), E = __ldg(v.row_ptr + n + 1) - e0;
        int nb = n, op;
        cx<R> cl{R(0), R(0)}, cr{R(0), R(0)};
        if (t == 0) {
            op = -3;  // damping: coefficient filled per element below
        } else if (t == 1) {
            op = -1;  // system superoperator: coefficients taken from s_val
        } else if (t <= E + 1) {
            const int4 raw = __ldg(reinterpret_cast<const int4 *>(v.ent) + e0 + t - 2);
            const int k = (int)(int16_t)(raw.y >> 16);
            const int dir = (int)(int16_t)(raw.z & 0xffff);
            const R ml = R((int16_t)(raw.z >> 16)), mr = R((int16_t)(raw.w & 0xffff));
            nb = raw.x;
            op = (int)(int16_t)(raw.y & 0xffff);
            if (dir > 0) {
                cl = cx<R>{R(0), -ml};
                cr = cx<R>{R(0), -mr};
            } else {
                const int64_t pk = (int64_t)set * v.K + k;
                cl = mul_mi(ml * ldc(v.coefL + pk));
                cr = mul_mi(mr * ldc(v.coefR + pk));
            }
        } else {
            op = -2;  // trace row of the steady-state system
            nb = 0;
            cl = cx<R>{aug, R(0)};
        }
        s_nb[q] = nb;
        s_op[q] = op;
        s_cl[q] = cl;
        s_cr[q] = cr;
    }
    __syncthreads();
    // ---------------- term count of every triple, ordered (p, e, t)
    for (int z = tid; z < n_triples; z += blockDim.x) {
        const int p = ado_of_pair(z / d2);  // triples of ADO p start at d2 * s_pb[p]
        const int E1 = s_pb[p + 1] - s_pb[p];
        const int loc = z - d2 * s_pb[p];
        const int e = loc / E1, t = loc - e * E1;
        const int op = s_op[s_pb[p] + t];
        int len;
        if (op >= 0) len = __ldg(v.t_ptr + op * d2 + e + 1) - __ldg(v.t_ptr + op * d2 + e);
        else if (op == -1) len = __ldg(v.s_ptr + e + 1) - __ldg(v.s_ptr + e);
        else if (op == -3) len = 1;
        else len = (e == 0 && n0 + p == 0 && aug != R(0)) ? d : 0;
        s_off[z] = len;
    }
    __syncthreads();
    // ---------------- exclusive scan of the counts (contiguous segment per thread)
    {
        const int per = (n_triples + blockDim.x - 1) / blockDim.x;
        const int z0 = tid * per, z1 = min(z0 + per, n_triples);
        int sum = 0;
        for (int z = z0; z < z1; ++z) sum += s_off[z];
        // block-wide exclusive scan of the per-thread sums: warp shuffles, then warp totals
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nbv = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += nbv;
        }
        if (lane == 31) s_scan[warp] = incl;
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int w = 0; w < nwarps; ++w) {
                const int tmp = s_scan[w];
                s_scan[w] = run;
                run += tmp;
            }
        }
        __syncthreads();
        int acc = s_scan[warp] + incl - sum;
        for (int z = z0; z < z1; ++z) {
            const int tmp = s_off[z];
            s_off[z] = acc;
            acc += tmp;
        }
        if (z1 == n_triples && z0 < z1) s_item[P * d2] = acc;
        if (n_triples == 0 && tid == 0) s_item[0] = 0;
    }
    __syncthreads();
    for (int i = tid; i < P * d2; i += blockDim.x) {
        const int p = i / d2, e = i - p * d2;
        s_item[i] = s_off[d2 * s_pb[p] + e * (s_pb[p + 1] - s_pb[p])];
    }
    // ---------------- fill the programs
    const cx<R> *sv = v.s_val + (int64_t)set * v.nS;
    for (int z = tid; z < n_triples; z += blockDim.x) {
        const int p = ado_of_pair(z / d2);
        const int E1 = s_pb[p + 1] - s_pb[p];
        const int loc = z - d2 * s_pb[p];
        const int e = loc / E1, t = loc - e * E1;
        const int q = s_pb[p] + t, op = s_op[q];
        int pos = s_off[z];
        const int32_t nbase = s_nb[q] * d2;
        if (op >= 0) {
            for (int j = __ldg(v.t_ptr + op * d2 + e), j1 = __ldg(v.t_ptr + op * d2 + e + 1); j < j1;
                 ++j, ++pos) {
                const int32_t src = __ldg(v.t_src + j);
                s_src[pos] = nbase + (src & 0xffff);
                s_coef[pos] = ((src >> 16) ? s_cr[q] : s_cl[q]) * ldc(v.t_val + j);
            }
        } else if (op == -1) {
            for (int j = __ldg(v.s_ptr + e), j1 = __ldg(v.s_ptr + e + 1); j < j1; ++j, ++pos) {
                s_src[pos] = nbase + __ldg(v.s_src + j);
                s_coef[pos] = ldc(sv + j);
            }
        } else if (op == -3) {
            const cx<R> dmp = damping_of(v, (int64_t)(n0 + p), set);
            s_src[pos] = (n0 + p) * d2 + e;
            s_coef[pos] = cx<R>{-dmp.re, -dmp.im};
        } else if (e == 0 && n0 + p == 0 && aug != R(0)) {
            for (int i = 0; i < d; ++i, ++pos) {
                s_src[pos] = i * d + i;
                s_coef[pos] = s_cl[q];
            }
        }
    }
    __syncthreads();

}

// Variants of the FP32 tiled kernel. P: float4 loads per lane and term (VC = 2P columns per
// lane; lane L reads columns 2L, 2L+1 of each 64-column half of its chunk, so every load
// instruction of a warp covers 512 contiguous bytes); U: terms per item loaded into registers
// together (their loads are in flight at once); KI: items (consecutive elements of one ADO,
// of similar term counts) in flight per warp; minb: the CTAs per SM the register budget is
// sized for. The kernel is bound by the latency of the neighbour gathers from L2, so what
// matters is the loads a warp keeps in flight times the warps an SM holds; the autotuner
// picks one variant per hierarchy. FP64 runs one (one double2 per lane, four terms, one
// item): the FP64 pipe bounds it. (Measured and dropped: a per-warp cp.async ring 8 to 24
// terms deep, with the terms of all the warp's items in one stream -- twice as slow: its
// per-term bookkeeping made it issue-bound.)
struct TileVariant {
    int P, U, KI, minb;
};
constexpr int kTileVariants = 6;
constexpr TileVariant kTileVariant[kTileVariants] = {
    {1, 4, 1, 3}, {1, 4, 1, 4}, {1, 3, 1, 4}, {1, 2, 1, 5}, {1, 6, 1, 3}, {2, 4, 1, 2}};

// Columns of one chunk (one warp-wide slice) of a variant.
template <class R>
inline int tile_cw(int var) {
    return sizeof(R) == 8 ? 32 : 64 * kTileVariant[var].P;
}

// Whether an epilogue mode sums per-column dot products (and needs the per-warp partials).
__host__ __device__ constexpr bool tile_mode_dots(int mode) {
    return mode == TM_BICG_V || mode == TM_BICG_T || mode == TM_RESID || mode == TM_NORMS;
}

// Shared-memory footprint of one CTA (one ADO range): per-warp dot partials (dot modes only),
// the FP32 broadcast coefficient records, the term programs.
template <class R>
__host__ __device__ inline size_t tile_smem_bytes(const DevView<R> &v, int cw, bool dots) {
    const size_t rec = sizeof(R) == 4 ? 16 * (size_t)v.range_terms : 0;
    return (dots ? kTileWarps * (size_t)cw * 3 * sizeof(double) : 0) + rec +
           prog_smem_bytes<R>(v.range_terms, v.range_slots, v.range_ados, v.d2);
}
template <class R>
inline size_t tile_smem_bytes_var(const DevView<R> &v, int var) {  // the largest (dot modes)
    return tile_smem_bytes(v, sizeof(R) == 8 ? 32 : 64 * kTileVariant[var].P, true);
}

// d = a * b + c on a pair of floats: one packed FP32 FMA (fma.rn.f32x2).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// A = sum cr (re, im), Bq = sum ci (re, im) over a term with record (cr, ci, row offset, -)
// and the two columns x = (re0, im0, re1, im1) of one float4.
__device__ __forceinline__ void term_f32(float4 c, float4 x, float2 &A0, float2 &B0, float2 &A1,
                                         float2 &B1) {
    const float2 cr = make_float2(c.x, c.x), ci = make_float2(c.y, c.y);
    const float2 x0 = make_float2(x.x, x.y), x1 = make_float2(x.z, x.w);
    A0 = ffma2(cr, x0, A0);
    B0 = ffma2(ci, x0, B0);
    A1 = ffma2(cr, x1, A1);
    B1 = ffma2(ci, x1, B1);
}

// Sum of the terms of KI items for the 2P columns of this lane (register path): item k's
// terms are jb[k] .. jb[k] + len[k] - 1 (its damping term excluded), taken U at a time from
// every item at once. Each term's record s_c4[j] = (cr, ci, row offset as int bits, 0) is one
// 16-byte broadcast read. With x = (re, im) per column the lane keeps A = sum cr (re, im) and
// Bq = sum ci (re, im) in packed pairs -- two f32x2 FMAs per term and column -- and forms
// sum c x = (A.re - Bq.im, A.im + Bq.re) at the end. Terms past an item's end are predicated
// off (no load, no arithmetic). pv[p]: pair p of this lane lies inside the batch (only the
// last chunk has invalid pairs).
template <int P, int U, int KI>
__device__ __forceinline__ void tile_terms_f32(const float4 *__restrict__ s_c4,
                                               const int32_t *__restrict__ s_off,
                                               const cx<float> *__restrict__ Xb,
                                               const int (&jb)[KI], const int (&len)[KI],
                                               int maxlen, const bool (&pv)[P],
                                               float2 (&A)[KI][2 * P], float2 (&Bq)[KI][2 * P]) {
    for (int t = 0; t < maxlen; t += U) {
        float4 cc[KI][U];
        float4 xv[KI][U][P];
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t + u < len[k]) {
                    cc[k][u] = s_c4[jb[k] + t + u];  // one shared-memory read per term
                    const float4 *p = reinterpret_cast<const float4 *>(Xb + __float_as_int(cc[k][u].z));
#pragma unroll
                    for (int q = 0; q < P; ++q)
                        xv[k][u][q] = pv[q] ? __ldg(p + 32 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (t + u < len[k]) {
#pragma unroll
                    for (int q = 0; q < P; ++q)
                        term_f32(cc[k][u], xv[k][u][q], A[k][2 * q], Bq[k][2 * q], A[k][2 * q + 1],
                                 Bq[k][2 * q + 1]);
                }
    }
}

// FP64: complex FMAs (GB300 has no packed FP64 FMA; the FP64 pipe bounds this path).
template <int U>
__device__ __forceinline__ void tile_terms_f64(const cx<double> *__restrict__ s_coef,
                                               const int32_t *__restrict__ s_off,
                                               const cx<double> *__restrict__ Xb, int j0, int j1,
                                               cx<double> &acc) {
    for (int j = j0; j < j1; j += U) {
        cx<double> cc[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < j1) {
                cc[u] = s_coef[j + u];
                const double2 t = __ldg(reinterpret_cast<const double2 *>(Xb + s_off[j + u]));
                xv[u] = cx<double>{t.x, t.y};
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < j1) fma_to(acc, cc[u], xv[u]);
    }
}

// The epilogue of one item: its output y (VC values of this lane) and own input xo, written
// or folded into the solver's per-column sums according to MODE. rb: the item's row at the
// chunk start; co(q): column offset of value q inside the chunk; pv: valid pairs.
template <class R, int MODE, int VC, int NP, class CO>
__device__ __forceinline__ void tile_epilogue(const TileArgs<R> &a, int64_t rb, const CO &co,
                                              const bool (&pv)[NP], const cx<R> (&y)[VC],
                                              const cx<R> (&xo)[VC], double (&dsum)[3][VC]) {
    constexpr bool F32 = sizeof(R) == 4;
    if constexpr (MODE == TM_STORE) {
        if constexpr (F32) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
                if (pv[p])
                    __stcs(reinterpret_cast<float4 *>(a.out + rb + co(2 * p)),
                           make_float4(y[2 * p].re, y[2 * p].im, y[2 * p + 1].re, y[2 * p + 1].im));
        } else {
            __stcs(reinterpret_cast<double2 *>(a.out + rb + co(0)), make_double2(y[0].re, y[0].im));
        }
    } else {
#pragma unroll
        for (int q = 0; q < VC; ++q) {
            if (!pv[F32 ? q >> 1 : 0]) continue;
            const int64_t i = rb + co(q);
            const cx<R> yj = y[q];
            if constexpr (MODE == TM_BICG_V) {
                a.out[i] = yj;
                const cx<double> yd = cast<double>(yj), wd = cast<double>(a.w[i]);
                dsum[0][q] += wd.re * yd.re + wd.im * yd.im;
                dsum[1][q] += wd.re * yd.im - wd.im * yd.re;
            } else if constexpr (MODE == TM_BICG_T) {
                a.out[i] = yj;
                const cx<double> yd = cast<double>(yj), wd = cast<double>(a.w[i]);
                dsum[0][q] += yd.re * wd.re + yd.im * wd.im;
                dsum[1][q] += yd.re * wd.im - yd.im * wd.re;
                dsum[2][q] += yd.re * yd.re + yd.im * yd.im;
            } else if constexpr (MODE == TM_RESID) {
                const cx<R> bb = a.w[i];
                const cx<R> r = bb - yj;
                a.out[i] = r;
                dsum[0][q] += (double)norm2(r);
                dsum[1][q] += (double)norm2(bb);
            } else if constexpr (MODE == TM_RK4) {
                const R dt = a.dt;
                if (a.stage == 1) {
                    a.acc[i] = yj;
                    a.out[i] = a.y[i] + (R(0.5) * dt) * yj;
                } else if (a.stage == 2) {
                    a.acc[i] = a.acc[i] + R(2) * yj;
                    a.out[i] = a.y[i] + (R(0.5) * dt) * yj;
                } else if (a.stage == 3) {
                    a.acc[i] = a.acc[i] + R(2) * yj;
                    a.out[i] = a.y[i] + dt * yj;
                } else {
                    a.y[i] = a.y[i] + (dt / R(6)) * (a.acc[i] + yj);
                }
            } else if constexpr (MODE == TM_NORMS) {
                dsum[0][q] += (double)norm2(yj);
                dsum[1][q] += (double)norm2(xo[q]);
            }
        }
    }
}

// One CTA per ADO range (persistent: all ranges resident at once). The CTA builds the term
// programs of its ADOs in shared memory once per launch and turns each term's source element
// into a row offset (source * B, 32-bit: the launch needs N d^2 B < 2^31) and, in FP32, a
// broadcast coefficient record; then it sweeps the batch columns in chunks of CW columns
// (FP32: 64 P; FP64: 32). Every CTA sweeps the chunks in the same order, so the data in use
// at any moment is one column chunk of every ADO (19 MB per vector for 2,325 ADOs of 4 x 4
// FP32 blocks at CW = 64), which L2 holds while the neighbours re-read it. The output row of
// item it is n0 d^2 + it. An item's first term is its damping term on its own element
// (build_programs), which also supplies the input element x_own. Value q of a lane is column
// c0 + 64 (q / 2) + 2 lane + q % 2 (FP32) or c0 + lane (FP64).
template <class R, int MODE, int P, int U, int KI, int MINB>
__global__ void __launch_bounds__(kTileWarps * 32, MINB) k_tile(TileArgs<R> a) {
    constexpr bool F32 = sizeof(R) == 4;
    constexpr int VC = F32 ? 2 * P : 1;   // values (columns) per lane
    constexpr int NP = F32 ? P : 1;       // 16-byte loads per lane and term
    constexpr int CW = F32 ? 64 * P : 32;
    constexpr int K = F32 ? KI : 1;       // items in flight per warp
    const DevView<R> &v = a.v;
    const int d2 = v.d2, set = a.set;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int64_t B = a.B;
    const int n0 = __ldg(v.cta_ado + blockIdx.x), n1 = __ldg(v.cta_ado + blockIdx.x + 1);
    const int P_ados = n1 - n0;

    extern __shared__ __align__(16) unsigned char smem[];
    double *s_red = reinterpret_cast<double *>(smem);  // [warps][CW][3] per-warp dot partials
    unsigned char *after_red = smem + (tile_mode_dots(MODE) ? (size_t)kTileWarps * CW * 3 * sizeof(double) : 0);
    float4 *s_c4 = reinterpret_cast<float4 *>(after_red);  // FP32 records [range_terms]
    ProgSmem<R> ps = prog_layout<R>(v.range_terms, v.range_slots, v.range_ados, d2,
                                    after_red + (F32 ? 16 * (size_t)v.range_terms : 0));
    build_programs<R>(v, ps, n0, n1, a.aug, set);
    const int n_items = P_ados * d2;
    const int n_terms = ps.item[n_items];
    // row offsets, and in FP32 one 16-byte record per term: (cr, ci, row offset, 0)
    for (int j = tid; j < n_terms; j += blockDim.x) {
        ps.src[j] = (int32_t)((int64_t)ps.src[j] * B);
        if constexpr (F32) {
            const cx<float> c = ps.coef[j];
            s_c4[j] = make_float4(c.re, c.im, __int_as_float(ps.src[j]), 0.f);
        }
    }
    __syncthreads();
    const int32_t *__restrict__ s_item = ps.item;
    const int32_t *__restrict__ s_off = ps.src;
    const cx<R> *__restrict__ s_coef = ps.coef;
    const int64_t row0 = (int64_t)n0 * d2;
    // column offset of value q inside a chunk
    auto co = [&](int q) -> int { return F32 ? (q >> 1) * 64 + 2 * lane + (q & 1) : lane; };

    // ---------------- sweep the column chunks
    for (int64_t c0 = 0; c0 < B; c0 += CW) {
        bool pv[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) pv[p] = c0 + co(2 * p) < B;  // B is even (FP32)
        const cx<R> *__restrict__ Xb = a.x + c0 + co(0);
        cx<R> shv[VC];
        double dsum[3][VC];
#pragma unroll
        for (int q = 0; q < VC; ++q) {
            const bool ok = pv[F32 ? q >> 1 : 0];
            shv[q] = (a.shift && ok) ? a.shift[c0 + co(q)] : cx<R>{R(0), R(0)};
            dsum[0][q] = dsum[1][q] = dsum[2][q] = 0.0;
        }
        if (pv[0]) {
            for (int it0 = warp * K; it0 < n_items; it0 += kTileWarps * K) {
                int jb[K], len[K], maxlen = 0;
                cx<R> xo[K][VC], y[K][VC];
                cx<R> cf0[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const bool ok = it0 + k < n_items;
                    const int j0 = ok ? s_item[it0 + k] : 0;
                    jb[k] = j0 + 1;
                    len[k] = ok ? s_item[it0 + k + 1] - j0 - 1 : 0;
                    maxlen = max(maxlen, len[k]);
                    cf0[k] = ok ? s_coef[j0] : cx<R>{R(0), R(0)};
                    // first term: damping (+ shift) on the item's own element
                    const cx<R> *pp = Xb + (ok ? s_off[j0] : 0);
                    if constexpr (F32) {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const float4 t = (ok && pv[p]) ? __ldg(reinterpret_cast<const float4 *>(pp) + 32 * p)
                                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                            xo[k][2 * p] = cx<R>{t.x, t.y};
                            xo[k][2 * p + 1] = cx<R>{t.z, t.w};
                        }
                    } else {
                        const double2 t = ok ? __ldg(reinterpret_cast<const double2 *>(pp)) : make_double2(0.0, 0.0);
                        xo[k][0] = cx<R>{t.x, t.y};
                    }
                }
                if constexpr (F32) {
                    float2 A[K][VC], Bq[K][VC];
#pragma unroll
                    for (int k = 0; k < K; ++k)
#pragma unroll
                        for (int q = 0; q < VC; ++q) {
                            const cx<float> f = (cf0[k] + shv[q]) * xo[k][q];
                            A[k][q] = make_float2(f.re, f.im);
                            Bq[k][q] = make_float2(0.f, 0.f);
                        }
                    tile_terms_f32<P, U, K>(s_c4, s_off, Xb, jb, len, maxlen, pv, A, Bq);
#pragma unroll
                    for (int k = 0; k < K; ++k)
#pragma unroll
                        for (int q = 0; q < VC; ++q)
                            y[k][q] = cx<R>{A[k][q].x - Bq[k][q].y, A[k][q].y + Bq[k][q].x};
                } else {
                    cx<double> acc = (cf0[0] + shv[0]) * xo[0][0];
                    tile_terms_f64<U>(reinterpret_cast<const cx<double> *>(s_coef), s_off,
                                      reinterpret_cast<const cx<double> *>(Xb), jb[0], jb[0] + len[0], acc);
                    y[0][0] = cx<R>{acc.re, acc.im};
                }
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (it0 + k < n_items)
                        tile_epilogue<R, MODE, VC, NP>(a, (row0 + it0 + k) * B + c0, co, pv, y[k], xo[k], dsum);
            }
        }
        // ---------------- per-column reductions of this chunk: one atomic per column and CTA
        if constexpr (tile_mode_dots(MODE)) {
#pragma unroll
            for (int q = 0; q < VC; ++q)
#pragma unroll
                for (int qv = 0; qv < 3; ++qv) s_red[(warp * CW + co(q)) * 3 + qv] = dsum[qv][q];
            __syncthreads();
            for (int t = tid; t < CW && c0 + t < B; t += blockDim.x) {
                double sum[3] = {0.0, 0.0, 0.0};
                for (int w = 0; w < kTileWarps; ++w)
#pragma unroll
                    for (int qv = 0; qv < 3; ++qv) sum[qv] += s_red[(w * CW + t) * 3 + qv];
                const int64_t col = c0 + t;
                if constexpr (MODE == TM_NORMS) {
                    atomicAdd(a.norms + 2 * col, sum[0]);
                    atomicAdd(a.norms + 2 * col + 1, sum[1]);
                } else {
                    ColState *sc = a.st + col;
                    if (sc->active) {
                        if constexpr (MODE == TM_BICG_V) {
                            atomicAdd(&sc->acc_rv.re, sum[0]);
                            atomicAdd(&sc->acc_rv.im, sum[1]);
                        } else if constexpr (MODE == TM_BICG_T) {
                            atomicAdd(&sc->acc_ts.re, sum[0]);
                            atomicAdd(&sc->acc_ts.im, sum[1]);
                            atomicAdd(&sc->acc_tt.re, sum[2]);
                            if (blockIdx.x == 0) {
                                sc->acc_rr = {0.0, 0.0};
                                sc->acc_nr = 0.0;
                            }
                        } else {
                            atomicAdd(&sc->acc_nr, sum[0]);
                            atomicAdd(&sc->bnorm2, sum[1]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Variant the tiled kernel runs for a launch of B columns: the hierarchy's (autotuned) FP32
// variant, or variant 0 (one float4 per lane) when B does not fill a 128-column chunk; FP64
// has one.
template <class R>
inline int tile_var_of(const DevView<R> &v, int64_t B) {
    if (sizeof(R) == 8) return 0;
    int var = v.tile_var;
    if (var < 0 || var >= kTileVariants) var = 0;
    if (kTileVariant[var].P == 2 && B < 128) var = 0;
    return var;
}

// Whether the tiled kernel can run this launch: one parameter set for all columns, enough
// columns to fill a warp, FP32 column count even (16-byte loads), 32-bit row offsets
// (N d^2 B < 2^31), every ADO range within its shared-memory budget.
template <class R>
inline bool tile_ok(const DevView<R> &v, int64_t B) {
    if (B < 16 || B < v.tile_min_b || v.n_sets != 1 || v.n_ranges < 1 || v.set_cap) return false;
    if (sizeof(R) == 4 && (B & 1)) return false;
    if ((double)v.N * v.d2 * (double)B >= 2147483647.0) return false;
    if (v.range_terms > kRangeTerms || v.range_slots > kRangeSlots) return false;
    return tile_smem_bytes_var(v, tile_var_of(v, B)) <= 200 * 1024;
}

// attr_only: set the dynamic shared-memory opt-in and launch nothing (needed before a launch
// is captured into a graph; not a stream operation)
template <class R, int MODE, int P, int U, int KI, int MINB>
inline cudaError_t launch_tile_var(const TileArgs<R> &a, cudaStream_t s, bool set_attr, bool attr_only) {
    constexpr int CW = sizeof(R) == 8 ? 32 : 64 * P;
    const size_t sm = tile_smem_bytes(a.v, CW, tile_mode_dots(MODE));
    if (set_attr || attr_only) {
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_tile<R, MODE, P, U, KI, MINB>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        // shared memory for the resident CTAs only: the rest of the SM's 256 KB of L1/shared
        // storage stays L1, which serves the neighbour re-reads
        const int pct = (int)std::min<size_t>(100, (MINB * (sm + 1024) * 100 + 232447) / 232448);
        cudaError_t e = cudaFuncSetAttribute(k_tile<R, MODE, P, U, KI, MINB>,
                                             cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        if (e != cudaSuccess) return e;
    }
    if (attr_only) return cudaSuccess;
    k_tile<R, MODE, P, U, KI, MINB><<<a.v.n_ranges, kTileWarps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

#define HEOM_TILE_VAR(i)                                                                    \
    launch_tile_var<R, MODE, kTileVariant[i].P, kTileVariant[i].U, kTileVariant[i].KI,       \
                    kTileVariant[i].minb>(a, s, set_attr, attr_only)

template <class R, int MODE>
inline cudaError_t launch_tile_dispatch(const TileArgs<R> &a, cudaStream_t s, bool set_attr,
                                        bool attr_only) {
    if constexpr (sizeof(R) == 8) {
        return launch_tile_var<R, MODE, 1, 4, 1, 3>(a, s, set_attr, attr_only);
    } else {
        switch (tile_var_of(a.v, a.B)) {
        case 0: return HEOM_TILE_VAR(0);
        case 1: return HEOM_TILE_VAR(1);
        case 2: return HEOM_TILE_VAR(2);
        case 3: return HEOM_TILE_VAR(3);
        case 4: return HEOM_TILE_VAR(4);
        default: return HEOM_TILE_VAR(5);
        }
    }
}
#undef HEOM_TILE_VAR

// the dynamic shared-memory opt-in of the kernel a launch of these arguments runs
template <class R, int MODE>
inline cudaError_t launch_tile_attr(const TileArgs<R> &a) {
    return launch_tile_dispatch<R, MODE>(a, 0, true, true);
}

template <class R, int MODE>
inline cudaError_t launch_tile(const TileArgs<R> &a, cudaStream_t s, bool set_attr = true) {
    return launch_tile_dispatch<R, MODE>(a, s, set_attr, false);
}

}  // namespace heom
