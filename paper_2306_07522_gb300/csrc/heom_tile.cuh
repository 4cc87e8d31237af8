// Tiled HEOM apply for batched columns (B >= 32): one CTA per (group of ADOs, chunk of up
// to 8 x 32 x VC columns), one warp per 32 x VC-column slice of the chunk.
//
// For each ADO n the CTA first writes the ADO's whole term program into shared memory:
// for every output element e of the d x d block the list of (source element, complex
// coefficient) pairs of Eq. HEOM -- the damping term, the system superoperator (commutator
// with H plus any Lindblad terms), and the left and right products of every raising / lowering neighbour with its coupling operator,
// coefficients already multiplied by the exponent factors and signs. Every warp then
// streams its columns through that program: one broadcast shared-memory read, one 16-byte
// coalesced load of VC complex values and 4*VC FMAs per term and lane. The warp-uniform
// work (decoding neighbour entries, operator structure, coefficients) is done once per ADO
// per CTA instead of once per lane and term.
//
// Program order per element: damping, system superoperator, then every neighbour entry (left
// products before right products), then the trace row -- the order in which the
// per-element kernel (apply_point) adds the same terms.
#pragma once

#include "heom_kernels.cuh"

namespace heom {

template <class R> struct VecT;
template <> struct VecT<float> {
    static constexpr int VC = 2;   // complex values per lane (one float4)
};
template <> struct VecT<double> {
    static constexpr int VC = 1;   // one double2
};

constexpr int kTileWarps = 8;
constexpr int kBatch = 8;  // term loads in flight per lane

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

// Shared-memory footprint of one CTA (one ADO range) for a hierarchy view.
template <class R>
__host__ __device__ inline size_t tile_smem_bytes(const DevView<R> &v) {
    const size_t cw = 32 * VecT<R>::VC;
    return kTileWarps * cw * 3 * sizeof(double) +  // per-warp dot partials
           prog_smem_bytes<R>(v.range_terms, v.range_slots, v.range_ados, v.d2);
}

// One CTA per ADO range (persistent: all ranges resident at once). The CTA builds the term
// programs of its ADOs in shared memory once per launch, then sweeps the batch columns in
// chunks of 32 x VC; every CTA sweeps the chunks in the same order, so the data in use at
// any moment is one column chunk of every ADO (about 19 MB per vector for 2,325 ADOs of
// 4 x 4 FP32 blocks), which L2 holds while the neighbours re-read it.
//
// Program layout: triples (ADO p, element e, entry t) in that order, entry t = 0 damping,
// t = 1 system commutator, t = 2 .. E_p + 1 neighbour entries, t = E_p + 2 trace row (ADO 0
// of the steady-state system only); an exclusive scan of their term counts gives every
// term's slot, so each (p, e) item's terms are contiguous and in the apply_point order.
template <class R, int MODE>
__global__ void __launch_bounds__(kTileWarps * 32, 5) k_tile(TileArgs<R> a) {
    constexpr int VC = VecT<R>::VC;
    constexpr int CW = 32 * VC;
    const DevView<R> &v = a.v;
    const int d = v.d, d2 = v.d2, set = a.set;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int64_t B = a.B;
    const int n0 = __ldg(v.cta_ado + blockIdx.x), n1 = __ldg(v.cta_ado + blockIdx.x + 1);
    const int P = n1 - n0;

    extern __shared__ __align__(16) unsigned char smem[];
    double *s_red = reinterpret_cast<double *>(smem);  // [warps][CW][3] per-warp dot partials
    ProgSmem<R> ps = prog_layout<R>(v.range_terms, v.range_slots, v.range_ados, d2,
                                    smem + (size_t)kTileWarps * CW * 3 * sizeof(double));
    build_programs<R>(v, ps, n0, n1, a.aug, set);
    const int32_t *s_item = ps.item;
    const int32_t *s_src = ps.src;
    const cx<R> *s_coef = ps.coef;
    (void)lane;

    // ---------------- sweep the column chunks
    const cx<R> *__restrict__ X = a.x;
    const int n_items = P * d2;
    for (int64_t c0 = 0; c0 < B; c0 += CW) {
        const int64_t b = c0 + (int64_t)lane * VC;
        const bool col_ok = b < B;  // B is a multiple of VC
        cx<R> shv[VC];
        double dsum[3][VC];
#pragma unroll
        for (int j = 0; j < VC; ++j) {
            shv[j] = (a.shift && col_ok) ? a.shift[b + j] : cx<R>{R(0), R(0)};
            dsum[0][j] = dsum[1][j] = dsum[2][j] = 0.0;
        }
        if (col_ok) {
            for (int it = warp; it < n_items; it += kTileWarps) {
                const int j0 = s_item[it], j1 = s_item[it + 1];
                cx<R> acc[VC], xo[VC];
                {
                    const cx<R> cf = s_coef[j0];
                    const cx<R> *pp = X + (int64_t)s_src[j0] * B + b;
#pragma unroll
                    for (int j = 0; j < VC; ++j) {
                        xo[j] = pp[j];
                        acc[j] = (cf + shv[j]) * xo[j];
                    }
                }
                // terms in batches of kBatch so that kBatch loads are in flight at once; the
                // last batch repeats the item's final term with a zero coefficient
                for (int jj = j0 + 1; jj < j1; jj += kBatch) {
                    cx<R> cf[kBatch];
                    const cx<R> *pp[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const bool ok = jj + u < j1;
                        const int idx = ok ? jj + u : j1 - 1;
                        cf[u] = ok ? s_coef[idx] : cx<R>{R(0), R(0)};
                        pp[u] = X + (int64_t)s_src[idx] * B + b;
                    }
                    cx<R> xv[kBatch][VC];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        if constexpr (VC == 2) {
                            const float4 tq = __ldg(reinterpret_cast<const float4 *>(pp[u]));
                            xv[u][0] = cx<R>{(R)tq.x, (R)tq.y};
                            xv[u][1] = cx<R>{(R)tq.z, (R)tq.w};
                        } else {
                            const double2 tq = __ldg(reinterpret_cast<const double2 *>(pp[u]));
                            xv[u][0] = cx<R>{(R)tq.x, (R)tq.y};
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u)
#pragma unroll
                        for (int j = 0; j < VC; ++j) fma_to(acc[j], cf[u], xv[u][j]);
                }
                const int p = it / d2, e = it - p * d2;
                const int64_t i = ((int64_t)(n0 + p) * d2 + e) * B + b;
#pragma unroll
                for (int j = 0; j < VC; ++j) {
                    const cx<R> y = acc[j];
                    if constexpr (MODE == TM_STORE) {
                        a.out[i + j] = y;
                    } else if constexpr (MODE == TM_BICG_V) {
                        a.out[i + j] = y;
                        const cx<double> yd = cast<double>(y), wd = cast<double>(a.w[i + j]);
                        dsum[0][j] += wd.re * yd.re + wd.im * yd.im;
                        dsum[1][j] += wd.re * yd.im - wd.im * yd.re;
                    } else if constexpr (MODE == TM_BICG_T) {
                        a.out[i + j] = y;
                        const cx<double> yd = cast<double>(y), wd = cast<double>(a.w[i + j]);
                        dsum[0][j] += yd.re * wd.re + yd.im * wd.im;
                        dsum[1][j] += yd.re * wd.im - yd.im * wd.re;
                        dsum[2][j] += yd.re * yd.re + yd.im * yd.im;
                    } else if constexpr (MODE == TM_RESID) {
                        const cx<R> bb = a.w[i + j];
                        const cx<R> r = bb - y;
                        a.out[i + j] = r;
                        dsum[0][j] += (double)norm2(r);
                        dsum[1][j] += (double)norm2(bb);
                    } else if constexpr (MODE == TM_RK4) {
                        const R dt = a.dt;
                        if (a.stage == 1) {
                            a.acc[i + j] = y;
                            a.out[i + j] = a.y[i + j] + (R(0.5) * dt) * y;
                        } else if (a.stage == 2) {
                            a.acc[i + j] = a.acc[i + j] + R(2) * y;
                            a.out[i + j] = a.y[i + j] + (R(0.5) * dt) * y;
                        } else if (a.stage == 3) {
                            a.acc[i + j] = a.acc[i + j] + R(2) * y;
                            a.out[i + j] = a.y[i + j] + dt * y;
                        } else {
                            a.y[i + j] = a.y[i + j] + (dt / R(6)) * (a.acc[i + j] + y);
                        }
                    } else if constexpr (MODE == TM_NORMS) {
                        dsum[0][j] += (double)norm2(y);
                        dsum[1][j] += (double)norm2(xo[j]);
                    }
                }
            }
        }
        // ---------------- per-column reductions of this chunk: one atomic per column and CTA
        if constexpr (MODE == TM_BICG_V || MODE == TM_BICG_T || MODE == TM_RESID || MODE == TM_NORMS) {
#pragma unroll
            for (int j = 0; j < VC; ++j)
#pragma unroll
                for (int qv = 0; qv < 3; ++qv) s_red[(warp * CW + lane * VC + j) * 3 + qv] = dsum[qv][j];
            __syncthreads();
            if (tid < CW && c0 + tid < B) {
                double sum[3] = {0.0, 0.0, 0.0};
                for (int w = 0; w < kTileWarps; ++w)
#pragma unroll
                    for (int qv = 0; qv < 3; ++qv) sum[qv] += s_red[(w * CW + tid) * 3 + qv];
                const int64_t col = c0 + tid;
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

// Whether the tiled kernel can run this launch: one parameter set for all columns, enough
// columns to fill a warp, FP32 column count even (float4 loads), every ADO range within
// its shared-memory budget.
template <class R>
inline bool tile_ok(const DevView<R> &v, int64_t B) {
    if (B < 16 || B < v.tile_min_b || v.n_sets != 1 || v.n_ranges < 1) return false;
    if (VecT<R>::VC == 2 && (B & 1)) return false;
    if (v.range_terms > kRangeTerms || v.range_slots > kRangeSlots) return false;
    return tile_smem_bytes(v) <= 200 * 1024;
}

// the dynamic shared-memory opt-in of k_tile<R, MODE> for this view (not a stream operation)
template <class R, int MODE>
inline cudaError_t launch_tile_attr(const TileArgs<R> &a) {
    const size_t sm = tile_smem_bytes(a.v);
    if (sm <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_tile<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <class R, int MODE>
inline cudaError_t launch_tile(const TileArgs<R> &a, cudaStream_t s, bool set_attr = true) {
    const size_t sm = tile_smem_bytes(a.v);
    if (set_attr && sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tile<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_tile<R, MODE><<<a.v.n_ranges, kTileWarps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace heom
