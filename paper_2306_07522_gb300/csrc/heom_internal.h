// Internal declarations shared by the host code (heom_host.cpp) and the CUDA kernels.
// Nothing here is part of the public ABI (include/heom.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/heom.h"

#if defined(__CUDACC__)
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
#endif

namespace heom {

// ------------------------------------------------------------------ complex arithmetic
template <class R>
struct alignas(2 * sizeof(R)) cx {
    R re, im;
};
template <class R> HD cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <class R> HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> HD cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> HD cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R> HD cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <class R> HD cx<R> mul_i(cx<R> a) { return {-a.im, a.re}; }         // i a
template <class R> HD cx<R> mul_mi(cx<R> a) { return {a.im, -a.re}; }        // -i a
template <class R> HD R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <class R> HD void fma_to(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.re += a.re * b.re - a.im * b.im;
    acc.im += a.re * b.im + a.im * b.re;
}
template <class R> HD cx<R> cdiv(cx<R> a, cx<R> b) {
    R den = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
template <class R, class S> HD cx<R> cast(cx<S> a) { return {R(a.re), R(a.im)}; }

// ------------------------------------------------------------------ tables
// One term of Eq. HEOM for a target ADO: (M X)_i += -i (mult_l a O X_nb + mult_r b X_nb O).
struct NbEntry {
    int32_t nb;      // neighbour ADO index
    int16_t op;      // operator slot
    int16_t k;       // global exponent index
    int16_t dir;     // +1 raised neighbour (a = b = 1), -1 lowered neighbour (a, b from params)
    int16_t mult_l;  // integer factor of the left product
    int16_t mult_r;  // integer factor of the right product
    int16_t pad;
};
static_assert(sizeof(NbEntry) == 16, "NbEntry must stay 16 bytes");

struct OccEntry {  // damping term: count * rate_k
    int16_t k;
    int16_t count;
};

// Device view of a hierarchy in one precision (R = double or float).
template <class R>
struct DevView {
    int64_t N;          // number of ADOs
    int d, d2, K, n_sets, nS;
    const int32_t *row_ptr;   // [N+1]
    const NbEntry *ent;       // [E]
    const int32_t *occ_ptr;   // [N+1]
    const OccEntry *occ;      // [Eo]
    const int32_t *op_rptr;   // [n_ops*(d+1)] absolute offsets into op_rcol/op_rval
    const int32_t *op_rcol;
    const cx<R> *op_rval;
    const int32_t *op_cptr;   // [n_ops*(d+1)] absolute offsets into op_crow/op_cval
    const int32_t *op_crow;
    const cx<R> *op_cval;
    const cx<R> *coefL;       // [n_sets][K]
    const cx<R> *coefR;       // [n_sets][K]
    const cx<R> *rate;        // [n_sets][K]
    const R *floor;           // [n_sets]      damping floor for undamped ADOs (preconditioner)
    // ADO-local system superoperator L_s X = -i (H X - X H) + sum_k gamma_k J(F_k)[X] (the
    // commutator of Eq. HEOM plus the Lindblad terms of Eq. Lindbladian), one term list per
    // output element: element e reads local element s_src[j] of the same ADO with coefficient
    // s_val[set * nS + j], j = s_ptr[e] .. s_ptr[e+1]-1. Terms with the same source element
    // are merged; terms that vanish in every parameter set are dropped.
    const int32_t *s_ptr;     // [d2 + 1]
    const int32_t *s_src;     // [nS]
    const cx<R> *s_val;       // [n_sets][nS]
    const cx<R> *sdiag;       // [n_sets][d2]  coefficient of element e on itself (preconditioner)
    // Per-element term lists of every operator, for the tiled kernels: for operator slot o
    // and output element e = r*d + c, terms t_ptr[o*d2+e] .. t_ptr[o*d2+e+1]-1 read local
    // element (t_src & 0xffff) of the source block, as a left product (bit 16 clear:
    // (O X)[r][c] needs X[l][c] O[r][l]) or a right product (bit 16 set: X[r][l] O[l][c]),
    // with operator value t_val.
    const int32_t *t_ptr;     // [n_ops*d2 + 1]
    const int32_t *t_src;
    const cx<R> *t_val;
    int max_terms;            // largest term program of one ADO (incl. damping, H, trace row)
    int max_entries;          // largest neighbour-entry count of one ADO
    // ADO ranges of the persistent tiled kernel (one CTA each, balanced by term count)
    const int32_t *cta_ado;   // [n_ranges + 1]
    int n_ranges;
    int64_t tile_min_b;       // smallest batch that takes the tiled kernel (autotuned, >= 16)
    int tile_var;             // FP32 variant of the tiled kernel (kTileVariant, autotuned)
    int range_terms;          // largest program of one range (terms)
    int range_slots;          // largest sum over a range of d2 * (entries + 3)
    int range_ados;           // largest number of ADOs in a range
    // ADO ranges of the cooperative persistent solvers: one range per SM, programs of the
    // whole hierarchy resident in shared memory (pers_ranges = 0 when they do not fit)
    const int32_t *pers_ado;  // [pers_ranges + 1]
    int pers_ranges, pers_terms, pers_slots, pers_ados;
    // Per-set truncation (heom_set_truncation; both null when unused): ADO n has fermionic
    // tier ado_tier[n] & 0xffff and bosonic tier ado_tier[n] >> 16; parameter set s keeps
    // the ADOs with fermionic tier <= set_cap[s] & 0xffff and bosonic tier <= set_cap[s] >> 16
    // and holds every other ADO at zero (the apply writes zero there).
    const int32_t *ado_tier;  // [N]
    const int32_t *set_cap;   // [n_sets]
    // Float-float copies {hi.re, hi.im, lo.re, lo.im} of the FP64 tables for the float-float
    // apply (FP64 view only; null in the FP32 view)
    const float4 *op_rvalf, *op_cvalf, *s_valf, *coefLf, *coefRf, *ratef;
};

// Whether ADO n lies beyond the truncation of parameter set s.
template <class R>
HD bool beyond_cap(const DevView<R> &v, int64_t n, int s) {
    if (!v.set_cap) return false;
    const int t = v.ado_tier[n], c = v.set_cap[s];
    return (t & 0xffff) > (c & 0xffff) || (t >> 16) > (c >> 16);
}

// Optional modifiers of the apply used by the solvers (all may be null / zero).
template <class R>
struct ApplyMods {
    const cx<R> *shift;   // [B]: y += shift_b x  (spectra: -+ i w)
    R aug;                // steady state: y_(0,(0,0)) += aug * Tr x_0
};

// A device buffer owned by the library.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace heom

// The opaque handle of the public ABI.
struct heom_hier {
    int device = 0;
    int d = 0, d2 = 0, K_b = 0, K_f = 0, K = 0, tier_b = 0, tier_f = 0, parity = 1;
    int n_sets = 1, n_ops = 0;
    int64_t N = 0, N_b = 0, N_f = 0, E = 0;
    // host copies (dictionary and table export)
    std::vector<std::vector<int>> bos;      // bosonic occupation vectors in order
    std::vector<uint64_t> fer;              // fermionic subsets (bit masks) in order
    // Importance pruning (heom_build_hierarchy_pruned): the ADOs are the kept subset of the
    // full product hierarchy (full index = bosonic rank * N_f + fermionic rank), in the same
    // order. Both maps are empty without pruning (ADO index = full index).
    double importance_th = 0.0;
    std::vector<int64_t> c2f;               // [N] full index of each ADO
    std::vector<int32_t> f2c;               // [N_b * N_f] ADO of each full index, -1 if dropped
    int64_t full_of(int64_t n) const { return c2f.empty() ? n : c2f[(size_t)n]; }
    int64_t compact_of(int64_t f) const { return f2c.empty() ? f : (int64_t)f2c[(size_t)f]; }
    std::vector<int32_t> row_ptr;
    std::vector<heom::NbEntry> ent;
    std::vector<int> exp_kind;              // heom_kind per global exponent
    std::vector<int> exp_bath;              // bath per global exponent
    std::vector<int> exp_nu;                // fermionic nu per global exponent (0 for bosons)
    std::vector<int> exp_partner;           // global index of the partner (fermions)
    std::vector<int> bath_slot;             // first operator slot of each bath (fermions: d, then d^dagger)
    std::vector<heom_c64> ops;              // [n_ops][d][d]
    std::vector<heom_c64> H0;               // [n_sets][d][d]
    std::vector<heom_c64> coef0, rate0;     // [n_sets][K] as given (before the kind mapping)
    std::vector<heom_c64> lind_F;           // [n_lind][d][d] Lindblad jump operators
    std::vector<double> lind_gamma;         // [n_lind] their rates
    std::vector<heom_c64> drive;            // [n_drive][d][d] drive operators H_k of H(t)
    int n_drive = 0;
    // device tables
    heom::DBuf d_row_ptr, d_ent, d_occ_ptr, d_occ;
    heom::DBuf d_op_rptr, d_op_rcol, d_op_cptr, d_op_crow, d_op_rval64, d_op_cval64,
        d_op_rval32, d_op_cval32, d_op_rvalff, d_op_cvalff;
    heom::DBuf d_s_ptr, d_s_src;
    heom::DBuf d_tdval64;                   // [n_drive][nS] system-term values of -i[H_k, .]
    int nS = 0;                             // system terms (all elements)
    // tiled-kernel term lists (see DevView)
    heom::DBuf d_t_ptr, d_t_src, d_t_val64, d_t_val32;
    std::vector<int> op_terms;              // total terms of operator slot o over all elements
    int max_terms = 0, max_entries = 0;
    heom::DBuf d_cta_ado, d_pers_ado;
    heom::DBuf d_ado_tier, d_set_cap;    // per-set truncation (heom_set_truncation)
    // When the sets' truncation tiers do not increase from one set to the next, the sets that
    // keep ADO n are sets 0 .. act_ado[n]-1 (has_act), so the columns of a vector that can be
    // nonzero in its rows are a leading block.
    std::vector<int32_t> act_ado;
    bool has_act = false;
    int64_t kept_rowsets = 0;            // sum over rows of the sets that keep the row's ADO
    std::vector<int64_t> set_kept;       // ADOs kept by each set (per-set truncation)
    // ADOs a parameter set keeps (all of them without per-set truncation)
    int64_t kept_of_set(int s) const {
        return has_caps && (size_t)s < set_kept.size() ? set_kept[(size_t)s] : N;
    }
    bool has_caps = false;
    int n_ranges = 0, range_terms = 0, range_slots = 0, range_ados = 0;
    int tile_per_sm = 2;        // tiled kernel: ADO ranges per SM (autotuned)
    int64_t tile_min_b = 16;    // tiled kernel from this batch on (autotuned)
    int tile_var = 0;           // FP32 tiled-kernel variant (autotuned)
    int pers_ranges = 0, pers_terms = 0, pers_slots = 0, pers_ados = 0;
    heom::DBuf d_ar_ado;        // ADO ranges of the persistent Arnoldi (elements weighted)
    int ar_ranges = 0, ar_terms = 0, ar_slots = 0, ar_ados = 0;
    // device parameters (per set), both precisions and float-float
    heom::DBuf d_sval64, d_sval32, d_coefL64, d_coefL32, d_coefR64, d_coefR32, d_rate64,
        d_rate32, d_sdiag64, d_sdiag32, d_floor64, d_floor32, d_svalff, d_coefLff, d_coefRff,
        d_rateff;
    // solver workspace (grown on demand)
    heom::DBuf ws;
    heom::DBuf ws_small;
    heom::DBuf ws_pers;  // cooperative persistent solver (vectors, block partials)
    heom::DevView<double> view64() const;
    heom::DevView<float> view32() const;
};

namespace heom {

// re-partition the ADO ranges of the tiled kernel for per_sm CTAs per SM (1..5) and upload
heom_status set_tile_partition(heom_hier *h, int per_sm);

// error reporting (thread-local message)
void set_error(const char *fmt, ...);
heom_status cuda_fail(cudaError_t e, const char *what);

#define HEOM_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return heom::cuda_fail(e__, #call); \
    } while (0)

// Makes a device current for the scope of an entry point and gives the calling thread its
// previous current device back when the scope ends, so a caller that drives several GPUs
// keeps its own thread state.
struct DeviceScope {
    int prev = -1;
    cudaError_t set(int device) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) {
            prev = -1;
            return e;
        }
        if (prev == device) {
            prev = -1;
            return cudaSuccess;
        }
        return cudaSetDevice(device);
    }
    DeviceScope() = default;
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
#define HEOM_DEVICE(dev)              \
    heom::DeviceScope device_scope__; \
    HEOM_CUDA(device_scope__.set(dev))

heom_status dalloc(DBuf &b, size_t bytes);  // the library's only cudaMalloc (counted)
long long wait_limit_cycles();               // bound of device-side waits (heom_set_wait_limit)
void dfree(DBuf &b);
heom_status ensure_ws(DBuf &b, size_t bytes);  // grows b, from the workspace cache when it can
void ws_release(DBuf &b, int device);           // hands b to the workspace cache
size_t ws_cached_total(int device);             // bytes of the cached workspaces on a device
void ws_release_all();

// bounds of one ADO range of the persistent tiled kernel (shared-memory budget)
constexpr int kRangeTerms = 4096;
constexpr int kRangeSlots = 8192;
constexpr int kRangeAdos = 64;
constexpr int kPersistTerms = 6144;  // terms of one persistent range (FP64: 20 B each)
constexpr int64_t kArElemWeight = 128;  // persistent Arnoldi: balance weight of one element

// launch geometry shared by every row x column kernel: block (bx, by), grid (gx, gy)
struct Geom {
    dim3 grid, block;
    int64_t rows, B;
};
Geom make_geom(int64_t rows, int64_t B, int max_blocks_x = 0);

// launch accounting: RAII bracket of one kernel launch (see heom_profile_enable)
bool prof_on();
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s, double units, double bytes, int kernels);
void prof_add(int cls, double units, double bytes);  // work known only after a launch
// The bracket covers `kernels` kernel launches of the library (default one); the device
// time between its two events is charged to class cls.
struct Prof {
    int cls;
    cudaStream_t s;
    double units, bytes;
    bool on;
    int kernels = 1;
    Prof(int c, cudaStream_t st, double u, double by = 0.0)
        : cls(c), s(st), units(u), bytes(by), on(prof_on()) {
        if (on) prof_begin(cls, s);
    }
    ~Prof() {
        if (on) prof_end(cls, s, units, bytes, kernels);
    }
};

// cudaMemcpyAsync that adds host<->device bytes to the accounting when it is on
cudaError_t memcpy_counted(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                           cudaStream_t s);

// kernels (heom_kernels.cu)
template <class R>
cudaError_t launch_apply(const DevView<R> &v, const cx<R> *x, cx<R> *y, int64_t B,
                         const ApplyMods<R> &mods, cudaStream_t s);

// shift-invariant GMRES (heom_shifted.cu): tier-0 blocks and residual estimates per shift
heom_status shifted_gmres(heom_hier *h, const cx<double> *bvec, int64_t B,
                          const std::vector<cx<double>> &shift, const std::vector<int> &col_of,
                          double tol, int mmax, std::vector<cx<double>> &x0,
                          std::vector<double> &res, int *steps, cudaStream_t s);

// cooperative persistent BiCGStab for one column (heom_persist.cu)
template <class R>
bool persist_ok(const heom_hier *h);
template <class R>
heom_status bicgstab_persistent(heom_hier *h, const cx<R> *b, cx<R> *x, bool x_zero,
                                const cx<R> *shift, R aug, double tol, int max_iter,
                                int stall_iters, int *iters, int *status, double *rel_res,
                                cudaStream_t s);

// persistent shift-invariant Arnoldi (heom_arnoldi.cu)
bool arnoldi_persistent_ok(const heom_hier *h, int64_t B, int max_steps);
int arnoldi_max_steps();
heom_status arnoldi_persistent(heom_hier *h, int64_t B, int mmax, int max_steps, float4 *Vf, cx<double> *V,
                               cx<double> *Hb, int64_t S, const cx<double> *shift, const int *col_of,
                               double *rot_c, cx<double> *rot_s, cx<double> *rdiag, cx<double> *g,
                               float2 *rot_cf, float4 *rot_sf, const double *beta, double *res,
                               double tol, int *steps, bool *converged, cudaStream_t s);

// one fused RK4 stage over all ADOs and columns (the launch heom_evolve uses)
template <class R>
cudaError_t launch_rk4_stage(const DevView<R> &v, const cx<R> *z_in, cx<R> *z_out, cx<R> *y,
                             cx<R> *acc, int64_t B, R dt, int stage, cudaStream_t s);

}  // namespace heom
