// Device building blocks shared by the kernels: the matrix-free HEOM apply at one point,
// the block-local preconditioner and block reductions into per-column FP64 accumulators.
#pragma once

#include "heom_internal.h"

namespace heom {

// BiCGStab restart rule: when |(rh, r)| < tau ||rh|| ||r|| the shadow residual rh has lost
// its grip on the Krylov space (the Lanczos biorthogonality behind the method has broken
// down in all but name); the iteration restarts with rh = r, p = r. tau = 1e-10. A sparse
// right-hand side such as the trace row of the stationary-state system makes the initial
// rh = b a poor shadow vector, and without the restart the recursion can stagnate.
constexpr double kRestartTau2 = 1e-20;

// Per-column solver state; every field is FP64 (Krylov scalars, dots, residuals).
struct ColState {
    cx<double> rho_old, alpha, omega;      // BiCGStab scalars
    cx<double> acc_rv, acc_ts, acc_tt, acc_rr;  // dot-product accumulators
    double acc_nr;                          // ||r||^2 accumulator
    double bnorm2;                          // ||b||^2
    double rhn;                             // ||rh||^2 of the current shadow residual
    int active;                             // 1 while the column iterates
    int flag;                               // breakdown marker
    int restart;                            // this iteration restarts (rh = r, p = r)
    int pad_;
};

template <class R>
__device__ __forceinline__ cx<R> ldc(const cx<R> *p) {
    if constexpr (sizeof(R) == 8) {
        double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        return cx<R>{t.x, t.y};
    } else {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        return cx<R>{t.x, t.y};
    }
}

template <class R>
__device__ __forceinline__ cx<R> damping_of(const DevView<R> &v, int64_t n, int set) {
    cx<R> dmp{R(0), R(0)};
    const int o1 = __ldg(v.occ_ptr + n + 1);
    for (int o = __ldg(v.occ_ptr + n); o < o1; ++o) {
        const int packed = __ldg(reinterpret_cast<const int *>(v.occ) + o);
        const int k = (int)(int16_t)(packed & 0xffff);
        const int cnt = (int)(int16_t)(packed >> 16);
        dmp = dmp + R(cnt) * ldc(v.rate + (int64_t)set * v.K + k);
    }
    return dmp;
}

// (M X)[n][e][b]: Eq. HEOM evaluated at ADO n, element e = r*d + c, batch column b.
// X points at the start of the ADO vector ([N][d2][B]). Zero for an ADO beyond the
// truncation of the column's parameter set (heom_set_truncation): with the input zero there
// too, this is the apply of that set's own, shallower hierarchy, whose ADOs are those of this
// one within the set's tiers, in the same relative order (neighbours beyond the tiers are
// not read: their couplings are the ones the truncation drops).
template <class R>
__device__ __forceinline__ cx<R> apply_point(const DevView<R> &v, const cx<R> *__restrict__ X,
                                             int64_t n, int e, int64_t b, int64_t B, int set,
                                             const cx<R> &damp) {
    if (beyond_cap(v, n, set)) return cx<R>{R(0), R(0)};  // held at zero by its set's truncation
    const int d = v.d;
    const int r = e / d, c = e - r * d;
    const cx<R> *Xn = X + n * v.d2 * B + b;
    const cx<R> x0 = Xn[(int64_t)e * B];
    cx<R> acc{-(damp.re * x0.re - damp.im * x0.im), -(damp.re * x0.im + damp.im * x0.re)};
    // system superoperator: -i (H X - X H) plus the Lindblad terms, one merged term list
    const cx<R> *sv = v.s_val + (int64_t)set * v.nS;
    for (int j = __ldg(v.s_ptr + e), j1 = __ldg(v.s_ptr + e + 1); j < j1; ++j)
        fma_to(acc, ldc(sv + j), Xn[(int64_t)__ldg(v.s_src + j) * B]);
    // couplings to the neighbouring ADOs
    const int cap = v.set_cap ? __ldg(v.set_cap + set) : 0;
    const int t1 = __ldg(v.row_ptr + n + 1);
    for (int t = __ldg(v.row_ptr + n); t < t1; ++t) {
        const int4 raw = __ldg(reinterpret_cast<const int4 *>(v.ent) + t);
        const int nb = raw.x;
        if (v.set_cap) {  // a neighbour beyond the set's tiers is not in its hierarchy
            const int tn = __ldg(v.ado_tier + nb);
            if ((tn & 0xffff) > (cap & 0xffff) || (tn >> 16) > (cap >> 16)) continue;
        }
        const int op = (int)(int16_t)(raw.y & 0xffff);
        const int k = (int)(int16_t)(raw.y >> 16);
        const int dir = (int)(int16_t)(raw.z & 0xffff);
        const R ml = R((int16_t)(raw.z >> 16));
        const R mr = R((int16_t)(raw.w & 0xffff));
        cx<R> cl, cr;  // -i * mult * (a | b)
        if (dir > 0) {
            cl = cx<R>{R(0), -ml};
            cr = cx<R>{R(0), -mr};
        } else {
            const int64_t pk = (int64_t)set * v.K + k;
            cl = mul_mi(ml * ldc(v.coefL + pk));
            cr = mul_mi(mr * ldc(v.coefR + pk));
        }
        const cx<R> *Xb = X + (int64_t)nb * v.d2 * B + b;
        const int base = op * (d + 1);
        for (int j = __ldg(v.op_rptr + base + r), j1 = __ldg(v.op_rptr + base + r + 1); j < j1; ++j)
            fma_to(acc, cl * ldc(v.op_rval + j), Xb[(int64_t)(__ldg(v.op_rcol + j) * d + c) * B]);
        for (int j = __ldg(v.op_cptr + base + c), j1 = __ldg(v.op_cptr + base + c + 1); j < j1; ++j)
            fma_to(acc, cr * ldc(v.op_cval + j), Xb[(int64_t)(r * d + __ldg(v.op_crow + j)) * B]);
    }
    return acc;
}

// Inverse of the ADO-local diagonal: 1 / (L_s[e][e] - damp + shift), with L_s[e][e] the
// coefficient of element e on itself in the system superoperator (-i (H_rr - H_cc) without
// Lindblad terms); the undamped tier-0 ADO is given the smallest positive rate as damping so
// the inverse stays bounded.
template <class R>
__device__ __forceinline__ cx<R> precond_inv(const DevView<R> &v, int64_t n, int e, int set,
                                             const cx<R> &damp, cx<R> shift) {
    cx<R> loc = ldc(v.sdiag + (int64_t)set * v.d2 + e) - damp + shift;
    if (__ldg(v.occ_ptr + n) == __ldg(v.occ_ptr + n + 1)) loc.re -= __ldg(v.floor + set);
    return cdiv(cx<R>{R(1), R(0)}, loc);
}

// Complex Givens rotation zeroing b in (a, b): G = [c s; -conj(s) c] with c real, so that
// G (a, b) = (r, 0). Built from two reciprocal square roots: an FP64 division or square root
// is a long instruction sequence on GB300's narrow FP64 pipe. With ia = 1/|a| and
// inr = 1/sqrt(|a|^2 + |b|^2): c = |a| inr, s = (a / |a|) conj(b) inr, r = (a / |a|) nr.
__device__ __forceinline__ void givens_rot(cx<double> a, cx<double> b, double &c, cx<double> &s,
                                           cx<double> &r) {
    const double a2 = norm2(a), b2 = norm2(b);
    if (b2 == 0.0) { c = 1.0; s = cx<double>{0.0, 0.0}; r = a; return; }
    if (a2 == 0.0) {
        const double ib = rsqrt(b2);
        c = 0.0;
        s = ib * conj(b);
        r = cx<double>{b2 * ib, 0.0};
        return;
    }
    const double ia = rsqrt(a2), inr = rsqrt(a2 + b2);
    c = a2 * ia * inr;
    s = (ia * inr) * (a * conj(b));
    r = ((a2 + b2) * inr * ia) * a;
}

// Sum a per-thread FP64 complex value over threadIdx.y and atomically add it to acc[col].
// Block is (bx, by) with by a power of two; every thread of the block must call this.
__device__ __forceinline__ void block_add(double re, double im, double *acc_re, double *acc_im,
                                          bool valid) {
    __shared__ double sre[256], sim[256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    sre[tid] = re;
    sim[tid] = im;
    __syncthreads();
    for (int s = blockDim.y >> 1; s > 0; s >>= 1) {
        if (threadIdx.y < s) {
            sre[tid] += sre[tid + s * blockDim.x];
            sim[tid] += sim[tid + s * blockDim.x];
        }
        __syncthreads();
    }
    if (threadIdx.y == 0 && valid) {
        atomicAdd(acc_re, sre[threadIdx.x]);
        if (acc_im) atomicAdd(acc_im, sim[threadIdx.x]);
    }
    __syncthreads();
}

}  // namespace heom
