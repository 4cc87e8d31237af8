// Solvers driven by the HEOM apply (package architecture: dynamics, stationary states,
// spectra): fixed-step RK4, batched right-preconditioned BiCGStab, FP64 iterative
// refinement around FP32 BiCGStab corrections, and the density-of-states readout
// (Methods, numerical computation of the spectrum).
//
// All batch columns are independent systems that iterate in lock-step; every Krylov scalar
// lives on the device per column (ColState, FP64), so an iteration is five kernel launches
// and no host round trip. The host reads the per-column residuals every few iterations to
// retire converged columns.
#include <algorithm>
#include <cmath>
#include <vector>

#include "heom_tile.cuh"

namespace heom {

// ------------------------------------------------------------------ block reduction
template <int NV>
__device__ __forceinline__ void reduce_add(double (&val)[NV], double *const (&dst)[NV],
                                           bool valid) {
    __shared__ double sh[NV][256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][tid] = val[i];
    __syncthreads();
    for (int s = blockDim.y >> 1; s > 0; s >>= 1) {
        if (threadIdx.y < s) {
#pragma unroll
            for (int i = 0; i < NV; ++i) sh[i][tid] += sh[i][tid + s * blockDim.x];
        }
        __syncthreads();
    }
    if (threadIdx.y == 0 && valid) {
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (dst[i]) atomicAdd(dst[i], sh[i][threadIdx.x]);
    }
}

// The parameter set of batch column b: (map ? map[b] : b) / cps, where map gives the original
// column of each column of a compacted working layout (null: the layout is the original).
struct ColSets {
    int64_t cps;
    const int *map;
    __host__ __device__ ColSets(int64_t c, const int *m = nullptr) : cps(c), map(m) {}
};

#define COLUMN_PROLOGUE                                                    \
    const int64_t b = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;      \
    const bool inb = b < B;                                                \
    const int64_t rows = v.N * v.d2;                                       \
    const int set = inb ? (int)((cps.map ? (int64_t)cps.map[b] : b) / cps.cps) : 0; \
    (void)set;

#define ROW_LOOP _Pragma("unroll 4") \
                 for (int64_t row = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; row < rows; \
                      row += (int64_t)gridDim.x * blockDim.y)

__device__ __forceinline__ bool designated() { return blockIdx.x == 0 && threadIdx.y == 0; }

// ------------------------------------------------------------------ RK4
// One fused stage of classical RK4: k = M z_in, then
//   stage 1: acc = k,       z_out = y + dt/2 k
//   stage 2: acc += 2k,     z_out = y + dt/2 k
//   stage 3: acc += 2k,     z_out = y + dt k
//   stage 4: y += dt/6 (acc + k)
template <class R>
__global__ void __launch_bounds__(256) k_rk4_stage(DevView<R> v, const cx<R> *__restrict__ z_in,
                                                   cx<R> *__restrict__ z_out, cx<R> *y,
                                                   cx<R> *__restrict__ acc, int64_t B,
                                                   ColSets cps, R dt, int stage) {
    COLUMN_PROLOGUE
    if (!inb) return;
    ROW_LOOP {
        const int64_t n = row / v.d2;
        const int e = (int)(row - n * v.d2);
        const cx<R> k = apply_point(v, z_in, n, e, b, B, set, damping_of(v, n, set));
        const int64_t i = row * B + b;
        if (stage == 1) {
            acc[i] = k;
            z_out[i] = y[i] + (R(0.5) * dt) * k;
        } else if (stage == 2) {
            acc[i] = acc[i] + R(2) * k;
            z_out[i] = y[i] + (R(0.5) * dt) * k;
        } else if (stage == 3) {
            acc[i] = acc[i] + R(2) * k;
            z_out[i] = y[i] + dt * k;
        } else {
            y[i] = y[i] + (dt / R(6)) * (acc[i] + k);
        }
    }
}

template <class R>
cudaError_t launch_rk4_stage(const DevView<R> &v, const cx<R> *z_in, cx<R> *z_out, cx<R> *y,
                             cx<R> *acc, int64_t B, R dt, int stage, cudaStream_t s) {
    const Geom g = make_geom(v.N * v.d2, B, 1 << 30);
    k_rk4_stage<R><<<g.grid, g.block, 0, s>>>(v, z_in, z_out, y, acc, B, B / v.n_sets, dt, stage);
    return cudaGetLastError();
}
template cudaError_t launch_rk4_stage<double>(const DevView<double> &, const cx<double> *,
                                              cx<double> *, cx<double> *, cx<double> *, int64_t,
                                              double, int, cudaStream_t);
template cudaError_t launch_rk4_stage<float>(const DevView<float> &, const cx<float> *,
                                             cx<float> *, cx<float> *, cx<float> *, int64_t,
                                             float, int, cudaStream_t);

// ------------------------------------------------------------------ BiCGStab
__global__ void k_state_init(ColState *st, int64_t B, const int *active) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    ColState c{};
    c.rho_old = {1.0, 0.0};
    c.alpha = {1.0, 0.0};
    c.omega = {1.0, 0.0};
    c.active = active ? active[b] : 1;
    st[b] = c;
}

// r = b - A x (or r = b when x is zero), rh = r, p = v = 0; acc_rr = (rh, r), acc_nr = |r|^2,
// bnorm2 = |b|^2.
template <class R>
__global__ void __launch_bounds__(256) k_bicg_init(DevView<R> v, const cx<R> *__restrict__ bb,
                                                   const cx<R> *__restrict__ x, cx<R> *r,
                                                   cx<R> *rh, cx<R> *p, cx<R> *vv, int64_t B,
                                                   ColSets cps, ApplyMods<R> mods, int x_zero,
                                                   ColState *st) {
    COLUMN_PROLOGUE
    const bool act = inb && st[b].active;
    double nr = 0, nb = 0;
    if (act) {
        ROW_LOOP {
            const int64_t i = row * B + b;
            cx<R> ri = bb[i];
            if (!x_zero) {
                const int64_t n = row / v.d2;
                const int e = (int)(row - n * v.d2);
                cx<R> ax = apply_point(v, x, n, e, b, B, set, damping_of(v, n, set));
                if (mods.shift) fma_to(ax, mods.shift[b], x[i]);
                if (mods.aug != R(0) && row == 0) {
                    cx<R> tr{R(0), R(0)};
                    for (int q = 0; q < v.d; ++q) tr = tr + x[(int64_t)(q * v.d + q) * B + b];
                    ax = ax + mods.aug * tr;
                }
                ri = ri - ax;
            }
            r[i] = ri;
            rh[i] = ri;
            p[i] = cx<R>{R(0), R(0)};
            vv[i] = cx<R>{R(0), R(0)};
            nr += (double)norm2(ri);
            nb += (double)norm2(bb[i]);
        }
    }
    double val[3] = {nr, nr, nb};
    double *const dst[3] = {act ? &st[b].acc_rr.re : nullptr, act ? &st[b].acc_nr : nullptr,
                            act ? &st[b].bnorm2 : nullptr};
    reduce_add<3>(val, dst, act);
}

// The per-column Krylov scalars are computed once per column and block (FP64 divisions are
// slow on GB300) by the threads of row 0 and shared with the block.
template <class R>
struct ColScalars {
    cx<R> a, b;      // two working-precision scalars of the kernel
    cx<double> keep; // an FP64 value to store back
    int on;          // column active
    int rs;          // restart this iteration (rh = r, p = r)
};

// p = r + beta (p - omega v), ph = P^-1 p, beta = (rho / rho_old)(alpha / omega); or, when
// the restart rule fires (rho small against ||rh|| ||r||), rh = r and p = r. The decision is
// taken from fields no kernel writes between here and k_bicg_s, which reads it back from
// st.restart.
template <class R>
__global__ void __launch_bounds__(256) k_bicg_p(DevView<R> v, const cx<R> *__restrict__ r,
                                                cx<R> *p, const cx<R> *__restrict__ vv,
                                                cx<R> *__restrict__ ph, cx<R> *rh, int64_t B,
                                                ColSets cps, const cx<R> *shift, int precond,
                                                ColState *st) {
    COLUMN_PROLOGUE
    __shared__ ColScalars<R> sc[32];
    if (threadIdx.y == 0) {
        ColScalars<R> c{};
        c.on = inb && st[b].active;
        if (c.on) {
            const ColState cs = st[b];
            c.rs = norm2(cs.acc_rr) < kRestartTau2 * cs.rhn * cs.acc_nr;
            c.a = cast<R>(cdiv(cs.acc_rr, cs.rho_old) * cdiv(cs.alpha, cs.omega));  // beta
            c.b = cast<R>(cs.omega);
        }
        sc[threadIdx.x] = c;
    }
    __syncthreads();
    const ColScalars<R> c = sc[threadIdx.x];
    if (!c.on) return;
    const cx<R> bt = c.a, om = c.b;
    const bool rs = c.rs != 0;
    const cx<R> shv = shift ? shift[b] : cx<R>{R(0), R(0)};
    ROW_LOOP {
        const int64_t i = row * B + b;
        const cx<R> ri = r[i];
        const cx<R> pi = rs ? ri : ri + bt * (p[i] - om * vv[i]);
        if (rs) rh[i] = ri;
        p[i] = pi;
        if (precond) {
            const int64_t n = row / v.d2;
            const int e = (int)(row - n * v.d2);
            ph[i] = pi * precond_inv(v, n, e, set, damping_of(v, n, set), shv);
        } else {
            ph[i] = pi;
        }
    }
    if (designated()) {
        st[b].acc_rv = {0.0, 0.0};
        st[b].restart = rs;
    }
}

// out = A in (apply with shift / trace augmentation), plus FP64 dots against two vectors:
//   mode 0 (v = A ph):  acc_rv += (rh, v)
//   mode 1 (t = A sh):  acc_ts += (t, s), acc_tt += (t, t)
template <class R>
__global__ void __launch_bounds__(256) k_bicg_apply(DevView<R> v, const cx<R> *__restrict__ in,
                                                    cx<R> *__restrict__ out,
                                                    const cx<R> *__restrict__ w, int64_t B,
                                                    ColSets cps, ApplyMods<R> mods, int mode,
                                                    ColState *st) {
    COLUMN_PROLOGUE
    const bool act = inb && st[b].active;
    double a_re = 0, a_im = 0, tt = 0;
    if (act) {
        ROW_LOOP {
            const int64_t n = row / v.d2;
            const int e = (int)(row - n * v.d2);
            const int64_t i = row * B + b;
            cx<R> y = apply_point(v, in, n, e, b, B, set, damping_of(v, n, set));
            if (mods.shift) fma_to(y, mods.shift[b], in[i]);
            if (mods.aug != R(0) && row == 0) {
                cx<R> tr{R(0), R(0)};
                for (int q = 0; q < v.d; ++q) tr = tr + in[(int64_t)(q * v.d + q) * B + b];
                y = y + mods.aug * tr;
            }
            out[i] = y;
            const cx<double> yd = cast<double>(y), wd = cast<double>(w[i]);
            if (mode == 0) {  // (rh, v) = sum conj(rh) v
                a_re += wd.re * yd.re + wd.im * yd.im;
                a_im += wd.re * yd.im - wd.im * yd.re;
            } else {          // (t, s) = sum conj(t) s ; (t, t)
                a_re += yd.re * wd.re + yd.im * wd.im;
                a_im += yd.re * wd.im - yd.im * wd.re;
                tt += yd.re * yd.re + yd.im * yd.im;
            }
        }
    }
    if (mode == 0) {
        double val[2] = {a_re, a_im};
        double *const dst[2] = {act ? &st[b].acc_rv.re : nullptr, act ? &st[b].acc_rv.im : nullptr};
        reduce_add<2>(val, dst, act);
    } else {
        double val[3] = {a_re, a_im, tt};
        double *const dst[3] = {act ? &st[b].acc_ts.re : nullptr, act ? &st[b].acc_ts.im : nullptr,
                                act ? &st[b].acc_tt.re : nullptr};
        reduce_add<3>(val, dst, act);
        if (act && designated()) {
            st[b].acc_rr = {0.0, 0.0};
            st[b].acc_nr = 0.0;
        }
    }
}

// alpha = rho / (rh, v); s = r - alpha v (in place in r); sh = P^-1 s
template <class R>
__global__ void __launch_bounds__(256) k_bicg_s(DevView<R> v, cx<R> *r, const cx<R> *__restrict__ vv,
                                                cx<R> *__restrict__ sh, int64_t B, ColSets cps,
                                                const cx<R> *shift, int precond, ColState *st) {
    COLUMN_PROLOGUE
    __shared__ ColScalars<R> sc[32];
    if (threadIdx.y == 0) {
        ColScalars<R> c{};
        c.on = inb && st[b].active;
        if (c.on) {
            const ColState cs = st[b];
            const bool bad = norm2(cs.acc_rv) == 0.0;
            const cx<double> rho = cs.restart ? cx<double>{cs.acc_nr, 0.0} : cs.acc_rr;
            c.keep = bad ? cx<double>{0.0, 0.0} : cdiv(rho, cs.acc_rv);  // alpha
            c.rs = cs.restart;
            c.a = cast<R>(c.keep);
            c.b = cx<R>{bad ? R(1) : R(0), R(0)};
        }
        sc[threadIdx.x] = c;
    }
    __syncthreads();
    const ColScalars<R> c = sc[threadIdx.x];
    if (!c.on) return;
    const cx<R> al = c.a;
    const cx<R> shf = shift ? shift[b] : cx<R>{R(0), R(0)};
    ROW_LOOP {
        const int64_t i = row * B + b;
        const cx<R> s = r[i] - al * vv[i];
        r[i] = s;
        if (precond) {
            const int64_t n = row / v.d2;
            const int e = (int)(row - n * v.d2);
            sh[i] = s * precond_inv(v, n, e, set, damping_of(v, n, set), shf);
        } else {
            sh[i] = s;
        }
    }
    if (designated()) {
        const cx<double> rr = c.rs ? cx<double>{st[b].acc_nr, 0.0} : st[b].acc_rr;
        if (c.rs) st[b].rhn = st[b].acc_nr;
        st[b].alpha = c.keep;
        st[b].rho_old = rr;
        st[b].acc_ts = {0.0, 0.0};
        st[b].acc_tt = {0.0, 0.0};
        if (c.b.re != R(0)) st[b].flag = 1;
    }
}

// omega = (t, s) / (t, t); x += alpha ph + omega sh; r = s - omega t;
// acc_rr += (rh, r), acc_nr += |r|^2
template <class R>
__global__ void __launch_bounds__(256) k_bicg_x(int64_t rows, cx<R> *x, const cx<R> *__restrict__ ph,
                                                const cx<R> *__restrict__ sh, cx<R> *r,
                                                const cx<R> *__restrict__ t,
                                                const cx<R> *__restrict__ rh, int64_t B,
                                                ColState *st) {
    const int64_t b = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    __shared__ ColScalars<R> sc[32];
    if (threadIdx.y == 0) {
        ColScalars<R> c{};
        c.on = b < B && st[b].active;
        if (c.on) {
            const ColState cs = st[b];
            const cx<double> omega =
                cs.acc_tt.re == 0.0 ? cx<double>{0.0, 0.0} : cdiv(cs.acc_ts, cs.acc_tt);
            const bool bad = !isfinite(omega.re) || !isfinite(omega.im) ||
                             !isfinite(cs.alpha.re) || !isfinite(cs.alpha.im);
            c.keep = omega;
            c.a = cast<R>(cs.alpha);
            c.b = cast<R>(omega);
            c.on = bad ? 2 : 1;
        }
        sc[threadIdx.x] = c;
    }
    __syncthreads();
    const ColScalars<R> c = sc[threadIdx.x];
    const bool act = c.on == 1;
    double rr_re = 0, rr_im = 0, nr = 0;
    if (act) {
        const cx<R> al = c.a, om = c.b;
        ROW_LOOP {
            const int64_t i = row * B + b;
            x[i] = x[i] + al * ph[i] + om * sh[i];
            const cx<R> ri = r[i] - om * t[i];
            r[i] = ri;
            const cx<double> rd = cast<double>(ri), hd = cast<double>(rh[i]);
            rr_re += hd.re * rd.re + hd.im * rd.im;
            rr_im += hd.re * rd.im - hd.im * rd.re;
            nr += rd.re * rd.re + rd.im * rd.im;
        }
    }
    double val[3] = {rr_re, rr_im, nr};
    double *const dst[3] = {act ? &st[b].acc_rr.re : nullptr, act ? &st[b].acc_rr.im : nullptr,
                            act ? &st[b].acc_nr : nullptr};
    reduce_add<3>(val, dst, act);
    if (c.on && designated()) {
        st[b].omega = c.keep;
        if (c.on == 2) st[b].flag = 1;
    }
}

// ------------------------------------------------------------------ refinement helpers
// r64 = b - A x64 in FP64 with |r|^2 -> acc_nr and |b|^2 -> bnorm2 of the outer state
__global__ void __launch_bounds__(256) k_residual64(DevView<double> v, const cx<double> *__restrict__ bb,
                                                    const cx<double> *__restrict__ x,
                                                    cx<double> *__restrict__ r, int64_t B,
                                                    ColSets cps, ApplyMods<double> mods,
                                                    ColState *st) {
    COLUMN_PROLOGUE
    const bool act = inb && st[b].active;
    double nr = 0, nb = 0;
    if (act) {
        ROW_LOOP {
            const int64_t n = row / v.d2;
            const int e = (int)(row - n * v.d2);
            const int64_t i = row * B + b;
            cx<double> ax = apply_point(v, x, n, e, b, B, set, damping_of(v, n, set));
            if (mods.shift) fma_to(ax, mods.shift[b], x[i]);
            if (mods.aug != 0.0 && row == 0) {
                cx<double> tr{0.0, 0.0};
                for (int q = 0; q < v.d; ++q) tr = tr + x[(int64_t)(q * v.d + q) * B + b];
                ax = ax + mods.aug * tr;
            }
            const cx<double> ri = bb[i] - ax;
            r[i] = ri;
            nr += norm2(ri);
            nb += norm2(bb[i]);
        }
    }
    double val[2] = {nr, nb};
    double *const dst[2] = {act ? &st[b].acc_nr : nullptr, act ? &st[b].bnorm2 : nullptr};
    reduce_add<2>(val, dst, act);
}

// rin = r64 / ||r64|| per active column, in the inner solver's precision
template <class RI>
__global__ void k_scale_to(int64_t rows, const cx<double> *__restrict__ r64,
                           cx<RI> *__restrict__ rin, int64_t B, const ColState *st) {
    const int64_t b = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (b >= B || !st[b].active) return;
    const double inv = 1.0 / std::sqrt(st[b].acc_nr);
    ROW_LOOP {
        const int64_t i = row * B + b;
        rin[i] = cx<RI>{RI(r64[i].re * inv), RI(r64[i].im * inv)};
    }
}

// x64 += ||r64|| d per active column
template <class RI>
__global__ void k_accum(int64_t rows, cx<double> *__restrict__ x, const cx<RI> *__restrict__ dv,
                        int64_t B, const ColState *st) {
    const int64_t b = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (b >= B || !st[b].active) return;
    const double s = std::sqrt(st[b].acc_nr);
    ROW_LOOP {
        const int64_t i = row * B + b;
        x[i].re += s * (double)dv[i].re;
        x[i].im += s * (double)dv[i].im;
    }
}

// per column: |M x|^2 and |x|^2 (FP64, no shift, no augmentation) into out[2*b], out[2*b+1]
__global__ void __launch_bounds__(256) k_apply_norms(DevView<double> v, const cx<double> *__restrict__ x,
                                                     int64_t B, ColSets cps, double *out) {
    COLUMN_PROLOGUE
    double mx = 0, xx = 0;
    if (inb) {
        ROW_LOOP {
            const int64_t n = row / v.d2;
            const int e = (int)(row - n * v.d2);
            const cx<double> y = apply_point(v, x, n, e, b, B, set, damping_of(v, n, set));
            mx += norm2(y);
            xx += norm2(x[row * B + b]);
        }
    }
    double val[2] = {mx, xx};
    double *const dst[2] = {inb ? out + 2 * b : nullptr, inb ? out + 2 * b + 1 : nullptr};
    reduce_add<2>(val, dst, inb);
}

// steady-state right-hand side: e_(0,(0,0)) in every column
template <class R>
__global__ void k_set_e00(int64_t total, cx<R> *bvec, int64_t B) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        bvec[i] = cx<R>{i < B ? R(1) : R(0), R(0)};
}

// spectrum right-hand sides: columns [0, nw) get O_plus rho_n, columns [nw, 2nw) O_minus rho_n
__global__ void k_dos_rhs(int64_t N, int d, const cx<double> *__restrict__ ss,
                          const cx<double> *__restrict__ op_plus, const cx<double> *__restrict__ op_minus,
                          cx<double> *__restrict__ bvec, int64_t nw) {
    const int64_t B = 2 * nw;
    const int64_t total = N * d * d * B;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i % B, row = i / B;
        const int64_t n = row / (d * d);
        const int e = (int)(row - n * d * d), r = e / d, c = e - r * d;
        const cx<double> *O = b < nw ? op_plus : op_minus;
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < d; ++l) fma_to(acc, O[r * d + l], ss[n * d * d + l * d + c]);
        bvec[i] = acc;
    }
}

// b[row][2s] = (op_plus rho_s)[row], b[row][2s+1] = (op_minus rho_s)[row] for the stationary
// states of ns parameter sets (ss [N][d][d][ns])
__global__ void k_dos_rhs_sets(int64_t N, int d, const cx<double> *__restrict__ ss,
                               const cx<double> *__restrict__ op_plus, const cx<double> *__restrict__ op_minus,
                               cx<double> *__restrict__ bvec, int64_t ns) {
    const int64_t B = 2 * ns;
    const int64_t total = N * d * d * B;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i % B, row = i / B, set = b >> 1;
        const int64_t n = row / (d * d);
        const int e = (int)(row - n * d * d), r = e / d, c = e - r * d;
        const cx<double> *O = (b & 1) ? op_minus : op_plus;
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < d; ++l) fma_to(acc, O[r * d + l], ss[(n * d * d + l * d + c) * ns + set]);
        bvec[i] = acc;
    }
}

template <class R>
__global__ void k_scale_cols(int64_t total, cx<R> *x, int64_t B, const cx<double> *fac) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const cx<R> f = cast<R>(fac[i % B]);
        x[i] = x[i] * f;
    }
}

template <class R, class S>
__global__ void k_convert(int64_t total, const cx<S> *__restrict__ in, cx<R> *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cast<R>(in[i]);
}

// batch-column gather / scatter: out[row][j] = in[row][map[j]] and out[row][map[j]] = in[row][j]
template <class R>
__global__ void k_gather_cols(int64_t rows, const cx<R> *__restrict__ in, int64_t Bin,
                              cx<R> *__restrict__ out, int64_t Bout, const int *__restrict__ map) {
    const int64_t total = rows * Bout;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / Bout, j = i - row * Bout;
        out[i] = in[row * Bin + map[j]];
    }
}

template <class R>
__global__ void k_scatter_cols(int64_t rows, const cx<R> *__restrict__ in, int64_t Bin,
                               cx<R> *__restrict__ out, int64_t Bout, const int *__restrict__ map) {
    const int64_t total = rows * Bin;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / Bin, j = i - row * Bin;
        out[row * Bout + map[j]] = in[i];
    }
}

// ------------------------------------------------------------------ host orchestration
namespace {

int flat_blocks(int64_t total) {
    int64_t g = (total + 255) / 256;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

template <class R> DevView<R> view_of(const heom_hier *h);
template <> DevView<double> view_of<double>(const heom_hier *h) { return h->view64(); }
template <> DevView<float> view_of<float>(const heom_hier *h) { return h->view32(); }

struct SolveOut {
    std::vector<int> iters;
    std::vector<int> status;
    std::vector<double> res;  // final relative residual sqrt(acc_nr / bnorm2)
};

// Batched right-preconditioned BiCGStab on A x = b, A = M + diag(shift) (+ trace aug).
// Columns with active[b] = 0 are left untouched. x holds the initial guess (x_zero: zero).
constexpr int kStallIters = 96;

// Batched right-preconditioned BiCGStab on A x = b, A = M + diag(shift) (+ trace aug).
// Columns with active[b] = 0 are left untouched. x holds the initial guess (x_zero: zero).
//
// The solver works on a compact copy of the active columns ([rows][Bc] with Bc <= B) and
// re-compacts whenever the still-active columns fall to 60 % of the working width, so that
// iteration cost follows the columns that still iterate (frequencies and parameter sets
// converge at different iterations; the kernels find each compact column's parameter set
// through the column map). Converged solutions are scattered back into x. Workspace: 13 vectors of
// rows x B (two sets of x, r, rh, p, v and the scratch ph, sh, t).
template <class R>
heom_status bicgstab(heom_hier *h, const cx<R> *bvec, cx<R> *x, int64_t B, const cx<R> *shift,
                     R aug, bool x_zero, double tol, int max_iter, const std::vector<int> &active,
                     cx<R> *work, ColState *st, int *d_map, int *d_lmap, cx<R> *shift_c,
                     SolveOut &out, cudaStream_t s) {
    const DevView<R> v = view_of<R>(h);
    const int64_t rows = h->N * h->d2, L = rows * B;
    cx<R> *set_a[5], *set_b[5];
    for (int i = 0; i < 5; ++i) { set_a[i] = work + i * L; set_b[i] = work + (5 + i) * L; }
    cx<R> *ph = work + 10 * L, *sh = work + 11 * L, *t = work + 12 * L;
    const int64_t cps_g = B / h->n_sets;  // columns per parameter set in the caller's layout
    out.iters.assign(B, 0);
    out.status.assign(B, HEOM_OK);
    out.res.assign(B, 0.0);
    // the initial column set
    std::vector<int> cols, alive;  // global column of each compact column; its activity
    for (int64_t b = 0; b < B; ++b)
        if (active[b]) { cols.push_back((int)b); alive.push_back(1); }
    if (cols.empty()) return HEOM_OK;
    if (sizeof(R) == 4 && (cols.size() & 1) && (int64_t)cols.size() < B) {
        for (int64_t b = 0; b < B; ++b)  // an even width keeps the float4 column loads aligned
            if (!active[b]) { cols.push_back((int)b); alive.push_back(0); break; }
    }
    int64_t Bc = (int64_t)cols.size();
    HEOM_CUDA(memcpy_counted(d_map, cols.data(), Bc * sizeof(int), cudaMemcpyHostToDevice, s));
    HEOM_CUDA(memcpy_counted(d_lmap, alive.data(), Bc * sizeof(int), cudaMemcpyHostToDevice, s));
    cx<R> **cur = set_a, **nxt = set_b;
    const cx<R> *shc = nullptr;
    {
        Prof pr(HEOM_KC_OTHER, s, (double)rows * Bc, (3.0 + (x_zero ? 0 : 2)) * rows * Bc * sizeof(cx<R>));
        pr.kernels = 1 + (x_zero ? 0 : 1) + (shift ? 1 : 0);
        k_gather_cols<R><<<flat_blocks(rows * Bc), 256, 0, s>>>(rows, bvec, B, t, Bc, d_map);
        if (x_zero) HEOM_CUDA(cudaMemsetAsync(cur[0], 0, rows * Bc * sizeof(cx<R>), s));
        else k_gather_cols<R><<<flat_blocks(rows * Bc), 256, 0, s>>>(rows, x, B, cur[0], Bc, d_map);
        if (shift) {
            k_gather_cols<R><<<flat_blocks(Bc), 256, 0, s>>>(1, shift, B, shift_c, Bc, d_map);
            shc = shift_c;
        }
    }
    {
        Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)Bc);
        k_state_init<<<(unsigned)((Bc + 255) / 256), 256, 0, s>>>(st, Bc, d_lmap);
    }
    auto geoms = [&](int64_t w, Geom &gd, Geom &gv) {
        // kernels with per-column dot products: a capped grid (few atomics per column);
        // pure vector updates: a larger grid
        gd = make_geom(rows, w, std::max<int64_t>(1, 4096 / ((w + 31) / 32)));
        gv = make_geom(rows, w, std::max<int64_t>(1, 16384 / ((w + 31) / 32)));
    };
    Geom gd, gv;
    geoms(Bc, gd, gv);
    {
        ApplyMods<R> mods{shc, aug};
        Prof pr(HEOM_KC_KRYLOV_VECTOR, s, (double)rows * Bc, (x_zero ? 5.0 : 6.0) * rows * Bc * sizeof(cx<R>));
        k_bicg_init<R><<<gd.grid, gd.block, 0, s>>>(v, t, cur[0], cur[1], cur[2], cur[3], cur[4],
                                                    Bc, ColSets(cps_g, d_map), mods, x_zero, st);
    }
    HEOM_CUDA(cudaGetLastError());
    std::vector<ColState> hs(Bc);
    const double tol2 = tol * tol;
    HEOM_CUDA(memcpy_counted(hs.data(), st, Bc * sizeof(ColState), cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    int n_act = 0;
    for (int64_t j = 0; j < Bc; ++j) {
        hs[j].rhn = hs[j].acc_nr;  // rh = r0
        if (!alive[j]) continue;
        const int b = cols[j];
        out.res[b] = hs[j].bnorm2 > 0 ? std::sqrt(hs[j].acc_nr / hs[j].bnorm2) : 0.0;
        if (hs[j].acc_nr <= tol2 * hs[j].bnorm2) { alive[j] = 0; hs[j].active = 0; }
        else ++n_act;
    }
    // stall / divergence guard: a column whose residual has not reached a new minimum for
    // kStallIters iterations, or has grown 1e12-fold above its minimum, stops; the caller's
    // refinement then restarts from its FP64 residual (or skips a correction that grew).
    std::vector<double> best(Bc);
    std::vector<int> best_it(Bc, 0);
    for (int64_t j = 0; j < Bc; ++j) best[j] = hs[j].acc_nr;
    int it = 0, check = 4;
    cudaGraphExec_t gexec = nullptr;  // one BiCGStab iteration as a graph (see below)
    cudaStream_t gcap = nullptr;
    const void *gkey_x = nullptr;
    int64_t gkey_B = -1;
    bool gkey_tiled = false;
    struct GraphRelease {
        cudaGraphExec_t &e;
        cudaStream_t &c;
        ~GraphRelease() {
            if (e) cudaGraphExecDestroy(e);
            if (c) cudaStreamDestroy(c);
        }
    } graph_release{gexec, gcap};
    while (n_act > 0 && it < max_iter) {
        // ---- re-compaction when the active columns fall to 60 % of the working width
        if (n_act <= 0.6 * Bc && Bc - n_act >= 16) {
            std::vector<int> keep;
            for (int64_t j = 0; j < Bc; ++j)
                if (alive[j]) keep.push_back((int)j);
            if (sizeof(R) == 4 && (keep.size() & 1)) {
                for (int64_t j = 0; j < Bc; ++j)
                    if (!alive[j]) { keep.push_back((int)j); break; }
            }
            std::sort(keep.begin(), keep.end());
            const int64_t Bn = (int64_t)keep.size();
            {   // solutions of every current column go home first
                Prof pr(HEOM_KC_OTHER, s, (double)rows * Bc, 2.0 * rows * Bc * sizeof(cx<R>));
                k_scatter_cols<R><<<flat_blocks(rows * Bc), 256, 0, s>>>(rows, cur[0], Bc, x, B, d_map);
            }
            HEOM_CUDA(memcpy_counted(d_lmap, keep.data(), Bn * sizeof(int), cudaMemcpyHostToDevice, s));
            {
                Prof pr(HEOM_KC_OTHER, s, 5.0 * rows * Bn, 10.0 * rows * Bn * sizeof(cx<R>));
                pr.kernels = 5;
                for (int i = 0; i < 5; ++i)
                    k_gather_cols<R><<<flat_blocks(rows * Bn), 256, 0, s>>>(rows, cur[i], Bc, nxt[i], Bn, d_lmap);
            }
            std::vector<int> ncols(Bn), nalive(Bn);
            std::vector<ColState> nhs(Bn);
            std::vector<double> nbest(Bn);
            std::vector<int> nbest_it(Bn);
            for (int64_t j = 0; j < Bn; ++j) {
                const int o = keep[j];
                ncols[j] = cols[o];
                nalive[j] = alive[o];
                nhs[j] = hs[o];
                nhs[j].active = alive[o];
                nbest[j] = best[o];
                nbest_it[j] = best_it[o];
            }
            cols.swap(ncols); alive.swap(nalive); hs.swap(nhs); best.swap(nbest); best_it.swap(nbest_it);
            std::swap(cur, nxt);
            Bc = Bn;
            HEOM_CUDA(memcpy_counted(d_map, cols.data(), Bc * sizeof(int), cudaMemcpyHostToDevice, s));
            if (shift) {
                Prof pr(HEOM_KC_OTHER, s, (double)Bc);
                k_gather_cols<R><<<flat_blocks(Bc), 256, 0, s>>>(1, shift, B, shift_c, Bc, d_map);
            }
            geoms(Bc, gd, gv);
        }
        HEOM_CUDA(memcpy_counted(st, hs.data(), Bc * sizeof(ColState), cudaMemcpyHostToDevice, s));
        const int steps = std::min(check, max_iter - it);
        const int kc_apply = sizeof(R) == 4 ? HEOM_KC_KRYLOV_APPLY32 : HEOM_KC_KRYLOV_APPLY64;
        ApplyMods<R> mods{shc, aug};
        const bool tiled = tile_ok(v, Bc);
        TileArgs<R> ta{};
        ta.v = v;
        ta.shift = shc;
        ta.aug = aug;
        ta.st = st;
        ta.B = Bc;
        cx<R> *xw = cur[0], *r = cur[1], *rh = cur[2], *p = cur[3], *vv = cur[4];
        const ColSets cps(cps_g, d_map);  // compact column -> the caller's column -> set
        // ADO-applies: the ADOs each running column's set keeps (idle padding columns excluded)
        double u_app = 0.0;
        for (int64_t j = 0; j < Bc; ++j)
            if (alive[(size_t)j]) u_app += (double)h->kept_of_set((int)(cols[(size_t)j] / cps_g));
        const double u_vec = (double)rows * Bc;
        const double sz = sizeof(cx<R>), e_vec = u_vec * sz;
        // one iteration: five kernels on stream q (event brackets when accounting is on)
        auto launch_iter = [&](cudaStream_t q, bool prof, bool set_attr) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            { Prof pr(HEOM_KC_KRYLOV_VECTOR, q, u_vec, 5.0 * e_vec); pr.on = pr.on && prof;
              k_bicg_p<R><<<gv.grid, gv.block, 0, q>>>(v, r, p, vv, ph, rh, Bc, cps, shc, 1, st); }
            { Prof pr(kc_apply, q, u_app, 3.0 * e_vec); pr.on = pr.on && prof;
              if (tiled) { ta.x = ph; ta.out = vv; ta.w = rh; e = launch_tile<R, TM_BICG_V>(ta, q, set_attr); }
              else k_bicg_apply<R><<<gd.grid, gd.block, 0, q>>>(v, ph, vv, rh, Bc, cps, mods, 0, st); }
            if (e != cudaSuccess) return e;
            { Prof pr(HEOM_KC_KRYLOV_VECTOR, q, u_vec, 4.0 * e_vec); pr.on = pr.on && prof;
              k_bicg_s<R><<<gv.grid, gv.block, 0, q>>>(v, r, vv, sh, Bc, cps, shc, 1, st); }
            { Prof pr(kc_apply, q, u_app, 3.0 * e_vec); pr.on = pr.on && prof;
              if (tiled) { ta.x = sh; ta.out = t; ta.w = r; e = launch_tile<R, TM_BICG_T>(ta, q, set_attr); }
              else k_bicg_apply<R><<<gd.grid, gd.block, 0, q>>>(v, sh, t, r, Bc, cps, mods, 1, st); }
            if (e != cudaSuccess) return e;
            { Prof pr(HEOM_KC_KRYLOV_VECTOR, q, u_vec, 8.0 * e_vec); pr.on = pr.on && prof;
              k_bicg_x<R><<<gd.grid, gd.block, 0, q>>>(rows, xw, ph, sh, r, t, rh, Bc, st); }
            return cudaGetLastError();
        };
        // Without launch accounting the iteration runs as a CUDA graph, captured once per
        // column layout on a private stream and replayed on s (five launches become one);
        // if capture or instantiation fails, the kernels are launched directly.
        bool graphed = false;
        if (!prof_on()) {
            if (!gexec || gkey_x != (const void *)cur[0] || gkey_B != Bc || gkey_tiled != tiled) {
                if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
                gkey_x = cur[0];
                gkey_B = Bc;
                gkey_tiled = tiled;
                if (!gcap) cudaStreamCreateWithFlags(&gcap, cudaStreamNonBlocking);
                if (gcap) {
                    if (tiled) {  // shared-memory opt-in set outside the capture
                        HEOM_CUDA((launch_tile_attr<R, TM_BICG_V>(ta)));
                        HEOM_CUDA((launch_tile_attr<R, TM_BICG_T>(ta)));
                    }
                    cudaGraph_t graph = nullptr;
                    if (cudaStreamBeginCapture(gcap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                        const cudaError_t e1 = launch_iter(gcap, false, false);
                        const cudaError_t e2 = cudaStreamEndCapture(gcap, &graph);
                        if (e1 == cudaSuccess && e2 == cudaSuccess && graph &&
                            cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess)
                            gexec = nullptr;
                        if (graph) cudaGraphDestroy(graph);
                    }
                    cudaGetLastError();  // a failed capture leaves no error behind
                }
            }
            if (gexec) {
                for (int k = 0; k < steps; ++k) HEOM_CUDA(cudaGraphLaunch(gexec, s));
                graphed = true;
            }
        }
        if (!graphed)
            for (int k = 0; k < steps; ++k) HEOM_CUDA(launch_iter(s, true, true));
        HEOM_CUDA(cudaGetLastError());
        it += steps;
        HEOM_CUDA(memcpy_counted(hs.data(), st, Bc * sizeof(ColState), cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(cudaStreamSynchronize(s));
        n_act = 0;
        for (int64_t j = 0; j < Bc; ++j) {
            if (!alive[j]) continue;
            const int b = cols[j];
            out.iters[b] = it;
            const double nr = hs[j].acc_nr;
            out.res[b] = hs[j].bnorm2 > 0 ? std::sqrt(nr / hs[j].bnorm2) : 0.0;
            if (!std::isfinite(nr) || hs[j].flag) {
                out.status[b] = HEOM_EBREAKDOWN;
                alive[j] = 0; hs[j].active = 0;
            } else if (nr <= tol2 * hs[j].bnorm2) {
                alive[j] = 0; hs[j].active = 0;
            } else if (nr < best[j]) {
                best[j] = nr;
                best_it[j] = it;
                ++n_act;
            } else if (it - best_it[j] >= kStallIters || nr > 1e12 * best[j]) {
                // stalled: usable if it still improved on the start, otherwise discard
                out.status[b] = nr < hs[j].bnorm2 ? HEOM_ENOCONV : HEOM_EBREAKDOWN;
                alive[j] = 0; hs[j].active = 0;
            } else {
                ++n_act;
            }
        }
        check = std::min(check * 2, 32);
    }
    for (int64_t j = 0; j < Bc; ++j)
        if (alive[j]) out.status[cols[j]] = HEOM_ENOCONV;
    {
        Prof pr(HEOM_KC_OTHER, s, (double)rows * Bc, 2.0 * rows * Bc * sizeof(cx<R>));
        k_scatter_cols<R><<<flat_blocks(rows * Bc), 256, 0, s>>>(rows, cur[0], Bc, x, B, d_map);
    }
    HEOM_CUDA(cudaGetLastError());
    return HEOM_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Solve {
    std::vector<int> iters, refine, status;
    std::vector<double> res;
};

// Solve (M + diag(shift) + aug e00 tr) x = b for all columns, FP64 output, by iterative
// refinement: r = b - A x in FP64, then BiCGStab on A d = r / ||r|| in the inner precision RI,
// x += ||r|| d, until the FP64 residual meets tol. RI = float is the mixed-precision path
// (inner tolerance 1e-5); RI = double is the plain FP64 path, whose inner tolerance asks for
// the whole remaining reduction at once and whose outer loop only guards against the drift
// between BiCGStab's recursive residual and the true one.
constexpr int kInnerCap = 400;     // FP32 BiCGStab iterations per refinement sweep
constexpr int kInnerCap64 = 1500;  // FP64 BiCGStab iterations per sweep (plain path)

// flagged columns: x = 0, r = b
__global__ void k_reset_cols(int64_t total, int64_t B, const int *flags, const cx<double> *b,
                             cx<double> *x, cx<double> *r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i % B]) {
            x[i] = cx<double>{0.0, 0.0};
            r[i] = b[i];
        }
}

template <class RI>
heom_status refine_solve(heom_hier *h, const cx<double> *b64, cx<double> *x64, int64_t B,
                         const cx<double> *shift64, double aug, bool x_zero, double tol,
                         int max_iter, Solve &res, cudaStream_t s,
                         const std::vector<int> *only = nullptr, bool strict = false) {
    const int64_t rows = h->N * h->d2, L = rows * B;
    const size_t bytes = align_up(L * sizeof(cx<double>)) + align_up(15 * L * sizeof(cx<RI>)) +
                         2 * align_up(B * sizeof(cx<RI>));
    heom_status stt = ensure_ws(h->ws, bytes);
    if (stt != HEOM_OK) return stt;
    stt = ensure_ws(h->ws_small, align_up(2 * B * sizeof(ColState)) + 3 * align_up(B * sizeof(int)));
    if (stt != HEOM_OK) return stt;
    ColState *st = (ColState *)h->ws_small.p;
    ColState *st_out = st + B;
    int *d_flags = (int *)((char *)h->ws_small.p + align_up(2 * B * sizeof(ColState)));
    int *d_map = (int *)((char *)d_flags + align_up(B * sizeof(int)));
    int *d_lmap = (int *)((char *)d_map + align_up(B * sizeof(int)));
    res.iters.assign(B, 0);
    res.refine.assign(B, 0);
    res.status.assign(B, HEOM_OK);
    res.res.assign(B, 0.0);
    std::vector<int> active(B, 1);
    if (only) active = *only;
    char *base = (char *)h->ws.p;
    cx<double> *r64 = (cx<double> *)base;
    cx<RI> *w = (cx<RI> *)(base + align_up(L * sizeof(cx<double>)));
    cx<RI> *rhs = w + 13 * L, *dv = w + 14 * L;
    cx<RI> *shift_in = (cx<RI> *)((char *)w + align_up(15 * L * sizeof(cx<RI>)));
    cx<RI> *shift_c = (cx<RI> *)((char *)shift_in + align_up(B * sizeof(cx<RI>)));
    if (shift64) {
        Prof pr(HEOM_KC_OTHER, s, (double)B);
        k_convert<RI, double><<<flat_blocks(B), 256, 0, s>>>(B, shift64, shift_in);
    }
    const DevView<double> v64 = h->view64();
    const int64_t cps = B / h->n_sets;
    const Geom gd = make_geom(rows, B, std::max<int64_t>(1, 2048 / ((B + 31) / 32)));
    ApplyMods<double> m64{shift64, aug};
    std::vector<ColState> hs(B);
    std::vector<int> breakdowns(B, 0);
    const bool plain = sizeof(RI) == 8;
    const int max_sweeps = plain ? 6 : 12;
    if (x_zero) HEOM_CUDA(cudaMemsetAsync(x64, 0, L * sizeof(cx<double>), s));
    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        HEOM_CUDA(memcpy_counted(d_flags, active.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
        int n_on = 0;
        double u_res = 0.0;  // ADO-applies of the residual: the ADOs each active column's set keeps
        for (int64_t b = 0; b < B; ++b)
            if (active[(size_t)b]) {
                ++n_on;
                u_res += (double)h->kept_of_set((int)(b / cps));
            }
        { Prof pr(HEOM_KC_OTHER, s, (double)B);
          k_state_init<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(st_out, B, d_flags); }
        { Prof pr(HEOM_KC_RESIDUAL64, s, u_res, 3.0 * rows * n_on * sizeof(cx<double>));
          if (tile_ok(v64, B)) {
              TileArgs<double> ta{};
              ta.v = v64; ta.x = x64; ta.out = r64; ta.w = b64; ta.shift = shift64; ta.aug = aug;
              ta.st = st_out; ta.B = B;
              HEOM_CUDA((launch_tile<double, TM_RESID>(ta, s)));
          } else {
              k_residual64<<<gd.grid, gd.block, 0, s>>>(v64, b64, x64, r64, B, cps, m64, st_out);
          } }
        HEOM_CUDA(cudaGetLastError());
        HEOM_CUDA(memcpy_counted(hs.data(), st_out, B * sizeof(ColState), cudaMemcpyDeviceToHost, s));
        HEOM_CUDA(cudaStreamSynchronize(s));
        if (sweep == 0 && !x_zero) {
            // a starting guess whose residual exceeds ||b|| is worse than the zero vector:
            // those columns start cold (x = 0, r = b)
            std::vector<int> reset(B, 0);
            int n_reset = 0;
            for (int64_t b = 0; b < B; ++b)
                if (active[b] && !(hs[b].acc_nr <= hs[b].bnorm2)) { reset[b] = 1; ++n_reset; hs[b].acc_nr = hs[b].bnorm2; }
            if (n_reset) {
                HEOM_CUDA(memcpy_counted(d_flags, reset.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
                Prof pr(HEOM_KC_OTHER, s, (double)L, 3.0 * L * sizeof(cx<double>));
                k_reset_cols<<<flat_blocks(L), 256, 0, s>>>(L, B, d_flags, b64, x64, r64);
            }
        }
        int n_act = 0;
        double worst = 0.0;
        for (int64_t b = 0; b < B; ++b) {
            if (!active[b]) continue;
            const double rel = hs[b].bnorm2 > 0 ? std::sqrt(hs[b].acc_nr / hs[b].bnorm2) : 0.0;
            res.res[b] = rel;
            if (!std::isfinite(rel)) { res.status[b] = HEOM_EBREAKDOWN; active[b] = 0; continue; }
            if (rel <= tol || res.iters[b] >= max_iter || sweep == max_sweeps) {
                if (rel > tol) res.status[b] = HEOM_ENOCONV;
                active[b] = 0;
                continue;
            }
            res.refine[b] = plain ? 0 : sweep + 1;
            worst = std::max(worst, rel);
            ++n_act;
        }
        if (n_act == 0) break;
        // keep each residual norm (acc_nr) for the scaling kernels; retire converged columns
        for (int64_t b = 0; b < B; ++b) hs[b].active = active[b];
        HEOM_CUDA(memcpy_counted(st_out, hs.data(), B * sizeof(ColState), cudaMemcpyHostToDevice, s));
        { Prof pr(HEOM_KC_OTHER, s, (double)rows * n_act, (16.0 + sizeof(cx<RI>)) * rows * n_act);
          k_scale_to<RI><<<gd.grid, gd.block, 0, s>>>(rows, r64, rhs, B, st_out); }
        HEOM_CUDA(cudaMemsetAsync(dv, 0, L * sizeof(cx<RI>), s));
        int inner_max = 0;
        for (int64_t b = 0; b < B; ++b)
            if (active[b]) inner_max = std::max(inner_max, max_iter - res.iters[b]);
        // One sweep never asks BiCGStab for more than its attainable accuracy (about 1e-5
        // relative in FP32, about 1e-10 in FP64 on these systems, limited by the size of
        // intermediate residuals); refinement from the FP64 residual supplies the rest.
        const double inner_tol = plain ? std::max(0.5 * tol / worst, 1e-10) : 1e-4;
        inner_max = std::min(inner_max, plain ? kInnerCap64 : kInnerCap);
        SolveOut o;
        if (B == 1 && !strict && persist_ok<RI>(h)) {
            // one column: the whole BiCGStab solve is one cooperative launch
            o.iters.assign(1, 0);
            o.status.assign(1, HEOM_OK);
            o.res.assign(1, 0.0);
            stt = bicgstab_persistent<RI>(h, rhs, dv, true, shift64 ? shift_in : nullptr, (RI)aug,
                                          inner_tol, inner_max, kStallIters, &o.iters[0],
                                          &o.status[0], &o.res[0], s);
        } else {
            stt = bicgstab<RI>(h, rhs, dv, B, shift64 ? shift_in : nullptr, (RI)aug, true, inner_tol,
                               inner_max, active, w, st, d_map, d_lmap, shift_c, o, s);
        }
        if (stt != HEOM_OK) return stt;
        bool skip_any = false;
        for (int64_t b = 0; b < B; ++b) {
            if (!active[b]) continue;
            res.iters[b] += o.iters[b];
            if (o.status[b] == HEOM_ETIMEOUT) {  // a device wait ran out: keep x64, stop
                hs[b].active = 0;
                skip_any = true;
                res.status[b] = HEOM_ETIMEOUT;
                active[b] = 0;
                continue;
            }
            if (o.status[b] == HEOM_EBREAKDOWN) {  // keep x64; retry from it next sweep
                hs[b].active = 0;
                skip_any = true;
                if (++breakdowns[b] >= 2) { res.status[b] = HEOM_EBREAKDOWN; active[b] = 0; }
            }
        }
        if (skip_any)
            HEOM_CUDA(memcpy_counted(st_out, hs.data(), B * sizeof(ColState), cudaMemcpyHostToDevice, s));
        { Prof pr(HEOM_KC_OTHER, s, (double)rows * n_act, (32.0 + sizeof(cx<RI>)) * rows * n_act);
          k_accum<RI><<<gd.grid, gd.block, 0, s>>>(rows, x64, dv, B, st_out); }
        HEOM_CUDA(cudaGetLastError());
    }
    return HEOM_OK;
}

// zero the batch columns flagged in keep (device int [B])
__global__ void k_zero_cols(int64_t total, cx<double> *x, int64_t B, const int *flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i % B]) x[i] = cx<double>{0.0, 0.0};
}

heom_status solve_system(heom_hier *h, const cx<double> *b64, cx<double> *x64, int64_t B,
                         const cx<double> *shift64, double aug, bool x_zero, double tol,
                         int max_iter, int prec, Solve &res, cudaStream_t s) {
    if (prec != HEOM_MIXED)  // HEOM_FP64_STRICT: no float-float persistent solve
        return refine_solve<double>(h, b64, x64, B, shift64, aug, x_zero, tol, max_iter, res, s,
                                    nullptr, prec == HEOM_FP64_STRICT);
    heom_status st = refine_solve<float>(h, b64, x64, B, shift64, aug, x_zero, tol, max_iter, res, s);
    if (st != HEOM_OK) return st;
    // columns whose FP32 corrections broke down (near-singular systems whose FP32 BiCGStab
    // overflows or stalls) are solved again from zero with FP64 inner solves
    std::vector<int> redo(B, 0);
    int n_redo = 0;
    for (int64_t b = 0; b < B; ++b)
        if (res.status[b] == HEOM_EBREAKDOWN) { redo[b] = 1; ++n_redo; }
    if (n_redo == 0) return HEOM_OK;
    DBuf flags;
    st = dalloc(flags, B * sizeof(int));
    if (st != HEOM_OK) return st;
    HEOM_CUDA(memcpy_counted(flags.p, redo.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    const int64_t L = h->N * h->d2 * B;
    { Prof pr(HEOM_KC_OTHER, s, (double)L);
      k_zero_cols<<<flat_blocks(L), 256, 0, s>>>(L, x64, B, (const int *)flags.p); }
    Solve r2;
    st = refine_solve<double>(h, b64, x64, B, shift64, aug, false, tol, max_iter, r2, s, &redo);
    dfree(flags);
    if (st != HEOM_OK) return st;
    for (int64_t b = 0; b < B; ++b)
        if (redo[b]) {
            res.iters[b] += r2.iters[b];
            res.res[b] = r2.res[b];
            res.status[b] = r2.status[b];
        }
    return HEOM_OK;
}

// System-term values of H(t) = H + sum_k f_k(t) H_k at cnt consecutive samples j0 .. j0+cnt-1
// of the drive table f [n_drive][T] (row-major): sv[j][set][t] = s_val[set][t] +
// sum_k f[k][j0 + j] td[k][t], formed in FP64 and stored in the apply's precision.
template <class R>
__global__ void k_td_sval(cx<R> *__restrict__ sv, const cx<double> *__restrict__ s_val,
                          const cx<double> *__restrict__ td, const double *__restrict__ f, int64_t T,
                          int64_t j0, int64_t cnt, int n_sets, int nS, int n_drive) {
    const int64_t per = (int64_t)n_sets * nS, total = cnt * per;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / per, r = i - j * per;
        const int t = (int)(r % nS);
        cx<double> v = s_val[r];
        for (int k = 0; k < n_drive; ++k) {
            const double fk = f[(int64_t)k * T + j0 + j];
            v.re += fk * td[(int64_t)k * nS + t].re;
            v.im += fk * td[(int64_t)k * nS + t].im;
        }
        sv[i] = cast<R>(v);
    }
}

// Classical RK4 over n_steps. With a drive table f (host, [n_drive][2 n_steps + 1], f_k at
// t0 + j dt / 2) the system terms follow H(t): stage 1 of step n reads sample 2n, stages 2
// and 3 sample 2n + 1, stage 4 sample 2n + 2; the values of up to kTdChunk samples are formed
// on the device at a time.
constexpr int64_t kTdChunk = 1025;

template <class R>
heom_status evolve_impl(heom_hier *h, cx<R> *y, int64_t B, double dt, int64_t n_steps,
                        int64_t save_every, cx<R> *traj, const double *f_host, cudaStream_t s) {
    const DevView<R> v = view_of<R>(h);
    const int64_t rows = h->N * h->d2, L = rows * B;
    heom_status st = ensure_ws(h->ws, 3 * L * sizeof(cx<R>));
    if (st != HEOM_OK) return st;
    cx<R> *za = (cx<R> *)h->ws.p, *zb = za + L, *acc = za + 2 * L;
    const Geom g = make_geom(rows, B, 1 << 30);
    const int64_t cps = B / h->n_sets;
    const size_t blk = (size_t)h->d2 * B * sizeof(cx<R>);
    int64_t saved = 0;
    if (traj) HEOM_CUDA(memcpy_counted(traj, y, blk, cudaMemcpyDeviceToDevice, s));
    const double u = (double)h->N * B, pass = (double)L * sizeof(cx<R>);
    const bool tiled = tile_ok(v, B);
    // time-dependent system terms: drive table and per-sample values on the device
    const bool td = f_host && h->n_drive > 0 && n_steps > 0;
    const int64_t T = 2 * n_steps + 1, per = (int64_t)h->n_sets * h->nS;
    DBuf tdbuf;
    double *fdev = nullptr;
    cx<R> *sv = nullptr;
    int64_t j0 = 0, jcnt = 0;
    if (td) {
        const int64_t fb = (int64_t)h->n_drive * T * sizeof(double);
        const int64_t ch = std::min(T, kTdChunk);
        if ((st = dalloc(tdbuf, fb + ch * std::max<int64_t>(per, 1) * sizeof(cx<R>) + 16)) != HEOM_OK) return st;
        fdev = (double *)tdbuf.p;
        sv = (cx<R> *)((char *)tdbuf.p + ((fb + 15) / 16) * 16);
        HEOM_CUDA(memcpy_counted(fdev, f_host, fb, cudaMemcpyHostToDevice, s));
    }
    auto view_at = [&](int64_t j) -> heom_status {  // values of sample j (refills the chunk)
        if (j < j0 || j >= j0 + jcnt) {
            j0 = j;
            jcnt = std::min(kTdChunk, T - j);
            Prof pr(HEOM_KC_OTHER, s, (double)(jcnt * per));
            k_td_sval<R><<<flat_blocks(jcnt * per), 256, 0, s>>>(
                sv, (const cx<double> *)h->d_sval64.p, (const cx<double> *)h->d_tdval64.p, fdev, T, j0,
                jcnt, h->n_sets, h->nS, h->n_drive);
            HEOM_CUDA(cudaGetLastError());
        }
        return HEOM_OK;
    };
    TileArgs<R> ta{};
    ta.v = v;
    ta.y = y;
    ta.acc = acc;
    ta.dt = (R)dt;
    ta.B = B;
    DevView<R> vt = v;
    auto stage = [&](const cx<R> *zi, cx<R> *zo, int st_no) -> cudaError_t {
        if (tiled) {
            ta.v = vt;
            ta.x = zi;
            ta.out = zo;
            ta.stage = st_no;
            return launch_tile<R, TM_RK4>(ta, s);
        }
        k_rk4_stage<R><<<g.grid, g.block, 0, s>>>(vt, zi, zo, y, acc, B, cps, (R)dt, st_no);
        return cudaGetLastError();
    };
    auto at = [&](int64_t j) -> heom_status {
        if (!td) return HEOM_OK;
        const heom_status r = view_at(j);
        if (r == HEOM_OK) vt.s_val = sv + (j - j0) * per;
        return r;
    };
    for (int64_t step = 1; step <= n_steps; ++step) {
        const int64_t j = 2 * (step - 1);
        if ((st = at(j)) != HEOM_OK) { dfree(tdbuf); return st; }
        { Prof pr(HEOM_KC_RK4, s, u, 3.0 * pass); HEOM_CUDA(stage(y, za, 1)); }
        if ((st = at(j + 1)) != HEOM_OK) { dfree(tdbuf); return st; }
        { Prof pr(HEOM_KC_RK4, s, u, 5.0 * pass); HEOM_CUDA(stage(za, zb, 2)); }
        { Prof pr(HEOM_KC_RK4, s, u, 5.0 * pass); HEOM_CUDA(stage(zb, za, 3)); }
        if ((st = at(j + 2)) != HEOM_OK) { dfree(tdbuf); return st; }
        { Prof pr(HEOM_KC_RK4, s, u, 4.0 * pass); HEOM_CUDA(stage(za, zb, 4)); }
        if (traj && step % save_every == 0) {
            ++saved;
            HEOM_CUDA(memcpy_counted((char *)traj + saved * blk, y, blk, cudaMemcpyDeviceToDevice, s));
        }
    }
    HEOM_CUDA(cudaGetLastError());
    HEOM_CUDA(cudaStreamSynchronize(s));
    dfree(tdbuf);
    return HEOM_OK;
}

}  // namespace
}  // namespace heom

using namespace heom;

extern "C" heom_status heom_evolve(heom_hier *h, void *ados, int64_t batch, double dt,
                                   int64_t n_steps, int64_t save_every, void *rho_traj, int prec,
                                   heom_stream s) {
    if (!h || !ados || batch < 1 || batch % h->n_sets != 0 || !std::isfinite(dt) || n_steps < 0 ||
        (rho_traj && save_every < 1) || (prec != HEOM_FP64 && prec != HEOM_FP32) ||
        batch > 65535LL * 32) {
        set_error("heom_evolve: need a hierarchy, ados, batch >= 1 (multiple of n_sets), finite dt, "
                  "n_steps >= 0, save_every >= 1 with a trajectory, prec FP64 or FP32");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    if (prec == HEOM_FP64)
        return evolve_impl<double>(h, (cx<double> *)ados, batch, dt, n_steps, save_every,
                                   (cx<double> *)rho_traj, nullptr, (cudaStream_t)s);
    return evolve_impl<float>(h, (cx<float> *)ados, batch, dt, n_steps, save_every,
                              (cx<float> *)rho_traj, nullptr, (cudaStream_t)s);
}

extern "C" heom_status heom_evolve_td(heom_hier *h, void *ados, int64_t batch, double dt,
                                      int64_t n_steps, const double *f, int64_t save_every,
                                      void *rho_traj, int prec, heom_stream s) {
    if (!h || !ados || batch < 1 || batch % h->n_sets != 0 || !std::isfinite(dt) || n_steps < 0 ||
        (rho_traj && save_every < 1) || (prec != HEOM_FP64 && prec != HEOM_FP32) ||
        batch > 65535LL * 32 || (h->n_drive > 0 && n_steps > 0 && !f)) {
        set_error("heom_evolve_td: need a hierarchy, ados, batch >= 1 (multiple of n_sets), finite "
                  "dt, n_steps >= 0, the drive table, save_every >= 1 with a trajectory, prec FP64 "
                  "or FP32");
        return HEOM_EINVAL;
    }
    if (h->n_drive > 0)
        for (int64_t i = 0; i < (int64_t)h->n_drive * (2 * n_steps + 1); ++i)
            if (!std::isfinite(f[i])) { set_error("heom_evolve_td: non-finite drive value"); return HEOM_EINVAL; }
    HEOM_DEVICE(h->device);
    if (prec == HEOM_FP64)
        return evolve_impl<double>(h, (cx<double> *)ados, batch, dt, n_steps, save_every,
                                   (cx<double> *)rho_traj, f, (cudaStream_t)s);
    return evolve_impl<float>(h, (cx<float> *)ados, batch, dt, n_steps, save_every,
                              (cx<float> *)rho_traj, f, (cudaStream_t)s);
}

static void fill_stats(heom_solve_stats *stats, const Solve &r, int64_t off, int64_t n) {
    if (!stats) return;
    for (int64_t b = 0; b < n; ++b) {
        stats[b].iterations = r.iters[off + b];
        stats[b].refinements = r.refine[off + b];
        stats[b].residual = r.res[off + b];
        stats[b].status = r.status[off + b];
    }
}

extern "C" heom_status heom_steady(heom_hier *h, const void *x0, void *x_out, int64_t batch,
                                   double tol, int max_iter, int prec, heom_solve_stats *stats,
                                   heom_stream s) {
    if (!h || !x_out || batch < 1 || batch % h->n_sets != 0 || !(tol > 0) || max_iter < 1 ||
        (prec != HEOM_FP64 && prec != HEOM_MIXED && prec != HEOM_FP64_STRICT) ||
        batch > 65535LL * 32 || h->parity != 1) {
        set_error("heom_steady: need an even-parity hierarchy, x_out, batch >= 1 (multiple of "
                  "n_sets), tol > 0, max_iter >= 1, prec FP64, FP64_STRICT or MIXED");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    cudaStream_t st = (cudaStream_t)s;
    const int64_t rows = h->N * h->d2, L = rows * batch;
    // the right-hand side e_(0,(0,0)) lives behind the solver workspace in ws_small's sibling
    DBuf bbuf;
    heom_status stt = dalloc(bbuf, L * sizeof(cx<double>));
    if (stt != HEOM_OK) return stt;
    cx<double> *b64 = (cx<double> *)bbuf.p, *x = (cx<double> *)x_out;
    { Prof pr(HEOM_KC_OTHER, st, (double)L);
      k_set_e00<double><<<flat_blocks(L), 256, 0, st>>>(L, b64, batch); }
    if (x0) {
        if (x0 != x_out) memcpy_counted(x, x0, L * sizeof(cx<double>), cudaMemcpyDeviceToDevice, st);
    }
    // drive ||b - A x|| below tol/10: then ||M x|| / ||x|| <= tol for ||x|| >= 0.2
    Solve r;
    stt = solve_system(h, b64, x, batch, nullptr, 1.0, x0 == nullptr, 0.1 * tol, max_iter, prec, r, st);
    dfree(bbuf);
    if (stt != HEOM_OK) return stt;
    // normalise Tr rho_sys = 1 and measure r_ss = ||M x|| / ||x||
    std::vector<cx<double>> top((size_t)h->d2 * batch);
    HEOM_CUDA(memcpy_counted(top.data(), x, top.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
    HEOM_CUDA(cudaStreamSynchronize(st));
    std::vector<cx<double>> fac(batch);
    for (int64_t b = 0; b < batch; ++b) {
        cx<double> tr{0.0, 0.0};
        for (int i = 0; i < h->d; ++i) tr = tr + top[(size_t)(i * h->d + i) * batch + b];
        fac[b] = (tr.re == 0.0 && tr.im == 0.0) ? cx<double>{1.0, 0.0} : cdiv(cx<double>{1.0, 0.0}, tr);
    }
    DBuf tmp;
    stt = dalloc(tmp, batch * (sizeof(cx<double>) + 2 * sizeof(double)));
    if (stt != HEOM_OK) return stt;
    cx<double> *dfac = (cx<double> *)tmp.p;
    double *norms = (double *)(dfac + batch);
    HEOM_CUDA(memcpy_counted(dfac, fac.data(), batch * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    { Prof pr(HEOM_KC_OTHER, st, (double)L);
      k_scale_cols<double><<<flat_blocks(L), 256, 0, st>>>(L, x, batch, dfac); }
    HEOM_CUDA(cudaMemsetAsync(norms, 0, 2 * batch * sizeof(double), st));
    const Geom gd = make_geom(rows, batch, std::max<int64_t>(1, 2048 / ((batch + 31) / 32)));
    { Prof pr(HEOM_KC_RESIDUAL64, st, (double)h->N * batch, (double)L * sizeof(cx<double>));
      if (tile_ok(h->view64(), batch)) {
          TileArgs<double> ta{};
          ta.v = h->view64(); ta.x = x; ta.norms = norms; ta.B = batch;
          HEOM_CUDA((launch_tile<double, TM_NORMS>(ta, st)));
      } else {
          k_apply_norms<<<gd.grid, gd.block, 0, st>>>(h->view64(), x, batch, batch / h->n_sets, norms);
      } }
    std::vector<double> hn(2 * batch);
    HEOM_CUDA(memcpy_counted(hn.data(), norms, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HEOM_CUDA(cudaStreamSynchronize(st));
    dfree(tmp);
    heom_status ret = HEOM_OK;
    for (int64_t b = 0; b < batch; ++b) {
        // r_ss = ||M x|| / ||x||; a zero iterate (a solve that never started) has none
        r.res[b] = hn[2 * b + 1] > 0.0 ? std::sqrt(hn[2 * b] / hn[2 * b + 1]) : INFINITY;
        if (r.status[b] == HEOM_OK && !(r.res[b] <= tol)) r.status[b] = HEOM_ENOCONV;
        if (r.status[b] != HEOM_OK && ret == HEOM_OK) ret = (heom_status)r.status[b];
    }
    fill_stats(stats, r, 0, batch);
    if (ret != HEOM_OK) set_error("heom_steady: some columns did not converge (see stats)");
    return ret;
}

// Density of states from shift-invariant Krylov processes: for parameter set s of the
// hierarchy, column 2s carries the x_+ family (right-hand side d^dag rho_s, shifts +i w) and
// column 2s+1 the x_- family (d rho_s, shifts -i w). A_out [n_sets][n_omega]; stats
// [n_sets][x_+ then x_-][n_omega].
static heom_status spectrum_shifted(heom_hier *odd, const void *ss_ados, const heom_c64 *op_d,
                                    const double *omega, int64_t n_omega, double tol,
                                    int max_iter, double *A_out, heom_solve_stats *stats,
                                    cudaStream_t st) {
    const int d = odd->d;
    const int64_t ns = odd->n_sets, B = 2 * ns;
    const int64_t rows = odd->N * odd->d2, L = rows * B;
    DBuf buf;
    heom_status stt = dalloc(buf, L * sizeof(cx<double>) + 2 * d * d * sizeof(cx<double>));
    if (stt != HEOM_OK) return stt;
    cx<double> *b64 = (cx<double> *)buf.p, *ops = b64 + L;
    std::vector<cx<double>> hops(2 * d * d);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            hops[r * d + c] = {op_d[c * d + r].re, -op_d[c * d + r].im};  // d^dagger
            hops[d * d + r * d + c] = {op_d[r * d + c].re, op_d[r * d + c].im};
        }
    HEOM_CUDA(memcpy_counted(ops, hops.data(), hops.size() * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    { Prof pr(HEOM_KC_OTHER, st, (double)L);
      k_dos_rhs_sets<<<flat_blocks(L), 256, 0, st>>>(odd->N, d, (const cx<double> *)ss_ados, ops, ops + d * d, b64, ns); }
    const int64_t S = 2 * n_omega * ns;
    std::vector<cx<double>> shift(S);
    std::vector<int> col_of(S);
    for (int64_t set = 0; set < ns; ++set)
        for (int64_t j = 0; j < n_omega; ++j) {
            const int64_t kp = set * 2 * n_omega + j, km = kp + n_omega;
            shift[kp] = {0.0, omega[j]};   // (M + i w) x_+ = d^dag rho
            col_of[kp] = (int)(2 * set);
            shift[km] = {0.0, -omega[j]};  // (M - i w) x_- = d rho
            col_of[km] = (int)(2 * set + 1);
        }
    std::vector<cx<double>> x0;
    std::vector<double> res;
    int steps = 0;
    stt = shifted_gmres(odd, b64, B, shift, col_of, 0.5 * tol, std::max(1, std::min(max_iter, 2000)),
                        x0, res, &steps, st);
    dfree(buf);
    if (stt == HEOM_ETIMEOUT) {  // a device wait ran out: no solution, every frequency flagged
        for (int64_t k = 0; k < ns * n_omega; ++k) A_out[k] = NAN;
        if (stats)
            for (int64_t k = 0; k < S; ++k) stats[k] = heom_solve_stats{steps, 0, NAN, HEOM_ETIMEOUT};
        return stt;
    }
    if (stt != HEOM_OK) return stt;
    heom_status ret = HEOM_OK;
    const int d2 = d * d;
    for (int64_t set = 0; set < ns; ++set)
        for (int64_t j = 0; j < n_omega; ++j) {
            const int64_t kp = set * 2 * n_omega + j, km = kp + n_omega;
            double acc = 0;
            for (int i = 0; i < d; ++i)
                for (int l = 0; l < d; ++l) {
                    const cx<double> xp = x0[(size_t)kp * d2 + l * d + i];
                    const cx<double> xm = x0[(size_t)km * d2 + l * d + i];
                    const cx<double> dd{op_d[i * d + l].re, op_d[i * d + l].im};
                    const cx<double> dh{op_d[l * d + i].re, -op_d[l * d + i].im};
                    acc += (dd * xp).re + (dh * xm).re;
                }
            A_out[set * n_omega + j] = -acc / M_PI;
        }
    for (int64_t k = 0; k < S; ++k) {
        const int status = (std::isfinite(res[k]) && res[k] <= tol) ? HEOM_OK : HEOM_ENOCONV;
        if (status != HEOM_OK && ret == HEOM_OK) ret = HEOM_ENOCONV;
        if (stats) stats[k] = heom_solve_stats{steps, 0, res[k], status};
    }
    if (ret != HEOM_OK) set_error("heom_spectrum: some frequencies did not converge (see stats)");
    return ret;
}

// b[row][s] = (a rho_s)[row]: left multiplication of every ADO of set s's stationary state
// (ss [N][d][d][ns]) by the d x d operator a
__global__ void k_psd_rhs(int64_t N, int d, const cx<double> *__restrict__ ss, const cx<double> *__restrict__ A,
                          cx<double> *__restrict__ bvec, int64_t ns) {
    const int64_t total = N * d * d * ns;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t set = i % ns, row = i / ns;
        const int64_t n = row / (d * d);
        const int e = (int)(row - n * d * d), r = e / d, c = e - r * d;
        cx<double> acc{0.0, 0.0};
        for (int l = 0; l < d; ++l) fma_to(acc, A[r * d + l], ss[(n * d * d + l * d + c) * ns + set]);
        bvec[i] = acc;
    }
}

extern "C" heom_status heom_psd(heom_hier *even, const void *ss_ados, const heom_c64 *op_a,
                                const double *omega, int64_t n_omega, double tol, int max_iter,
                                double *S_out, heom_solve_stats *stats, heom_stream s) {
    if (!even || !ss_ados || !op_a || !omega || n_omega < 1 || !(tol > 0) || max_iter < 1 || !S_out ||
        even->parity != 1) {
        set_error("heom_psd: need an even-parity hierarchy, ss_ados, op_a, omega[n_omega >= 1], S_out, "
                  "tol > 0 and max_iter >= 1");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(even->device);
    cudaStream_t st = (cudaStream_t)s;
    const int d = even->d, d2 = d * d;
    const int64_t ns = even->n_sets, B = ns, rows = even->N * even->d2, L = rows * B;
    DBuf buf;
    heom_status stt = dalloc(buf, L * sizeof(cx<double>) + d2 * sizeof(cx<double>));
    if (stt != HEOM_OK) return stt;
    cx<double> *b64 = (cx<double> *)buf.p, *A = b64 + L;
    HEOM_CUDA(memcpy_counted(A, op_a, d2 * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    { Prof pr(HEOM_KC_OTHER, st, (double)L);
      k_psd_rhs<<<flat_blocks(L), 256, 0, st>>>(even->N, d, (const cx<double> *)ss_ados, A, b64, ns); }
    const int64_t S = n_omega * ns;
    std::vector<cx<double>> shift(S);
    std::vector<int> col_of(S);
    for (int64_t set = 0; set < ns; ++set)
        for (int64_t j = 0; j < n_omega; ++j) {
            shift[set * n_omega + j] = {0.0, -omega[j]};  // (M - i w) x = a rho
            col_of[set * n_omega + j] = (int)set;
        }
    std::vector<cx<double>> x0;
    std::vector<double> res;
    int steps = 0;
    stt = shifted_gmres(even, b64, B, shift, col_of, 0.5 * tol, std::max(1, std::min(max_iter, 2000)), x0,
                        res, &steps, st);
    dfree(buf);
    if (stt == HEOM_ETIMEOUT) {  // a device wait ran out: no solution, every frequency flagged
        for (int64_t k = 0; k < S; ++k) {
            S_out[k] = NAN;
            if (stats) stats[k] = heom_solve_stats{steps, 0, NAN, HEOM_ETIMEOUT};
        }
        return stt;
    }
    if (stt != HEOM_OK) return stt;
    heom_status ret = HEOM_OK;
    for (int64_t k = 0; k < S; ++k) {
        // pi S(w) = -Re Tr[a^dag x_0], Tr[a^dag X] = sum_{i,l} conj(a[l][i]) X[l][i]
        double acc = 0.0;
        for (int i = 0; i < d; ++i)
            for (int l = 0; l < d; ++l) {
                const cx<double> xv = x0[(size_t)k * d2 + l * d + i];
                const cx<double> ah{op_a[l * d + i].re, -op_a[l * d + i].im};
                acc += (ah * xv).re;
            }
        S_out[k] = -acc / M_PI;
        const int status = (std::isfinite(res[k]) && res[k] <= tol) ? HEOM_OK : HEOM_ENOCONV;
        if (status != HEOM_OK && ret == HEOM_OK) ret = HEOM_ENOCONV;
        if (stats) stats[k] = heom_solve_stats{steps, 0, res[k], status};
    }
    if (ret != HEOM_OK) set_error("heom_psd: some frequencies did not converge (see stats)");
    return ret;
}

extern "C" heom_status heom_spectrum_batched(int n_hier, heom_hier *const *odd, const void *const *ss_ados,
                                             const heom_c64 *const *op_d, const double *omega,
                                             int64_t n_omega, double tol, int max_iter, double *A_out,
                                             int prec, heom_solve_stats *stats, heom_stream s) {
    if (n_hier < 1 || !odd || !ss_ados || !op_d || !omega || n_omega < 1 || !A_out) {
        set_error("heom_spectrum_batched: need n_hier >= 1 and the per-hierarchy arrays, omega, A_out");
        return HEOM_EINVAL;
    }
    for (int h = 0; h < n_hier; ++h)
        if (!odd[h] || !ss_ados[h] || !op_d[h] || odd[h]->parity != -1) {
            set_error("heom_spectrum_batched: hierarchy %d: need an odd-parity hierarchy, its "
                      "stationary state and its operator", h);
            return HEOM_EINVAL;
        }
    heom_status first = HEOM_OK;
    int64_t row = 0;
    for (int h = 0; h < n_hier; ++h) {
        const int64_t ns = odd[h]->n_sets;
        const heom_status st = heom_spectrum(odd[h], ss_ados[h], op_d[h], omega, n_omega, tol, max_iter,
                                             A_out + row * n_omega, prec,
                                             stats ? stats + 2 * row * n_omega : nullptr, s);
        if (st != HEOM_OK && first == HEOM_OK) first = st;
        if (st == HEOM_EINVAL || st == HEOM_ECUDA || st == HEOM_ENOMEM) return st;
        row += ns;
    }
    return first;
}

extern "C" heom_status heom_spectrum(heom_hier *odd, const void *ss_ados, const heom_c64 *op_d,
                                     const double *omega, int64_t n_omega, double tol,
                                     int max_iter, double *A_out, int prec,
                                     heom_solve_stats *stats, heom_stream s) {
    if (!odd || !ss_ados || !op_d || !omega || n_omega < 1 || !(tol > 0) || max_iter < 1 ||
        !A_out || (prec != HEOM_FP64 && prec != HEOM_MIXED && prec != HEOM_SHIFTED) ||
        (odd->n_sets != 1 && prec != HEOM_SHIFTED) || 2 * n_omega > 65535LL * 32 ||
        2LL * odd->n_sets > 65535LL * 32) {
        set_error("heom_spectrum: need an odd-parity hierarchy (several parameter sets only with "
                  "SHIFTED), ss_ados, op_d, omega[n_omega >= 1], A_out, tol > 0, max_iter >= 1, "
                  "prec FP64, MIXED or SHIFTED");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(odd->device);
    cudaStream_t st = (cudaStream_t)s;
    const int d = odd->d;
    if (prec == HEOM_SHIFTED) return spectrum_shifted(odd, ss_ados, op_d, omega, n_omega, tol,
                                                      max_iter, A_out, stats, st);
    const int64_t B = 2 * n_omega, rows = odd->N * odd->d2, L = rows * B;
    DBuf buf;
    heom_status stt = dalloc(buf, L * 2 * sizeof(cx<double>) + B * sizeof(cx<double>) +
                                      2 * d * d * sizeof(cx<double>));
    if (stt != HEOM_OK) return stt;
    cx<double> *b64 = (cx<double> *)buf.p, *x64 = b64 + L, *shift = x64 + L, *ops = shift + B;
    std::vector<cx<double>> hops(2 * d * d), hshift(B);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            hops[r * d + c] = {op_d[c * d + r].re, -op_d[c * d + r].im};  // d^dagger
            hops[d * d + r * d + c] = {op_d[r * d + c].re, op_d[r * d + c].im};
        }
    for (int64_t j = 0; j < n_omega; ++j) {
        hshift[j] = {0.0, omega[j]};             // (M + i w) x_+ = d^dag rho
        hshift[n_omega + j] = {0.0, -omega[j]};  // (M - i w) x_- = d rho
    }
    HEOM_CUDA(memcpy_counted(ops, hops.data(), hops.size() * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    HEOM_CUDA(memcpy_counted(shift, hshift.data(), B * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    { Prof pr(HEOM_KC_OTHER, st, (double)L);
      k_dos_rhs<<<flat_blocks(L), 256, 0, st>>>(odd->N, d, (const cx<double> *)ss_ados, ops, ops + d * d, b64, n_omega); }
    Solve r;
    stt = solve_system(odd, b64, x64, B, shift, 0.0, true, tol, max_iter, prec, r, st);
    if (stt != HEOM_OK) { dfree(buf); return stt; }
    std::vector<cx<double>> top((size_t)d * d * B);
    HEOM_CUDA(memcpy_counted(top.data(), x64, top.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
    HEOM_CUDA(cudaStreamSynchronize(st));
    dfree(buf);
    heom_status ret = HEOM_OK;
    for (int64_t j = 0; j < n_omega; ++j) {
        // -Re{Tr[d x_+] + Tr[d^dag x_-]} / pi with Tr[O X] = sum_{i,l} O[i][l] X[l][i]
        double acc = 0;
        for (int i = 0; i < d; ++i)
            for (int l = 0; l < d; ++l) {
                const cx<double> xp = top[(size_t)(l * d + i) * B + j];
                const cx<double> xm = top[(size_t)(l * d + i) * B + n_omega + j];
                const cx<double> dd{op_d[i * d + l].re, op_d[i * d + l].im};
                const cx<double> dh{op_d[l * d + i].re, -op_d[l * d + i].im};
                acc += (dd * xp).re + (dh * xm).re;
            }
        A_out[j] = -acc / M_PI;
    }
    for (int64_t b = 0; b < B; ++b)
        if (r.status[b] != HEOM_OK && ret == HEOM_OK) ret = (heom_status)r.status[b];
    fill_stats(stats, r, 0, B);
    if (ret != HEOM_OK) set_error("heom_spectrum: some frequencies did not converge (see stats)");
    return ret;
}

// ------------------------------------------------------------------ electronic current
namespace heom {
namespace {

// I[b] = Re(i sum_t sign_t Tr[O_t rho_{ado_t}]) for batch column b: one block per column,
// threads over (term, row, column) triples, a fixed-order block reduction.
__global__ void __launch_bounds__(128) k_current(int n_terms, int d, const int *__restrict__ ado,
                                                 const int *__restrict__ sign, const cx<double> *__restrict__ O,
                                                 const cx<double> *__restrict__ x, int64_t B, double *__restrict__ out) {
    const int64_t b = blockIdx.x;
    const int d2 = d * d;
    __shared__ double s_im[128];
    double acc = 0.0;  // Im of the signed trace sum
    for (int w = threadIdx.x; w < n_terms * d2; w += blockDim.x) {
        const int t = w / d2, e = w - t * d2, r = e / d, l = e - r * d;
        // Tr[O rho] = sum_{r,l} O[r][l] rho[l][r]
        const cx<double> o = O[(int64_t)t * d2 + r * d + l];
        const cx<double> rho = x[((int64_t)ado[t] * d2 + l * d + r) * B + b];
        acc += sign[t] * (o.re * rho.im + o.im * rho.re);
    }
    s_im[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 64; k > 0; k >>= 1) {
        if (threadIdx.x < k) s_im[threadIdx.x] += s_im[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = -s_im[0];  // Re(i z) = -Im z
}

}  // namespace
}  // namespace heom

extern "C" heom_status heom_current(const heom_hier *h, const void *x, int64_t batch, const int *baths,
                                    int n_baths, double *I_out, heom_stream s) {
    using namespace heom;
    if (!h || !x || !I_out || batch < 1 || n_baths < 1 || !baths || h->parity != 1 || h->tier_f < 1) {
        set_error("heom_current: need an even-parity hierarchy with fermionic tier >= 1, x, batch >= 1, "
                  "baths[n_baths >= 1] and I_out");
        return HEOM_EINVAL;
    }
    std::vector<char> in_lead(h->bath_slot.size(), 0);
    for (int i = 0; i < n_baths; ++i) {
        if (baths[i] < 0 || baths[i] >= (int)h->bath_slot.size()) {
            set_error("heom_current: bath index %d out of range", baths[i]);
            return HEOM_EINVAL;
        }
        in_lead[baths[i]] = 1;
    }
    // tier-1 fermionic ADO {q} (bosonic part 0) of every exponent of the lead, with
    // O = d^{-nu} (slot of d for nu = +1, of d^dagger for nu = -1) and sign nu
    const int d = h->d, d2 = h->d2;
    std::vector<int> ado, sign;
    std::vector<heom_c64> O;
    for (int q = 0; q < h->K_f; ++q) {
        const int g = h->K_b + q, bath = h->exp_bath[g];
        if (h->exp_kind[g] != HEOM_FERMION || !in_lead[bath]) continue;
        int64_t idx = -1;
        for (int64_t f = 0; f < h->N_f; ++f)
            if (h->fer[f] == (1ULL << q)) { idx = h->compact_of(f); break; }  // bosonic rank 0
        if (idx < 0) continue;
        const int nu = h->exp_nu[g];
        const int slot = h->bath_slot[bath] + (nu == 1 ? 0 : 1);
        ado.push_back((int)idx);
        sign.push_back(nu);
        O.insert(O.end(), h->ops.begin() + (size_t)slot * d2, h->ops.begin() + (size_t)(slot + 1) * d2);
    }
    if (ado.empty()) {
        set_error("heom_current: the baths hold no fermionic exponents");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    cudaStream_t st = (cudaStream_t)s;
    const int nt = (int)ado.size();
    const size_t obytes = O.size() * sizeof(cx<double>), ooff = (obytes + (size_t)nt * 8 + 15) & ~size_t(15);
    DBuf buf;
    heom_status r = dalloc(buf, ooff + batch * sizeof(double));
    if (r != HEOM_OK) return r;
    char *base = (char *)buf.p;
    cx<double> *dO = (cx<double> *)base;
    int *dado = (int *)(base + obytes);
    int *dsign = dado + nt;
    double *dout = (double *)(base + ooff);
    HEOM_CUDA(memcpy_counted(dO, O.data(), obytes, cudaMemcpyHostToDevice, st));
    HEOM_CUDA(memcpy_counted(dado, ado.data(), nt * 4, cudaMemcpyHostToDevice, st));
    HEOM_CUDA(memcpy_counted(dsign, sign.data(), nt * 4, cudaMemcpyHostToDevice, st));
    {
        Prof pr(HEOM_KC_OTHER, st, (double)batch * nt * d2);
        k_current<<<(unsigned)batch, 128, 0, st>>>(nt, d, dado, dsign, dO, (const cx<double> *)x, batch, dout);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = memcpy_counted(I_out, dout, batch * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "heom_current");
    return HEOM_OK;
}

extern "C" heom_status heom_conductance(heom_hier *h, const double *dphi, const int *baths, int n_baths,
                                        double tol, int max_iter, int prec, double *G_out, double *I_out,
                                        heom_solve_stats *stats, heom_stream s) {
    using namespace heom;
    if (!h || !dphi || !G_out || h->n_sets < 2 || (h->n_sets & 1) || h->parity != 1) {
        set_error("heom_conductance: need an even-parity hierarchy holding bias pairs (an even "
                  "number >= 2 of parameter sets), dphi[n_sets / 2] and G_out");
        return HEOM_EINVAL;
    }
    const int64_t B = h->n_sets, npair = B / 2;
    for (int64_t k = 0; k < npair; ++k)
        if (!(std::isfinite(dphi[k]) && dphi[k] != 0.0)) {
            set_error("heom_conductance: dphi[%lld] must be finite and non-zero", (long long)k);
            return HEOM_EINVAL;
        }
    HEOM_DEVICE(h->device);
    DBuf xbuf;
    heom_status st = dalloc(xbuf, (size_t)h->N * h->d2 * B * sizeof(cx<double>));
    if (st != HEOM_OK) return st;
    std::vector<heom_solve_stats> ss(B);
    st = heom_steady(h, nullptr, xbuf.p, B, tol, max_iter, prec, ss.data(), s);
    std::vector<double> I(B, 0.0);
    const heom_status sc = (st == HEOM_OK || st == HEOM_ENOCONV || st == HEOM_EBREAKDOWN)
                               ? heom_current(h, xbuf.p, B, baths, n_baths, I.data(), s)
                               : st;
    dfree(xbuf);
    if (sc != HEOM_OK) return sc;
    for (int64_t k = 0; k < npair; ++k) G_out[k] = (I[2 * k + 1] - I[2 * k]) / dphi[k];
    if (I_out) for (int64_t b = 0; b < B; ++b) I_out[b] = I[b];
    if (stats) for (int64_t b = 0; b < B; ++b) stats[b] = ss[b];
    return st;
}
