// Persistent shift-invariant Arnoldi (Methods, numerical computation of the spectrum): the
// steps of the Krylov process that serves every frequency of a spectrum, run in one
// cooperative launch. Each CTA owns one ADO range (one per SM) and keeps that range's term
// programs of Eq. HEOM in shared memory for the whole solve, their coefficients turned into
// float-float once. One Arnoldi step:
//
//   1. w = M v_j on the CTA's own rows (float-float term programs; neighbour rows of v_j
//      through L2);
//   2. classical Gram-Schmidt on the own rows: partial dot products of w with v_0 .. v_j and
//      with itself -> grid barrier -> each CTA reduces a slice of the partials -> barrier ->
//      every CTA reads h; w -= sum_i v_i h_i; a second pass only when the first kept less
//      than 5 % of |w| (the same decision in every CTA);
//   3. |w| by partials -> barrier -> v_{j+1} = w / |w| (FP64 and float-float copies);
//   4. every thread advances the Givens QR of its shifts by the new Hessenberg column
//      (the column is in every CTA's shared memory) and records the residual estimate;
//      the largest estimate over the grid decides, identically in every CTA, whether the
//      solve has converged.
//
// The state it leaves (basis, Hessenberg matrix, rotations, g) is the one the per-step path
// of heom_shifted.cu keeps, so that path can continue where this launch stopped.
#include <algorithm>
#include <cmath>

#include "heom_ff.cuh"
#include "heom_grid.cuh"
#include "heom_tile.cuh"

namespace heom {

namespace {

constexpr int kArThreads = 512;
constexpr int kArMaxSteps = 192;  // Hessenberg column held in shared memory
constexpr int kArMaxB = 8;        // columns (B divides 32)
constexpr double kArKeep2 = 0.05 * 0.05;

struct ArnoldiArgs {
    DevView<double> v;
    int64_t B, L, S;
    int mmax, max_steps;
    int hcap;  // (max_steps + 2) * B: entries of the shared-memory Hessenberg column
    float4 *Vf;
    cx<double> *V, *Hb;
    const cx<double> *shift;
    const int *col_of;
    double *rot_c;
    cx<double> *rot_s, *rdiag, *g;
    float2 *rot_cf;    // the rotations again, split into float-float for the chains
    float4 *rot_sf;
    const double *beta;
    double *res;
    double tol;
    double *part;      // per CTA: dot partials [2][kArMaxSteps + 2][B] complex, norm [B], res max
    cx<double> *hred;  // reduced h of the two passes [2][kArMaxSteps + 2][B]
    GridBar *bar;
    long long wait_cycles;  // bound of every grid-barrier wait (SM clock cycles)
    int *out;          // [0] steps done, [1] converged, [2] barrier failure
};

constexpr int kPartStride = 2 * 2 * (kArMaxSteps + 2) * kArMaxB + kArMaxB + 2;  // doubles per CTA

__device__ __forceinline__ float4 ld_l2_f4(const float4 *p) { return __ldcg(p); }


// Partial dot products conj(V_i) w over the CTA's own elements for i < nv (w is V_nv-1 +1
// slot when self is wanted), into this CTA's slot of part: warp per i, lanes over own
// elements (element = row * B + b; B divides 32, so a lane always sees the same column).
__device__ void own_dots(const ArnoldiArgs &a, const float4 *W, int nv, int64_t e0, int nel,
                         double *mypart) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int B = (int)a.B;
    for (int i = warp; i < nv; i += nw) {
        const float4 *Vi = a.Vf + (int64_t)i * a.L + e0;
        const float4 *Wo = W + e0;
        // float-float accumulation over the lane's elements, one conversion to FP64 at the end
        // (GB300's FP64 pipe is the scarce one)
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        int t = lane;
        for (; t + 96 < nel; t += 128) {  // four elements per lane, eight loads in flight
            float4 x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = Vi[t + 32 * u];
                y[u] = Wo[t + 32 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ff_mac(rh, rl, x[u].x, x[u].z, y[u].x, y[u].z);
                ff_mac(rh, rl, x[u].y, x[u].w, y[u].y, y[u].w);
                ff_mac(ih, il, x[u].x, x[u].z, y[u].y, y[u].w);
                ff_mac(ih, il, -x[u].y, -x[u].w, y[u].x, y[u].z);
            }
        }
        for (; t < nel; t += 32) {
            const float4 x = Vi[t], y = Wo[t];
            ff_mac(rh, rl, x.x, x.z, y.x, y.z);
            ff_mac(rh, rl, x.y, x.w, y.y, y.w);
            ff_mac(ih, il, x.x, x.z, y.y, y.w);
            ff_mac(ih, il, -x.y, -x.w, y.x, y.z);
        }
        // lanes with the same column: reduce over the lane bits above log2(B), in float-float
        // (a tree of dependent FP64 additions is slow on GB300), then one conversion
        ff_norm(rh, rl);
        ff_norm(ih, il);
        for (int o = 16; o >= B; o >>= 1) {
            const float a0 = __shfl_down_sync(0xffffffffu, rh, o), a1 = __shfl_down_sync(0xffffffffu, rl, o);
            const float b0 = __shfl_down_sync(0xffffffffu, ih, o), b1 = __shfl_down_sync(0xffffffffu, il, o);
            ff_add(rh, rl, a0, a1);
            ff_add(ih, il, b0, b1);
        }
        if (lane < B) {
            mypart[2 * (i * B + lane)] = (double)rh + (double)rl;
            mypart[2 * (i * B + lane) + 1] = (double)ih + (double)il;
        }
    }
}

// After the barrier: CTA c reduces pairs p = c, c + G, ... of the nv * B dot products over
// all CTAs (fixed order) into hred; then (after the next barrier) every CTA reads them.
__device__ void slice_reduce(const ArnoldiArgs &a, int pass, int nv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int B = (int)a.B, G = gridDim.x;
    const int np = nv * B;
    for (int p = blockIdx.x + warp * G; p < np; p += nw * G) {
        double re = 0.0, im = 0.0;
        for (int gidx = lane; gidx < G; gidx += 32) {
            const double *pp = a.part + (int64_t)gidx * kPartStride + pass * 2 * (kArMaxSteps + 2) * kArMaxB;
            re += __ldcg(pp + 2 * p);
            im += __ldcg(pp + 2 * p + 1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) a.hred[(int64_t)pass * (kArMaxSteps + 2) * kArMaxB + p] = cx<double>{re, im};
    }
}

__global__ void __launch_bounds__(kArThreads, 1) k_arnoldi(ArnoldiArgs a) {
    unsigned gen = 0;
    const DevView<double> &v = a.v;
    const int d2 = v.d2, B = (int)a.B, G = gridDim.x;
    const int n0 = __ldg(v.pers_ado + blockIdx.x), n1 = __ldg(v.pers_ado + blockIdx.x + 1);
    const int items = (n1 - n0) * d2, nel = items * B;
    const int64_t e0 = (int64_t)n0 * d2 * B;
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    cx<double> *s_hcol = reinterpret_cast<cx<double> *>(smem);    // [max_steps + 2][B]
    float4 *s_hf = reinterpret_cast<float4 *>(s_hcol + a.hcap);   // its float-float split
    double *s_red = reinterpret_cast<double *>(s_hf + a.hcap);     // [32][kArMaxB]
    double *s_nrm = s_red + 32 * kArMaxB;                              // [kArMaxB]
    double *s_ib2 = s_nrm + kArMaxB;                                   // [kArMaxB] 1 / beta^2
    int *s_flag = reinterpret_cast<int *>(s_ib2 + kArMaxB);           // [2 + kArMaxB]
    ProgSmem<double> ps = prog_layout<double>(v.pers_terms, v.pers_slots, v.pers_ados, d2,
                                              reinterpret_cast<unsigned char *>(s_flag + 4));
    if (threadIdx.x < B) {
        const double bt = a.beta[threadIdx.x];
        s_ib2[threadIdx.x] = bt > 0.0 ? 1.0 / (bt * bt) : 0.0;
    }
    build_programs<double>(v, ps, n0, n1, 0.0, 0);
    // coefficients to float-float, in place (a cx<double> and a float4 are both 16 bytes)
    {
        const int nt = ps.item[items];
        float4 *cf = reinterpret_cast<float4 *>(ps.coef);
        for (int t = tid; t < nt; t += bd) {  // each thread rewrites only its own slots
            const cx<double> c = ps.coef[t];
            cf[t] = ff_split(c);
        }
    }
    __syncthreads();
    const float4 *coef = reinterpret_cast<const float4 *>(ps.coef);
    double *mypart = a.part + (int64_t)blockIdx.x * kPartStride;
    int status = 0, steps = 0, converged = 0;

    for (int j = 0; j < a.max_steps; ++j) {
        const float4 *Vj = a.Vf + (int64_t)j * a.L;
        float4 *W = a.Vf + (int64_t)(j + 1) * a.L;
        // ---- 1. w = M v_j on the own elements
        for (int idx = tid; idx < nel; idx += bd) {
            const int it = idx / B, b = idx - it * B;
            const int j0 = ps.item[it], j1 = ps.item[it + 1];
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            for (int t = j0; t < j1; t += 8) {  // 8 loads in flight
                float4 c[8], x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int tt = t + u < j1 ? t + u : j1 - 1;
                    c[u] = t + u < j1 ? coef[tt] : make_float4(0.f, 0.f, 0.f, 0.f);
                    x[u] = ld_l2_f4(Vj + (int64_t)ps.src[tt] * B + b);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) ff_cmac(rh, rl, ih, il, c[u], x[u]);
            }
            ff_norm(rh, rl);
            ff_norm(ih, il);
            W[e0 + idx] = make_float4(rh, ih, rl, il);
        }
        __syncthreads();
        // ---- 2. Gram-Schmidt pass 1 (+ |w|^2 as the dot of w with itself, slot j + 1)
        own_dots(a, W, j + 2, e0, nel, mypart);
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
        slice_reduce(a, 0, j + 2);
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
        for (int p = tid; p < (j + 2) * B; p += bd) {  // written by other CTAs: through L2
            const double2 hv = __ldcg(reinterpret_cast<const double2 *>(a.hred + p));
            const cx<double> h{hv.x, hv.y};
            s_hcol[p] = h;
            s_hf[p] = ff_split(h);
        }
        __syncthreads();
        // second pass needed? warp b tests column b: sum of |h_i|^2 in float (a threshold
        // test), lane-strided with a fixed tree, so every CTA takes the same decision
        if (warp < B) {
            float sacc = 0.f;
            for (int i = lane; i <= j; i += 32) {
                const cx<double> hv = s_hcol[i * B + warp];
                const float hr = (float)hv.re, hi = (float)hv.im;
                sacc += hr * hr + hi * hi;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
            if (lane == 0) {
                const float w2 = (float)s_hcol[(j + 1) * B + warp].re;
                s_flag[2 + warp] = !(w2 - sacc >= (float)kArKeep2 * w2);
            }
        }
        __syncthreads();
        int need2 = 0;
        for (int b = 0; b < B; ++b) need2 |= s_flag[2 + b];
        for (int pass = 0; pass < 1 + need2; ++pass) {
            if (pass == 1) {
                own_dots(a, W, j + 1, e0, nel, mypart + 2 * (kArMaxSteps + 2) * kArMaxB);
                if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
                slice_reduce(a, 1, j + 1);
                if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
                for (int p = tid; p < (j + 1) * B; p += bd) {
                    const double2 hv = __ldcg(reinterpret_cast<const double2 *>(
                        a.hred + (int64_t)(kArMaxSteps + 2) * kArMaxB + p));
                    const cx<double> h2{hv.x, hv.y};
                    s_hcol[p] = s_hcol[p] + h2;
                    s_hf[p] = ff_split(h2);
                }
                __syncthreads();
            }
            // w -= sum_{i <= j} v_i h_i on the own elements
            for (int idx = tid; idx < nel; idx += bd) {
                const int b = idx % B;
                const float4 w0 = W[e0 + idx];
                float rh = w0.x, rl = w0.z, ih = w0.y, il = w0.w;
                for (int i0 = 0; i0 <= j; i0 += 8) {  // 8 basis loads in flight
                    float4 vv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        vv[u] = i0 + u <= j ? a.Vf[(int64_t)(i0 + u) * a.L + e0 + idx] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (i0 + u > j) break;
                        const float4 hv = s_hf[(i0 + u) * B + b];
                        ff_mac(rh, rl, -vv[u].x, -vv[u].z, hv.x, hv.z);
                        ff_mac(rh, rl, vv[u].y, vv[u].w, hv.y, hv.w);
                        ff_mac(ih, il, -vv[u].x, -vv[u].z, hv.y, hv.w);
                        ff_mac(ih, il, -vv[u].y, -vv[u].w, hv.x, hv.z);
                    }
                }
                ff_norm(rh, rl);
                ff_norm(ih, il);
                W[e0 + idx] = make_float4(rh, ih, rl, il);
            }
            __syncthreads();
        }
        if (status) break;
        // ---- 3. |w| (float-float within a warp, FP64 across warps and CTAs; fixed order)
        {
            // |w|^2 of the own elements in float-float (FP32 pipe), one conversion per warp;
            // a thread's elements all have column tid % B when B | bd
            float ah = 0.f, al = 0.f;
            for (int idx = tid; idx < nel; idx += bd) {
                const float4 x = W[e0 + idx];
                ff_mac(ah, al, x.x, x.z, x.x, x.z);
                ff_mac(ah, al, x.y, x.w, x.y, x.w);
            }
            ff_norm(ah, al);
            for (int o = 16; o >= B; o >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, ah, o), ol = __shfl_down_sync(0xffffffffu, al, o);
                ff_add(ah, al, oh, ol);
            }
            if (lane < B) s_red[warp * kArMaxB + lane] = (double)ah + (double)al;
            __syncthreads();
            if (warp < B) {  // warp b adds column b over the CTA's warps (a tree, not a chain)
                double sacc = lane < (bd >> 5) ? s_red[lane * kArMaxB + warp] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
                if (lane == 0) mypart[4 * (kArMaxSteps + 2) * kArMaxB + warp] = sacc;
            }
        }
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
        if (warp < B) {  // warp b adds column b's partials of all CTAs: lane-strided, fixed tree
            double sacc = 0.0;
            for (int gi = lane; gi < G; gi += 32)
                sacc += __ldcg(a.part + (int64_t)gi * kPartStride + 4 * (kArMaxSteps + 2) * kArMaxB + warp);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
            if (lane == 0) {
                const double n = std::sqrt(sacc);
                s_nrm[warp] = n > 0.0 ? 1.0 / n : 0.0;  // the inverse, used by every element
                s_hcol[(j + 1) * B + warp] = cx<double>{n, 0.0};
            }
        }
        __syncthreads();
        // v_{j+1} = w / |w| in float-float for the next steps; the FP64 copy only of the
        // tier-0 rows (elements below d2 * B), which the final combination x_0 = V_0 y reads,
        // so that the basis held in L2 is the float-float one alone
        for (int idx = tid; idx < nel; idx += bd) {
            const cx<double> x = s_nrm[idx % B] * ff_join(W[e0 + idx]);  // zero norm: zeros
            if (e0 + idx < (int64_t)d2 * B) a.V[(int64_t)(j + 1) * a.L + e0 + idx] = x;
            W[e0 + idx] = ff_split(x);
        }
        // Hessenberg column j to global memory (CTA 0); its rows 0 .. j split into float-float
        // for the rotation chains (s_hf is free again: the Gram-Schmidt update has used it)
        if (blockIdx.x == 0)
            for (int p = tid; p < (j + 2) * B; p += bd) {
                const int i = p / B, b = p - i * B;
                a.Hb[((int64_t)j * (a.mmax + 1) + i) * a.B + b] = s_hcol[p];
            }
        for (int p = tid; p < (j + 1) * B; p += bd) s_hf[p] = ff_split(s_hcol[p]);
        __syncthreads();
        // ---- 4. Givens QR of every shift, one thread per shift, shifts dealt round-robin over
        // the CTAs. The chain that brings column j up to date with the earlier rotations runs
        // in float-float (FP32 pipe; the FP64 instructions of GB300 are few and slow to
        // complete); the new rotation itself and g stay FP64.
        float rmax = 0.f;  // largest (|g_{j+1}| / beta)^2 of the CTA's shifts (a threshold test)
        for (int64_t k = (int64_t)tid * G + blockIdx.x; k < a.S; k += (int64_t)G * bd) {
            const int b = a.col_of[k];
            const cx<double> shk = a.shift[k];
            double *rc = a.rot_c + k * a.mmax;
            cx<double> *rs = a.rot_s + k * a.mmax;
            float2 *rcf = a.rot_cf + k * a.mmax;
            float4 *rsf = a.rot_sf + k * a.mmax;
            cx<double> *gk = a.g + k * (a.mmax + 1);
            const float4 shf = ff_split(shk);
            float4 h = s_hf[b];
            if (j == 0) {
                ff_add(h.x, h.z, shf.x, shf.z);
                ff_add(h.y, h.w, shf.y, shf.w);
            }
            for (int i0 = 0; i0 < j; i0 += 8) {  // the rotations, 8 loads in flight
                float2 cr[8];
                float4 sr[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u < j ? i0 + u : j - 1;
                    cr[u] = rcf[i];
                    sr[u] = rsf[i];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u;
                    if (i >= j) break;
                    float4 hi1 = s_hf[(i + 1) * B + b];
                    if (i + 1 == j) {
                        ff_add(hi1.x, hi1.z, shf.x, shf.z);
                        ff_add(hi1.y, hi1.w, shf.y, shf.w);
                    }
                    h = ff_rot_step(cr[u], sr[u], hi1, h);
                }
            }
            const cx<double> hj = ff_join(h);
            const cx<double> hsub = s_hcol[(j + 1) * B + b];
            double c;
            cx<double> sn, r;
            givens_rot(hj, hsub, c, sn, r);
            rc[j] = c;
            rs[j] = sn;
            {
                const float ch = __double2float_rn(c);
                rcf[j] = make_float2(ch, __double2float_rn(c - (double)ch));
                rsf[j] = ff_split(sn);
            }
            a.rdiag[k * a.mmax + j] = r;
            const cx<double> gj = gk[j];
            gk[j] = c * gj;
            const cx<double> gn = cx<double>{0.0, 0.0} - conj(sn) * gj;
            gk[j + 1] = gn;
            const double rk2 = norm2(gn) * s_ib2[b];  // (|g_{j+1}| / beta)^2
            a.res[k] = (double)sqrtf((float)rk2);     // reported estimate
            rmax = fmaxf(rmax, isfinite(rk2) ? (float)rk2 : 3.0e38f);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
        float *s_redf = reinterpret_cast<float *>(s_red);
        if (lane == 0) s_redf[warp] = rmax;
        __syncthreads();
        if (warp == 0) {
            float mx = lane < (bd >> 5) ? s_redf[lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
            if (lane == 0) mypart[4 * (kArMaxSteps + 2) * kArMaxB + kArMaxB] = (double)mx;
        }
        steps = j + 1;
        if (!grid_barrier(a.bar, gen, a.wait_cycles)) { status = 1; break; }
        if (warp == 0) {  // largest residual estimate over all CTAs
            float mx = 0.f;
            for (int gi = lane; gi < G; gi += 32)
                mx = fmaxf(mx, (float)__ldcg(a.part + (int64_t)gi * kPartStride + 4 * (kArMaxSteps + 2) * kArMaxB + kArMaxB));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
            if (lane == 0) s_flag[1] = mx <= (float)(a.tol * a.tol);
        }
        __syncthreads();
        if (s_flag[1]) { converged = 1; break; }
    }
    // the last basis vector in FP64 as a whole: the step-by-step continuation starts from it
    if (!status)
        for (int idx = tid; idx < nel; idx += bd)
            a.V[(int64_t)steps * a.L + e0 + idx] = ff_join(a.Vf[(int64_t)steps * a.L + e0 + idx]);
    if (blockIdx.x == 0 && tid == 0) {
        a.out[0] = steps;
        a.out[1] = converged;
        a.out[2] = status;
    }
}

size_t arnoldi_smem(const DevView<double> &v, int hcap) {
    return (size_t)hcap * (sizeof(cx<double>) + sizeof(float4)) +
           32 * kArMaxB * sizeof(double) + 2 * kArMaxB * sizeof(double) + (2 + kArMaxB) * sizeof(int) +
           prog_smem_bytes<double>(v.pers_terms, v.pers_slots, v.pers_ados, v.d2) + 64;
}

// The FP64 view with the Arnoldi's own ADO ranges in place of the persistent solver's.
DevView<double> arnoldi_view(const heom_hier *h) {
    DevView<double> v = h->view64();
    v.pers_ado = (const int32_t *)h->d_ar_ado.p;
    v.pers_ranges = h->ar_ranges;
    v.pers_terms = h->ar_terms;
    v.pers_slots = h->ar_slots;
    v.pers_ados = h->ar_ados;
    return v;
}

}  // namespace

bool arnoldi_persistent_ok(const heom_hier *h, int64_t B, int max_steps) {
    // the resident term programs carry one parameter set's coefficients
    if (h->n_sets != 1 || h->has_caps) return false;
    if (h->ar_ranges < 1 || B < 1 || B > kArMaxB || (32 % B) != 0 || (kArThreads % B) != 0) return false;
    const int steps = std::min(max_steps, kArMaxSteps);
    return arnoldi_smem(arnoldi_view(h), (steps + 2) * (int)B) <= 200 * 1024;
}

int arnoldi_max_steps() { return kArMaxSteps; }

// Runs Arnoldi steps j = 0 .. max_steps-1 (max_steps <= kArMaxSteps) of the shift-invariant
// solve in one cooperative launch. V_0 (FP64 and split), g (beta in row 0) and the zeroed
// Hessenberg matrix must be in place. Returns the steps done and whether every shift's
// residual estimate reached tol.
heom_status arnoldi_persistent(heom_hier *h, int64_t B, int mmax, int max_steps, float4 *Vf, cx<double> *V,
                               cx<double> *Hb, int64_t S, const cx<double> *shift, const int *col_of,
                               double *rot_c, cx<double> *rot_s, cx<double> *rdiag, cx<double> *g,
                               float2 *rot_cf, float4 *rot_sf, const double *beta, double *res,
                               double tol, int *steps, bool *converged, cudaStream_t s) {
    const int G = h->ar_ranges;
    const size_t part_bytes = (size_t)G * kPartStride * sizeof(double);
    const size_t hred_bytes = (size_t)2 * (kArMaxSteps + 2) * kArMaxB * sizeof(cx<double>);
    heom_status st = ensure_ws(h->ws_pers, part_bytes + hred_bytes + 512);
    if (st != HEOM_OK) return st;
    char *base = (char *)h->ws_pers.p;
    ArnoldiArgs a{};
    a.v = arnoldi_view(h);
    a.B = B;
    a.L = h->N * h->d2 * B;
    a.S = S;
    a.mmax = mmax;
    a.max_steps = std::min(max_steps, std::min(mmax, kArMaxSteps));
    a.hcap = (a.max_steps + 2) * (int)B;
    a.Vf = Vf;
    a.V = V;
    a.Hb = Hb;
    a.shift = shift;
    a.col_of = col_of;
    a.rot_c = rot_c;
    a.rot_s = rot_s;
    a.rdiag = rdiag;
    a.g = g;
    a.rot_cf = rot_cf;
    a.rot_sf = rot_sf;
    a.beta = beta;
    a.res = res;
    a.tol = tol;
    a.part = (double *)base;
    a.hred = (cx<double> *)(base + part_bytes);
    a.bar = (GridBar *)(base + part_bytes + hred_bytes);
    a.out = (int *)(base + part_bytes + hred_bytes + 256);
    a.wait_cycles = wait_limit_cycles();
    HEOM_CUDA(cudaMemsetAsync(a.bar, 0, 512, s));
    const size_t sm = arnoldi_smem(a.v, a.hcap);
    HEOM_CUDA(cudaFuncSetAttribute(k_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    void *args[] = {&a};
    {
        Prof pr(HEOM_KC_KRYLOV_APPLY64, s, 0.0, 0.0);
        HEOM_CUDA(cudaLaunchCooperativeKernel((const void *)k_arnoldi, dim3(G), dim3(kArThreads), args, sm, s));
    }
    int out[3] = {0, 0, 0};
    HEOM_CUDA(memcpy_counted(out, a.out, sizeof(out), cudaMemcpyDeviceToHost, s));
    HEOM_CUDA(cudaStreamSynchronize(s));
    *steps = out[0];
    if (out[2]) {  // every CTA has left the launch; the device stays usable
        *converged = false;
        set_error("persistent Arnoldi: a grid-barrier wait ran out after %lld cycles",
                  (long long)a.wait_cycles);
        return HEOM_ETIMEOUT;
    }
    *converged = out[1] != 0;
    // launch accounting: one apply of B columns per step
    prof_add(HEOM_KC_KRYLOV_APPLY64, (double)out[0] * h->N * B, (double)out[0] * 2.0 * a.L * 16.0);
    return HEOM_OK;
}

}  // namespace heom
