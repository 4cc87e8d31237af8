// Learned warm start for stationary states (no counterpart in the paper): a multilayer
// perceptron maps the physical parameters of a model to its reduced density matrix and its
// first-tier ADOs, which seed the stationary-state Krylov solve. Everything here -- forward
// pass, loss, back-propagation, Adam -- runs in this file's kernels.
//
// Numerics: parameters and activations live in FP32; every matrix product rounds its two
// operands to BF16 (round to nearest even) and accumulates in FP32 on the tensor cores
// (mma.sync m16n8k16, BF16 in, FP32 out). Hidden layers use tanh; the output layer is linear.
// Inputs and targets are standardised with host-supplied means and deviations. Loss: mean
// squared error over the batch and the outputs of the standardised targets.
//
// The networks are small (widths of a few hundred, batches of a few thousand): one product
// is a few hundred MFLOP at most, microseconds on this GPU next to the milliseconds of a
// stationary solve, so the products use the synchronous warp-level MMA with plain shared-
// memory staging rather than an asynchronous TMA / tcgen05 pipeline.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "heom_internal.h"

struct heom_mlp {
    int device = 0;
    int n_layers = 0;
    std::vector<int> width;            // n_layers + 1
    std::vector<int64_t> w_off, b_off;  // offsets of W_l ([in][out] row-major) and b_l
    int64_t n_params = 0;
    int64_t adam_t = 0;
    heom::DBuf params, grads, adam_m, adam_v;  // FP32, flat
    heom::DBuf norm;                           // in_mean, in_std, out_mean, out_std
    heom::DBuf ws;                             // activations and gradients
};

namespace heom {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kPad = 8;

enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_TANH = 2, EPI_DTANH = 3 };

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

// C[M][N] (row-major, ldc) = op(A) op(B) with an epilogue. op(A) is M x K: element (m, k) at
// A[m lda + k], or at A[k lda + m] when transA; op(B) is K x N: element (k, n) at B[k ldb + n],
// or at B[n ldb + k] when transB. Operands are rounded to BF16 when staged into shared memory.
// Epilogues: STORE C = acc; BIAS C = acc + bias[n]; TANH C = tanh(acc + bias[n]);
// DTANH C = acc (1 - aux[m ldc + n]^2) (back-propagation through a tanh layer whose output
// is aux). Block: 128 threads = 2 x 2 warps, 64 x 64 tile, each warp 32 x 32 as 2 x 4 MMA
// tiles of 16 x 8.
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              int transA, const float *__restrict__ B, int ldb, int transB,
                                              float *__restrict__ C, int ldc, const float *__restrict__ bias,
                                              const float *__restrict__ aux) {
    __shared__ __align__(16) __nv_bfloat16 As[kBM][kBK + kPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN][kBK + kPad];  // n-major: Bs[n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kBK) {
        for (int idx = tid; idx < kBM * kBK; idx += 128) {
            int r, c;
            if (transA) { c = idx / kBM; r = idx - c * kBM; }  // consecutive threads: consecutive m
            else { r = idx / kBK; c = idx - r * kBK; }         // consecutive threads: consecutive k
            const int m = m0 + r, k = k0 + c;
            float val = 0.f;
            if (m < M && k < K) val = transA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            As[r][c] = __float2bfloat16_rn(val);
        }
        for (int idx = tid; idx < kBN * kBK; idx += 128) {
            int n, c;
            if (transB) { n = idx / kBK; c = idx - n * kBK; }  // consecutive k
            else { c = idx / kBN; n = idx - c * kBN; }         // consecutive n
            const int nn = n0 + n, k = k0 + c;
            float val = 0.f;
            if (nn < N && k < K) val = transB ? B[(int64_t)nn * ldb + k] : B[(int64_t)k * ldb + nn];
            Bs[n][c] = __float2bfloat16_rn(val);
        }
        __syncthreads();
        uint32_t af[2][4], bf[4][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int rb = wm * 32 + mt * 16;
            af[mt][0] = ld_pair(&As[rb + gq][2 * tq]);
            af[mt][1] = ld_pair(&As[rb + gq + 8][2 * tq]);
            af[mt][2] = ld_pair(&As[rb + gq][2 * tq + 8]);
            af[mt][3] = ld_pair(&As[rb + gq + 8][2 * tq + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int cb = wn * 32 + nt * 8;
            bf[nt][0] = ld_pair(&Bs[cb + gq][2 * tq]);
            bf[nt][1] = ld_pair(&Bs[cb + gq][2 * tq + 8]);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                float *d = acc[mt][nt];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                    "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                    : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]),
                      "r"(bf[nt][0]), "r"(bf[nt][1]));
            }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm * 32 + mt * 16 + gq + (q >> 1) * 8;
                const int n = n0 + wn * 32 + nt * 8 + 2 * tq + (q & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mt][nt][q];
                if constexpr (EPI == EPI_BIAS) v += bias[n];
                if constexpr (EPI == EPI_TANH) v = tanhf(v + bias[n]);
                if constexpr (EPI == EPI_DTANH) {
                    const float a = aux[(int64_t)m * ldc + n];
                    v *= 1.f - a * a;
                }
                C[(int64_t)m * ldc + n] = v;
            }
}

// out[m][i] = (x[m][i] - mean[i]) / sd[i]
__global__ void k_standardise(int64_t M, int n, const float *__restrict__ x, const float *__restrict__ mean,
                              const float *__restrict__ sd, float *__restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < M * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n);
        out[t] = (x[t] - mean[i]) / sd[i];
    }
}

// out[m][i] = y[m][i] sd[i] + mean[i]
__global__ void k_destandardise(int64_t M, int n, const float *__restrict__ y, const float *__restrict__ mean,
                                const float *__restrict__ sd, float *__restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < M * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n);
        out[t] = y[t] * sd[i] + mean[i];
    }
}

// g = 2 (y - t) / (M n); per-block partial sums of (y - t)^2 into part[block]
__global__ void __launch_bounds__(256) k_mse_grad(int64_t total, const float *__restrict__ y,
                                                  const float *__restrict__ t, float *__restrict__ g,
                                                  double *__restrict__ part) {
    __shared__ double sh[256];
    double acc = 0.0;
    const float scale = 2.f / (float)total;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float dlt = y[i] - t[i];
        g[i] = scale * dlt;
        acc += (double)dlt * dlt;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[0] = sum of part[0 .. n) / total (one block, fixed order)
__global__ void k_loss_finish(int n, const double *__restrict__ part, double total, double *__restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] / total;
}

// db[n] = sum_m g[m][n] (one thread per output column, fixed order)
__global__ void k_colsum(int M, int N, const float *__restrict__ g, float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) acc += g[(int64_t)m * N + n];
    db[n] = acc;
}

// Adam (Kingma & Ba), bias-corrected: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Warm-start features of a stationary state (set b of x [N][d2][B], complex128):
// f[b][0 .. d^2): rho_sys as d diagonal reals then, for i < j in row-major order, Re and Im
// of rho[i][j]; then for every tier-1 ADO q (ados[q]) its d^2 elements, Re and Im interleaved.
// to_x = 0: features from x; to_x = 1: x from features (Hermitian rho_sys, tier-1 ADOs; the
// rest of x is left as it is).
__global__ void k_features(int64_t B, int d, int n1, const int *__restrict__ ados, int nf,
                           cx<double> *__restrict__ x, float *__restrict__ f, int to_x) {
    const int d2 = d * d;
    const int per = d2 + n1 * d2;  // work items per set: rho elements + tier-1 elements
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < B * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / per;
        const int w = (int)(t - b * per);
        float *fb = f + b * nf;
        if (w < d2) {  // rho_sys element (r, c)
            const int r = w / d, c = w - r * d;
            cx<double> &xe = x[(int64_t)(r * d + c) * B + b];
            if (r == c) {
                if (to_x) xe = cx<double>{(double)fb[r], 0.0};
                else fb[r] = (float)xe.re;
            } else {
                const int i = r < c ? r : c, j = r < c ? c : r;
                const int pair = i * d - i * (i + 1) / 2 + (j - i - 1);  // rank of (i, j), i < j
                const int o = d + 2 * pair;
                if (to_x) {
                    const double re = fb[o], im = fb[o + 1];
                    xe = r < c ? cx<double>{re, im} : cx<double>{re, -im};
                } else if (r < c) {
                    fb[o] = (float)xe.re;
                    fb[o + 1] = (float)xe.im;
                }
            }
        } else {
            const int q = (w - d2) / d2, e = (w - d2) - q * d2;
            cx<double> &xe = x[((int64_t)ados[q] * d2 + e) * B + b];
            const int o = d2 + 2 * (q * d2 + e);
            if (to_x) xe = cx<double>{(double)fb[o], (double)fb[o + 1]};
            else {
                fb[o] = (float)xe.re;
                fb[o + 1] = (float)xe.im;
            }
        }
    }
}

int nblk(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 8); }

template <int EPI>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, int tA, const float *B, int ldb, int tB,
                 float *C, int ldc, const float *bias, const float *aux, cudaStream_t s) {
    dim3 grid((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM));
    k_gemm<EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, bias, aux);
    return cudaGetLastError();
}

// splitmix64 (Steele, Lea, Flood 2014): the parameter initialisation stream
uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

struct Work {
    std::vector<float *> act;  // act[0] standardised input, act[l] layer outputs, act[L] = y
    float *tn, *g0, *g1;       // standardised targets, two gradient buffers
    double *part, *loss;
    int nblocks;
};

heom_status work_for(heom_mlp *net, int64_t M, Work &w) {
    const int L = net->n_layers;
    int maxw = 0;
    for (int x : net->width) maxw = std::max(maxw, x);
    const int nb = nblk(M * net->width[L]);
    size_t off = 0;
    std::vector<size_t> aoff(L + 1);
    for (int l = 0; l <= L; ++l) { aoff[l] = off; off += (size_t)M * net->width[l] * 4; off = (off + 255) & ~size_t(255); }
    const size_t otn = off; off += (size_t)M * net->width[L] * 4; off = (off + 255) & ~size_t(255);
    const size_t og0 = off; off += (size_t)M * maxw * 4; off = (off + 255) & ~size_t(255);
    const size_t og1 = off; off += (size_t)M * maxw * 4; off = (off + 255) & ~size_t(255);
    const size_t opart = off; off += (size_t)nb * 8 + 8; off = (off + 255) & ~size_t(255);
    heom_status st = ensure_ws(net->ws, off);
    if (st != HEOM_OK) return st;
    char *base = (char *)net->ws.p;
    w.act.resize(L + 1);
    for (int l = 0; l <= L; ++l) w.act[l] = (float *)(base + aoff[l]);
    w.tn = (float *)(base + otn);
    w.g0 = (float *)(base + og0);
    w.g1 = (float *)(base + og1);
    w.part = (double *)(base + opart);
    w.loss = w.part + nb;
    w.nblocks = nb;
    return HEOM_OK;
}

const float *norm_ptr(const heom_mlp *net, int which) {  // 0 in_mean 1 in_sd 2 out_mean 3 out_sd
    const int in = net->width[0], out = net->width[net->n_layers];
    const float *p = (const float *)net->norm.p;
    switch (which) {
        case 0: return p;
        case 1: return p + in;
        case 2: return p + 2 * in;
        default: return p + 2 * in + out;
    }
}

// forward pass on raw inputs x [M][in]; leaves the standardised output in w.act[L]
heom_status forward(heom_mlp *net, const float *x, int64_t M, Work &w, cudaStream_t s) {
    const int L = net->n_layers, in = net->width[0];
    k_standardise<<<nblk(M * in), 256, 0, s>>>(M, in, x, norm_ptr(net, 0), norm_ptr(net, 1), w.act[0]);
    HEOM_CUDA(cudaGetLastError());
    const float *P = (const float *)net->params.p;
    for (int l = 0; l < L; ++l) {
        const int K = net->width[l], N = net->width[l + 1];
        const float *W = P + net->w_off[l], *b = P + net->b_off[l];
        if (l + 1 < L) HEOM_CUDA(gemm<EPI_TANH>((int)M, N, K, w.act[l], K, 0, W, N, 0, w.act[l + 1], N, b, nullptr, s));
        else HEOM_CUDA(gemm<EPI_BIAS>((int)M, N, K, w.act[l], K, 0, W, N, 0, w.act[l + 1], N, b, nullptr, s));
    }
    return HEOM_OK;
}

// loss and gradients (into net->grads) for raw inputs x and raw targets t
heom_status backward(heom_mlp *net, const float *x, const float *t, int64_t M, Work &w, cudaStream_t s) {
    const int L = net->n_layers, out = net->width[L];
    heom_status st = forward(net, x, M, w, s);
    if (st != HEOM_OK) return st;
    k_standardise<<<nblk(M * out), 256, 0, s>>>(M, out, t, norm_ptr(net, 2), norm_ptr(net, 3), w.tn);
    k_mse_grad<<<w.nblocks, 256, 0, s>>>(M * out, w.act[L], w.tn, w.g0, w.part);
    k_loss_finish<<<1, 256, 0, s>>>(w.nblocks, w.part, (double)M * out, w.loss);
    HEOM_CUDA(cudaGetLastError());
    const float *P = (const float *)net->params.p;
    float *G = (float *)net->grads.p;
    float *g = w.g0, *gp = w.g1;
    for (int l = L - 1; l >= 0; --l) {
        const int K = net->width[l], N = net->width[l + 1];
        // dW_l = act_l^T g (K x N), db_l = column sums of g
        HEOM_CUDA(gemm<EPI_STORE>(K, N, (int)M, w.act[l], K, 1, g, N, 0, G + net->w_off[l], N, nullptr, nullptr, s));
        k_colsum<<<(N + 127) / 128, 128, 0, s>>>((int)M, N, g, G + net->b_off[l]);
        HEOM_CUDA(cudaGetLastError());
        if (l > 0) {  // g_{l-1} = (g W_l^T) * (1 - act_l^2)
            HEOM_CUDA(gemm<EPI_DTANH>((int)M, K, N, g, N, 0, P + net->w_off[l], N, 1, gp, K, nullptr, w.act[l], s));
            std::swap(g, gp);
        }
    }
    return HEOM_OK;
}

}  // namespace
}  // namespace heom

using heom::set_error;

extern "C" heom_status heom_mlp_create(int n_layers, const int *widths, uint64_t seed, heom_mlp **out) {
    if (!out || n_layers < 1 || n_layers > 16 || !widths) {
        set_error("heom_mlp_create: need 1..16 layers, widths[n_layers + 1] and out");
        return HEOM_EINVAL;
    }
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 1 || widths[l] > 65536) {
            set_error("heom_mlp_create: widths must be in 1..65536");
            return HEOM_EINVAL;
        }
    heom_mlp *net = new heom_mlp();
    cudaGetDevice(&net->device);
    net->n_layers = n_layers;
    net->width.assign(widths, widths + n_layers + 1);
    int64_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
        net->w_off.push_back(off);
        off += (int64_t)widths[l] * widths[l + 1];
        net->b_off.push_back(off);
        off += widths[l + 1];
    }
    net->n_params = off;
    // Glorot-uniform weights, zero biases; identity standardisation
    std::vector<float> p(off, 0.f);
    uint64_t state = seed;
    for (int l = 0; l < n_layers; ++l) {
        const double a = std::sqrt(6.0 / (widths[l] + widths[l + 1]));
        for (int64_t i = 0; i < (int64_t)widths[l] * widths[l + 1]; ++i) {
            const double u = (double)(heom::splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
            p[net->w_off[l] + i] = (float)(a * (2.0 * u - 1.0));
        }
    }
    const int in = widths[0], o = widths[n_layers];
    std::vector<float> nm(2 * in + 2 * o, 0.f);
    for (int i = 0; i < in; ++i) nm[in + i] = 1.f;
    for (int i = 0; i < o; ++i) nm[2 * in + o + i] = 1.f;
    heom_status st;
    if ((st = heom::dalloc(net->params, off * 4)) != HEOM_OK || (st = heom::dalloc(net->grads, off * 4)) != HEOM_OK ||
        (st = heom::dalloc(net->adam_m, off * 4)) != HEOM_OK || (st = heom::dalloc(net->adam_v, off * 4)) != HEOM_OK ||
        (st = heom::dalloc(net->norm, nm.size() * 4)) != HEOM_OK) {
        heom_mlp_destroy(net);
        return st;
    }
    if (cudaMemcpy(net->params.p, p.data(), off * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->adam_m.p, 0, off * 4) != cudaSuccess || cudaMemset(net->adam_v.p, 0, off * 4) != cudaSuccess ||
        cudaMemset(net->grads.p, 0, off * 4) != cudaSuccess ||
        cudaMemcpy(net->norm.p, nm.data(), nm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        heom_mlp_destroy(net);
        set_error("heom_mlp_create: upload failed");
        return HEOM_ECUDA;
    }
    *out = net;
    return HEOM_OK;
}

extern "C" void heom_mlp_destroy(heom_mlp *net) {
    if (!net) return;
    heom::dfree(net->params);
    heom::dfree(net->grads);
    heom::dfree(net->adam_m);
    heom::dfree(net->adam_v);
    heom::dfree(net->norm);
    heom::dfree(net->ws);
    delete net;
}

extern "C" heom_status heom_mlp_info(const heom_mlp *net, int64_t *n_params, int *n_in, int *n_out) {
    if (!net) { set_error("heom_mlp_info: null network"); return HEOM_EINVAL; }
    if (n_params) *n_params = net->n_params;
    if (n_in) *n_in = net->width[0];
    if (n_out) *n_out = net->width[net->n_layers];
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_set_standardisation(heom_mlp *net, const float *in_mean, const float *in_sd,
                                                     const float *out_mean, const float *out_sd) {
    if (!net || !in_mean || !in_sd || !out_mean || !out_sd) {
        set_error("heom_mlp_set_standardisation: null argument");
        return HEOM_EINVAL;
    }
    const int in = net->width[0], o = net->width[net->n_layers];
    std::vector<float> nm(2 * in + 2 * o);
    for (int i = 0; i < in; ++i) {
        if (!(in_sd[i] > 0.f)) { set_error("heom_mlp_set_standardisation: deviations must be > 0"); return HEOM_EINVAL; }
        nm[i] = in_mean[i];
        nm[in + i] = in_sd[i];
    }
    for (int i = 0; i < o; ++i) {
        if (!(out_sd[i] > 0.f)) { set_error("heom_mlp_set_standardisation: deviations must be > 0"); return HEOM_EINVAL; }
        nm[2 * in + i] = out_mean[i];
        nm[2 * in + o + i] = out_sd[i];
    }
    HEOM_DEVICE(net->device);
    HEOM_CUDA(cudaMemcpy(net->norm.p, nm.data(), nm.size() * 4, cudaMemcpyHostToDevice));
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_get_params(const heom_mlp *net, float *host_out) {
    if (!net || !host_out) { set_error("heom_mlp_get_params: null argument"); return HEOM_EINVAL; }
    HEOM_DEVICE(net->device);
    HEOM_CUDA(cudaMemcpy(host_out, net->params.p, net->n_params * 4, cudaMemcpyDeviceToHost));
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_set_params(heom_mlp *net, const float *host_in) {
    if (!net || !host_in) { set_error("heom_mlp_set_params: null argument"); return HEOM_EINVAL; }
    HEOM_DEVICE(net->device);
    HEOM_CUDA(cudaMemcpy(net->params.p, host_in, net->n_params * 4, cudaMemcpyHostToDevice));
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_forward(heom_mlp *net, const float *x, float *y, int64_t batch, heom_stream s) {
    if (!net || !x || !y || batch < 1 || batch > (1 << 24)) {
        set_error("heom_mlp_forward: need a network, x, y and 1 <= batch <= 2^24");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(net->device);
    cudaStream_t st = (cudaStream_t)s;
    heom::Work w;
    heom_status r = heom::work_for(net, batch, w);
    if (r != HEOM_OK) return r;
    {
        heom::Prof pr(HEOM_KC_OTHER, st, (double)batch);
        pr.kernels = net->n_layers + 2;
        if ((r = heom::forward(net, x, batch, w, st)) != HEOM_OK) return r;
        const int o = net->width[net->n_layers];
        heom::k_destandardise<<<heom::nblk(batch * o), 256, 0, st>>>(batch, o, w.act[net->n_layers],
                                                                     heom::norm_ptr(net, 2), heom::norm_ptr(net, 3), y);
    }
    HEOM_CUDA(cudaGetLastError());
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_gradients(heom_mlp *net, const float *x, const float *t, int64_t batch,
                                          float *grad_out, double *loss, heom_stream s) {
    if (!net || !x || !t || batch < 1 || batch > (1 << 24)) {
        set_error("heom_mlp_gradients: need a network, x, t and 1 <= batch <= 2^24");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(net->device);
    cudaStream_t st = (cudaStream_t)s;
    heom::Work w;
    heom_status r = heom::work_for(net, batch, w);
    if (r != HEOM_OK) return r;
    {
        heom::Prof pr(HEOM_KC_OTHER, st, (double)batch);
        pr.kernels = 4 + 4 * net->n_layers;
        if ((r = heom::backward(net, x, t, batch, w, st)) != HEOM_OK) return r;
    }
    if (grad_out) HEOM_CUDA(cudaMemcpyAsync(grad_out, net->grads.p, net->n_params * 4, cudaMemcpyDeviceToDevice, st));
    if (loss) {
        HEOM_CUDA(heom::memcpy_counted(loss, w.loss, 8, cudaMemcpyDeviceToHost, st));
        HEOM_CUDA(cudaStreamSynchronize(st));
    }
    return HEOM_OK;
}

extern "C" heom_status heom_mlp_train_step(heom_mlp *net, const float *x, const float *t, int64_t batch,
                                           float lr, double *loss, heom_stream s) {
    if (!(lr > 0.f)) { set_error("heom_mlp_train_step: lr must be > 0"); return HEOM_EINVAL; }
    heom_status r = heom_mlp_gradients(net, x, t, batch, nullptr, nullptr, s);
    if (r != HEOM_OK) return r;
    cudaStream_t st = (cudaStream_t)s;
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->adam_t), c2 = 1.f - std::pow(b2, (float)net->adam_t);
    {
        heom::Prof pr(HEOM_KC_OTHER, st, (double)net->n_params);
        heom::k_adam<<<heom::nblk(net->n_params), 256, 0, st>>>(net->n_params, (float *)net->params.p,
                                                                (const float *)net->grads.p, (float *)net->adam_m.p,
                                                                (float *)net->adam_v.p, lr, b1, b2, 1e-8f, c1, c2);
    }
    HEOM_CUDA(cudaGetLastError());
    if (loss) {
        heom::Work w;
        if ((r = heom::work_for(net, batch, w)) != HEOM_OK) return r;
        HEOM_CUDA(heom::memcpy_counted(loss, w.loss, 8, cudaMemcpyDeviceToHost, st));
        HEOM_CUDA(cudaStreamSynchronize(st));
    }
    return HEOM_OK;
}

// tier-1 ADO indices of a hierarchy, in the hierarchy's order
static std::vector<int> tier1_ados(const heom_hier *h) {
    std::vector<int> out;
    for (int64_t n = 0; n < h->N; ++n) {
        const int64_t full = h->full_of(n), bi = full / h->N_f, fi = full % h->N_f;
        int tier = __builtin_popcountll(h->fer[fi]);
        for (int m : h->bos[bi]) tier += m;
        if (tier == 1) out.push_back((int)n);
    }
    return out;
}

static heom_status feature_call(const heom_hier *h, void *x, float *f, int64_t n_sets, int nf, int to_x,
                                cudaStream_t st, const char *who) {
    const std::vector<int> t1 = tier1_ados(h);
    const int need = h->d2 + 2 * (int)t1.size() * h->d2;
    if (nf != need) {
        set_error("%s: %d features expected (d^2 + 2 d^2 x %d tier-1 ADOs), got %d", who, need, (int)t1.size(), nf);
        return HEOM_EINVAL;
    }
    heom::DBuf idx;
    heom_status r = heom::dalloc(idx, std::max<size_t>(t1.size(), 1) * 4);
    if (r != HEOM_OK) return r;
    if (!t1.empty()) HEOM_CUDA(heom::memcpy_counted(idx.p, t1.data(), t1.size() * 4, cudaMemcpyHostToDevice, st));
    {
        heom::Prof pr(HEOM_KC_OTHER, st, (double)n_sets * need);
        heom::k_features<<<heom::nblk(n_sets * (h->d2 + (int64_t)t1.size() * h->d2)), 256, 0, st>>>(
            n_sets, h->d, (int)t1.size(), (const int *)idx.p, nf, (heom::cx<double> *)x, f, to_x);
    }
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    heom::dfree(idx);
    if (e != cudaSuccess) return heom::cuda_fail(e, who);
    return HEOM_OK;
}

extern "C" heom_status heom_warm_start_features(const heom_hier *h, const void *x, int64_t n_sets, float *f,
                                                int n_features, heom_stream s) {
    if (!h || !x || !f || n_sets < 1) {
        set_error("heom_warm_start_features: need a hierarchy, x, f and n_sets >= 1");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    return feature_call(h, const_cast<void *>(x), f, n_sets, n_features, 0, (cudaStream_t)s,
                        "heom_warm_start_features");
}

extern "C" heom_status heom_warm_start(const heom_hier *h, heom_mlp *net, const float *params, int64_t n_sets,
                                       void *x_out, heom_stream s) {
    if (!h || !net || !params || !x_out || n_sets < 1) {
        set_error("heom_warm_start: need a hierarchy, a network, params, x_out and n_sets >= 1");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    cudaStream_t st = (cudaStream_t)s;
    const int nf = net->width[net->n_layers];
    heom::DBuf y;
    heom_status r = heom::dalloc(y, (size_t)n_sets * nf * 4);
    if (r != HEOM_OK) return r;
    if ((r = heom_mlp_forward(net, params, (float *)y.p, n_sets, s)) != HEOM_OK) { heom::dfree(y); return r; }
    const size_t bytes = (size_t)h->N * h->d2 * n_sets * sizeof(heom::cx<double>);
    if (cudaMemsetAsync(x_out, 0, bytes, st) != cudaSuccess) { heom::dfree(y); set_error("heom_warm_start: memset"); return HEOM_ECUDA; }
    r = feature_call(h, x_out, (float *)y.p, n_sets, nf, 1, st, "heom_warm_start");
    heom::dfree(y);
    return r;
}

// ------------------------------------------------------------------ selected elements
namespace heom {
namespace {
// f[s][2k], f[s][2k+1] = Re, Im of element elems[k] of column s (to_x = 0), or the reverse
// (to_x = 1: x already zeroed by the caller)
__global__ void k_elements(int64_t n_sets, const int64_t *__restrict__ elems, int64_t n_el,
                           cx<double> *__restrict__ x, float *__restrict__ f, int to_x) {
    const int64_t total = n_sets * n_el;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / n_el, k = i - s * n_el;
        const int64_t e = elems[k] * n_sets + s;
        float *fp = f + s * 2 * n_el + 2 * k;
        if (to_x) {
            x[e] = cx<double>{(double)fp[0], (double)fp[1]};
        } else {
            fp[0] = (float)x[e].re;
            fp[1] = (float)x[e].im;
        }
    }
}

heom_status elements_call(const heom_hier *h, void *x, const int64_t *elems, int64_t n_el, float *f,
                          int64_t n_sets, int to_x, cudaStream_t st, const char *who) {
    std::vector<int64_t> he((size_t)n_el);
    HEOM_CUDA(memcpy_counted(he.data(), elems, (size_t)n_el * 8, cudaMemcpyDeviceToHost, st));
    HEOM_CUDA(cudaStreamSynchronize(st));
    const int64_t total = h->N * h->d2;
    for (int64_t k = 0; k < n_el; ++k)
        if (he[k] < 0 || he[k] >= total) {
            set_error("%s: element index %lld outside [0, N d^2 = %lld)", who, (long long)he[k], (long long)total);
            return HEOM_EINVAL;
        }
    Prof pr(HEOM_KC_OTHER, st, (double)n_sets * n_el);
    k_elements<<<nblk(n_sets * n_el), 256, 0, st>>>(n_sets, elems, n_el, (cx<double> *)x, f, to_x);
    HEOM_CUDA(cudaGetLastError());
    HEOM_CUDA(cudaStreamSynchronize(st));
    return HEOM_OK;
}
}  // namespace
}  // namespace heom

extern "C" heom_status heom_gather_elements(const heom_hier *h, const void *x, int64_t n_sets,
                                            const int64_t *elems, int64_t n_elems, float *f,
                                            heom_stream s) {
    if (!h || !x || !elems || !f || n_sets < 1 || n_elems < 1) {
        set_error("heom_gather_elements: need a hierarchy, x, elems[n_elems >= 1], f and n_sets >= 1");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    return heom::elements_call(h, const_cast<void *>(x), elems, n_elems, f, n_sets, 0, (cudaStream_t)s,
                               "heom_gather_elements");
}

extern "C" heom_status heom_warm_start_elements(const heom_hier *h, heom_mlp *net, const float *params,
                                                int64_t n_sets, const int64_t *elems, int64_t n_elems,
                                                void *x_out, heom_stream s) {
    if (!h || !net || !params || !elems || !x_out || n_sets < 1 || n_elems < 1) {
        set_error("heom_warm_start_elements: need a hierarchy, a network, params, elems[n_elems >= 1], "
                  "x_out and n_sets >= 1");
        return HEOM_EINVAL;
    }
    const int nf = net->width[net->n_layers];
    if ((int64_t)nf != 2 * n_elems) {
        set_error("heom_warm_start_elements: the network has %d outputs, 2 n_elems = %lld needed", nf,
                  (long long)(2 * n_elems));
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    cudaStream_t st = (cudaStream_t)s;
    heom::DBuf y;
    heom_status r = heom::dalloc(y, (size_t)n_sets * nf * 4);
    if (r != HEOM_OK) return r;
    if ((r = heom_mlp_forward(net, params, (float *)y.p, n_sets, s)) != HEOM_OK) { heom::dfree(y); return r; }
    const size_t bytes = (size_t)h->N * h->d2 * n_sets * sizeof(heom::cx<double>);
    if (cudaMemsetAsync(x_out, 0, bytes, st) != cudaSuccess) {
        heom::dfree(y);
        set_error("heom_warm_start_elements: memset");
        return HEOM_ECUDA;
    }
    r = heom::elements_call(h, x_out, elems, n_elems, (float *)y.p, n_sets, 1, st, "heom_warm_start_elements");
    heom::dfree(y);
    return r;
}
