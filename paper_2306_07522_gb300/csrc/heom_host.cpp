// Host side of libheom: exponent helpers, ADO enumeration, neighbour/sign tables, device
// upload, the hierarchy dictionary and error reporting.
//
// Paper passages: Eq. HEOM and its multi-index notation (which ADO couples to which, with
// which sign), the definitions of A, B, C, D and P_s below it; Methods (exponents of the
// Lorentzian and Drude-Lorentz baths). The enumeration here is combinatorial ranking
// (compositions for bosons, the combinatorial number system for fermionic subsets), so a
// neighbour's index is computed, not looked up; with importance pruning (Eq. importance) the
// computed full index goes through one table to the kept ADO's index.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <atomic>
#include <mutex>
#include <new>

#include "heom_internal.h"

using heom::cx;
using heom::DBuf;
using heom::NbEntry;
using heom::OccEntry;

namespace heom {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

heom_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return HEOM_ECUDA;
}

// Process-wide counts for heom_profile_allocs: device allocations made, workspace buffers
// taken (from the cache or newly allocated).
std::atomic<int64_t> g_dev_allocs{0}, g_dev_alloc_bytes{0}, g_ws_takes{0};

// Bound, in SM clock cycles, of every device-side wait (heom_set_wait_limit).
constexpr long long kDefaultWaitCycles = 4000000000LL;
std::atomic<long long> g_wait_cycles{kDefaultWaitCycles};
long long wait_limit_cycles() { return g_wait_cycles.load(); }

heom_status dalloc(DBuf &b, size_t bytes) {
    dfree(b);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HEOM_ENOMEM : HEOM_ECUDA;
    }
    b.bytes = bytes;
    g_dev_allocs.fetch_add(1);
    g_dev_alloc_bytes.fetch_add((int64_t)bytes);
    return HEOM_OK;
}

void dfree(DBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Process-wide cache of solver workspaces, per device. A destroyed hierarchy hands its
// workspace buffers (up to gigabytes: the Krylov bases) to the cache instead of cudaFree,
// which is slow for such buffers and synchronises the whole device; the next workspace
// request on the same device takes the smallest cached buffer that is large enough. At
// most kWsCacheMax buffers are kept (the oldest is freed beyond that);
// heom_release_workspace_cache frees them all, and a failed allocation frees the device's
// cached buffers and tries once more.
namespace {
struct WsEntry {
    int device;
    DBuf buf;
};
std::mutex g_ws_mu;
std::vector<WsEntry> g_ws_cache;
constexpr size_t kWsCacheMax = 8;

void free_on_device(const WsEntry &e) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != e.device) cudaSetDevice(e.device);
    cudaFree(e.buf.p);
    if (cur != e.device) cudaSetDevice(cur);
}

void release_cached(int device) {  // device < 0: every device
    std::vector<WsEntry> out;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        for (size_t i = 0; i < g_ws_cache.size();) {
            if (device < 0 || g_ws_cache[i].device == device) {
                out.push_back(g_ws_cache[i]);
                g_ws_cache.erase(g_ws_cache.begin() + (std::ptrdiff_t)i);
            } else {
                ++i;
            }
        }
    }
    for (const WsEntry &e : out) free_on_device(e);
}
}  // namespace

size_t ws_cached_total(int device) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    size_t m = 0;
    for (const WsEntry &e : g_ws_cache)
        if (e.device == device) m += e.buf.bytes;
    return m;
}

void ws_release(DBuf &b, int device) {
    if (!b.p) return;
    WsEntry evict{-1, DBuf{}};
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        g_ws_cache.push_back(WsEntry{device, b});
        if (g_ws_cache.size() > kWsCacheMax) {
            evict = g_ws_cache.front();
            g_ws_cache.erase(g_ws_cache.begin());
        }
    }
    b = DBuf{};
    if (evict.buf.p) free_on_device(evict);
}

heom_status ensure_ws(DBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return HEOM_OK;
    g_ws_takes.fetch_add(1);
    int dev = 0;
    cudaGetDevice(&dev);
    if (b.p) ws_release(b, dev);
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        size_t best = g_ws_cache.size();
        for (size_t i = 0; i < g_ws_cache.size(); ++i)
            if (g_ws_cache[i].device == dev && g_ws_cache[i].buf.bytes >= bytes &&
                (best == g_ws_cache.size() || g_ws_cache[i].buf.bytes < g_ws_cache[best].buf.bytes))
                best = i;
        if (best < g_ws_cache.size()) {
            b = g_ws_cache[best].buf;
            g_ws_cache.erase(g_ws_cache.begin() + (std::ptrdiff_t)best);
            return HEOM_OK;
        }
    }
    heom_status st = dalloc(b, bytes);
    if (st == HEOM_ENOMEM) {
        release_cached(dev);
        cudaGetLastError();  // clear the failed allocation's error
        st = dalloc(b, bytes);
    }
    return st;
}

void ws_release_all() { release_cached(-1); }

}  // namespace heom

using heom::set_error;

// ======================================================================= exponents
namespace {

// Number of eigenvalues smaller than x of the symmetric tridiagonal matrix with zero
// diagonal and off-diagonal b (Sturm sequence of the LDL^T pivots).
int sturm_count(const std::vector<double> &b, double x) {
    int n = (int)b.size() + 1, cnt = 0;
    double q = -x;
    if (q < 0) cnt++;
    for (int i = 1; i < n; ++i) {
        double prev = (q == 0.0) ? 1e-300 : q;
        q = -x - b[i - 1] * b[i - 1] / prev;
        if (q < 0) cnt++;
    }
    return cnt;
}

// The m largest eigenvalues, descending, by bisection (all eigenvalues lie in [-2max|b|, 2max|b|]).
std::vector<double> top_eigs(const std::vector<double> &b, int m) {
    int n = (int)b.size() + 1;
    double bound = 0;
    for (double v : b) bound = std::max(bound, 2.0 * std::fabs(v));
    bound += 1e-12;
    std::vector<double> out;
    for (int j = 0; j < m; ++j) {
        // eigenvalue of rank n-1-j (0-based ascending): smallest x with count(x) >= n-j
        int target = n - j;
        double lo = -bound, hi = bound;
        for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
            double mid = 0.5 * (lo + hi);
            if (sturm_count(b, mid) >= target) hi = mid; else lo = mid;
        }
        out.push_back(0.5 * (lo + hi));
    }
    return out;
}

void decomposition(int N, bool fermi, bool pade, std::vector<double> &kappa,
                   std::vector<double> &zeta) {
    kappa.assign(N, 1.0);
    zeta.assign(N, 0.0);
    if (N == 0) return;
    if (!pade) {  // Matsubara poles
        for (int j = 1; j <= N; ++j) zeta[j - 1] = fermi ? (2 * j - 1) * M_PI : 2 * M_PI * j;
        return;
    }
    auto bm = [fermi](int m) { return fermi ? 2.0 * m - 1.0 : 2.0 * m + 1.0; };
    std::vector<double> off(2 * N - 1), off_t(std::max(0, 2 * N - 2));
    for (int m = 1; m < 2 * N; ++m) off[m - 1] = 1.0 / std::sqrt(bm(m) * bm(m + 1));
    for (int m = 1; m < 2 * N - 1; ++m) off_t[m - 1] = 1.0 / std::sqrt(bm(m + 1) * bm(m + 2));
    std::vector<double> lam = top_eigs(off, N);
    std::vector<double> lt = N > 1 ? top_eigs(off_t, N - 1) : std::vector<double>();
    for (int j = 0; j < N; ++j) zeta[j] = 2.0 / lam[j];
    for (int j = 0; j < N; ++j) {
        double num = 1.0, den = 1.0;
        for (double l : lt) {
            double z = 2.0 / l;
            num *= z * z - zeta[j] * zeta[j];
        }
        for (int k = 0; k < N; ++k)
            if (k != j) den *= zeta[k] * zeta[k] - zeta[j] * zeta[j];
        kappa[j] = 0.5 * N * bm(N + 1) * num / den;
    }
}

}  // namespace

extern "C" heom_status heom_pade_constants(int n_poles, int fermi, int pade, double *kappa,
                                           double *zeta) {
    if (n_poles < 0 || n_poles > 2000 || (n_poles > 0 && (!kappa || !zeta))) {
        set_error("heom_pade_constants: n_poles must be in [0, 2000] with output arrays");
        return HEOM_EINVAL;
    }
    std::vector<double> k, z;
    decomposition(n_poles, fermi != 0, pade != 0, k, z);
    for (int j = 0; j < n_poles; ++j) { kappa[j] = k[j]; zeta[j] = z[j]; }
    return HEOM_OK;
}

extern "C" heom_status heom_exp_drude_lorentz(double lam, double W, double kT, int n_poles,
                                              int pade, heom_c64 *xi, heom_c64 *chi) {
    if (!(kT > 0) || !(W > 0) || !std::isfinite(lam) || n_poles < 0 || n_poles > 2000 || !xi ||
        !chi) {
        set_error("heom_exp_drude_lorentz: need kT > 0, W > 0, finite lam, n_poles in [0,2000]");
        return HEOM_EINVAL;
    }
    std::vector<double> kap, zet;
    decomposition(n_poles, false, pade != 0, kap, zet);
    xi[0] = {lam * W / std::tan(W / (2.0 * kT)), -lam * W};
    chi[0] = {W, 0.0};
    for (int l = 0; l < n_poles; ++l) {
        double zk = zet[l] * kT;
        xi[l + 1] = {-2.0 * kap[l] * kT * 2.0 * lam * W * zk / (W * W - zk * zk), 0.0};
        chi[l + 1] = {zk, 0.0};
    }
    return HEOM_OK;
}

extern "C" heom_status heom_exp_lorentz_fermion(double Gamma, double W, double mu, double kT,
                                                int n_poles, int pade, int nu, heom_c64 *eta,
                                                heom_c64 *gamma) {
    if (!(kT > 0) || !(W > 0) || !std::isfinite(Gamma) || !std::isfinite(mu) || n_poles < 0 ||
        n_poles > 2000 || (nu != 1 && nu != -1) || !eta || !gamma) {
        set_error("heom_exp_lorentz_fermion: need kT > 0, W > 0, finite Gamma/mu, nu = +-1");
        return HEOM_EINVAL;
    }
    std::vector<double> kap, zet;
    decomposition(n_poles, true, pade != 0, kap, zet);
    // n(x) at x = i W / kT of the truncated Fermi function 1/2 - sum 2 kappa x/(x^2+zeta^2)
    std::complex<double> x(0.0, W / kT), n(0.5, 0.0);
    for (int h = 0; h < n_poles; ++h) n -= 2.0 * kap[h] * x / (x * x + zet[h] * zet[h]);
    std::complex<double> e1 = 0.5 * Gamma * W * n;
    eta[0] = {e1.real(), e1.imag()};
    gamma[0] = {W, -nu * mu};
    for (int h = 0; h < n_poles; ++h) {
        double zk = zet[h] * kT;
        eta[h + 1] = {0.0, -kap[h] * kT * Gamma * W * W / (W * W - zk * zk)};
        gamma[h + 1] = {zk, -nu * mu};
    }
    return HEOM_OK;
}

// ======================================================================= enumeration
namespace {

uint64_t binom(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    k = std::min(k, n - k);
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (unsigned __int128)(n - k + i) / i;
    return (uint64_t)r;
}

// compositions of s into p >= 1 non-negative parts
uint64_t ncomp(int s, int p) { return p <= 0 ? (s == 0) : binom(s + p - 1, p - 1); }

struct Ranker {
    int Kb, Kf, tb, tf;
    std::vector<uint64_t> bos_off;  // bos_off[t] = # bosonic vectors of tier < t
    std::vector<uint64_t> fer_off;  // fer_off[n] = # fermionic subsets of size < n
    uint64_t Nb = 0, Nf = 0;

    void init(int Kb_, int Kf_, int tb_, int tf_) {
        Kb = Kb_; Kf = Kf_; tb = Kb_ > 0 ? tb_ : 0; tf = std::min(tf_, Kf_);
        bos_off.assign(tb + 2, 0);
        for (int t = 0; t <= tb; ++t) bos_off[t + 1] = bos_off[t] + (Kb > 0 ? ncomp(t, Kb) : (t == 0));
        Nb = bos_off[tb + 1];
        fer_off.assign(tf + 2, 0);
        for (int n = 0; n <= tf; ++n) fer_off[n + 1] = fer_off[n] + binom(Kf, n);
        Nf = fer_off[tf + 1];
    }
    // rank of m among all bosonic vectors (tier ascending, lex descending inside a tier)
    int64_t rank_bos(const int *m) const {
        int t = 0;
        for (int i = 0; i < Kb; ++i) t += m[i];
        if (t > tb) return -1;
        uint64_t cnt = 0;
        int rem = t;
        for (int i = 0; i + 1 < Kb; ++i) {
            for (int v = m[i] + 1; v <= rem; ++v) cnt += ncomp(rem - v, Kb - 1 - i);
            rem -= m[i];
        }
        return (int64_t)(bos_off[t] + cnt);
    }
    // rank of the subset with bit mask S (size ascending, lex ascending inside a size)
    int64_t rank_fer(uint64_t S) const {
        int n = __builtin_popcountll(S);
        if (n > tf) return -1;
        uint64_t r = binom(Kf, n) - 1;
        int i = 0;
        for (int c = 0; c < Kf; ++c)
            if (S >> c & 1ULL) { r -= binom(Kf - 1 - c, n - i); ++i; }
        return (int64_t)(fer_off[n] + r);
    }
};

// next bosonic vector of the same tier in lex-descending order; false at the end
bool next_comp(std::vector<int> &m) {
    int K = (int)m.size();
    for (int i = K - 2; i >= 0; --i) {
        if (m[i] > 0) {
            int tail = 0;
            for (int j = i + 1; j < K; ++j) { tail += m[j]; m[j] = 0; }
            m[i] -= 1;
            m[i + 1] = tail + 1;
            return true;
        }
    }
    return false;
}

bool finite(const heom_c64 &z) { return std::isfinite(z.re) && std::isfinite(z.im); }

template <class T>
// A copy from pageable host memory has staged the data when it returns, so v may go at once;
// the callers synchronise stream 0 once after their last upload, so that the tables are on
// the device before the call returns (kernels on other streams may read them next).
heom_status upload(DBuf &b, const std::vector<T> &v) {
    heom_status st = heom::dalloc(b, v.size() * sizeof(T));
    if (st != HEOM_OK) return st;
    if (!v.empty())
        HEOM_CUDA(heom::memcpy_counted(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, 0));
    return HEOM_OK;
}

template <class R>
std::vector<cx<R>> to_cx(const std::vector<heom_c64> &v) {
    std::vector<cx<R>> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = cx<R>{R(v[i].re), R(v[i].im)};
    return o;
}

// float-float {hi.re, hi.im, lo.re, lo.im} of each value (hi = nearest float, lo = the
// nearest float to the rest)
std::vector<float4> to_ff(const std::vector<heom_c64> &v) {
    std::vector<float4> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float hr = (float)v[i].re, hi = (float)v[i].im;
        o[i] = make_float4(hr, hi, (float)(v[i].re - (double)hr), (float)(v[i].im - (double)hi));
    }
    return o;
}

// bosonic (a, b) of D X = a V X - b X V for one exponent of the given kind
void boson_ab(int kind, heom_c64 c, heom_c64 &a, heom_c64 &b) {
    if (kind == HEOM_BOSON_R) { a = c; b = c; }
    else if (kind == HEOM_BOSON_I) { a = {-c.im, c.re}; b = {c.im, -c.re}; }
    else { a = c; b = {c.re, -c.im}; }
}

}  // namespace

heom::DevView<double> heom_hier::view64() const {
    heom::DevView<double> v{};
    v.N = N; v.d = d; v.d2 = d2; v.K = K; v.n_sets = n_sets; v.nS = nS;
    v.row_ptr = (const int32_t *)d_row_ptr.p; v.ent = (const NbEntry *)d_ent.p;
    v.occ_ptr = (const int32_t *)d_occ_ptr.p; v.occ = (const OccEntry *)d_occ.p;
    v.op_rptr = (const int32_t *)d_op_rptr.p; v.op_rcol = (const int32_t *)d_op_rcol.p;
    v.op_rval = (const cx<double> *)d_op_rval64.p;
    v.op_cptr = (const int32_t *)d_op_cptr.p; v.op_crow = (const int32_t *)d_op_crow.p;
    v.op_cval = (const cx<double> *)d_op_cval64.p;
    v.s_ptr = (const int32_t *)d_s_ptr.p; v.s_src = (const int32_t *)d_s_src.p;
    v.s_val = (const cx<double> *)d_sval64.p; v.sdiag = (const cx<double> *)d_sdiag64.p;
    v.coefL = (const cx<double> *)d_coefL64.p; v.coefR = (const cx<double> *)d_coefR64.p;
    v.rate = (const cx<double> *)d_rate64.p;
    v.floor = (const double *)d_floor64.p;
    v.t_ptr = (const int32_t *)d_t_ptr.p; v.t_src = (const int32_t *)d_t_src.p;
    v.t_val = (const cx<double> *)d_t_val64.p;
    v.max_terms = max_terms; v.max_entries = max_entries;
    v.cta_ado = (const int32_t *)d_cta_ado.p; v.n_ranges = n_ranges; v.range_terms = range_terms;
    v.range_slots = range_slots; v.range_ados = range_ados; v.tile_min_b = tile_min_b;
    v.tile_var = tile_var;
    v.ado_tier = has_caps ? (const int32_t *)d_ado_tier.p : nullptr;
    v.set_cap = has_caps ? (const int32_t *)d_set_cap.p : nullptr;
    v.pers_ado = (const int32_t *)d_pers_ado.p; v.pers_ranges = pers_ranges;
    v.pers_terms = pers_terms; v.pers_slots = pers_slots; v.pers_ados = pers_ados;
    v.op_rvalf = (const float4 *)d_op_rvalff.p; v.op_cvalf = (const float4 *)d_op_cvalff.p;
    v.s_valf = (const float4 *)d_svalff.p; v.coefLf = (const float4 *)d_coefLff.p;
    v.coefRf = (const float4 *)d_coefRff.p; v.ratef = (const float4 *)d_rateff.p;
    return v;
}

heom::DevView<float> heom_hier::view32() const {
    heom::DevView<float> v{};
    v.N = N; v.d = d; v.d2 = d2; v.K = K; v.n_sets = n_sets; v.nS = nS;
    v.row_ptr = (const int32_t *)d_row_ptr.p; v.ent = (const NbEntry *)d_ent.p;
    v.occ_ptr = (const int32_t *)d_occ_ptr.p; v.occ = (const OccEntry *)d_occ.p;
    v.op_rptr = (const int32_t *)d_op_rptr.p; v.op_rcol = (const int32_t *)d_op_rcol.p;
    v.op_rval = (const cx<float> *)d_op_rval32.p;
    v.op_cptr = (const int32_t *)d_op_cptr.p; v.op_crow = (const int32_t *)d_op_crow.p;
    v.op_cval = (const cx<float> *)d_op_cval32.p;
    v.s_ptr = (const int32_t *)d_s_ptr.p; v.s_src = (const int32_t *)d_s_src.p;
    v.s_val = (const cx<float> *)d_sval32.p; v.sdiag = (const cx<float> *)d_sdiag32.p;
    v.coefL = (const cx<float> *)d_coefL32.p; v.coefR = (const cx<float> *)d_coefR32.p;
    v.rate = (const cx<float> *)d_rate32.p;
    v.floor = (const float *)d_floor32.p;
    v.t_ptr = (const int32_t *)d_t_ptr.p; v.t_src = (const int32_t *)d_t_src.p;
    v.t_val = (const cx<float> *)d_t_val32.p;
    v.max_terms = max_terms; v.max_entries = max_entries;
    v.cta_ado = (const int32_t *)d_cta_ado.p; v.n_ranges = n_ranges; v.range_terms = range_terms;
    v.range_slots = range_slots; v.range_ados = range_ados; v.tile_min_b = tile_min_b;
    v.tile_var = tile_var;
    v.ado_tier = has_caps ? (const int32_t *)d_ado_tier.p : nullptr;
    v.set_cap = has_caps ? (const int32_t *)d_set_cap.p : nullptr;
    v.pers_ado = (const int32_t *)d_pers_ado.p; v.pers_ranges = pers_ranges;
    v.pers_terms = pers_terms; v.pers_slots = pers_slots; v.pers_ados = pers_ados;
    return v;
}

namespace {

void free_all(heom_hier *h) {
    DBuf *bufs[] = {&h->d_row_ptr, &h->d_ent, &h->d_occ_ptr, &h->d_occ, &h->d_op_rptr,
                    &h->d_op_rcol, &h->d_op_cptr, &h->d_op_crow, &h->d_op_rval64,
                    &h->d_op_cval64, &h->d_op_rval32, &h->d_op_cval32, &h->d_s_ptr,
                    &h->d_s_src, &h->d_sval64, &h->d_sval32, &h->d_coefL64, &h->d_coefL32,
                    &h->d_coefR64, &h->d_coefR32, &h->d_rate64, &h->d_rate32, &h->d_sdiag64,
                    &h->d_sdiag32, &h->d_tdval64, &h->d_floor64, &h->d_floor32, &h->ws,
                    &h->ws_small,
                    &h->d_t_ptr, &h->d_t_src, &h->d_t_val64, &h->d_t_val32, &h->d_cta_ado,
                    &h->d_pers_ado, &h->d_ar_ado, &h->ws_pers, &h->d_ado_tier, &h->d_set_cap,
                    &h->d_op_rvalff, &h->d_op_cvalff, &h->d_svalff, &h->d_coefLff, &h->d_coefRff,
                    &h->d_rateff};
    for (DBuf *b : bufs) heom::dfree(*b);
}

// Term count and shared-memory slots of every ADO's program (damping 1 per element, H, the
// neighbour terms, the trace row of ADO 0).
struct RangeCosts {
    std::vector<int64_t> terms, slots;
    int64_t total = 0;
};
RangeCosts range_costs(const heom_hier *h) {
    RangeCosts rc;
    rc.terms.resize(h->N);
    rc.slots.resize(h->N);
    for (int64_t i = 0; i < h->N; ++i) {
        int64_t t = h->d2 + h->nS + (i == 0 ? h->d : 0);
        for (int32_t k = h->row_ptr[i]; k < h->row_ptr[i + 1]; ++k) t += h->op_terms[h->ent[k].op];
        rc.terms[i] = t;
        rc.slots[i] = (int64_t)h->d2 * (h->row_ptr[i + 1] - h->row_ptr[i] + 3);
        rc.total += t;
    }
    return rc;
}

// At most `resident` contiguous ranges; a range closes once it reaches the target term count
// (or a shared-memory bound). Returns whether every range fits within the bounds.
// Balance on weight[i] when given (its sum in wtotal), else on the term counts; the bounds
// always apply to the real term and slot counts.
bool partition_ranges(const heom_hier *h, const RangeCosts &rc, int64_t resident, int64_t cap_terms,
                      std::vector<int32_t> &rg, int64_t &rt, int64_t &rs, int64_t &rn,
                      const std::vector<int64_t> *weight = nullptr, int64_t wtotal = 0,
                      bool nearest = false) {
    const int64_t total = weight ? wtotal : rc.total;
    int64_t target = std::max<int64_t>(1, (total + resident - 1) / resident);
    for (int attempt = 0; attempt < 64; ++attempt) {
        rg.assign(1, 0);
        int64_t cur_t = 0, cur_s = 0, cur_n = 0, cur_w = 0;
        rt = rs = rn = 0;
        for (int64_t i = 0; i < h->N; ++i) {
            // a range closes once it reaches the target weight, or (nearest) once taking the
            // next ADO would overshoot the target by more than half of that ADO's weight: ranges
            // of a few heavy ADOs then stay near the target instead of near twice it
            const int64_t wi = weight ? (*weight)[i] : rc.terms[i];
            const bool reached = nearest ? cur_w + wi / 2 > target : cur_w >= target;
            const bool full = cur_n > 0 && (reached || cur_t + rc.terms[i] > cap_terms ||
                                            cur_s + rc.slots[i] > heom::kRangeSlots ||
                                            cur_n >= heom::kRangeAdos);
            if (full) {
                rg.push_back((int32_t)i);
                cur_t = cur_s = cur_n = cur_w = 0;
            }
            cur_t += rc.terms[i]; cur_s += rc.slots[i]; ++cur_n;
            cur_w += wi;
            rt = std::max(rt, cur_t); rs = std::max(rs, cur_s); rn = std::max(rn, cur_n);
        }
        rg.push_back((int32_t)h->N);
        if ((int64_t)rg.size() - 1 <= resident) return true;
        target += target / 8 + 1;
    }
    return false;
}

// ADO ranges of the tiled kernel: balanced on the terms plus a per-item cost of the item's
// own work (its first load, the accumulator set-up and the epilogue, about kTileItemWeight
// terms), nearest-target closing.
constexpr int64_t kTileItemWeight = 2;
bool tile_partition(const heom_hier *h, const RangeCosts &rc, int64_t resident,
                    std::vector<int32_t> &rg, int64_t &rt, int64_t &rs, int64_t &rn) {
    std::vector<int64_t> w(h->N);
    int64_t wt = 0;
    for (int64_t i = 0; i < h->N; ++i) {
        w[i] = rc.terms[i] + kTileItemWeight * h->d2;
        wt += w[i];
    }
    return partition_ranges(h, rc, resident, heom::kRangeTerms, rg, rt, rs, rn, &w, wt, true);
}

// Most system-superoperator terms (all elements together) a hierarchy may carry.
constexpr int kMaxSystemTerms = 1 << 22;

// Upload the parameter-dependent arrays for n_sets sets: the system superoperator's term
// lists and values (H and the Lindblad terms), the (a, b) pairs and rates of the exponents,
// the preconditioner's diagonal and damping floor; then re-partition the ADO ranges, whose
// term counts depend on the system terms.
heom_status upload_params(heom_hier *h, int n_sets, const heom_c64 *H, const heom_c64 *coef,
                          const heom_c64 *rate) {
    const int d = h->d, d2 = h->d2, K = h->K;
    const int n_lind = (int)h->lind_gamma.size();
    // System superoperator per set: L_s X = -i (H X - X H) + sum_k g_k (F_k X F_k^+ -
    // 1/2 {F_k^+ F_k, X}) (Eq. HEOM's commutator, Eq. Lindbladian). With G = 1/2 sum_k g_k
    // F_k^+ F_k, element (r, c) reads
    //   X[l][c] with (-i H[r][l] - G[r][l]),   X[r][l] with (i H[l][c] - G[l][c]),
    //   X[l][m] with sum_k g_k F_k[r][l] conj(F_k[c][m]).
    // Terms are accumulated per (element, source element), so each source appears once.
    std::vector<heom_c64> G((size_t)d * d, heom_c64{0.0, 0.0});
    for (int k = 0; k < n_lind; ++k) {
        const heom_c64 *F = h->lind_F.data() + (size_t)k * d * d;
        const double g = 0.5 * h->lind_gamma[k];
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                double re = 0.0, im = 0.0;  // (F^+ F)[r][c] = sum_l conj(F[l][r]) F[l][c]
                for (int l = 0; l < d; ++l) {
                    const heom_c64 a = F[(size_t)l * d + r], b = F[(size_t)l * d + c];
                    re += a.re * b.re + a.im * b.im;
                    im += a.re * b.im - a.im * b.re;
                }
                G[(size_t)r * d + c].re += g * re;
                G[(size_t)r * d + c].im += g * im;
            }
    }
    // per element: source element -> value in each set, then in each drive operator H_k of
    // H(t) = H + sum_k f_k(t) H_k (-i H_k[r][l] left, i H_k[l][c] right), ordered by source
    const int n_drive = h->n_drive, n_val = n_sets + n_drive;
    std::vector<std::map<int, std::vector<heom_c64>>> terms(d2);
    auto add = [&](int e, int src, int set, double re, double im) {
        if (re == 0.0 && im == 0.0) return;
        auto &vals = terms[e][src];
        if (vals.empty()) vals.assign(n_val, heom_c64{0.0, 0.0});
        vals[set].re += re;
        vals[set].im += im;
    };
    for (int k = 0; k < n_drive; ++k) {
        const heom_c64 *Hk = h->drive.data() + (size_t)k * d * d;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c)
                for (int l = 0; l < d; ++l) {
                    const heom_c64 hl = Hk[(size_t)r * d + l], hr = Hk[(size_t)l * d + c];
                    add(r * d + c, l * d + c, n_sets + k, hl.im, -hl.re);
                    add(r * d + c, r * d + l, n_sets + k, -hr.im, hr.re);
                }
    }
    for (int s = 0; s < n_sets; ++s) {
        const heom_c64 *Hs = H + (size_t)s * d * d;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                const int e = r * d + c;
                for (int l = 0; l < d; ++l) {
                    const heom_c64 hl = Hs[(size_t)r * d + l], gl = G[(size_t)r * d + l];
                    add(e, l * d + c, s, hl.im - gl.re, -hl.re - gl.im);   // -i H[r][l] - G[r][l]
                    const heom_c64 hr = Hs[(size_t)l * d + c], gr = G[(size_t)l * d + c];
                    add(e, r * d + l, s, -hr.im - gr.re, hr.re - gr.im);   // i H[l][c] - G[l][c]
                }
                for (int k = 0; k < n_lind; ++k) {
                    const heom_c64 *F = h->lind_F.data() + (size_t)k * d * d;
                    const double g = h->lind_gamma[k];
                    for (int l = 0; l < d; ++l) {
                        const heom_c64 a = F[(size_t)r * d + l];
                        if (a.re == 0.0 && a.im == 0.0) continue;
                        for (int m = 0; m < d; ++m) {
                            const heom_c64 b = F[(size_t)c * d + m];  // conj(F[c][m])
                            if (b.re == 0.0 && b.im == 0.0) continue;
                            add(e, l * d + m, s, g * (a.re * b.re + a.im * b.im),
                                g * (a.im * b.re - a.re * b.im));
                        }
                    }
                }
            }
    }
    std::vector<int32_t> sptr(d2 + 1, 0), ssrc;
    std::vector<std::vector<heom_c64>> scols;  // per kept term: values per set
    std::vector<heom_c64> sd((size_t)n_sets * d2, heom_c64{0.0, 0.0});
    for (int e = 0; e < d2; ++e) {
        for (auto &kv : terms[e]) {
            bool nz = false;
            for (const heom_c64 &v : kv.second) nz = nz || v.re != 0.0 || v.im != 0.0;
            if (!nz) continue;
            if (kv.first == e)
                for (int s = 0; s < n_sets; ++s) sd[(size_t)s * d2 + e] = kv.second[s];
            ssrc.push_back(kv.first);
            scols.push_back(kv.second);
        }
        sptr[e + 1] = (int32_t)ssrc.size();
        if (ssrc.size() > (size_t)kMaxSystemTerms) {
            set_error("system superoperator has more than %d terms (jump operators too dense)",
                      kMaxSystemTerms);
            return HEOM_EINVAL;
        }
    }
    const int nS = (int)ssrc.size();
    std::vector<heom_c64> sval((size_t)n_sets * std::max(nS, 1), heom_c64{0.0, 0.0});
    std::vector<heom_c64> tdval((size_t)std::max(n_drive, 1) * std::max(nS, 1), heom_c64{0.0, 0.0});
    for (int j = 0; j < nS; ++j) {
        for (int s = 0; s < n_sets; ++s) sval[(size_t)s * nS + j] = scols[j][s];
        for (int k = 0; k < n_drive; ++k) tdval[(size_t)k * nS + j] = scols[j][n_sets + k];
    }
    std::vector<heom_c64> cl((size_t)n_sets * K), cr((size_t)n_sets * K), rt((size_t)n_sets * K);
    std::vector<double> fl(n_sets);
    for (int s = 0; s < n_sets; ++s) {
        double floor = 0;
        bool first = true;
        for (int k = 0; k < K; ++k) {
            heom_c64 c = coef[(size_t)s * K + k];
            heom_c64 a, b;
            if (k < h->K_b) {
                boson_ab(h->exp_kind[k], c, a, b);
            } else {
                heom_c64 p = coef[(size_t)s * K + h->exp_partner[k]];
                a = c;
                b = {p.re, -p.im};
            }
            cl[(size_t)s * K + k] = a;
            cr[(size_t)s * K + k] = b;
            rt[(size_t)s * K + k] = rate[(size_t)s * K + k];
            double re = rate[(size_t)s * K + k].re;
            if (re > 0 && (first || re < floor)) { floor = re; first = false; }
        }
        fl[s] = first ? 1.0 : floor;
    }
    std::vector<float> fl32(fl.begin(), fl.end());
    h->nS = nS;
    // largest term program of one ADO: damping (1 per element) + system terms + neighbour
    // terms + trace row
    {
        int mt = 0, me = 0;
        for (int64_t i = 0; i < h->N; ++i) {
            int t = h->d2 + h->nS + d;
            for (int32_t k = h->row_ptr[i]; k < h->row_ptr[i + 1]; ++k) t += h->op_terms[h->ent[k].op];
            mt = std::max(mt, t);
            me = std::max(me, (int)(h->row_ptr[i + 1] - h->row_ptr[i]));
        }
        h->max_terms = mt;
        h->max_entries = me;
    }
    // ADO ranges: contiguous, about equal term counts, each range's program and bookkeeping
    // bounded for shared memory. Tiled kernel: tile_per_sm CTAs per SM (two unless the
    // autotuner chose otherwise), all resident at once. Cooperative persistent solvers: one
    // range per SM.
    std::vector<int32_t> ranges, pranges, arranges;
    {
        RangeCosts rc = range_costs(h);
        int n_sm = 152;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
        int64_t rt, rs, rn;
        tile_partition(h, rc, (int64_t)n_sm * h->tile_per_sm, ranges, rt, rs, rn);
        h->n_ranges = (int)ranges.size() - 1;
        h->range_terms = (int)std::min<int64_t>(rt, INT32_MAX);
        h->range_slots = (int)std::min<int64_t>(rs, INT32_MAX);
        h->range_ados = (int)rn;
        const bool pfit = partition_ranges(h, rc, n_sm, heom::kPersistTerms, pranges, rt, rs, rn);
        h->pers_ranges = (pfit && rt <= heom::kPersistTerms && rs <= heom::kRangeSlots) ? (int)pranges.size() - 1 : 0;
        h->pers_terms = (int)std::min<int64_t>(rt, INT32_MAX);
        h->pers_slots = (int)std::min<int64_t>(rs, INT32_MAX);
        h->pers_ados = (int)rn;
        // The persistent Arnoldi's Gram-Schmidt work grows with the elements a range owns
        // (about 2 (j + 1) float-float multiply-adds per element and step), the apply with its
        // terms: its ranges balance terms + kArElemWeight * d2 per ADO. Without a fitting
        // partition it keeps the one above.
        std::vector<int64_t> w(h->N);
        int64_t wt = 0;
        for (int64_t i = 0; i < h->N; ++i) { w[i] = rc.terms[i] + heom::kArElemWeight * h->d2; wt += w[i]; }
        std::vector<int32_t> ar;
        const bool afit = partition_ranges(h, rc, n_sm, heom::kPersistTerms, ar, rt, rs, rn, &w, wt) &&
                          rt <= heom::kPersistTerms && rs <= heom::kRangeSlots;
        if (afit) {
            arranges = ar;
            h->ar_ranges = (int)ar.size() - 1;
            h->ar_terms = (int)rt;
            h->ar_slots = (int)rs;
            h->ar_ados = (int)rn;
        } else {
            arranges = pranges;
            h->ar_ranges = h->pers_ranges;
            h->ar_terms = h->pers_terms;
            h->ar_slots = h->pers_slots;
            h->ar_ados = h->pers_ados;
        }
    }
    heom_status st;
#define UP(buf, vec) if ((st = upload(h->buf, vec)) != HEOM_OK) return st
    UP(d_cta_ado, ranges); UP(d_pers_ado, pranges); UP(d_ar_ado, arranges);
    UP(d_s_ptr, sptr); UP(d_s_src, ssrc);
    UP(d_sval64, to_cx<double>(sval)); UP(d_sval32, to_cx<float>(sval)); UP(d_svalff, to_ff(sval));
    UP(d_coefLff, to_ff(cl)); UP(d_coefRff, to_ff(cr)); UP(d_rateff, to_ff(rt));
    UP(d_sdiag64, to_cx<double>(sd)); UP(d_sdiag32, to_cx<float>(sd));
    UP(d_tdval64, to_cx<double>(tdval));
    UP(d_coefL64, to_cx<double>(cl)); UP(d_coefL32, to_cx<float>(cl));
    UP(d_coefR64, to_cx<double>(cr)); UP(d_coefR32, to_cx<float>(cr));
    UP(d_rate64, to_cx<double>(rt)); UP(d_rate32, to_cx<float>(rt));
    UP(d_floor64, fl); UP(d_floor32, fl32);
#undef UP
    HEOM_CUDA(cudaStreamSynchronize(0));  // every upload of this call (and of the build) landed
    h->n_sets = n_sets;
    h->H0.assign(H, H + (size_t)n_sets * d * d);
    h->coef0.assign(coef, coef + (size_t)n_sets * K);
    h->rate0.assign(rate, rate + (size_t)n_sets * K);
    return HEOM_OK;
}

}  // namespace

namespace {

// Largest full hierarchy (bosonic x fermionic product) that importance pruning enumerates.
constexpr int64_t kMaxPruneFull = int64_t(1) << 29;

// Eq. importance, evaluated in one fixed sequence: the bosonic multiset j listed by
// ascending exponent index (exponent k repeated m_k times), then the fermionic set q by
// ascending index; each member multiplies the running product by |c / (Re r * cum)| with cum
// the running sum of Re r within its part. A zero denominator makes the importance infinite.
struct Importance {
    const heom_c64 *coef, *rate;  // global exponent order (bosonic first)
    int Kb;
    double bosonic(const std::vector<int> &m) const {
        double val = 1.0, cum = 0.0;
        for (int k = 0; k < Kb; ++k)
            for (int c = 0; c < m[k]; ++c) {
                const double r = rate[k].re;
                cum += r;
                const double den = r * cum;
                if (den == 0.0) return INFINITY;
                val *= std::hypot(coef[k].re / den, coef[k].im / den);
            }
        return val;
    }
    // continue the running product val of the bosonic part over the fermionic set S
    double with_fermionic(double val, uint64_t S) const {
        if (std::isinf(val)) return val;
        double cum = 0.0;
        for (uint64_t T = S; T; T &= T - 1) {
            const int g = Kb + __builtin_ctzll(T);
            const double r = rate[g].re;
            cum += r;
            const double den = r * cum;
            if (den == 0.0) return INFINITY;
            val *= std::hypot(coef[g].re / den, coef[g].im / den);
        }
        return val;
    }
};

// Levels (m, n) in {0, 1} x {0, 1} are never pruned; every other ADO is kept when its
// importance reaches the threshold.
bool keep_ado(const Importance &imp, double bos_val, int tb, uint64_t S, double th) {
    const int n = __builtin_popcountll(S);
    if (tb <= 1 && n <= 1) return true;
    return imp.with_fermionic(bos_val, S) >= th;
}

// Every fermionic subset of {0..Kf-1} with at most tf elements: size ascending, then
// lexicographically ascending (the canonical order).
template <class F>
void for_each_subset(int Kf, int tf, F &&fn) {
    for (int n = 0; n <= tf; ++n) {
        if (n == 0) { fn(0ULL); continue; }
        std::vector<int> c(n);
        for (int i = 0; i < n; ++i) c[i] = i;
        while (true) {
            uint64_t S = 0;
            for (int v : c) S |= 1ULL << v;
            fn(S);
            int i = n - 1;
            while (i >= 0 && c[i] == Kf - n + i) --i;
            if (i < 0) break;
            ++c[i];
            for (int j = i + 1; j < n; ++j) c[j] = c[j - 1] + 1;
        }
    }
}

// Every bosonic occupation vector with |m| <= tb: tier ascending, lexicographically
// descending inside a tier (the canonical order).
template <class F>
void for_each_occupation(int Kb, int tb, F &&fn) {
    for (int t = 0; t <= tb; ++t) {
        std::vector<int> m(Kb, 0);
        if (Kb == 0) { if (t == 0) fn(m); continue; }
        m[0] = t;
        do { fn(m); } while (next_comp(m));
    }
}

heom_status build_impl(int d, const heom_c64 *H, int n_baths, const heom_bath *baths, int tier_b,
                       int tier_f, int parity, double th, heom_hier **out);

}  // namespace

extern "C" heom_status heom_build_hierarchy(int d, const heom_c64 *H, int n_baths,
                                            const heom_bath *baths, int tier_b, int tier_f,
                                            int parity, int flags, heom_hier **out) {
    if (flags != 0) { set_error("heom_build_hierarchy: flags must be 0"); return HEOM_EINVAL; }
    return build_impl(d, H, n_baths, baths, tier_b, tier_f, parity, 0.0, out);
}

extern "C" heom_status heom_build_hierarchy_pruned(int d, const heom_c64 *H, int n_baths,
                                                   const heom_bath *baths, int tier_b, int tier_f,
                                                   int parity, double importance_th,
                                                   heom_hier **out) {
    if (!(importance_th >= 0.0) || !std::isfinite(importance_th)) {
        set_error("heom_build_hierarchy_pruned: importance_th must be finite and >= 0");
        return HEOM_EINVAL;
    }
    return build_impl(d, H, n_baths, baths, tier_b, tier_f, parity, importance_th, out);
}

namespace {

heom_status build_impl(int d, const heom_c64 *H, int n_baths, const heom_bath *baths, int tier_b,
                       int tier_f, int parity, double th, heom_hier **out) {
    if (!out) { set_error("heom_build_hierarchy: out is NULL"); return HEOM_EINVAL; }
    *out = nullptr;
    if (d < 1 || d > 64 || !H || n_baths < 0 || (n_baths > 0 && !baths) || tier_b < 0 ||
        tier_f < 0 || (parity != 1 && parity != -1)) {
        set_error("heom_build_hierarchy: need 1 <= d <= 64, H, tiers >= 0, parity = +-1");
        return HEOM_EINVAL;
    }
    for (int i = 0; i < d * d; ++i)
        if (!finite(H[i])) { set_error("heom_build_hierarchy: H has a non-finite entry"); return HEOM_EINVAL; }
    heom_hier *h = new (std::nothrow) heom_hier();
    if (!h) { set_error("heom_build_hierarchy: out of host memory"); return HEOM_ENOMEM; }
    h->d = d; h->d2 = d * d; h->tier_b = tier_b; h->tier_f = tier_f; h->parity = parity;
    cudaGetDevice(&h->device);

    // ---- exponents: bosonic first (bath order), then fermionic (bath order)
    std::vector<heom_c64> coef, rate;
    std::vector<int> op_slot_of_bath(n_baths, -1);
    std::vector<int> fer_first_global(n_baths, -1);
    int n_ops = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int b = 0; b < n_baths; ++b) {
            const heom_bath &B = baths[b];
            bool fer = B.kind == HEOM_FERMION;
            if (B.kind < 0 || B.kind > 3 || B.n_exp < 0 || (B.n_exp > 0 && (!B.coef || !B.rate)) || !B.op) {
                set_error("heom_build_hierarchy: bath %d: bad kind, n_exp or NULL arrays", b);
                delete h; return HEOM_EINVAL;
            }
            if ((pass == 0) == fer) continue;
            for (int i = 0; i < d * d; ++i)
                if (!finite(B.op[i])) { set_error("bath %d: non-finite operator", b); delete h; return HEOM_EINVAL; }
            op_slot_of_bath[b] = n_ops;
            for (int i = 0; i < d * d; ++i) h->ops.push_back(B.op[i]);
            ++n_ops;
            if (fer) {  // second slot: d^dagger
                for (int r = 0; r < d; ++r)
                    for (int c = 0; c < d; ++c) {
                        heom_c64 z = B.op[c * d + r];
                        h->ops.push_back({z.re, -z.im});
                    }
                ++n_ops;
                if (!B.nu || !B.partner) { set_error("bath %d: fermionic bath needs nu and partner", b); delete h; return HEOM_EINVAL; }
                fer_first_global[b] = (int)h->exp_kind.size();
            }
            for (int k = 0; k < B.n_exp; ++k) {
                if (!finite(B.coef[k]) || !finite(B.rate[k])) {
                    set_error("bath %d exponent %d: non-finite coefficient or rate", b, k);
                    delete h; return HEOM_EINVAL;
                }
                h->exp_kind.push_back(B.kind);
                h->exp_bath.push_back(b);
                coef.push_back(B.coef[k]);
                rate.push_back(B.rate[k]);
                if (fer) {
                    int p = B.partner[k];
                    if (B.nu[k] != 1 && B.nu[k] != -1) { set_error("bath %d exponent %d: nu must be +-1", b, k); delete h; return HEOM_EINVAL; }
                    if (p < 0 || p >= B.n_exp || B.partner[p] != k || B.nu[p] != -B.nu[k]) {
                        set_error("bath %d exponent %d: partner map must be an involution flipping nu", b, k);
                        delete h; return HEOM_EINVAL;
                    }
                    h->exp_nu.push_back(B.nu[k]);
                    h->exp_partner.push_back(fer_first_global[b] + p);
                } else {
                    h->exp_nu.push_back(0);
                    h->exp_partner.push_back(-1);
                }
            }
            if (pass == 0) h->K_b += B.n_exp; else h->K_f += B.n_exp;
        }
    }
    h->K = h->K_b + h->K_f;
    h->n_ops = n_ops;
    h->bath_slot = op_slot_of_bath;
    if (h->K_f > 64) { set_error("heom_build_hierarchy: at most 64 fermionic exponents"); delete h; return HEOM_EINVAL; }
    if (h->K_b == 0) h->tier_b = 0;
    if (h->K_f < h->tier_f) h->tier_f = h->K_f;
    const int Kb = h->K_b, Kf = h->K_f;

    // ---- enumerate
    Ranker rk;
    rk.init(Kb, Kf, h->tier_b, h->tier_f);
    h->N_b = (int64_t)rk.Nb; h->N_f = (int64_t)rk.Nf;
    if ((double)rk.Nb * (double)rk.Nf > 2.0e9) { set_error("heom_build_hierarchy: more than 2e9 ADOs"); delete h; return HEOM_EINVAL; }
    h->N = h->N_b * h->N_f;
    try {
        h->bos.reserve(rk.Nb);
        for_each_occupation(Kb, h->tier_b, [&](const std::vector<int> &m) { h->bos.push_back(m); });
        h->fer.reserve(rk.Nf);
        for_each_subset(Kf, h->tier_f, [&](uint64_t S) { h->fer.push_back(S); });
        // ---- importance pruning (Eq. importance): keep the ADOs that reach the threshold
        if (th > 0.0) {
            if (h->N > kMaxPruneFull) {
                set_error("heom_build_hierarchy_pruned: the full hierarchy has more than 2^29 ADOs");
                delete h; return HEOM_EINVAL;
            }
            const Importance imp{coef.data(), rate.data(), Kb};
            h->importance_th = th;
            h->f2c.assign((size_t)h->N, -1);
            for (int64_t ib = 0; ib < h->N_b; ++ib) {
                const std::vector<int> &m = h->bos[ib];
                int tb = 0;
                for (int v : m) tb += v;
                const double bv = imp.bosonic(m);
                for (int64_t jf = 0; jf < h->N_f; ++jf)
                    if (keep_ado(imp, bv, tb, h->fer[jf], th)) {
                        h->f2c[(size_t)(ib * h->N_f + jf)] = (int32_t)h->c2f.size();
                        h->c2f.push_back(ib * h->N_f + jf);
                    }
            }
            h->N = (int64_t)h->c2f.size();
        }
        // ---- neighbour / sign tables (an entry whose neighbour was pruned is left out)
        const int p = parity;
        std::vector<int32_t> occ_ptr(h->N + 1, 0);
        std::vector<OccEntry> occ;
        h->row_ptr.assign(h->N + 1, 0);
        std::vector<int> mm(Kb);
        for (int64_t i = 0; i < h->N; ++i) {
            const int64_t full = h->full_of(i), ib = full / h->N_f, jf = full % h->N_f;
            const std::vector<int> &m = h->bos[ib];
            int tb = 0;
            for (int v : m) tb += v;
            const uint64_t S = h->fer[jf];
            const int n = __builtin_popcountll(S);
            const int sigma = ((n & 1) ? -p : p);
            if (tb < h->tier_b) {
                for (int k = 0; k < Kb; ++k) {
                    mm = m; mm[k] += 1;
                    const int64_t j = h->compact_of(rk.rank_bos(mm.data()) * h->N_f + jf);
                    if (j < 0) continue;
                    h->ent.push_back({(int32_t)j, (int16_t)op_slot_of_bath[h->exp_bath[k]], (int16_t)k, 1, 1, -1, 0});
                }
            }
            for (int k = 0; k < Kb; ++k) {
                if (m[k] == 0) continue;
                mm = m; mm[k] -= 1;
                const int64_t j = h->compact_of(rk.rank_bos(mm.data()) * h->N_f + jf);
                if (j < 0) continue;
                h->ent.push_back({(int32_t)j, (int16_t)op_slot_of_bath[h->exp_bath[k]], (int16_t)k, -1,
                                  (int16_t)m[k], (int16_t)(-m[k]), 0});
            }
            for (int q = 0; q < Kf; ++q) {
                const int g = Kb + q;
                const int slot = op_slot_of_bath[h->exp_bath[g]];
                const int nu = h->exp_nu[g];
                const int eps = (__builtin_popcountll(S & ((1ULL << q) - 1ULL)) & 1) ? -1 : 1;
                if (S >> q & 1ULL) {  // lowered neighbour: C term, O = d^{nu}
                    const int64_t j = h->compact_of(ib * h->N_f + rk.rank_fer(S & ~(1ULL << q)));
                    if (j < 0) continue;
                    h->ent.push_back({(int32_t)j, (int16_t)(slot + (nu == 1 ? 1 : 0)), (int16_t)g, -1,
                                      (int16_t)(p * eps), (int16_t)(p * eps * sigma), 0});
                } else if (n < h->tier_f) {  // raised neighbour: A term, O = d^{-nu}
                    const int64_t j = h->compact_of(ib * h->N_f + rk.rank_fer(S | (1ULL << q)));
                    if (j < 0) continue;
                    h->ent.push_back({(int32_t)j, (int16_t)(slot + (nu == 1 ? 0 : 1)), (int16_t)g, 1,
                                      (int16_t)(p * eps), (int16_t)(-p * eps * sigma), 0});
                }
            }
            h->row_ptr[i + 1] = (int32_t)h->ent.size();
            for (int k = 0; k < Kb; ++k)
                if (m[k]) occ.push_back({(int16_t)k, (int16_t)m[k]});
            for (int q = 0; q < Kf; ++q)
                if (S >> q & 1ULL) occ.push_back({(int16_t)(Kb + q), 1});
            occ_ptr[i + 1] = (int32_t)occ.size();
        }
        h->E = (int64_t)h->ent.size();
        if (h->E > INT32_MAX) { set_error("heom_build_hierarchy: table too large"); delete h; return HEOM_EINVAL; }
        // ---- operators, CSR and CSC with absolute offsets
        std::vector<int32_t> orp, orc, ocp, ocr;
        std::vector<heom_c64> orv, ocv;
        for (int o = 0; o < n_ops; ++o) {
            const heom_c64 *A = &h->ops[(size_t)o * d * d];
            orp.push_back((int32_t)orc.size());
            for (int r = 0; r < d; ++r) {
                for (int c = 0; c < d; ++c)
                    if (A[r * d + c].re != 0.0 || A[r * d + c].im != 0.0) { orc.push_back(c); orv.push_back(A[r * d + c]); }
                orp.push_back((int32_t)orc.size());
            }
            ocp.push_back((int32_t)ocr.size());
            for (int c = 0; c < d; ++c) {
                for (int r = 0; r < d; ++r)
                    if (A[r * d + c].re != 0.0 || A[r * d + c].im != 0.0) { ocr.push_back(r); ocv.push_back(A[r * d + c]); }
                ocp.push_back((int32_t)ocr.size());
            }
        }
        heom_status st;
#define UP(buf, vec) if ((st = upload(h->buf, vec)) != HEOM_OK) { free_all(h); delete h; return st; }
        UP(d_row_ptr, h->row_ptr); UP(d_ent, h->ent); UP(d_occ_ptr, occ_ptr); UP(d_occ, occ);
        UP(d_op_rptr, orp); UP(d_op_rcol, orc); UP(d_op_cptr, ocp); UP(d_op_crow, ocr);
        UP(d_op_rval64, to_cx<double>(orv)); UP(d_op_cval64, to_cx<double>(ocv));
        UP(d_op_rval32, to_cx<float>(orv)); UP(d_op_cval32, to_cx<float>(ocv));
        UP(d_op_rvalff, to_ff(orv)); UP(d_op_cvalff, to_ff(ocv));
        // per-element term lists of every operator slot (tiled kernels)
        std::vector<int32_t> tp(1, 0), tsrc;
        std::vector<heom_c64> tval;
        h->op_terms.assign(n_ops, 0);
        for (int o = 0; o < n_ops; ++o) {
            const heom_c64 *A = &h->ops[(size_t)o * d * d];
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) {
                    for (int l = 0; l < d; ++l)
                        if (A[r * d + l].re != 0.0 || A[r * d + l].im != 0.0) {
                            tsrc.push_back(l * d + c); tval.push_back(A[r * d + l]);
                        }
                    for (int l = 0; l < d; ++l)
                        if (A[l * d + c].re != 0.0 || A[l * d + c].im != 0.0) {
                            tsrc.push_back((r * d + l) | (1 << 16)); tval.push_back(A[l * d + c]);
                        }
                    tp.push_back((int32_t)tsrc.size());
                }
            h->op_terms[o] = tp.back() - tp[(size_t)o * d * d];
        }
        UP(d_t_ptr, tp); UP(d_t_src, tsrc);
        UP(d_t_val64, to_cx<double>(tval)); UP(d_t_val32, to_cx<float>(tval));
#undef UP
        if ((st = upload_params(h, 1, H, coef.data(), rate.data())) != HEOM_OK) { free_all(h); delete h; return st; }
    } catch (const std::bad_alloc &) {
        set_error("heom_build_hierarchy: out of host memory");
        free_all(h); delete h;
        return HEOM_ENOMEM;
    }
    *out = h;
    return HEOM_OK;
}

}  // namespace

extern "C" heom_status heom_count_ados(int n_baths, const heom_bath *baths, int tier_b, int tier_f,
                                       double importance_th, int64_t *count) {
    if (!count || n_baths < 0 || (n_baths > 0 && !baths) || tier_b < 0 || tier_f < 0 ||
        !(importance_th >= 0.0) || !std::isfinite(importance_th)) {
        set_error("heom_count_ados: need count, baths, tiers >= 0 and a finite importance_th >= 0");
        return HEOM_EINVAL;
    }
    // exponents in the global order: bosonic baths first, then fermionic, each in call order
    std::vector<heom_c64> coef, rate;
    int Kb = 0, Kf = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int b = 0; b < n_baths; ++b) {
            const heom_bath &B = baths[b];
            if (B.kind < 0 || B.kind > 3 || B.n_exp < 0 || (B.n_exp > 0 && (!B.coef || !B.rate))) {
                set_error("heom_count_ados: bath %d: bad kind, n_exp or NULL arrays", b);
                return HEOM_EINVAL;
            }
            if ((pass == 0) == (B.kind == HEOM_FERMION)) continue;
            for (int k = 0; k < B.n_exp; ++k) {
                if (!finite(B.coef[k]) || !finite(B.rate[k])) {
                    set_error("heom_count_ados: bath %d exponent %d: non-finite value", b, k);
                    return HEOM_EINVAL;
                }
                coef.push_back(B.coef[k]);
                rate.push_back(B.rate[k]);
            }
            (pass == 0 ? Kb : Kf) += B.n_exp;
        }
    if (Kf > 64) { set_error("heom_count_ados: at most 64 fermionic exponents"); return HEOM_EINVAL; }
    Ranker rk;
    rk.init(Kb, Kf, tier_b, tier_f);
    if (importance_th == 0.0) {
        if ((double)rk.Nb * (double)rk.Nf > 9.0e18) { set_error("heom_count_ados: count overflows"); return HEOM_EINVAL; }
        *count = (int64_t)(rk.Nb * rk.Nf);
        return HEOM_OK;
    }
    if ((double)rk.Nb * (double)rk.Nf > 4.0e10) {
        set_error("heom_count_ados: more than 4e10 ADOs to rate");
        return HEOM_EINVAL;
    }
    const Importance imp{coef.data(), rate.data(), Kb};
    int64_t n_keep = 0;
    for_each_occupation(Kb, rk.tb, [&](const std::vector<int> &m) {
        int tb = 0;
        for (int v : m) tb += v;
        const double bv = imp.bosonic(m);
        for_each_subset(Kf, rk.tf, [&](uint64_t S) { n_keep += keep_ado(imp, bv, tb, S, importance_th); });
    });
    *count = n_keep;
    return HEOM_OK;
}

extern "C" heom_status heom_set_params(heom_hier *h, int n_sets, const heom_c64 *H,
                                       const heom_c64 *coef, const heom_c64 *rate) {
    if (!h || n_sets < 1 || !H || (h->K > 0 && (!coef || !rate))) {
        set_error("heom_set_params: need a hierarchy, n_sets >= 1 and H/coef/rate arrays");
        return HEOM_EINVAL;
    }
    for (size_t i = 0; i < (size_t)n_sets * h->d2; ++i)
        if (!finite(H[i])) { set_error("heom_set_params: non-finite H"); return HEOM_EINVAL; }
    for (size_t i = 0; i < (size_t)n_sets * h->K; ++i)
        if (!finite(coef[i]) || !finite(rate[i])) { set_error("heom_set_params: non-finite exponent"); return HEOM_EINVAL; }
    HEOM_DEVICE(h->device);
    // a new set count invalidates per-set truncation tiers
    h->has_caps = h->has_act = false;
    heom::dfree(h->d_set_cap);
    return upload_params(h, n_sets, H, coef, rate);
}

extern "C" heom_status heom_set_truncation(heom_hier *h, const int *tier_b, const int *tier_f) {
    if (!h) {
        set_error("heom_set_truncation: need a hierarchy");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    if (!tier_b && !tier_f) {  // remove
        h->has_caps = h->has_act = false;
        heom::dfree(h->d_set_cap);
        return HEOM_OK;
    }
    if (!tier_b || !tier_f) {
        set_error("heom_set_truncation: need both tier arrays (or neither, to remove)");
        return HEOM_EINVAL;
    }
    std::vector<int32_t> cap(h->n_sets);
    for (int s = 0; s < h->n_sets; ++s) {
        if (tier_b[s] < 0 || tier_b[s] > h->tier_b || tier_f[s] < 0 || tier_f[s] > h->tier_f) {
            set_error("heom_set_truncation: set %d asks for tiers (%d, %d) outside [0, %d] x [0, %d]",
                      s, tier_b[s], tier_f[s], h->tier_b, h->tier_f);
            return HEOM_EINVAL;
        }
        cap[s] = tier_f[s] | (tier_b[s] << 16);
    }
    heom_status st;
    std::vector<int32_t> at(h->N);
    for (int64_t n = 0; n < h->N; ++n) {
        const int64_t f = h->full_of(n);
        const std::vector<int> &m = h->bos[(size_t)(f / h->N_f)];
        int nb = 0;
        for (int k : m) nb += k;
        const int nf = __builtin_popcountll(h->fer[(size_t)(f % h->N_f)]);
        at[n] = nf | (nb << 16);
    }
    if (!h->d_ado_tier.p && (st = upload(h->d_ado_tier, at)) != HEOM_OK) return st;
    if ((st = upload(h->d_set_cap, cap)) != HEOM_OK) return st;
    // caps that never increase from one set to the next: each ADO is kept by a leading run of
    // sets, whose length the Gram-Schmidt kernels use to skip the columns held at zero
    h->kept_rowsets = 0;
    h->set_kept.assign((size_t)h->n_sets, 0);
    for (int64_t n = 0; n < h->N; ++n)
        for (int s = 0; s < h->n_sets; ++s)
            if ((at[n] & 0xffff) <= tier_f[s] && (at[n] >> 16) <= tier_b[s]) {
                h->kept_rowsets += h->d2;
                ++h->set_kept[(size_t)s];
            }
    bool mono = true;
    for (int s = 1; s < h->n_sets; ++s)
        mono = mono && tier_b[s] <= tier_b[s - 1] && tier_f[s] <= tier_f[s - 1];
    h->has_act = false;
    h->act_ado.clear();
    if (mono) {
        h->act_ado.resize(h->N);
        for (int64_t n = 0; n < h->N; ++n) {
            int k = 0;
            while (k < h->n_sets && (at[n] & 0xffff) <= tier_f[k] && (at[n] >> 16) <= tier_b[k]) ++k;
            h->act_ado[n] = k;
        }
        h->has_act = true;
    }
    HEOM_CUDA(cudaStreamSynchronize(0));
    h->has_caps = true;
    return HEOM_OK;
}

extern "C" heom_status heom_set_lindblad(heom_hier *h, int n_ops, const heom_c64 *F,
                                         const double *gamma) {
    if (!h || n_ops < 0 || (n_ops > 0 && (!F || !gamma))) {
        set_error("heom_set_lindblad: need a hierarchy, n_ops >= 0 and F/gamma arrays");
        return HEOM_EINVAL;
    }
    for (size_t i = 0; i < (size_t)n_ops * h->d2; ++i)
        if (!finite(F[i])) { set_error("heom_set_lindblad: non-finite jump operator"); return HEOM_EINVAL; }
    for (int k = 0; k < n_ops; ++k)
        if (!std::isfinite(gamma[k])) { set_error("heom_set_lindblad: non-finite rate"); return HEOM_EINVAL; }
    HEOM_DEVICE(h->device);
    std::vector<heom_c64> oldF, Hs = h->H0, cs = h->coef0, rs = h->rate0;
    std::vector<double> oldg;
    oldF.swap(h->lind_F);
    oldg.swap(h->lind_gamma);
    h->lind_F.assign(F, F + (size_t)n_ops * h->d2);
    h->lind_gamma.assign(gamma, gamma + n_ops);
    const heom_status st = upload_params(h, h->n_sets, Hs.data(), cs.data(), rs.data());
    if (st != HEOM_OK) {
        h->lind_F.swap(oldF);
        h->lind_gamma.swap(oldg);
    }
    return st;
}

extern "C" heom_status heom_set_drive(heom_hier *h, int n_drive, const heom_c64 *Hk) {
    if (!h || n_drive < 0 || n_drive > 64 || (n_drive > 0 && !Hk)) {
        set_error("heom_set_drive: need a hierarchy, 0 <= n_drive <= 64 and the operators");
        return HEOM_EINVAL;
    }
    for (size_t i = 0; i < (size_t)n_drive * h->d2; ++i)
        if (!finite(Hk[i])) { set_error("heom_set_drive: non-finite drive operator"); return HEOM_EINVAL; }
    HEOM_DEVICE(h->device);
    std::vector<heom_c64> old, Hs = h->H0, cs = h->coef0, rs = h->rate0;
    old.swap(h->drive);
    const int old_n = h->n_drive;
    h->drive.assign(Hk, Hk + (size_t)n_drive * h->d2);
    h->n_drive = n_drive;
    const heom_status st = upload_params(h, h->n_sets, Hs.data(), cs.data(), rs.data());
    if (st != HEOM_OK) {
        h->drive.swap(old);
        h->n_drive = old_n;
    }
    return st;
}

extern "C" heom_status heom_hier_info(const heom_hier *h, int64_t *n_ado, int *d, int *k_b,
                                      int *k_f, int *n_sets, int64_t *n_entries) {
    if (!h) { set_error("heom_hier_info: NULL hierarchy"); return HEOM_EINVAL; }
    if (n_ado) *n_ado = h->N;
    if (d) *d = h->d;
    if (k_b) *k_b = h->K_b;
    if (k_f) *k_f = h->K_f;
    if (n_sets) *n_sets = h->n_sets;
    if (n_entries) *n_entries = h->E;
    return HEOM_OK;
}

extern "C" heom_status heom_ado_index(const heom_hier *h, const int *occ, int64_t *idx) {
    if (!h || !occ || !idx) { set_error("heom_ado_index: NULL argument"); return HEOM_EINVAL; }
    Ranker rk;
    rk.init(h->K_b, h->K_f, h->tier_b, h->tier_f);
    uint64_t S = 0;
    for (int k = 0; k < h->K_b; ++k)
        if (occ[k] < 0) { *idx = -1; return HEOM_OK; }
    for (int q = 0; q < h->K_f; ++q) {
        int v = occ[h->K_b + q];
        if (v != 0 && v != 1) { *idx = -1; return HEOM_OK; }
        if (v) S |= 1ULL << q;
    }
    int64_t ib = rk.rank_bos(occ), jf = rk.rank_fer(S);
    *idx = (ib < 0 || jf < 0) ? -1 : h->compact_of(ib * h->N_f + jf);
    return HEOM_OK;
}

extern "C" heom_status heom_ado_label(const heom_hier *h, int64_t idx, int *occ_out) {
    if (!h || !occ_out || idx < 0 || idx >= h->N) {
        set_error("heom_ado_label: index out of range or NULL argument");
        return HEOM_EINVAL;
    }
    const int64_t full = h->full_of(idx);
    const std::vector<int> &m = h->bos[full / h->N_f];
    uint64_t S = h->fer[full % h->N_f];
    for (int k = 0; k < h->K_b; ++k) occ_out[k] = m[k];
    for (int q = 0; q < h->K_f; ++q) occ_out[h->K_b + q] = (int)(S >> q & 1ULL);
    return HEOM_OK;
}

extern "C" heom_status heom_export_tables(const heom_hier *h, int32_t *row_ptr, int32_t *nb,
                                          int32_t *k, int32_t *dir, int32_t *mult_l,
                                          int32_t *mult_r) {
    if (!h) { set_error("heom_export_tables: NULL hierarchy"); return HEOM_EINVAL; }
    if (row_ptr) std::copy(h->row_ptr.begin(), h->row_ptr.end(), row_ptr);
    for (int64_t t = 0; t < h->E; ++t) {
        const NbEntry &e = h->ent[t];
        if (nb) nb[t] = e.nb;
        if (k) k[t] = e.k;
        if (dir) dir[t] = e.dir;
        if (mult_l) mult_l[t] = e.mult_l;
        if (mult_r) mult_r[t] = e.mult_r;
    }
    return HEOM_OK;
}

extern "C" void heom_destroy(heom_hier *h) {
    if (!h) return;
    heom::DeviceScope scope;
    scope.set(h->device);
    // the solver workspaces go to the process-wide cache (every solver has synchronised
    // its stream before returning, so no kernel still uses them)
    heom::ws_release(h->ws, h->device);
    heom::ws_release(h->ws_small, h->device);
    heom::ws_release(h->ws_pers, h->device);
    free_all(h);
    delete h;
}

extern "C" heom_status heom_release_workspace_cache(void) {
    heom::ws_release_all();
    return HEOM_OK;
}

extern "C" const char *heom_last_error(void) { return heom::g_err.c_str(); }

// ======================================================================= launch accounting
namespace {
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double units;
};
struct ProfState {
    bool on = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    int64_t launches[HEOM_KC_COUNT] = {};
    double ms[HEOM_KC_COUNT] = {};
    double units[HEOM_KC_COUNT] = {};
    double bytes[HEOM_KC_COUNT] = {};
    int64_t h2d = 0, d2h = 0;
    cudaEvent_t open_ev = nullptr;
};
ProfState g_prof;

cudaEvent_t prof_event() {
    if (!g_prof.pool.empty()) {
        cudaEvent_t e = g_prof.pool.back();
        g_prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_drain() {
    for (ProfRec &r : g_prof.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess)
            g_prof.ms[r.cls] += t;
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.pending.clear();
}
}  // namespace

namespace heom {
bool prof_on() { return g_prof.on; }
cudaError_t memcpy_counted(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                           cudaStream_t s) {
    if (g_prof.on) {
        if (kind == cudaMemcpyHostToDevice) g_prof.h2d += (int64_t)bytes;
        if (kind == cudaMemcpyDeviceToHost) g_prof.d2h += (int64_t)bytes;
    }
    return cudaMemcpyAsync(dst, src, bytes, kind, s);
}
void prof_begin(int cls, cudaStream_t s) {
    (void)cls;
    g_prof.open_ev = prof_event();
    cudaEventRecord(g_prof.open_ev, s);
}
void prof_end(int cls, cudaStream_t s, double units, double bytes, int kernels) {
    cudaEvent_t e = prof_event();
    cudaEventRecord(e, s);
    g_prof.pending.push_back({cls, g_prof.open_ev, e, units});
    g_prof.launches[cls] += kernels;
    g_prof.units[cls] += units;
    g_prof.bytes[cls] += bytes;
    if (g_prof.pending.size() > 4096) prof_drain();
}
void prof_add(int cls, double units, double bytes) {
    if (!g_prof.on) return;
    g_prof.units[cls] += units;
    g_prof.bytes[cls] += bytes;
}
}  // namespace heom

namespace heom {
heom_status set_tile_partition(heom_hier *h, int per_sm) {
    if (per_sm < 1 || per_sm > 5) {
        set_error("tile partition: 1..5 CTAs per SM");
        return HEOM_EINVAL;
    }
    HEOM_DEVICE(h->device);
    RangeCosts rc = range_costs(h);
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    std::vector<int32_t> ranges;
    int64_t rt, rs, rn;
    tile_partition(h, rc, (int64_t)n_sm * per_sm, ranges, rt, rs, rn);
    dfree(h->d_cta_ado);
    heom_status st = upload(h->d_cta_ado, ranges);
    if (st != HEOM_OK) return st;
    HEOM_CUDA(cudaStreamSynchronize(0));
    h->n_ranges = (int)ranges.size() - 1;
    h->range_terms = (int)std::min<int64_t>(rt, INT32_MAX);
    h->range_slots = (int)std::min<int64_t>(rs, INT32_MAX);
    h->range_ados = (int)rn;
    h->tile_per_sm = per_sm;
    return HEOM_OK;
}
}  // namespace heom

extern "C" heom_status heom_set_wait_limit(int64_t cycles) {
    heom::g_wait_cycles.store(cycles > 0 ? (long long)cycles : heom::kDefaultWaitCycles);
    return HEOM_OK;
}

extern "C" heom_status heom_profile_allocs(int64_t *device_allocs, int64_t *device_bytes,
                                           int64_t *workspace_takes) {
    if (device_allocs) *device_allocs = heom::g_dev_allocs.load();
    if (device_bytes) *device_bytes = heom::g_dev_alloc_bytes.load();
    if (workspace_takes) *workspace_takes = heom::g_ws_takes.load();
    return HEOM_OK;
}

extern "C" heom_status heom_profile_enable(int on) {
    prof_drain();
    if (on) {
        for (int c = 0; c < HEOM_KC_COUNT; ++c) {
            g_prof.launches[c] = 0;
            g_prof.ms[c] = 0;
            g_prof.units[c] = 0;
            g_prof.bytes[c] = 0;
        }
        g_prof.h2d = 0;
        g_prof.d2h = 0;
    }
    g_prof.on = on != 0;
    return HEOM_OK;
}

extern "C" heom_status heom_profile_read(int cls, int64_t *launches, double *device_ms,
                                         double *units, double *bytes) {
    if (cls < 0 || cls >= HEOM_KC_COUNT) {
        set_error("heom_profile_read: class out of range");
        return HEOM_EINVAL;
    }
    prof_drain();
    if (launches) *launches = g_prof.launches[cls];
    if (device_ms) *device_ms = g_prof.ms[cls];
    if (units) *units = g_prof.units[cls];
    if (bytes) *bytes = g_prof.bytes[cls];
    return HEOM_OK;
}

extern "C" heom_status heom_profile_copies(int64_t *h2d_bytes, int64_t *d2h_bytes) {
    if (h2d_bytes) *h2d_bytes = g_prof.h2d;
    if (d2h_bytes) *d2h_bytes = g_prof.d2h;
    return HEOM_OK;
}
