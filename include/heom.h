/*
 * heom.h -- C ABI of the GB300 HEOM library (libheom.so).
 *
 * The library applies the HEOM Liouvillian superoperator M of the hierarchical equations
 * of motion (Eq. HEOM of arXiv 2306.07522 with the superoperators A, B, C, D, P_s defined
 * below it) to the vector of all auxiliary density operators (ADOs), matrix-free on one
 * GPU, and drives it in three solvers: RK4 time evolution, stationary states and spectra.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are (re, im) pairs of doubles (heom_c64, the memory layout of
 *   torch.complex128 / std::complex<double>). FP32 device buffers are (re, im) float pairs
 *   (torch.complex64).
 * - Operators are d x d, row-major.
 * - An ADO vector is a device buffer laid out [N][d][d][batch]: ADO n, row r, column c,
 *   batch column b at element ((n*d + r)*d + c)*batch + b. With batch = 1 this is a plain
 *   array of N row-major d x d blocks. ADO n = 0 is the reduced density matrix rho_sys.
 * - ADO order (the "hierarchy dictionary", Fig. 1e): bosonic occupation vectors m
 *   (|m| <= tier_b) by tier ascending then lexicographically descending, fermionic index
 *   sets S (|S| <= tier_f) by size ascending then lexicographically ascending as sorted
 *   tuples; ADO index = bosonic index * N_f + fermionic index (in an importance-pruned
 *   hierarchy the kept ADOs in this order, renumbered 0 .. N-1). Exponents are numbered in
 *   bath order, then in order within each bath; bosonic exponents come first
 *   (0 .. K_b-1), fermionic ones after (K_b .. K_b+K_f-1) in the occupation arrays below.
 * - Ownership: every input array is copied by the call that receives it. Device vectors are
 *   caller-allocated and caller-owned; the library never frees them. A heom_hier owns its
 *   device tables and workspace until heom_destroy.
 * - Streams: every device entry point takes a CUDA stream (a cudaStream_t; 0 = legacy
 *   default stream) and enqueues its work there. Solvers synchronise that stream before
 *   they return (they read convergence flags on the host); heom_apply does not.
 * - Errors: every call returns a heom_status. No exception crosses the ABI. On failure the
 *   message of the last error on the calling thread is available from heom_last_error().
 *   There is no CPU fallback: without a usable CUDA device the device entry points return
 *   HEOM_ECUDA.
 */
#ifndef HEOM_H
#define HEOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } heom_c64;
typedef struct heom_hier heom_hier;
typedef struct CUstream_st *heom_stream; /* binary-compatible with cudaStream_t */

typedef enum {
    HEOM_OK = 0,
    HEOM_EINVAL = 1,      /* invalid argument (message says which)                      */
    HEOM_ENOMEM = 2,      /* host or device allocation failed                           */
    HEOM_ECUDA = 3,       /* CUDA runtime error, or no usable device                    */
    HEOM_ENOCONV = 4,     /* a solver reached max_iter; stats hold the last residual    */
    HEOM_EBREAKDOWN = 5,  /* Krylov breakdown or a non-finite value in a solver         */
    HEOM_ENOTSUP = 6,     /* valid request the library does not implement              */
    HEOM_ETIMEOUT = 7     /* a device-side wait (a grid barrier of a persistent solver)
                             ran out (heom_set_wait_limit); every CTA left the launch, the
                             device and the hierarchy stay usable, stats are filled       */
} heom_status;

/* Kinds of exponent lists (one per bath). Results: Eqs. C_beta_RI and C_beta_u; D_j. */
typedef enum {
    HEOM_BOSON_R = 0,   /* real part:       D X = c [V, X]                             */
    HEOM_BOSON_I = 1,   /* imaginary part:  D X = i c {V, X}                           */
    HEOM_BOSON_RI = 2,  /* both, real rates: D X = Re(c) [V, X] + i Im(c) {V, X}       */
    HEOM_FERMION = 3    /* fermionic: A_q, C_q with eta = coef, gamma = rate            */
} heom_kind;

/* Arithmetic of a call. */
typedef enum {
    HEOM_FP64 = 0,   /* complex FP64 storage and arithmetic (the plain path); the
                        single-column stationary solve runs its Krylov applies in
                        float-float (about 48 significant bits), its residuals in FP64  */
    HEOM_FP32 = 1,   /* complex FP32 storage and arithmetic                            */
    HEOM_MIXED = 2,  /* solvers: FP32 inner Krylov solves inside FP64 iterative
                        refinement; FP64 residuals, dot products and normalisation      */
    HEOM_SHIFTED = 3, /* heom_spectrum: one Arnoldi process per right-hand side serves
                        every frequency (the shifted systems share one Krylov space):
                        apply, Gram-Schmidt and rotation chains in float-float (about
                        48 significant bits), Hessenberg matrix, rotations and solutions
                        FP64; residual per frequency from its shifted Hessenberg problem */
    HEOM_FP64_STRICT = 4 /* heom_steady: FP64 storage and arithmetic in every step, the
                        single-column solve included (never the float-float persistent
                        kernel): the plain reference path                                */
} heom_prec;

/* One bath = one coupling operator + its exponent list (Fig. 1b). */
typedef struct {
    int kind;               /* heom_kind                                                */
    const heom_c64 *op;     /* d x d: V (bosonic, Hermitian) or d (fermionic annihilator) */
    int n_exp;              /* number of exponents of this bath                         */
    const heom_c64 *coef;   /* bosonic: c (R / I) or xi (RI); fermionic: eta             */
    const heom_c64 *rate;   /* bosonic chi, fermionic gamma                              */
    const int *nu;          /* fermionic only: +1 (d^dagger) / -1 (d) per exponent       */
    const int *partner;     /* fermionic only: index within this bath of the exponent
                               with the same (alpha, h, sigma) and opposite nu; must be an
                               involution that flips nu                                  */
} heom_bath;

/* Per-solve statistics (one per batch column). */
typedef struct {
    int iterations;    /* Krylov iterations (inner ones summed over refinement sweeps) */
    int refinements;   /* FP64 refinement sweeps (0 for HEOM_FP64 / HEOM_FP32)          */
    double residual;   /* final FP64 residual, as defined by the solver                */
    int status;        /* heom_status of this column                                   */
} heom_solve_stats;

/* ---------------------------------------------------------------- exponents (host) */

/* Pade ([N-1/N], pade = 1) or Matsubara (pade = 0) constants of the Fermi (fermi = 1) or
 * Bose (fermi = 0) function: 1/(e^x+1) ~ 1/2 - sum_j 2 kappa_j x/(x^2+zeta_j^2) and
 * 1/(e^x-1) ~ 1/x - 1/2 + sum_j 2 kappa_j x/(x^2+zeta_j^2) (Methods, the two Pade forms;
 * the constants are from the Pade spectrum decomposition the paper cites). kappa, zeta:
 * caller arrays of n_poles doubles. n_poles in [0, 2000]. */
heom_status heom_pade_constants(int n_poles, int fermi, int pade, double *kappa, double *zeta);

/* Drude-Lorentz bosonic bath J(w) = 4 lam W w / (w^2 + W^2) (Methods, Eq. Drude-Lorentz):
 * xi_1 = lam W [cot(W/2kT) - i], chi_1 = W; xi_l = -2 kappa_l kT 2 lam W zeta_l kT /
 * (W^2 - (zeta_l kT)^2), chi_l = zeta_l kT. Writes n_poles+1 entries to xi and chi (RI
 * kind exponents). kT > 0, W > 0. */
heom_status heom_exp_drude_lorentz(double lam, double W, double kT, int n_poles, int pade,
                                   heom_c64 *xi, heom_c64 *chi);

/* Lorentzian fermionic lead J(w) = Gamma W^2/((w-mu)^2 + W^2) (Methods, Eq. Lorentz):
 * eta_1 = (Gamma W/2) n(iW/kT) with n the Pade (or Matsubara) Fermi function,
 * gamma_1 = W - nu i mu; eta_h = -i kappa_h kT Gamma W^2/(W^2 - (zeta_h kT)^2),
 * gamma_h = zeta_h kT - nu i mu. Writes n_poles+1 entries to eta and gamma. nu = +1 | -1. */
heom_status heom_exp_lorentz_fermion(double Gamma, double W, double mu, double kT,
                                     int n_poles, int pade, int nu,
                                     heom_c64 *eta, heom_c64 *gamma);

/* ---------------------------------------------------------------- hierarchy */

/* Enumerate the ADOs (Eq. HEOM multi-indices, Pauli exclusion for fermions, truncation at
 * tier_b / tier_f), build the neighbour and sign tables of M for parity p = +1 (even) or
 * -1 (odd), and copy tables, operators and coefficients to the current CUDA device.
 * H: d x d Hermitian system Hamiltonian. flags: 0. On success *out owns everything.
 * Errors: HEOM_EINVAL for d < 1, tiers < 0, non-finite inputs, a non-involutive partner
 * map, nu not +-1, more than 64 fermionic exponents; HEOM_ENOMEM; HEOM_ECUDA. */
heom_status heom_build_hierarchy(int d, const heom_c64 *H, int n_baths, const heom_bath *baths,
                                 int tier_b, int tier_f, int parity, int flags,
                                 heom_hier **out);

/* heom_build_hierarchy with importance pruning (Eq. importance): of the full hierarchy, keep
 * every ADO at levels (m, n) in {0, 1} x {0, 1} and every other ADO whose importance
 *   I = |prod_r xi_{j_r} / (Re chi_{j_r} sum_{x<=r} Re chi_{j_x})|
 *     x |prod_w eta_{q_w} / (Re gamma_{q_w} sum_{x<=w} Re gamma_{q_x})|
 * reaches importance_th. The members of j and q are taken in ascending exponent order (the
 * order that reproduces the paper's Table 3 counts); a zero denominator counts as infinite
 * importance. The kept ADOs stay in canonical order and are numbered 0 .. N-1; couplings
 * to dropped ADOs are left out (a dropped ADO is zero). The importance uses the exponents
 * given here: later heom_set_params calls change values, not the kept set.
 * importance_th = 0 is heom_build_hierarchy. Errors as heom_build_hierarchy, plus HEOM_EINVAL
 * for a negative or non-finite threshold or a full hierarchy above 2^29 ADOs. */
heom_status heom_build_hierarchy_pruned(int d, const heom_c64 *H, int n_baths,
                                        const heom_bath *baths, int tier_b, int tier_f,
                                        int parity, double importance_th, heom_hier **out);

/* Number of ADOs the hierarchy of these baths has at tiers tier_b / tier_f after importance
 * pruning at importance_th (0: no pruning), on the host, without building it (Table 3's
 * counts). Only the kinds, exponent counts, coefficients and rates of the baths are read.
 * Errors: HEOM_EINVAL for bad arguments or more than 4e10 ADOs to rate. */
heom_status heom_count_ados(int n_baths, const heom_bath *baths, int tier_b, int tier_f,
                            double importance_th, int64_t *count);

/* Replace the parameter sets of a hierarchy by n_sets sets that share its structure
 * (operators, exponent kinds, nu, partner map, tiers) and differ in H and in the
 * exponent values: H [n_sets][d][d], coef [n_sets][K], rate [n_sets][K] with K = K_b + K_f
 * in the global exponent order. Batch column b of every later call then uses parameter
 * set b / (batch / n_sets); batch must be a multiple of n_sets. */
heom_status heom_set_params(heom_hier *h, int n_sets, const heom_c64 *H,
                            const heom_c64 *coef, const heom_c64 *rate);

/* Per-set truncation: parameter set s (heom_set_params) keeps only the ADOs with bosonic
 * tier <= tier_b[s] and fermionic tier <= tier_f[s] (host arrays of n_sets entries, each at
 * most the hierarchy's own tiers) and holds every other ADO at zero. The hierarchy truncated
 * at tiers (t_b, t_f) is the restriction of this one to those ADOs (in the same relative
 * canonical order; for a single kind of bath they are the leading ADOs; truncation (Eq. HEOM)
 * drops exactly the couplings into the dropped tiers), so every later call -- apply, RK4,
 * stationary states, spectra -- computes
 * set s's own, shallower hierarchy, and parameter sets of different depths share one batched
 * call. Input vectors must be zero beyond a set's tiers (the solvers' are); the apply writes
 * zero there and reads nothing there. Tables are not rebuilt. NULL, NULL removes the truncation; heom_set_params
 * removes it too. Errors: HEOM_EINVAL for tiers out of range or one NULL array. */
heom_status heom_set_truncation(heom_hier *h, const int *tier_b, const int *tier_f);

/* Lindblad terms (Eq. Lindbladian, J(F)[X] = F X F^dagger - 1/2 {F^dagger F, X}): replace
 * the hierarchy's jump operators by n_ops operators F [n_ops][d][d] (row-major, host) with
 * real rates gamma [n_ops] (host). Every later call then adds
 *   sum_k gamma_k J(F_k)[X]
 * to the equation of every ADO X, in every parameter set and in either parity, without
 * adding ADOs (the weakly coupled baths the terms stand for carry no hierarchy). The
 * operators survive heom_set_params. n_ops = 0 removes them. The arrays are copied.
 * Errors: HEOM_EINVAL for n_ops < 0, NULL arrays with n_ops > 0, non-finite entries, or jump
 * operators so dense that the system superoperator exceeds 2^22 element terms (the previous
 * operators then stay); HEOM_ENOMEM; HEOM_ECUDA. */
heom_status heom_set_lindblad(heom_hier *h, int n_ops, const heom_c64 *F, const double *gamma);

/* Sizes: number of ADOs, system dimension, bosonic / fermionic exponent counts, number of
 * parameter sets, number of neighbour-table entries. Any pointer may be NULL. */
heom_status heom_hier_info(const heom_hier *h, int64_t *n_ado, int *d, int *k_b, int *k_f,
                           int *n_sets, int64_t *n_entries);

/* Hierarchy dictionary (Fig. 1e). occ: K_b bosonic occupations then K_f fermionic 0/1
 * occupations. heom_ado_index returns -1 in *idx for a multi-index outside the hierarchy. */
heom_status heom_ado_index(const heom_hier *h, const int *occ, int64_t *idx);
heom_status heom_ado_label(const heom_hier *h, int64_t idx, int *occ_out);

/* Export the neighbour and sign tables (host copies, for inspection and tests).
 * For ADO i the entries row_ptr[i] .. row_ptr[i+1]-1 each describe one term of Eq. HEOM:
 *   (M X)_i += -i ( mult_l * a * O X_nb  +  mult_r * b * X_nb O )
 * with exponent k, dir = +1 when X_nb is the ADO raised in k (A or B term: a = b = 1,
 * O = V_k or d_k^{-nu_k}) and dir = -1 when it is lowered in k (D or C term: bosonic
 * (a, b) = (c, c) | (ic, -ic) | (xi, xi^*) for kinds R | I | RI, O = V_k; fermionic
 * a = eta_k, b = conj(eta_partner(k)), O = d_k^{nu_k}). The integers carry the tier
 * multiplicity m_k, the parity sign (-1)^{delta_{p,-}}, the ordering sign
 * (-1)^{#{r in S : r < k}} and the P_s sign p (-1)^n. Arrays: row_ptr [N+1]; nb, k, dir,
 * mult_l, mult_r [n_entries]. */
heom_status heom_export_tables(const heom_hier *h, int32_t *row_ptr, int32_t *nb, int32_t *k,
                               int32_t *dir, int32_t *mult_l, int32_t *mult_r);

void heom_destroy(heom_hier *h);

/* Solver workspaces (Krylov bases and vectors, up to gigabytes) of destroyed hierarchies are
 * kept in a process-wide cache per device, at most 8 buffers, and reused by later solves of
 * any hierarchy on that device: cudaFree of such buffers is slow and synchronises the device.
 * This call frees every cached buffer. A workspace allocation that fails frees the device's
 * cached buffers and tries again by itself. Call it only while no library call is running. */
heom_status heom_release_workspace_cache(void);

/* Bound, in SM clock cycles, of every device-side wait the library's kernels make: the grid
 * barriers of the persistent stationary-state and spectrum solvers, the only spin-waits in
 * the library. cycles <= 0 restores the default, 4e9 (about 2 s at 2 GHz). A wait that runs
 * out raises a flag on which every CTA of the launch leaves its wait, the launch ends, and
 * the call returns HEOM_ETIMEOUT with its statistics filled (stationary state: the true
 * residual of the current iterate per column; spectrum: status HEOM_ETIMEOUT per
 * frequency); the device and the hierarchy stay usable. Process-wide, read at each launch.
 * For tests of this failure path and for callers that need a tighter bound. The paper has no
 * counterpart. */
heom_status heom_set_wait_limit(int64_t cycles);

/* Message of the last error on the calling thread ("" if none). */
const char *heom_last_error(void);

/* ---------------------------------------------------------------- apply (the hot path) */

/* y = M x for every batch column (Eq. HEOM right-hand side), matrix-free.
 * x, y: device ADO vectors [N][d][d][batch], complex128 (prec = HEOM_FP64) or complex64
 * (prec = HEOM_FP32); must not overlap. batch >= 1 and a multiple of n_sets.
 * Enqueued on stream s; returns without synchronising. */
heom_status heom_apply(const heom_hier *h, const void *x, void *y, int64_t batch, int prec,
                       heom_stream s);

/* ---------------------------------------------------------------- solvers */

/* RK4 time evolution d/dt x = M x (fixed step dt, n_steps steps) of every batch column.
 * ados: device ADO vector, in: state at t0, out: state at t0 + n_steps dt, complex128
 * (HEOM_FP64) or complex64 (HEOM_FP32). If rho_traj is not NULL it receives the tier-0
 * block (rho_sys, all batch columns) at steps 0, save_every, 2 save_every, ...:
 * n_steps / save_every + 1 device blocks of [d][d][batch], same precision as ados.
 * Library workspace is allocated on first use and kept in h. Synchronises s. */
heom_status heom_evolve(heom_hier *h, void *ados, int64_t batch, double dt, int64_t n_steps,
                        int64_t save_every, void *rho_traj, int prec, heom_stream s);

/* Time-dependent system Hamiltonian H_s(t) (Eq. H_total; the commutator L_s(t) = [H_s(t), .]
 * of Eq. HEOM acts on every ADO): H_s(t) = H + sum_k f_k(t) H_k, with H the hierarchy's
 * Hamiltonian (of each parameter set) and H_k the n_drive operators given here
 * ([n_drive][d][d], row-major, host; copied). The scalar functions f_k are supplied per call
 * to heom_evolve_td; every other call (apply, evolve, solvers, spectra) uses f_k = 0.
 * n_drive = 0 removes them. Errors: HEOM_EINVAL for n_drive outside [0, 64], NULL operators
 * with n_drive > 0 or non-finite entries (the previous operators then stay); HEOM_ENOMEM;
 * HEOM_ECUDA. */
heom_status heom_set_drive(heom_hier *h, int n_drive, const heom_c64 *Hk);

/* heom_evolve with H_s(t) = H + sum_k f_k(t) H_k (heom_set_drive). f: host array
 * [n_drive][2 n_steps + 1], f[k][j] = f_k(t0 + j dt / 2) for the start time t0 of the call;
 * stage 1 of step n (n = 0 .. n_steps-1) uses sample 2n, stages 2 and 3 sample 2n + 1 and
 * stage 4 sample 2n + 2 (classical RK4 evaluates the right-hand side at t, t + dt/2 twice and
 * t + dt). f may be NULL when the hierarchy has no drive operators. Other arguments, layout
 * and errors as heom_evolve, plus HEOM_EINVAL for a non-finite f. Allocates the drive table
 * and the values of up to 1,025 samples on the device. Synchronises s. */
heom_status heom_evolve_td(heom_hier *h, void *ados, int64_t batch, double dt, int64_t n_steps,
                           const double *f, int64_t save_every, void *rho_traj, int prec,
                           heom_stream s);

/* heom_evolve without any allocation. The paper has no counterpart: this serves callers
 * that cannot let a library call cudaMalloc or cudaFree -- a process whose device memory is
 * held by another allocator (a framework's caching pool, a fixed budget) can see cudaMalloc
 * fail, and cudaFree waits for the whole device. Same arguments, layout and results as
 * heom_evolve, but the three RK4 stage buffers come from one static 16 MiB device array of
 * the library, so 3 * N * d * d * batch * (16 bytes for HEOM_FP64, 8 for HEOM_FP32) must not
 * exceed 16 MiB; larger requests return HEOM_EINVAL and allocate nothing. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current). Under the CUDA runtime's lazy module loading (the default since CUDA 12.2) that
 * lookup is what makes the runtime reserve the 16 MiB on that device, which it then holds
 * until the process exits; if the device has no room left the call returns HEOM_ENOMEM.
 * So make one call with n_steps = 0 on each device at start-up, before the other allocator
 * fills device memory and before any stream capture. All calls share the one array: calls
 * whose work overlaps on the GPU (other threads, other streams) race on it and must be
 * serialised by the caller. Synchronises s. */
heom_status heom_evolve_noalloc(heom_hier *h, void *ados, int64_t batch, double dt,
                                int64_t n_steps, int64_t save_every, void *rho_traj, int prec,
                                heom_stream s);

/* Stationary state of every batch column: M x = 0 with Tr rho_sys = 1 (package
 * architecture: stationary states by a linear solve; the trace condition is added to the
 * (0,0) equation of the tier-0 ADO, which M leaves redundant because it preserves the
 * trace). x0: optional device warm start (complex128, NULL for a cold start); a column whose
 * x0 has a residual ||b - A x0|| above ||b|| starts from zero instead. x_out:
 * device complex128 [N][d][d][batch]. Converged when ||M x||_2 / ||x||_2 <= tol for x
 * normalised to Tr rho_sys = 1. prec: HEOM_FP64 (FP64 BiCGStab; a single column runs in one
 * cooperative launch whose applies are float-float), HEOM_FP64_STRICT (FP64 BiCGStab, FP64
 * applies everywhere) or HEOM_MIXED (FP32 BiCGStab corrections inside FP64 iterative
 * refinement). stats: host array of
 * batch entries or NULL. Returns HEOM_ENOCONV if any column missed tol within max_iter
 * Krylov iterations. Synchronises s. */
heom_status heom_steady(heom_hier *h, const void *x0, void *x_out, int64_t batch, double tol,
                        int max_iter, int prec, heom_solve_stats *stats, heom_stream s);

/* Density of states of the fermionic mode op_d (Methods, numerical computation of the
 * spectrum): for every omega, (M + i w) x_+ = d^dag rho and (M - i w) x_- = d rho with M
 * of the odd-parity hierarchy `odd` and b built from every ADO of the even stationary
 * state ss_ados (device complex128 [N][d][d], batch 1); pi A(w) = -Re{Tr[d x_+,0] +
 * Tr[d^dag x_-,0]}. op_d: host d x d. omega: host [n_omega]; A_out: host [n_omega].
 * Converged when ||b - (M -+ i w) x|| / ||b|| <= tol. prec: HEOM_FP64 or HEOM_MIXED (one
 * BiCGStab solve per frequency and sign, batched as columns, as for heom_steady) or
 * HEOM_SHIFTED (two Arnoldi processes, one per sign, up to max_iter steps; the residual of
 * each frequency is the least-squares residual of its shifted Hessenberg problem, which
 * equals ||b - (M -+ i w) x|| up to the rounding of the Arnoldi relation; the basis is kept
 * within 60 % of the free device memory, which may lower max_iter).
 * Parameter sets (HEOM_SHIFTED only): when `odd` holds n_sets > 1 sets (heom_set_params),
 * ss_ados is [N][d][d][n_sets] (set s's stationary state in column s), every set gets its own
 * pair of Arnoldi processes, A_out is [n_sets][n_omega] and stats run set by set.
 * stats: host array of 2*n_omega*n_sets entries (per set: x_+ then x_-) or NULL.
 * Synchronises s. */
heom_status heom_spectrum(heom_hier *odd, const void *ss_ados, const heom_c64 *op_d,
                          const double *omega, int64_t n_omega, double tol, int max_iter,
                          double *A_out, int prec, heom_solve_stats *stats, heom_stream s);

/* Densities of states of n_hier odd-parity hierarchies of different shapes (tiers, exponent
 * counts, d) on one frequency grid (Methods, spectrum). Hierarchy h takes its stationary
 * state ss_ados[h] (device, [N_h][d_h][d_h][n_sets_h]) and its mode op_d[h] (host,
 * d_h x d_h). Each hierarchy is the heom_spectrum call with the same tol, max_iter and
 * prec; the calls run one after the other on s, and each fills the GPU (parameter sets of
 * one structure belong in one hierarchy, where they share one launch). Outputs are
 * concatenated in hierarchy order: A_out (host) holds n_sets_h rows of n_omega per
 * hierarchy; stats (host, or NULL) holds 2 * n_omega * n_sets_h entries per hierarchy. A
 * solver status (HEOM_ENOCONV, HEOM_EBREAKDOWN) of one hierarchy does not stop the others,
 * and the first status other than HEOM_OK is returned; an argument, memory or CUDA error
 * stops at that hierarchy (HEOM_EINVAL before any solve when the arrays are invalid).
 * Synchronises s. */
heom_status heom_spectrum_batched(int n_hier, heom_hier *const *odd, const void *const *ss_ados,
                                  const heom_c64 *const *op_d, const double *omega,
                                  int64_t n_omega, double tol, int max_iter, double *A_out,
                                  int prec, heom_solve_stats *stats, heom_stream s);

/* Power spectral density of the mode op_a (Methods, numerical computation of the spectrum,
 * bosonic case): pi S(w) = -Re Tr[a^dag x_0] with (M - i w) x = a rho over every ADO, M of the
 * even-parity hierarchy `even` whose stationary state is ss_ados (device complex128
 * [N][d][d][n_sets]). Solved by the shift-invariant Krylov method of HEOM_SHIFTED (one
 * process per parameter set serves every frequency). op_a: host d x d; omega: host
 * [n_omega]; S_out: host [n_sets][n_omega]; stats: host [n_sets][n_omega] or NULL.
 * Converged when the residual estimate ||b - (M - i w) x|| / ||b|| <= tol. At w = 0 the
 * system is singular (M has the stationary state as null vector) unless Tr[a rho] = 0;
 * such a frequency returns HEOM_ENOCONV in its stats. Synchronises s. */
heom_status heom_psd(heom_hier *even, const void *ss_ados, const heom_c64 *op_a, const double *omega,
                     int64_t n_omega, double tol, int max_iter, double *S_out,
                     heom_solve_stats *stats, heom_stream s);

/* Autotuner of the apply for one batch width (measurement of this GPU; the paper has no
 * counterpart). Times heom_apply on a library-allocated test vector of `batch` columns in
 * precision prec with the per-element kernel and with the tiled kernel at 1..5 ADO ranges
 * per SM -- in FP32 each with every kernel variant (columns per lane / terms per item in
 * flight / items per warp in flight / CTAs per SM the registers are sized for -- 0: 2/4/1/3;
 * 1: 2/4/1/4; 2: 2/3/1/4; 3: 2/2/1/5; 4: 2/6/1/3; 5: 4/4/1/2) -- and keeps the fastest in h: the tiled granularity and variant for every later
 * batched apply and solve, or, when the per-element kernel wins, the per-element kernel for
 * batches up to `batch` columns. candidates_us: host [6] or NULL (index 0 per-element,
 * p = 1..5 the fastest variant of the tiled kernel with p ranges per SM, -1 where not
 * applicable); tiled, ctas_per_sm, best_us, variant (-1 when the per-element kernel won):
 * host or NULL. Results do not depend on the granularity (the same terms, summed in the
 * same order); the tiled and per-element kernels agree to rounding. Allocates two vectors
 * of N d^2 batch elements for the duration of the call. Synchronises s. */
heom_status heom_autotune(heom_hier *h, int64_t batch, int prec, double *candidates_us,
                          int *tiled, int *ctas_per_sm, double *best_us, int *variant,
                          heom_stream s);

/* Pin the configuration the autotuner would choose (the paper has no counterpart): the
 * tiled kernel for every batch of 16 or more columns, at ctas_per_sm ADO ranges per SM
 * (1..5) and FP32 variant `variant` (0..5, as listed for heom_autotune; FP64 ignores it). For
 * reproducible timings and for tests of each variant. Results agree with every other
 * configuration to rounding. Errors: HEOM_EINVAL for arguments out of range. */
heom_status heom_set_tile_config(heom_hier *h, int ctas_per_sm, int variant);

/* Electronic current into lead alpha (Methods, electronic current; e = 1):
 * <I_alpha> = Re( i sum_q s_q Tr[d^{-nu_q} rho_q] ) over the fermionic exponents q of the
 * baths that form the lead, rho_q the tier-1 ADO with S = {q} (bosonic occupations zero),
 * s_q = +1 for nu = +1 and -1 for nu = -1 ((-1)^{delta_{nu,-}}). x: device complex128
 * [N][d][d][batch] stationary states of the even-parity hierarchy h (columns = parameter
 * sets or repeats); baths: host [n_baths] indices of the lead's baths in the order given
 * to heom_build_hierarchy; I_out: host [batch]. heom_conductance forms conductances from
 * currents at neighbouring biases. Synchronises s. */
heom_status heom_current(const heom_hier *h, const void *x, int64_t batch, const int *baths,
                         int n_baths, double *I_out, heom_stream s);

/* Differential conductance G = dI_alpha / dPhi (Methods, electronic current; Example 1's
 * conductance) as difference quotients over bias pairs: h holds 2 P parameter sets
 * (heom_set_params), set 2k at bias Phi_k and set 2k + 1 at Phi_k + dphi[k] (the exponents of
 * the leads follow the bias through their chemical potentials). One batched stationary solve
 * of all 2 P sets (tol, max_iter, prec as heom_steady), the current of the lead made of
 * `baths` for every set (as heom_current), then G_out[k] = (I_{2k+1} - I_{2k}) / dphi[k].
 * dphi: host [P], finite and non-zero; G_out: host [P]; I_out: host [2 P] or NULL; stats:
 * host [2 P] or NULL (the stationary solves). Allocates the 2 P stationary states for the call.
 * Returns heom_steady's status (the quotients are still formed on HEOM_ENOCONV /
 * HEOM_EBREAKDOWN: see stats). Synchronises s. */
heom_status heom_conductance(heom_hier *h, const double *dphi, const int *baths, int n_baths,
                             double tol, int max_iter, int prec, double *G_out, double *I_out,
                             heom_solve_stats *stats, heom_stream s);

/* ---------------------------------------------------------------- learned warm start */

/* A multilayer perceptron trained on stationary states the library computes, predicting the
 * reduced density matrix and the first-tier ADOs of a model from its physical parameters;
 * the prediction seeds heom_steady (x0). The paper has no counterpart: it solves every
 * stationary state from scratch. Layers: width[0] inputs -> ... -> width[n_layers] outputs,
 * tanh on hidden layers, linear output. Every matrix product rounds both operands to BF16
 * and accumulates in FP32 (tensor cores); parameters, activations, gradients and the Adam
 * state are FP32. Inputs and targets are standardised ((v - mean) / sd) inside the network;
 * the loss is the mean squared error of the standardised targets. Parameters are one flat
 * FP32 array: for each layer W ([in][out], row-major) then b ([out]). The network lives on
 * the device that is current at creation; all pointers below are device pointers unless
 * marked host. Not thread-safe per network. */
typedef struct heom_mlp heom_mlp;

/* widths: host [n_layers + 1], each 1..65536; 1 <= n_layers <= 16. Weights Glorot-uniform
 * from a splitmix64 stream started at seed, biases zero, identity standardisation. */
heom_status heom_mlp_create(int n_layers, const int *widths, uint64_t seed, heom_mlp **out);
void heom_mlp_destroy(heom_mlp *net);
heom_status heom_mlp_info(const heom_mlp *net, int64_t *n_params, int *n_in, int *n_out);
/* host arrays: in_mean/in_sd [n_in], out_mean/out_sd [n_out]; deviations > 0 */
heom_status heom_mlp_set_standardisation(heom_mlp *net, const float *in_mean, const float *in_sd,
                                         const float *out_mean, const float *out_sd);
/* flat FP32 parameters, host [n_params] */
heom_status heom_mlp_get_params(const heom_mlp *net, float *host_out);
heom_status heom_mlp_set_params(heom_mlp *net, const float *host_in);
/* y [batch][n_out] = net(x [batch][n_in]) in raw (de-standardised) units */
heom_status heom_mlp_forward(heom_mlp *net, const float *x, float *y, int64_t batch, heom_stream s);
/* Gradient of the loss with respect to the flat parameters for inputs x [batch][n_in] and
 * raw targets t [batch][n_out]: grad_out (device [n_params], or NULL) and the loss (host,
 * or NULL; synchronises s when given). */
heom_status heom_mlp_gradients(heom_mlp *net, const float *x, const float *t, int64_t batch,
                               float *grad_out, double *loss, heom_stream s);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) at learning rate lr on
 * the gradient of (x, t); loss as in heom_mlp_gradients, before the step. */
heom_status heom_mlp_train_step(heom_mlp *net, const float *x, const float *t, int64_t batch,
                                float lr, double *loss, heom_stream s);
/* Warm-start features of n_sets states x (device complex128 [N][d][d][n_sets], columns =
 * parameter sets) into f (device FP32 [n_sets][n_features]): rho_sys as d diagonal reals,
 * then Re and Im of rho[i][j] for i < j in row-major order (d^2 reals), then every tier-1
 * ADO of h in hierarchy order, its d^2 elements row-major with Re and Im interleaved.
 * n_features must equal d^2 (1 + 2 x number of tier-1 ADOs). Synchronises s. */
heom_status heom_warm_start_features(const heom_hier *h, const void *x, int64_t n_sets, float *f,
                                     int n_features, heom_stream s);
/* x_out (device complex128 [N][d][d][n_sets]) = the ADO vector the network predicts for
 * the parameter rows params (device FP32 [n_sets][n_in]): rho_sys (Hermitian) and the
 * tier-1 ADOs from the features above, every other ADO zero. Synchronises s. */
heom_status heom_warm_start(const heom_hier *h, heom_mlp *net, const float *params, int64_t n_sets,
                            void *x_out, heom_stream s);

/* Selected elements as features: f (device FP32 [n_sets][2 n_elems]) holds Re and Im of
 * element elems[k] (device int64 [n_elems], flat indices n d^2 + r d + c of the ADO vector) of
 * every column of x (device complex128 [N][d][d][n_sets]). A network that predicts them can
 * cover whole ADO vectors: the elements a caller lists are those that vary over its training
 * states (the others vanish in every state, by the symmetry of the model). Synchronises s. */
heom_status heom_gather_elements(const heom_hier *h, const void *x, int64_t n_sets,
                                 const int64_t *elems, int64_t n_elems, float *f, heom_stream s);
/* x_out (device complex128 [N][d][d][n_sets]) = the network's prediction for the parameter
 * rows params (device FP32 [n_sets][n_in]) written to the listed elements (layout as
 * heom_gather_elements; the network has 2 n_elems outputs), every other element zero: a
 * whole-vector warm start for heom_steady. Synchronises s. */
heom_status heom_warm_start_elements(const heom_hier *h, heom_mlp *net, const float *params,
                                     int64_t n_sets, const int64_t *elems, int64_t n_elems,
                                     void *x_out, heom_stream s);

/* ---------------------------------------------------------------- launch accounting */

/* Measurement support for benchmarks; the paper has no counterpart. While enabled, every
 * kernel the library launches is counted in one of these classes and bracketed by a pair of
 * CUDA events on its stream. heom_profile_read waits for those events and returns, for one
 * class, the number of launches, their summed device time in milliseconds, the work units
 * they processed (ADO-applies -- one d x d output block of one batch column -- for the apply
 * classes, vector elements for the others) and their algorithmic bytes: the compulsory
 * reads and writes of the vectors each kernel streams, one pass per vector, with the
 * neighbour re-reads of the apply counted as zero. heom_profile_enable(1) resets every
 * counter; heom_profile_enable(0) stops recording. Not thread-safe; meant for one
 * benchmarking thread. */
typedef enum {
    HEOM_KC_APPLY = 0,           /* heom_apply                                       */
    HEOM_KC_RK4 = 1,             /* fused RK4 stages (one apply each)                */
    HEOM_KC_KRYLOV_APPLY32 = 2,  /* apply + dot products inside FP32 BiCGStab         */
    HEOM_KC_KRYLOV_APPLY64 = 3,  /* FP64 BiCGStab applies; the Arnoldi applies (FP64
                                    or float-float)                                  */
    HEOM_KC_KRYLOV_VECTOR = 4,   /* BiCGStab vector updates and start-up; Arnoldi
                                    Gram-Schmidt                                      */
    HEOM_KC_RESIDUAL64 = 5,      /* FP64 residual applies (refinement, final norms)   */
    HEOM_KC_OTHER = 6,           /* right-hand sides, scaling, normalisation          */
    HEOM_KC_COUNT = 7
} heom_kernel_class;

heom_status heom_profile_enable(int on);
heom_status heom_profile_read(int cls, int64_t *launches, double *device_ms, double *units,
                              double *bytes);
/* Bytes the library copied host -> device and device -> host while accounting was on
 * (table and parameter uploads, right-hand sides, convergence flags, results). */
heom_status heom_profile_copies(int64_t *h2d_bytes, int64_t *d2h_bytes);

/* Process-wide allocation counts since the library was loaded (always on, any pointer may
 * be NULL): device_allocs = cudaMalloc calls the library made (tables, workspaces, test
 * vectors; every device allocation of the library goes through one counted routine),
 * device_bytes = their total size, workspace_takes = times a solver workspace was grown
 * (taken from the workspace cache or newly allocated). */
heom_status heom_profile_allocs(int64_t *device_allocs, int64_t *device_bytes,
                                int64_t *workspace_takes);

#ifdef __cplusplus
}
#endif
#endif /* HEOM_H */
