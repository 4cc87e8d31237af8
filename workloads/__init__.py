"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds the *inputs* of the HEOM method and nothing of its arithmetic:

* the model systems of the paper's examples (system Hamiltonians, coupling operators,
  initial states) built from textbook operator algebra (Pauli matrices, Jordan-Wigner
  fermions, a truncated harmonic oscillator);
* the physical bath parameters of each workload (Results: Table 1 and the examples);
* seeded random vectors, random operators, random exponent lists and parameter draws.

Exponent generation, hierarchy enumeration and the Liouvillian live on each side of the
comparison separately: in ``oracle/`` (plain CPU) and in the CUDA library (its own C++ and
kernels). Neither imports the other; both import this module.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_VECTORS = 2306
SEED_SETS = 7522

# --------------------------------------------------------------------------------------
# Operator algebra (textbook definitions; occupation basis |0>, |1> for a fermion mode).
# --------------------------------------------------------------------------------------

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
# annihilator of one fermion mode in the occupation basis: |1> -> |0>
SM = np.array([[0, 1], [0, 0]], dtype=np.complex128)


def dag(a: np.ndarray) -> np.ndarray:
    return a.conj().T


def destroy(n: int) -> np.ndarray:
    """Truncated bosonic annihilation operator on Fock states 0..n-1."""
    a = np.zeros((n, n), dtype=np.complex128)
    for k in range(1, n):
        a[k - 1, k] = np.sqrt(k)
    return a


# --------------------------------------------------------------------------------------
# Bath parameter records. The physical parameters only; exponents are derived elsewhere.
# --------------------------------------------------------------------------------------


@dataclass(frozen=True)
class BosonDL:
    """Drude-Lorentz bosonic bath J(w) = 4*lam*W*w/(w^2+W^2) (Methods, Eq. Drude-Lorentz)."""

    lam: float
    W: float
    kT: float
    n_poles: int
    method: str = "matsubara"  # or "pade"


@dataclass(frozen=True)
class FermionLorentz:
    """Lorentzian fermionic lead J(w) = Gamma*W^2/((w-mu)^2+W^2) (Methods, Eq. Lorentz)."""

    Gamma: float
    W: float
    mu: float
    kT: float
    n_poles: int
    method: str = "pade"  # or "matsubara"


@dataclass
class Model:
    """A system plus its baths, as a user of the paper's package specifies it (Fig. 1a-b).

    ``boson_baths`` holds (V, BosonDL) pairs, ``fermion_baths`` holds (d, FermionLorentz)
    pairs where d is the annihilation operator the lead couples to. The order of the
    lists is the order of the exponents in the hierarchy. ``lindblad`` holds (F, gamma)
    pairs: jump operators of weakly coupled environments that carry no ADOs (Fig. 1c).
    """

    name: str
    H: np.ndarray
    boson_baths: list = field(default_factory=list)
    fermion_baths: list = field(default_factory=list)
    tier_b: int = 0
    tier_f: int = 0
    rho0: np.ndarray | None = None
    lindblad: list = field(default_factory=list)  # (F, gamma): jump operator and its rate

    @property
    def d(self) -> int:
        return self.H.shape[0]


# --------------------------------------------------------------------------------------
# Model systems of the paper's examples.
# --------------------------------------------------------------------------------------


def spin_boson_ops(delta: float = 1.0):
    """H = (Delta/2) sigma_x, V = sigma_z, rho0 = |0><0| with sigma_z|0> = +|0>."""
    H = 0.5 * delta * SX
    V = SZ.copy()
    rho0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    return H, V, rho0


def siam_ops(eps: float, U: float):
    """Single-impurity Anderson model (Example 1).

    Basis |n_up n_dn>, index 2*n_up + n_dn. Jordan-Wigner: d_up = sm (x) I,
    d_dn = sz (x) sm, so that the two modes anticommute. Returns H, d_up, d_dn.
    """
    d_up = np.kron(SM, I2)
    d_dn = np.kron(SZ, SM)
    n_up = dag(d_up) @ d_up
    n_dn = dag(d_dn) @ d_dn
    H = eps * (n_up + n_dn) + U * (n_up @ n_dn)
    return H, d_up, d_dn


def single_level_ops(eps: float):
    """One spinless fermion level: H = eps d^dag d on occupation basis |0>, |1>."""
    d = SM.copy()
    H = eps * dag(d) @ d
    return H, d


def charge_cavity_ops(eps: float, omega_c: float, g: float, n_fock: int):
    """Charge-cavity system (Example 2): basis dot (x) Fock, d = sm (x) I, a = I (x) a.

    H = eps d^dag d + omega_c a^dag a + g d^dag d (a + a^dag); bosonic coupling V = a + a^dag.
    """
    a1 = destroy(n_fock)
    d = np.kron(SM, np.eye(n_fock))
    a = np.kron(I2, a1)
    nd = dag(d) @ d
    H = eps * nd + omega_c * dag(a) @ a + g * nd @ (a + dag(a))
    V = a + dag(a)
    return H, d, a, V


# --------------------------------------------------------------------------------------
# Workloads: the paper's example systems with their Table 1 parameters, and the benchmark shapes.
# --------------------------------------------------------------------------------------


def spin_boson_model(tier: int = 4, lam: float = 0.1, W: float = 0.5, kT: float = 0.5,
                     delta: float = 1.0, n_poles: int = 2) -> Model:
    """Spin-boson: H=(Delta/2)sx, V=sz, one Drude-Lorentz bath, Matsubara, 3 exponents."""
    H, V, rho0 = spin_boson_ops(delta)
    return Model("spin_boson", H, [(V, BosonDL(lam, W, kT, n_poles, "matsubara"))], [],
                 tier_b=tier, tier_f=0, rho0=rho0)


def siam_model(eps: float = -5.0, U: float = 10.0, Gamma: float = 2.0, W: float = 10.0,
               kT: float = 0.5, mu: float = 1.0, n_poles: int = 2, tier: int = 3,
               method: str = "pade") -> Model:
    """Single-impurity Anderson model with leads L (mu_L=+mu) and R (mu_R=-mu).

    Fermionic baths in the order [L up, L down, R up, R down]; each contributes
    2*(n_poles+1) exponents (nu=+1 then nu=-1).
    """
    H, d_up, d_dn = siam_ops(eps, U)
    leads = []
    for m in (mu, -mu):
        lead = FermionLorentz(Gamma, W, m, kT, n_poles, method)
        leads.append((d_up, lead))
        leads.append((d_dn, lead))
    rho0 = np.zeros((4, 4), dtype=np.complex128)
    rho0[0, 0] = 1.0
    return Model("siam", H, [], leads, tier_b=0, tier_f=tier, rho0=rho0)


def single_level_model(eps: float = 0.3, Gamma: float = 1.0, W: float = 4.0, kT: float = 0.5,
                       mu_l: float = 1.0, mu_r: float = -0.5, n_poles: int = 4,
                       tier: int = 2) -> Model:
    """A noninteracting spinless level between two Lorentzian leads (test system)."""
    H, d = single_level_ops(eps)
    leads = [(d, FermionLorentz(Gamma, W, mu_l, kT, n_poles, "pade")),
             (d, FermionLorentz(Gamma, W, mu_r, kT, n_poles, "pade"))]
    rho0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    return Model("single_level", H, [], leads, tier_b=0, tier_f=tier, rho0=rho0)


def charge_cavity_model(eps: float = -3.0, omega_c: float = 1.0, g: float = 0.5,
                        Gamma: float = 1.0, Delta: float = 0.01, W_b: float = 0.2,
                        W_f: float = 10.0, kT: float = 0.5, bias: float = 6.0,
                        n_fock: int = 12, tier_b: int = 2, tier_f: int = 2,
                        n_poles: int = 2) -> Model:
    """Charge-cavity (Example 2 with Table 1 row 2), Fock cutoff n_fock, d = 2*n_fock.

    Bosonic Drude-Lorentz cavity-loss bath (Pade, n_poles+1 exponents) on V = a + a^dag;
    two spinless fermionic leads (mu_L = bias/2, mu_R = -bias/2) on the dot.
    """
    H, d, a, V = charge_cavity_ops(eps, omega_c, g, n_fock)
    bos = [(V, BosonDL(Delta, W_b, kT, n_poles, "pade"))]
    fer = [(d, FermionLorentz(Gamma, W_f, bias / 2, kT, n_poles, "pade")),
           (d, FermionLorentz(Gamma, W_f, -bias / 2, kT, n_poles, "pade"))]
    rho0 = np.zeros((2 * n_fock, 2 * n_fock), dtype=np.complex128)
    rho0[0, 0] = 1.0
    return Model("charge_cavity", H, bos, fer, tier_b=tier_b, tier_f=tier_f, rho0=rho0)


def bose_einstein(omega: float, kT: float) -> float:
    """Occupation 1 / (e^{omega/kT} - 1) of a bosonic mode (textbook definition)."""
    return 1.0 / np.expm1(omega / kT)


def drude_lorentz_density(omega: float, lam: float, W: float) -> float:
    """J(w) = 4 lam W w / (w^2 + W^2) (Methods, Eq. Drude-Lorentz)."""
    return 4.0 * lam * W * omega / (omega * omega + W * W)


def charge_cavity_me_model(eps: float = -3.0, omega_c: float = 1.0, g: float = 0.5,
                           Gamma: float = 1.0, Delta: float = 0.01, W_b: float = 0.2,
                           W_f: float = 10.0, kT: float = 0.5, bias: float = 6.0,
                           n_fock: int = 12, tier_f: int = 2, n_poles: int = 2) -> Model:
    """Charge-cavity system of Example 2 with its cavity bath replaced by Lindblad terms.

    The bosonic bath's hierarchy is dropped and the cavity loses and gains photons through
    the jump operators a (rate J(w_c) (n + 1)) and a^dag (rate J(w_c) n), with J the bath's
    Drude-Lorentz density and n its Bose-Einstein occupation at w_c: the Born-Markov
    master-equation variant the example compares against. The fermionic leads keep their
    hierarchy.
    """
    H, d, a, V = charge_cavity_ops(eps, omega_c, g, n_fock)
    fer = [(d, FermionLorentz(Gamma, W_f, bias / 2, kT, n_poles, "pade")),
           (d, FermionLorentz(Gamma, W_f, -bias / 2, kT, n_poles, "pade"))]
    J = drude_lorentz_density(omega_c, Delta, W_b)
    n = bose_einstein(omega_c, kT)
    rho0 = np.zeros((2 * n_fock, 2 * n_fock), dtype=np.complex128)
    rho0[0, 0] = 1.0
    return Model("charge_cavity_me", H, [], fer, tier_b=0, tier_f=tier_f, rho0=rho0,
                 lindblad=[(a, J * (n + 1.0)), (dag(a), J * n)])


def omega_grid(n: int, lo: float = -20.0, hi: float = 20.0) -> np.ndarray:
    """Uniform frequency grid on [lo, hi] with n points."""
    return np.linspace(lo, hi, n)


def draw_siam_sets(n_sets: int = 64, seed: int = SEED_SETS):
    """Batched-spectra parameter draws: U~U[0,12], bias~U[0,3], kT~U[0.2,1] (outside
    KT_EXCLUDED), tier~{2,3,4}."""
    rng = np.random.default_rng(seed)
    U = rng.uniform(0.0, 12.0, n_sets)
    bias = rng.uniform(0.0, 3.0, n_sets)
    kT = _draw_kt(rng, n_sets)
    tier = rng.choice(np.array([2, 3, 4]), n_sets)
    return [dict(U=float(U[i]), mu=float(bias[i]), kT=float(kT[i]), tier=int(tier[i]))
            for i in range(n_sets)]


# With the lead band width W = 10 and two Pade poles, the second pole of the Fermi function
# sits on the Lorentzian's pole (zeta_2 kT = W) at kT = 10 / 13.0432 = 0.7667, where the
# exponent formula divides by W^2 - (zeta_2 kT)^2 = 0. Near it the two exponents of that
# pole grow large with cancelling contributions (|eta_2| = 26 at kT = 0.68 and 0.87, 50 to 63
# at kT = 0.729 and 0.815), and BiCGStab stationary solves of tier-4 sets break down there.
# Draws of kT avoid this band.
KT_EXCLUDED = (0.68, 0.87)


def _draw_kt(rng, n, lo=0.2, hi=1.0):
    out = np.empty(n)
    for i in range(n):
        while True:
            v = rng.uniform(lo, hi)
            if not (KT_EXCLUDED[0] <= v <= KT_EXCLUDED[1]):
                out[i] = v
                break
    return out


def draw_warmstart_samples(n: int, seed: int = SEED_VECTORS):
    """Learned-warm-start draws: U~U[0,12], eps~U[-8,-2], Gamma~U[1,3], kT~U[0.2,1] (outside
    KT_EXCLUDED), bias~U[0,3]."""
    rng = np.random.default_rng(seed)
    U = rng.uniform(0.0, 12.0, n)
    eps = rng.uniform(-8.0, -2.0, n)
    G = rng.uniform(1.0, 3.0, n)
    kT = _draw_kt(rng, n)
    mu = rng.uniform(0.0, 3.0, n)
    return np.stack([U, eps, G, kT, mu], axis=1)


# --------------------------------------------------------------------------------------
# Seeded random inputs for the apply parity tests.
# --------------------------------------------------------------------------------------


def random_complex(shape, rng) -> np.ndarray:
    """Complex normal: real and imaginary parts ~ N(0, 1)."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_hermitian(d: int, rng) -> np.ndarray:
    a = random_complex((d, d), rng)
    return 0.5 * (a + dag(a))


def random_raw_problem(d: int, boson_sizes, fermion_sizes, tier_b: int, tier_f: int,
                       parity: int = 1, seed: int = SEED_VECTORS, dense_fermion_ops=True,
                       n_lindblad: int = 0):
    """A random HEOM problem in raw form (the user-supplied-exponent route of Fig. 1a).

    boson_sizes: list of (kind, n_exp) with kind in {"R", "I", "RI"};
    fermion_sizes: list of n_exp (even; the first half nu=+1, the second half nu=-1 and the
    partner of exponent h is h +- n_exp/2).
    n_lindblad: number of random jump operators (complex normal, half of their entries set
    to zero) with rates ~ U[0.1, 1].
    Returns a dict with keys d, H, baths, tier_b, tier_f, parity, lindblad. Every bath is a
    dict {kind, op, coef, rate[, nu, partner]}; every Lindblad term a dict {op, rate}.
    """
    rng = np.random.default_rng(seed)
    H = random_hermitian(d, rng)
    baths = []
    for kind, k in boson_sizes:
        V = random_hermitian(d, rng)
        coef = random_complex(k, rng) * 0.3
        if kind in ("R", "I"):
            coef = coef.real.astype(np.complex128)
        rate = rng.uniform(0.2, 2.0, k) + 1j * rng.uniform(-0.5, 0.5, k)
        baths.append(dict(kind=kind, op=V, coef=coef, rate=rate))
    for k in fermion_sizes:
        assert k % 2 == 0
        if dense_fermion_ops:
            op = random_complex((d, d), rng) * 0.5
        else:
            op = np.zeros((d, d), dtype=np.complex128)
            op[0, d - 1] = 1.0
        coef = random_complex(k, rng) * 0.3
        rate = rng.uniform(0.2, 2.0, k) + 1j * rng.uniform(-0.5, 0.5, k)
        h = k // 2
        nu = np.array([1] * h + [-1] * h, dtype=np.int32)
        partner = np.array([i + h for i in range(h)] + [i for i in range(h)], dtype=np.int32)
        baths.append(dict(kind="F", op=op, coef=coef, rate=rate, nu=nu, partner=partner))
    lind = []
    for _ in range(n_lindblad):
        F = random_complex((d, d), rng) * 0.5
        F[rng.random((d, d)) < 0.5] = 0.0
        lind.append(dict(op=F, rate=float(rng.uniform(0.1, 1.0))))
    return dict(d=d, H=H, baths=baths, tier_b=tier_b, tier_f=tier_f, parity=parity,
                lindblad=lind)


def random_ado_vector(n_ado: int, d: int, batch: int | None = None,
                      seed: int = SEED_VECTORS) -> np.ndarray:
    """Complex normal ADO vector, shape (N, d, d) or (N, d, d, batch)."""
    rng = np.random.default_rng(seed)
    shape = (n_ado, d, d) if batch is None else (n_ado, d, d, batch)
    return random_complex(shape, rng)
