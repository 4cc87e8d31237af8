"""Python binding of libheom.so: argument marshalling only.

Every function here forwards to the C ABI declared in ``include/heom.h`` under the same
name (without the ``heom_`` prefix). Device buffers are torch tensors (PyTorch supplies
device memory and streams); every step of the HEOM path runs in the library's CUDA kernels.
There is no fallback: if ``libheom.so`` is missing or fails to load, importing this package
raises, and every device entry point needs a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libheom.so")

if not os.path.exists(LIBRARY_PATH):
    raise ImportError(f"libheom.so is not built ({LIBRARY_PATH}); run "
                      "`python paper_2306_07522_gb300/build.py` or __graft_entry__.build()")
_lib = C.CDLL(LIBRARY_PATH)

# ------------------------------------------------------------------------- ABI types
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ENOTSUP, ETIMEOUT = range(8)
BOSON_R, BOSON_I, BOSON_RI, FERMION = range(4)
FP64, FP32, MIXED, SHIFTED, FP64_STRICT = range(5)
KERNEL_CLASSES = ("apply", "rk4", "krylov_apply_fp32", "krylov_apply_fp64", "krylov_vector",
                  "residual_fp64", "other")
APPLY_CLASSES = ("apply", "rk4", "krylov_apply_fp32", "krylov_apply_fp64", "residual_fp64")
KIND = {"R": BOSON_R, "I": BOSON_I, "RI": BOSON_RI, "F": FERMION}
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
                ENOCONV: "ENOCONV", EBREAKDOWN: "EBREAKDOWN", ENOTSUP: "ENOTSUP",
                ETIMEOUT: "ETIMEOUT"}


class c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Bath(C.Structure):
    _fields_ = [("kind", C.c_int), ("op", C.POINTER(c64)), ("n_exp", C.c_int),
                ("coef", C.POINTER(c64)), ("rate", C.POINTER(c64)),
                ("nu", C.POINTER(C.c_int)), ("partner", C.POINTER(C.c_int))]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("residual", C.c_double),
                ("status", C.c_int)]


class HeomError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.heom_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_P = C.c_void_p
_sig = {
    "heom_pade_constants": [C.c_int, C.c_int, C.c_int, _P, _P],
    "heom_exp_drude_lorentz": [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _P, _P],
    "heom_exp_lorentz_fermion": [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                 C.c_int, C.c_int, _P, _P],
    "heom_build_hierarchy": [C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                             C.POINTER(_P)],
    "heom_set_params": [_P, C.c_int, _P, _P, _P],
    "heom_set_truncation": [_P, _P, _P],
    "heom_set_lindblad": [_P, C.c_int, _P, _P],
    "heom_set_drive": [_P, C.c_int, _P],
    "heom_evolve_td": [_P, _P, C.c_int64, C.c_double, C.c_int64, _P, C.c_int64, _P, C.c_int, _P],
    "heom_build_hierarchy_pruned": [C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.POINTER(_P)],
    "heom_count_ados": [C.c_int, _P, C.c_int, C.c_int, C.c_double, _P],
    "heom_hier_info": [_P, _P, _P, _P, _P, _P, _P],
    "heom_ado_index": [_P, _P, _P],
    "heom_ado_label": [_P, C.c_int64, _P],
    "heom_export_tables": [_P, _P, _P, _P, _P, _P, _P],
    "heom_apply": [_P, _P, _P, C.c_int64, C.c_int, _P],
    "heom_evolve": [_P, _P, C.c_int64, C.c_double, C.c_int64, C.c_int64, _P, C.c_int, _P],
    "heom_evolve_noalloc": [_P, _P, C.c_int64, C.c_double, C.c_int64, C.c_int64, _P, C.c_int,
                            _P],
    "heom_steady": [_P, _P, _P, C.c_int64, C.c_double, C.c_int, C.c_int, _P, _P],
    "heom_spectrum": [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_int, _P, C.c_int, _P, _P],
    "heom_spectrum_batched": [C.c_int, _P, _P, _P, _P, C.c_int64, C.c_double, C.c_int, _P, C.c_int,
                              _P, _P],
    "heom_current": [_P, _P, C.c_int64, _P, C.c_int, _P, _P],
    "heom_psd": [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_int, _P, _P, _P],
    "heom_conductance": [_P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_int, _P, _P, _P, _P],
    "heom_autotune": [_P, C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P],
    "heom_set_tile_config": [_P, C.c_int, C.c_int],
    "heom_mlp_create": [C.c_int, _P, C.c_uint64, C.POINTER(_P)],
    "heom_mlp_info": [_P, _P, _P, _P],
    "heom_mlp_set_standardisation": [_P, _P, _P, _P, _P],
    "heom_mlp_get_params": [_P, _P],
    "heom_mlp_set_params": [_P, _P],
    "heom_mlp_forward": [_P, _P, _P, C.c_int64, _P],
    "heom_mlp_gradients": [_P, _P, _P, C.c_int64, _P, _P, _P],
    "heom_mlp_train_step": [_P, _P, _P, C.c_int64, C.c_float, _P, _P],
    "heom_warm_start_features": [_P, _P, C.c_int64, _P, C.c_int, _P],
    "heom_warm_start": [_P, _P, _P, C.c_int64, _P, _P],
    "heom_gather_elements": [_P, _P, C.c_int64, _P, C.c_int64, _P, _P],
    "heom_warm_start_elements": [_P, _P, _P, C.c_int64, _P, C.c_int64, _P, _P],
    "heom_release_workspace_cache": [],
    "heom_profile_enable": [C.c_int],
    "heom_profile_read": [C.c_int, _P, _P, _P, _P],
    "heom_profile_copies": [_P, _P],
    "heom_profile_allocs": [_P, _P, _P],
    "heom_set_wait_limit": [C.c_int64],
}
EXPORTED = sorted(list(_sig) + ["heom_destroy", "heom_last_error", "heom_mlp_destroy"])
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.heom_destroy.argtypes = [_P]
_lib.heom_destroy.restype = None
_lib.heom_mlp_destroy.argtypes = [_P]
_lib.heom_mlp_destroy.restype = None
_lib.heom_last_error.argtypes = []
_lib.heom_last_error.restype = C.c_char_p


def _check(status: int, where: str) -> int:
    if status != OK:
        raise HeomError(status, where)
    return status


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------------- exponents
def pade_constants(n_poles: int, fermi: bool = True, pade: bool = True):
    kappa = np.zeros(max(n_poles, 1))
    zeta = np.zeros(max(n_poles, 1))
    _check(_lib.heom_pade_constants(n_poles, int(fermi), int(pade), _ptr(kappa), _ptr(zeta)),
           "heom_pade_constants")
    return kappa[:n_poles], zeta[:n_poles]


def exp_drude_lorentz(lam, W, kT, n_poles, pade=True):
    xi = np.zeros(n_poles + 1, np.complex128)
    chi = np.zeros(n_poles + 1, np.complex128)
    _check(_lib.heom_exp_drude_lorentz(lam, W, kT, n_poles, int(pade), _ptr(xi), _ptr(chi)),
           "heom_exp_drude_lorentz")
    return xi, chi


def exp_lorentz_fermion(Gamma, W, mu, kT, n_poles, pade=True, nu=1):
    eta = np.zeros(n_poles + 1, np.complex128)
    gam = np.zeros(n_poles + 1, np.complex128)
    _check(_lib.heom_exp_lorentz_fermion(Gamma, W, mu, kT, n_poles, int(pade), nu, _ptr(eta),
                                         _ptr(gam)), "heom_exp_lorentz_fermion")
    return eta, gam


def problem_from_model(model, parity: int = 1) -> dict:
    """Raw problem (bath list with exponents) of a physical model, exponents from the library."""
    baths = []
    for V, p in model.boson_baths:
        xi, chi = exp_drude_lorentz(p.lam, p.W, p.kT, p.n_poles, p.method == "pade")
        baths.append(dict(kind="RI", op=_c64(V), coef=xi, rate=chi))
    for dop, p in model.fermion_baths:
        ep, gp = exp_lorentz_fermion(p.Gamma, p.W, p.mu, p.kT, p.n_poles, p.method == "pade", 1)
        em, gm = exp_lorentz_fermion(p.Gamma, p.W, p.mu, p.kT, p.n_poles, p.method == "pade", -1)
        h = len(ep)
        baths.append(dict(kind="F", op=_c64(dop), coef=np.concatenate([ep, em]),
                          rate=np.concatenate([gp, gm]),
                          nu=np.array([1] * h + [-1] * h, np.int32),
                          partner=np.array(list(range(h, 2 * h)) + list(range(h)), np.int32)))
    return dict(d=model.d, H=_c64(model.H), baths=baths, tier_b=model.tier_b,
                tier_f=model.tier_f, parity=parity,
                lindblad=[dict(op=_c64(F), rate=float(g)) for F, g in model.lindblad])


# ------------------------------------------------------------------------- hierarchy
class Hierarchy:
    """Owner of a ``heom_hier*`` (freed by ``heom_destroy`` when collected)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep
        n_ado, d, kb, kf, ns, ne = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        _check(_lib.heom_hier_info(self._h, C.byref(n_ado), C.byref(d), C.byref(kb), C.byref(kf),
                                   C.byref(ns), C.byref(ne)), "heom_hier_info")
        self.n_ado, self.d, self.k_b, self.k_f = n_ado.value, d.value, kb.value, kf.value
        self.n_sets, self.n_entries = ns.value, ne.value
        if not hasattr(self, "device"):
            # the library builds a hierarchy on the device current at the call
            import torch
            self.device = torch.cuda.current_device() if torch.cuda.is_available() else None

    @property
    def handle(self):
        return self._h

    def refresh(self):
        self.__init__(self._h, self._keep)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.heom_destroy(self._h)
            self._h = None


def _bath_array(baths, keep):
    arr = (Bath * max(len(baths), 1))()
    for i, b in enumerate(baths):
        coef = _c64(b["coef"])
        rate = _c64(b["rate"])
        keep += [coef, rate]
        if b.get("op") is not None:  # heom_count_ados reads no operator
            op = _c64(b["op"])
            keep.append(op)
            arr[i].op = op.ctypes.data_as(C.POINTER(c64))
        arr[i].kind = KIND[b["kind"]]
        arr[i].n_exp = len(coef)
        arr[i].coef = coef.ctypes.data_as(C.POINTER(c64))
        arr[i].rate = rate.ctypes.data_as(C.POINTER(c64))
        if b["kind"] == "F":
            nu = np.ascontiguousarray(b["nu"], np.int32)
            partner = np.ascontiguousarray(b["partner"], np.int32)
            keep += [nu, partner]
            arr[i].nu = nu.ctypes.data_as(C.POINTER(C.c_int))
            arr[i].partner = partner.ctypes.data_as(C.POINTER(C.c_int))
    return arr


def build_hierarchy(problem: dict) -> Hierarchy:
    """heom_build_hierarchy, or heom_build_hierarchy_pruned when the problem carries
    importance_th > 0; then heom_set_lindblad for its Lindblad terms."""
    d = int(problem["d"])
    H = _c64(problem["H"])
    keep = [H]
    arr = _bath_array(problem["baths"], keep)
    out = C.c_void_p()
    th = float(problem.get("importance_th", 0.0))
    args = (d, _ptr(H), len(problem["baths"]), C.cast(arr, C.c_void_p), int(problem["tier_b"]),
            int(problem["tier_f"]), int(problem.get("parity", 1)))
    if th > 0.0:
        _check(_lib.heom_build_hierarchy_pruned(*args, th, C.byref(out)),
               "heom_build_hierarchy_pruned")
    else:
        _check(_lib.heom_build_hierarchy(*args, 0, C.byref(out)), "heom_build_hierarchy")
    h = Hierarchy(out, None)
    if problem.get("lindblad"):
        set_lindblad(h, [t["op"] for t in problem["lindblad"]],
                     [t["rate"] for t in problem["lindblad"]])
    return h


def count_ados(baths, tier_b: int, tier_f: int, importance_th: float = 0.0) -> int:
    """heom_count_ados: hierarchy size after importance pruning, computed on the host."""
    keep = []
    arr = _bath_array(baths, keep)
    n = C.c_int64()
    _check(_lib.heom_count_ados(len(baths), C.cast(arr, C.c_void_p), int(tier_b), int(tier_f),
                                float(importance_th), C.byref(n)), "heom_count_ados")
    return n.value


def set_lindblad(h: Hierarchy, ops, rates):
    """Jump operators F_k [n, d, d] and real rates gamma_k [n] (Eq. Lindbladian) added to every
    ADO's equation; empty lists remove them."""
    n = len(rates)
    F = _c64(np.reshape(ops, (n, h.d, h.d)) if n else np.zeros((1, h.d, h.d)))
    g = np.ascontiguousarray(rates if n else [0.0], np.float64)
    _check(_lib.heom_set_lindblad(h.handle, n, _ptr(F), _ptr(g)), "heom_set_lindblad")


def set_params(h: Hierarchy, H, coef, rate):
    """H [n_sets, d, d], coef / rate [n_sets, K] in the global exponent order."""
    H = _c64(H)
    coef = _c64(coef)
    rate = _c64(rate)
    n_sets = H.shape[0]
    _check(_lib.heom_set_params(h.handle, n_sets, _ptr(H), _ptr(coef), _ptr(rate)),
           "heom_set_params")
    h.refresh()


def set_params_from_models(h: Hierarchy, models, parity: int = 1):
    """heom_set_params with one parameter set per model of h's structure (exponents from the
    library's helpers, as problem_from_model)."""
    Hs, coefs, rates = [], [], []
    for m in models:
        p = problem_from_model(m, parity)
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in p["baths"]]) if p["baths"] else np.zeros(0))
        rates.append(np.concatenate([b["rate"] for b in p["baths"]]) if p["baths"] else np.zeros(0))
    set_params(h, np.array(Hs), np.array(coefs), np.array(rates))


def set_truncation(h: Hierarchy, tier_b=None, tier_f=None):
    """heom_set_truncation: per parameter set tiers [n_sets] (both None: remove)."""
    if tier_b is None and tier_f is None:
        _check(_lib.heom_set_truncation(h.handle, None, None), "heom_set_truncation")
        return
    tb = np.ascontiguousarray(tier_b, np.int32)
    tf = np.ascontiguousarray(tier_f, np.int32)
    if tb.shape != (h.n_sets,) or tf.shape != (h.n_sets,):
        raise ValueError(f"tier arrays need one entry per parameter set ({h.n_sets})")
    _check(_lib.heom_set_truncation(h.handle, _ptr(tb), _ptr(tf)), "heom_set_truncation")


def ado_index(h: Hierarchy, occ) -> int:
    occ = np.ascontiguousarray(occ, np.int32)
    idx = C.c_int64()
    _check(_lib.heom_ado_index(h.handle, _ptr(occ), C.byref(idx)), "heom_ado_index")
    return idx.value


def ado_label(h: Hierarchy, idx: int) -> np.ndarray:
    out = np.zeros(h.k_b + h.k_f, np.int32)
    _check(_lib.heom_ado_label(h.handle, idx, _ptr(out)), "heom_ado_label")
    return out


def export_tables(h: Hierarchy) -> dict:
    E = h.n_entries
    row_ptr = np.zeros(h.n_ado + 1, np.int32)
    cols = {k: np.zeros(max(E, 1), np.int32) for k in ("nb", "k", "dir", "mult_l", "mult_r")}
    _check(_lib.heom_export_tables(h.handle, _ptr(row_ptr), *[_ptr(cols[k]) for k in
                                                              ("nb", "k", "dir", "mult_l", "mult_r")]),
           "heom_export_tables")
    out = {k: v[:E] for k, v in cols.items()}
    out["row_ptr"] = row_ptr
    return out


# ------------------------------------------------------------------------- device calls
def _prec_of(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return FP64
    if t.dtype == torch.complex64:
        return FP32
    raise TypeError("ADO vectors must be complex128 or complex64 tensors")


def _batch_of(h: Hierarchy, t) -> int:
    """Batch width of an ADO vector of hierarchy h, after checking that its shape is
    (N, d, d) or (N, d, d, batch) with h's N and d, that it is contiguous and that it lives on
    h's device: the library indexes N d^2 batch elements from h's tables, so a tensor of any
    other shape would be read and written out of bounds."""
    if t.dim() not in (3, 4):
        raise ValueError("ADO vector shape must be (N, d, d) or (N, d, d, batch)")
    if tuple(t.shape[:3]) != (h.n_ado, h.d, h.d):
        raise ValueError(f"ADO vector shape {tuple(t.shape)} does not match the hierarchy "
                         f"(N, d, d) = ({h.n_ado}, {h.d}, {h.d})")
    if t.dim() == 4 and t.shape[3] < 1:
        raise ValueError("ADO vector batch must be >= 1")
    if not t.is_contiguous():
        raise ValueError("ADO vectors must be contiguous")
    if not t.is_cuda:
        raise ValueError("ADO vectors must be CUDA tensors")
    dev = getattr(h, "device", None)
    if dev is not None and t.device.index != dev:
        raise ValueError(f"ADO vector on cuda:{t.device.index}, hierarchy on cuda:{dev}")
    return 1 if t.dim() == 3 else t.shape[3]


def apply(h: Hierarchy, x, y, stream=None):
    """y = M x (x, y: CUDA complex tensors (N, d, d[, batch]), same dtype)."""
    prec = _prec_of(x)
    if y.dtype != x.dtype or y.shape != x.shape:
        raise ValueError("x and y must have the same shape and dtype")
    _check(_lib.heom_apply(h.handle, _dptr(x), _dptr(y), _batch_of(h, x), prec, _stream(stream)),
           "heom_apply")
    return y


def evolve(h: Hierarchy, ados, dt: float, n_steps: int, save_every: int = 0, stream=None):
    """RK4 in place on ``ados``; returns the rho_sys snapshots (n_saves, d, d[, batch]) or None."""
    import torch
    prec = _prec_of(ados)
    B = _batch_of(h, ados)
    traj = None
    if save_every:
        shape = (n_steps // save_every + 1, h.d, h.d) + ((B,) if ados.dim() == 4 else ())
        traj = torch.empty(shape, dtype=ados.dtype, device=ados.device)
    _check(_lib.heom_evolve(h.handle, _dptr(ados), B, dt, n_steps, max(save_every, 1),
                            _dptr(traj) if traj is not None else None, prec, _stream(stream)),
           "heom_evolve")
    return traj


def set_drive(h: Hierarchy, ops):
    """Drive operators H_k of H(t) = H + sum_k f_k(t) H_k ([n, d, d]); [] removes them."""
    n = len(ops)
    Hk = _c64(np.reshape(ops, (n, h.d, h.d)) if n else np.zeros((1, h.d, h.d)))
    _check(_lib.heom_set_drive(h.handle, n, _ptr(Hk)), "heom_set_drive")
    h.n_drive = n


def evolve_td(h: Hierarchy, ados, dt: float, n_steps: int, f, save_every: int = 0, stream=None):
    """RK4 in place with H(t) = H + sum_k f_k(t) H_k; f [n_drive, 2 n_steps + 1] holds
    f_k(t0 + j dt / 2). Returns the rho_sys snapshots (n_saves, d, d[, batch]) or None."""
    import torch
    prec = _prec_of(ados)
    B = _batch_of(h, ados)
    fa = np.ascontiguousarray(f, np.float64).reshape(-1)
    if fa.size != getattr(h, "n_drive", 0) * (2 * n_steps + 1):
        raise ValueError("f must have shape (n_drive, 2 n_steps + 1)")
    traj = None
    if save_every:
        shape = (n_steps // save_every + 1, h.d, h.d) + ((B,) if ados.dim() == 4 else ())
        traj = torch.empty(shape, dtype=ados.dtype, device=ados.device)
    _check(_lib.heom_evolve_td(h.handle, _dptr(ados), B, dt, n_steps,
                               _ptr(fa) if fa.size else None, max(save_every, 1),
                               _dptr(traj) if traj is not None else None, prec, _stream(stream)),
           "heom_evolve_td")
    return traj


def _check_traj(h: Hierarchy, ados, B: int, n_steps: int, save_every: int, traj):
    """A caller-owned snapshot buffer must hold n_steps // save_every + 1 blocks of d x d x B
    elements of the ADO vector's dtype, contiguous, on its device: the library writes that many
    elements and nothing checks the buffer on the device side."""
    if traj is None:
        if save_every:
            raise ValueError("evolve_noalloc needs a caller-owned traj tensor when save_every > 0")
        return
    if not save_every:
        raise ValueError("traj given with save_every = 0: no snapshot would be written")
    if save_every < 0 or n_steps < 0:
        raise ValueError("save_every and n_steps must be >= 0")
    need = (n_steps // save_every + 1) * h.d * h.d * B
    if traj.dtype != ados.dtype:
        raise ValueError(f"traj dtype {traj.dtype} differs from the ADO vector's {ados.dtype}")
    if traj.numel() < need:
        raise ValueError(f"traj holds {traj.numel()} elements; {need} are written")
    if not traj.is_contiguous():
        raise ValueError("traj must be contiguous")
    if traj.device != ados.device:
        raise ValueError("traj must be on the ADO vector's device")


def evolve_noalloc(h: Hierarchy, ados, dt: float, n_steps: int, save_every: int = 0,
                   traj=None, stream=None):
    """heom_evolve_noalloc: RK4 in place on ``ados`` with no allocation in the library; the
    optional snapshot buffer ``traj`` is the caller's (this wrapper allocates nothing either)."""
    prec = _prec_of(ados)
    B = _batch_of(h, ados)
    _check_traj(h, ados, B, n_steps, save_every, traj)
    _check(_lib.heom_evolve_noalloc(h.handle, _dptr(ados), B, dt, n_steps, max(save_every, 1),
                                    _dptr(traj) if save_every else None, prec, _stream(stream)),
           "heom_evolve_noalloc")
    return traj


def _need_c128(t, name: str):
    import torch
    if t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a complex128 tensor")


def _check_sets(h: Hierarchy, ss, name: str = "ss"):
    """An ADO vector with one column per parameter set of h (complex128)."""
    _need_c128(ss, name)
    cols = ss.shape[3] if ss.dim() == 4 else 1
    if cols != h.n_sets:
        raise ValueError(f"{name} must be (N, d, d) or (N, d, d, n_sets) with n_sets = {h.n_sets}")
    _batch_of(h, ss)


def _stats_list(arr):
    return [dict(iterations=s.iterations, refinements=s.refinements, residual=s.residual,
                 status=s.status) for s in arr]


def steady(h: Hierarchy, x_out, x0=None, tol: float = 1e-8, max_iter: int = 2000,
           prec: int = MIXED, stream=None, raise_on_error: bool = True):
    """Stationary state into x_out (complex128). Returns (status, per-column stats)."""
    B = _batch_of(h, x_out)
    _need_c128(x_out, "x_out")
    if x0 is not None:
        _need_c128(x0, "x0")
        if tuple(x0.shape) != tuple(x_out.shape) or _batch_of(h, x0) != B:
            raise ValueError("x0 must have the shape of x_out")
    stats = (SolveStats * B)()
    st = _lib.heom_steady(h.handle, _dptr(x0) if x0 is not None else None, _dptr(x_out), B, tol,
                          max_iter, prec, C.cast(stats, C.c_void_p), _stream(stream))
    if raise_on_error:
        _check(st, "heom_steady")
    return st, _stats_list(stats)


def spectrum(odd: Hierarchy, ss, op_d, omegas, tol: float = 1e-8, max_iter: int = 2000,
             prec: int = MIXED, stream=None, raise_on_error: bool = True):
    """Density of states A(w) of mode op_d; returns (A, status, stats of x_+ then x_-).
    With a hierarchy holding several parameter sets (SHIFTED only), ss is (N, d, d, n_sets),
    A is (n_sets, n_omega) and the stats run set by set."""
    _check_sets(odd, ss)
    op = _c64(op_d)
    om = np.ascontiguousarray(omegas, np.float64)
    A = np.zeros(len(om)) if odd.n_sets == 1 else np.zeros((odd.n_sets, len(om)))
    stats = (SolveStats * (2 * len(om) * odd.n_sets))()
    st = _lib.heom_spectrum(odd.handle, _dptr(ss), _ptr(op), _ptr(om), len(om), tol, max_iter,
                            _ptr(A), prec, C.cast(stats, C.c_void_p), _stream(stream))
    if raise_on_error:
        _check(st, "heom_spectrum")
    return A, st, _stats_list(stats)


def spectrum_batched(odds, sss, ops, omegas, tol: float = 1e-8, max_iter: int = 2000,
                     prec: int = SHIFTED, stream=None, raise_on_error: bool = True):
    """heom_spectrum_batched: densities of states of several odd hierarchies of different
    shapes on one grid. Returns (list of A per hierarchy, (n_sets, n_omega) or (n_omega,),
    status, stats concatenated in hierarchy order)."""
    n = len(odds)
    if len(sss) != n or len(ops) != n:
        raise ValueError("one stationary state and one mode operator per hierarchy")
    for o, x in zip(odds, sss):
        _check_sets(o, x)
    om = np.ascontiguousarray(omegas, np.float64)
    rows = [o.n_sets for o in odds]
    A = np.zeros((sum(rows), len(om)))
    stats = (SolveStats * (2 * len(om) * sum(rows)))()
    keep = [_c64(op) for op in ops]
    hp = (C.c_void_p * n)(*[C.cast(o.handle, C.c_void_p).value for o in odds])
    sp = (C.c_void_p * n)(*[_dptr(x).value for x in sss])
    opp = (C.c_void_p * n)(*[k.ctypes.data for k in keep])
    st = _lib.heom_spectrum_batched(n, C.cast(hp, C.c_void_p), C.cast(sp, C.c_void_p),
                                    C.cast(opp, C.c_void_p), _ptr(om), len(om), tol, max_iter,
                                    _ptr(A), prec, C.cast(stats, C.c_void_p), _stream(stream))
    if raise_on_error:
        _check(st, "heom_spectrum_batched")
    out, r = [], 0
    for ns in rows:
        out.append(A[r] if ns == 1 else A[r:r + ns])
        r += ns
    return out, st, _stats_list(stats)


def autotune(h: Hierarchy, batch: int, prec: int = FP32, stream=None) -> dict:
    """heom_autotune: time the apply's kernel choices for `batch` columns, keep the fastest."""
    cand = np.zeros(6)
    t, p, best, var = C.c_int(), C.c_int(), C.c_double(), C.c_int()
    _check(_lib.heom_autotune(h.handle, batch, prec, _ptr(cand), C.byref(t), C.byref(p),
                              C.byref(best), C.byref(var), _stream(stream)), "heom_autotune")
    return {"tiled": bool(t.value), "ctas_per_sm": p.value, "variant": var.value,
            "best_us": best.value, "candidates_us": cand.tolist()}


def set_tile_config(h: Hierarchy, ctas_per_sm: int, variant: int):
    """heom_set_tile_config: pin the tiled kernel's ranges per SM and FP32 variant."""
    _check(_lib.heom_set_tile_config(h.handle, ctas_per_sm, variant), "heom_set_tile_config")


def psd(even: Hierarchy, ss, op_a, omegas, tol: float = 1e-8, max_iter: int = 2000, stream=None,
        raise_on_error: bool = True):
    """Power spectral density S(w) of mode op_a; returns (S, status, stats). With several
    parameter sets, ss is (N, d, d, n_sets) and S is (n_sets, n_omega)."""
    _check_sets(even, ss)
    op = _c64(op_a)
    om = np.ascontiguousarray(omegas, np.float64)
    S = np.zeros(len(om)) if even.n_sets == 1 else np.zeros((even.n_sets, len(om)))
    stats = (SolveStats * (len(om) * even.n_sets))()
    st = _lib.heom_psd(even.handle, _dptr(ss), _ptr(op), _ptr(om), len(om), tol, max_iter, _ptr(S),
                       C.cast(stats, C.c_void_p), _stream(stream))
    if raise_on_error:
        _check(st, "heom_psd")
    return S, st, _stats_list(stats)


def current(h: Hierarchy, x, baths, stream=None) -> np.ndarray:
    """Electronic current into the lead made of ``baths`` for stationary states x
    (N, d, d[, batch], complex128); one value per batch column."""
    B = _batch_of(h, x)
    _need_c128(x, "x")
    idx = np.ascontiguousarray(baths, np.int32)
    out = np.zeros(B)
    _check(_lib.heom_current(h.handle, _dptr(x), B, _ptr(idx), len(idx), _ptr(out), _stream(stream)),
           "heom_current")
    return out


def conductance(h: Hierarchy, dphi, baths, tol: float = 1e-10, max_iter: int = 4000,
                prec: int = FP64, stream=None, raise_on_error: bool = True):
    """heom_conductance over bias pairs (sets 2k, 2k + 1 of h): returns (G [P], I [2 P],
    status, stats)."""
    d = np.ascontiguousarray(dphi, np.float64)
    if d.shape != (h.n_sets // 2,) or h.n_sets % 2:
        raise ValueError("dphi needs one entry per bias pair (n_sets / 2)")
    idx = np.ascontiguousarray(baths, np.int32)
    G = np.zeros(len(d))
    I = np.zeros(h.n_sets)
    stats = (SolveStats * h.n_sets)()
    st = _lib.heom_conductance(h.handle, _ptr(d), _ptr(idx), len(idx), tol, max_iter, prec,
                               _ptr(G), _ptr(I), C.cast(stats, C.c_void_p), _stream(stream))
    if raise_on_error:
        _check(st, "heom_conductance")
    return G, I, st, _stats_list(stats)


# ------------------------------------------------------------------------- launch accounting
def set_wait_limit(cycles: int = 0):
    """heom_set_wait_limit: bound (SM clock cycles) of the persistent solvers' grid-barrier
    waits; 0 restores the default."""
    _check(_lib.heom_set_wait_limit(int(cycles)), "heom_set_wait_limit")


def release_workspace_cache():
    """heom_release_workspace_cache: free the solver workspaces kept for reuse."""
    _check(_lib.heom_release_workspace_cache(), "heom_release_workspace_cache")


def profile_enable(on: bool = True):
    _check(_lib.heom_profile_enable(int(on)), "heom_profile_enable")


def profile_read() -> dict:
    """{class name: dict(launches, ms, units, bytes)} for every kernel class."""
    out = {}
    for i, name in enumerate(KERNEL_CLASSES):
        n, ms, u, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        _check(_lib.heom_profile_read(i, C.byref(n), C.byref(ms), C.byref(u), C.byref(by)),
               "heom_profile_read")
        out[name] = dict(launches=n.value, ms=ms.value, units=u.value, bytes=by.value)
    return out


def profile_allocs() -> dict:
    """heom_profile_allocs: the library's device allocations (count, bytes) and workspace
    grows since it was loaded."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.heom_profile_allocs(C.byref(a), C.byref(b), C.byref(c)), "heom_profile_allocs")
    return {"device_allocs": a.value, "device_bytes": b.value, "workspace_takes": c.value}


def profile_copies():
    """(host->device bytes, device->host bytes) copied by the library while accounting was on."""
    a, b = C.c_int64(), C.c_int64()
    _check(_lib.heom_profile_copies(C.byref(a), C.byref(b)), "heom_profile_copies")
    return a.value, b.value


# ------------------------------------------------------------------------- learned warm start
def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class Mlp:
    """heom_mlp_*: a network that predicts warm-start features from model parameters."""

    def __init__(self, widths, seed: int = 0):
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        h = C.c_void_p()
        _check(_lib.heom_mlp_create(len(w) - 1, _ptr(w), seed, C.byref(h)), "heom_mlp_create")
        self._h = h
        n, i, o = C.c_int64(), C.c_int(), C.c_int()
        _check(_lib.heom_mlp_info(self._h, C.byref(n), C.byref(i), C.byref(o)), "heom_mlp_info")
        self.widths = [int(x) for x in w]
        self.n_params, self.n_in, self.n_out = n.value, i.value, o.value

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.heom_mlp_destroy(self._h)
            self._h = None

    def set_standardisation(self, in_mean, in_sd, out_mean, out_sd):
        arrs = [_f32(a) for a in (in_mean, in_sd, out_mean, out_sd)]
        _check(_lib.heom_mlp_set_standardisation(self._h, *[_ptr(a) for a in arrs]),
               "heom_mlp_set_standardisation")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(_lib.heom_mlp_get_params(self._h, _ptr(out)), "heom_mlp_get_params")
        return out

    def set_params(self, p):
        p = _f32(p)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(_lib.heom_mlp_set_params(self._h, _ptr(p)), "heom_mlp_set_params")

    def forward(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        _check(_lib.heom_mlp_forward(self._h, _dptr(x), _dptr(y), x.shape[0], _stream(stream)),
               "heom_mlp_forward")
        return y

    def gradients(self, x, t, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = C.c_double()
        _check(_lib.heom_mlp_gradients(self._h, _dptr(x), _dptr(t), x.shape[0], _dptr(g),
                                       C.byref(loss), _stream(stream)), "heom_mlp_gradients")
        return g, loss.value

    def train_step(self, x, t, lr: float, want_loss: bool = False, stream=None):
        loss = C.c_double()
        _check(_lib.heom_mlp_train_step(self._h, _dptr(x), _dptr(t), x.shape[0], lr,
                                        C.byref(loss) if want_loss else None, _stream(stream)),
               "heom_mlp_train_step")
        return loss.value if want_loss else None


def warm_start_features(h: "Hierarchy", x, n_features: int, stream=None):
    """Features (torch float32 [n_sets][n_features]) of states x (N, d, d[, n_sets])."""
    import torch
    _need_c128(x, "x")
    n_sets = _batch_of(h, x)
    f = torch.empty((n_sets, n_features), dtype=torch.float32, device=x.device)
    _check(_lib.heom_warm_start_features(h.handle, _dptr(x), n_sets, _dptr(f), n_features,
                                         _stream(stream)), "heom_warm_start_features")
    return f


def warm_start(h: "Hierarchy", net: Mlp, params, x_out, stream=None):
    """x_out (N, d, d[, n_sets], complex128) = the ADO vector net predicts for params."""
    _need_c128(x_out, "x_out")
    n_sets = _batch_of(h, x_out)
    if params.shape[0] != n_sets:
        raise ValueError("params must have one row per column of x_out")
    _check(_lib.heom_warm_start(h.handle, net.handle, _dptr(params), n_sets, _dptr(x_out),
                                _stream(stream)), "heom_warm_start")
    return x_out


def gather_elements(h: Hierarchy, x, elems, stream=None):
    """Features (torch float32 [n_sets][2 n_elems]) of the listed elements (torch int64, CUDA)
    of states x (N, d, d[, n_sets], complex128)."""
    import torch
    _need_c128(x, "x")
    n_sets = _batch_of(h, x)
    f = torch.empty((n_sets, 2 * elems.numel()), dtype=torch.float32, device=x.device)
    _check(_lib.heom_gather_elements(h.handle, _dptr(x), n_sets, _dptr(elems), elems.numel(),
                                     _dptr(f), _stream(stream)), "heom_gather_elements")
    return f


def warm_start_elements(h: Hierarchy, net: Mlp, params, elems, x_out, stream=None):
    """x_out (N, d, d[, n_sets], complex128) = net's prediction for params on the listed
    elements, zero elsewhere."""
    _need_c128(x_out, "x_out")
    n_sets = _batch_of(h, x_out)
    if params.shape[0] != n_sets:
        raise ValueError("params must have one row per column of x_out")
    _check(_lib.heom_warm_start_elements(h.handle, net.handle, _dptr(params), n_sets, _dptr(elems),
                                         elems.numel(), _dptr(x_out), _stream(stream)),
           "heom_warm_start_elements")
    return x_out
