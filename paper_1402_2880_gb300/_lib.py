"""ctypes binding of libsscf (argument marshalling only).

Every function here forwards to the C-ABI declared in ``include/sscf.h``;
no step of the sparse SCF is computed in Python. The library is built
in-tree by ``paper_1402_2880_gb300.build`` and loading fails loudly when it
is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsscf.so")

SSCF_OK = 0
SSCF_FP64 = 0
SSCF_MIXED = 1
SSCF_ORTHO_ALL = 0
SSCF_ORTHO_OCC = 1

ERRORS = {
    -1: "SSCF_ERR_INVALID_ARG", -2: "SSCF_ERR_OOM", -3: "SSCF_ERR_CUDA", -4: "SSCF_ERR_NONFINITE",
    -5: "SSCF_ERR_CAPACITY", -6: "SSCF_ERR_NOT_CONVERGED", -7: "SSCF_ERR_TIMEOUT", -8: "SSCF_ERR_STATE",
}

EXPORTED = [
    "sscf_create", "sscf_destroy", "sscf_strerror", "sscf_set_allocator", "sscf_set_thresholds",
    "sscf_get_dims", "sscf_guess", "sscf_orthonormalise", "sscf_build_fock", "sscf_rotate_sweep",
    "sscf_density", "sscf_reset_charges", "sscf_step", "sscf_run", "sscf_get_C_dense",
    "sscf_set_C_dense", "sscf_get_H_dense", "sscf_get_F_dense", "sscf_get_charges",
    "sscf_set_charges", "sscf_get_colouring", "sscf_get_pairs", "sscf_profile", "sscf_profile_read",
    "sscf_select_pairs_noalloc", "sscf_gradients", "sscf_get_cluster_results",
    "sscf_enable_graph", "sscf_get_C_rows", "sscf_get_blocks",
    "sscf_get_C_cols", "sscf_get_F_entries", "sscf_get_C_tiles", "sscf_set_C_tiles", "sscf_autotune",
    "sscf_set_precision", "sscf_set_fock_blocks", "sscf_get_density_blocks", "sscf_get_overlap_dense",
    "sscf_group_molecules", "sscf_run_from_current",
]


class SscfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {ERRORS.get(status, status)}")


class System(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("species", ctypes.POINTER(ctypes.c_int)),
                ("xyz", ctypes.POINTER(ctypes.c_double)), ("group_of_mol", ctypes.POINTER(ctypes.c_int)),
                ("cluster_of_mol", ctypes.POINTER(ctypes.c_int))]


class Params(ctypes.Structure):
    _fields_ = [("onsite", ctypes.c_double * 3), ("V0", ctypes.c_double * 4), ("S0", ctypes.c_double * 4),
                ("r_decay", ctypes.c_double), ("r_cut", ctypes.c_double), ("U", ctypes.c_double * 2),
                ("q0", ctypes.c_double * 2), ("eps", ctypes.c_double), ("dq_tol", ctypes.c_double),
                ("e_tol", ctypes.c_double), ("group_cut", ctypes.c_double), ("rot_cap_factor", ctypes.c_double),
                ("mix_beta", ctypes.c_double), ("max_scc", ctypes.c_int), ("precision", ctypes.c_int),
                ("ortho_every", ctypes.c_int), ("cap_tiles", ctypes.c_int), ("cap_y", ctypes.c_int),
                ("apply_variant", ctypes.c_int), ("closure_mode", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("dq_max", ctypes.c_double), ("dE", ctypes.c_double),
                ("max_fov", ctypes.c_double), ("eta", ctypes.c_double), ("n_rot", ctypes.c_int64),
                ("n_combo", ctypes.c_int64), ("nnz_c", ctypes.c_int64), ("nnz_occ", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("upd_rot", ctypes.c_int64), ("upd_combo", ctypes.c_int64),
                ("iteration", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree libsscf.so (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsscf.so not built ({LIB_PATH}); run paper_1402_2880_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    c_int, c_double, c_i64, c_vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "sscf_create": (c_int, [P(System), P(Params), c_vp, P(c_vp)]),
        "sscf_destroy": (None, [c_vp]),
        "sscf_strerror": (ctypes.c_char_p, [c_int]),
        "sscf_set_allocator": (c_int, [ALLOC_FN, FREE_FN, c_vp]),
        "sscf_set_thresholds": (c_int, [c_vp, c_double, c_double, c_double]),
        "sscf_get_dims": (c_int, [c_vp] + [P(c_int)] * 6),
        "sscf_guess": (c_int, [c_vp]),
        "sscf_orthonormalise": (c_int, [c_vp, c_int, c_int, P(c_int), P(c_double)]),
        "sscf_build_fock": (c_int, [c_vp]),
        "sscf_rotate_sweep": (c_int, [c_vp, P(c_i64), P(c_double)]),
        "sscf_density": (c_int, [c_vp, P(c_double), P(c_double), P(c_double)]),
        "sscf_reset_charges": (c_int, [c_vp, P(c_double)]),
        "sscf_step": (c_int, [c_vp, P(StepInfo)]),
        "sscf_run": (c_int, [c_vp, P(StepInfo)]),
        "sscf_run_from_current": (c_int, [c_vp, P(StepInfo)]),
        "sscf_get_C_dense": (c_int, [c_vp, P(c_double)]),
        "sscf_set_C_dense": (c_int, [c_vp, P(c_double)]),
        "sscf_get_H_dense": (c_int, [c_vp, P(c_double), P(c_double), P(c_double)]),
        "sscf_get_F_dense": (c_int, [c_vp, P(c_double), P(c_double)]),
        "sscf_get_charges": (c_int, [c_vp, P(c_double), P(c_double), P(c_double)]),
        "sscf_set_charges": (c_int, [c_vp, P(c_double), P(c_double), P(c_double)]),
        "sscf_get_colouring": (c_int, [c_vp, P(c_int)]),
        "sscf_get_pairs": (c_int, [c_vp, c_i64, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                                   P(ctypes.c_int32), P(c_i64)]),
        "sscf_profile": (c_int, [c_vp, c_int]),
        "sscf_profile_read": (c_int, [c_vp, c_int, ctypes.c_char_p, P(c_double), P(c_i64), P(c_int)]),
        "sscf_select_pairs_noalloc": (c_int, [c_vp, c_i64, c_double, c_i64, c_vp, P(c_i64), c_vp]),
        "sscf_gradients": (c_int, [c_vp, P(c_double), P(c_double)]),
        "sscf_get_cluster_results": (c_int, [c_vp, P(c_double), P(c_double), P(c_int)]),
        "sscf_enable_graph": (c_int, [c_vp, c_int]),
        "sscf_get_C_rows": (c_int, [c_vp, c_int, P(c_int), P(c_double)]),
        "sscf_get_C_cols": (c_int, [c_vp, c_int, P(c_int), P(c_double)]),
        "sscf_autotune": (c_int, [c_vp, P(c_int)]),
        "sscf_set_precision": (c_int, [c_vp, c_int]),
        "sscf_set_fock_blocks": (c_int, [c_vp, P(c_double)]),
        "sscf_get_overlap_dense": (c_int, [c_vp, P(c_double), P(c_int)]),
        "sscf_group_molecules": (c_int, [c_int, P(c_double), c_int, c_int, c_double, c_vp, P(c_int), P(c_int),
                                         P(c_int)]),
        "sscf_get_density_blocks": (c_int, [c_vp, P(c_double)]),
        "sscf_get_C_tiles": (c_int, [c_vp, P(ctypes.c_int32), P(ctypes.c_int32), P(c_double), P(c_i64)]),
        "sscf_set_C_tiles": (c_int, [c_vp, P(ctypes.c_int32), P(ctypes.c_int32), P(c_double)]),
        "sscf_get_F_entries": (c_int, [c_vp, c_int, P(c_int), P(c_int), P(c_double)]),
        "sscf_get_blocks": (c_int, [c_vp, P(c_int), P(c_double), P(c_double), P(c_double), P(c_i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray | None, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(status: int, what: str):
    if status != SSCF_OK:
        raise SscfError(status, what)


def make_params(p: dict, precision: int = SSCF_FP64, ortho_every: int = 1, cap_tiles: int = 0, cap_y: int = 0,
                apply_variant: int = 0, closure_mode: int = 0) -> Params:
    q = Params()
    q.onsite[:] = [p["onsite_O_s"], p["onsite_O_p"], p["onsite_H_s"]]
    q.V0[:] = list(p["V0"])
    q.S0[:] = list(p["S0"])
    q.r_decay, q.r_cut = p["r_decay"], p["r_cut"]
    q.U[:] = [p["U_O"], p["U_H"]]
    q.q0[:] = [p["q0_O"], p["q0_H"]]
    q.eps, q.dq_tol, q.e_tol = p["eps_mo"], p["dq_tol"], p["e_tol"]
    q.group_cut, q.rot_cap_factor, q.mix_beta = p["group_cut"], p["rot_cap_factor"], p["mix_beta"]
    q.max_scc, q.precision, q.ortho_every, q.cap_tiles = int(p["max_scc"]), precision, ortho_every, cap_tiles
    q.cap_y, q.apply_variant, q.closure_mode = cap_y, apply_variant, closure_mode
    return q


def select_pairs_noalloc(f_dev_ptr: int, n: int, tau: float, k_max: int, keep_dev_ptr: int,
                         stream: int | None = None) -> int:
    """Pair selection on caller-owned device arrays, without any device allocation.

    ``f_dev_ptr`` points to n doubles, ``keep_dev_ptr`` to n bytes (both
    device memory owned by the caller). Returns the number of kept entries.
    """
    lib = load()
    kept = ctypes.c_int64()
    _check(lib.sscf_select_pairs_noalloc(ctypes.c_void_p(f_dev_ptr), int(n), float(tau), int(k_max),
                                         ctypes.c_void_p(keep_dev_ptr), ctypes.byref(kept),
                                         ctypes.c_void_p(stream or 0)), "sscf_select_pairs_noalloc")
    return kept.value


def group_molecules(xyz, n_link: int = 8, max_iter: int = 100, tol: float = 1e-3, stream: int | None = None):
    """MO groups of a water-like system (atoms O, H, H per molecule) by the
    GPU's constrained k-means: (group_of_mol, n_groups, iterations)."""
    lib = load()
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    n_atoms = x.size // 3
    groups = np.empty(n_atoms // 3, dtype=np.int32)
    ng, it = ctypes.c_int(), ctypes.c_int()
    _check(lib.sscf_group_molecules(int(n_atoms), _ptr(x), int(n_link), int(max_iter), float(tol),
                                    ctypes.c_void_p(stream or 0), _ptr(groups, ctypes.c_int), ctypes.byref(ng),
                                    ctypes.byref(it)), "sscf_group_molecules")
    return groups, ng.value, it.value


class Context:
    """One cluster on the GPU (wraps an ``sscf_ctx``)."""

    def __init__(self, species, xyz, group_of_mol, params: dict, precision: int = SSCF_FP64,
                 stream: int | None = None, ortho_every: int = 1, cap_tiles: int = 0, cluster_of_mol=None,
                 cap_y: int = 0, apply_variant: int = 0, closure_mode: int = 0):
        self.lib = load()
        self._species = np.ascontiguousarray(species, dtype=np.int32)
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        self._groups = np.ascontiguousarray(group_of_mol, dtype=np.int32)
        self._clusters = None if cluster_of_mol is None else np.ascontiguousarray(cluster_of_mol, dtype=np.int32)
        sysc = System(n_atoms=int(self._species.size), species=_ptr(self._species, ctypes.c_int),
                      xyz=_ptr(self._xyz), group_of_mol=_ptr(self._groups, ctypes.c_int),
                      cluster_of_mol=_ptr(self._clusters, ctypes.c_int))
        self.params = make_params(params, precision, ortho_every, cap_tiles, cap_y, apply_variant, closure_mode)
        h = ctypes.c_void_p()
        _check(self.lib.sscf_create(ctypes.byref(sysc), ctypes.byref(self.params),
                                    ctypes.c_void_p(stream or 0), ctypes.byref(h)), "sscf_create")
        self.h = h
        dims = [ctypes.c_int() for _ in range(6)]
        _check(self.lib.sscf_get_dims(self.h, *[ctypes.byref(d) for d in dims]), "sscf_get_dims")
        (self.n_ao, self.n_mo, self.n_occ, self.n_groups, self.n_tiles, self.n_colours) = [d.value for d in dims]
        self.n_atoms = int(self._species.size)

    @classmethod
    def from_system(cls, sysm, params: dict, **kw):
        clusters = getattr(sysm, "cluster_of_mol", None)
        if clusters is not None and "cluster_of_mol" not in kw:
            kw["cluster_of_mol"] = clusters
        return cls(sysm.species, sysm.xyz, sysm.group_of_mol, params, **kw)

    def cluster_results(self):
        """(energy, max |q - q_prev|) of every cluster after the last charge update."""
        n = ctypes.c_int()
        _check(self.lib.sscf_get_cluster_results(self.h, None, None, ctypes.byref(n)), "sscf_get_cluster_results")
        e = np.empty(n.value)
        d = np.empty(n.value)
        _check(self.lib.sscf_get_cluster_results(self.h, _ptr(e), _ptr(d), None), "sscf_get_cluster_results")
        return e, d

    def close(self):
        if getattr(self, "h", None):
            self.lib.sscf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- steps ----
    def set_thresholds(self, eps: float, dq_tol: float, e_tol: float):
        _check(self.lib.sscf_set_thresholds(self.h, eps, dq_tol, e_tol), "sscf_set_thresholds")

    def guess(self):
        _check(self.lib.sscf_guess(self.h), "sscf_guess")

    def orthonormalise(self, which: int = SSCF_ORTHO_ALL, max_pass: int = 200):
        n, eta = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.sscf_orthonormalise(self.h, which, max_pass, ctypes.byref(n), ctypes.byref(eta)),
               "sscf_orthonormalise")
        return n.value, eta.value

    def set_precision(self, precision: int):
        """Widen (SSCF_FP64) or narrow (SSCF_MIXED) the context's storage in place."""
        _check(self.lib.sscf_set_precision(self.h, int(precision)), "sscf_set_precision")

    def build_fock(self):
        _check(self.lib.sscf_build_fock(self.h), "sscf_build_fock")

    def rotate_sweep(self):
        n, mx = ctypes.c_int64(), ctypes.c_double()
        _check(self.lib.sscf_rotate_sweep(self.h, ctypes.byref(n), ctypes.byref(mx)), "sscf_rotate_sweep")
        return n.value, mx.value

    def density(self):
        q = np.empty(self.n_atoms)
        E, dq = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.sscf_density(self.h, _ptr(q), ctypes.byref(E), ctypes.byref(dq)), "sscf_density")
        return q, E.value, dq.value

    def reset_charges(self) -> float:
        E = ctypes.c_double()
        _check(self.lib.sscf_reset_charges(self.h, ctypes.byref(E)), "sscf_reset_charges")
        return E.value

    def enable_graph(self, enable: bool = True):
        _check(self.lib.sscf_enable_graph(self.h, 1 if enable else 0), "sscf_enable_graph")

    def step(self) -> dict:
        info = StepInfo()
        _check(self.lib.sscf_step(self.h, ctypes.byref(info)), "sscf_step")
        return info.as_dict()

    def run(self, allow_not_converged: bool = False) -> dict:
        info = StepInfo()
        s = self.lib.sscf_run(self.h, ctypes.byref(info))
        if not (s == SSCF_OK or (allow_not_converged and s == -6)):
            _check(s, "sscf_run")
        d = info.as_dict()
        d["converged"] = s == SSCF_OK
        return d

    def run_from_current(self, allow_not_converged: bool = False) -> dict:
        """The user-threshold SCF from the MOs already in the context (a restart)."""
        info = StepInfo()
        s = self.lib.sscf_run_from_current(self.h, ctypes.byref(info))
        if not (s == SSCF_OK or (allow_not_converged and s == -6)):
            _check(s, "sscf_run_from_current")
        d = info.as_dict()
        d["converged"] = s == SSCF_OK
        return d

    def gradients(self):
        """(dE/dxyz (n_atoms, 3) in Ha/bohr, dE/d(V0[0..3], S0[0..3])) at the current MOs."""
        g = np.empty((self.n_atoms, 3))
        dp = np.empty(8)
        _check(self.lib.sscf_gradients(self.h, _ptr(g), _ptr(dp)), "sscf_gradients")
        return g, dp

    # ---- state ----
    def get_C(self) -> np.ndarray:
        C = np.empty((self.n_ao, self.n_mo))
        _check(self.lib.sscf_get_C_dense(self.h, _ptr(C)), "sscf_get_C_dense")
        return C

    def set_C(self, C: np.ndarray):
        C = np.ascontiguousarray(C, dtype=np.float64)
        assert C.shape == (self.n_ao, self.n_mo)
        _check(self.lib.sscf_set_C_dense(self.h, _ptr(C)), "sscf_set_C_dense")

    def get_C_rows(self, rows) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rows.size, self.n_mo))
        _check(self.lib.sscf_get_C_rows(self.h, int(rows.size), _ptr(rows, ctypes.c_int), _ptr(out)),
               "sscf_get_C_rows")
        return out

    def autotune(self) -> int:
        """Pick the transform's launch shape by timing it on the current state; returns the choice."""
        s = ctypes.c_int()
        _check(self.lib.sscf_autotune(self.h, ctypes.byref(s)), "sscf_autotune")
        return s.value

    def get_C_tiles(self):
        """Checkpoint of C: (nt per row block, tile ids, values as (n_stored, 6, 16))."""
        n = ctypes.c_int64()
        _check(self.lib.sscf_get_C_tiles(self.h, None, None, None, ctypes.byref(n)), "sscf_get_C_tiles")
        nt = np.empty(self.n_ao // 6, dtype=np.int32)
        tiles = np.empty(n.value, dtype=np.int32)
        vals = np.empty((n.value, 6, 16))
        _check(self.lib.sscf_get_C_tiles(self.h, _ptr(nt, ctypes.c_int32), _ptr(tiles, ctypes.c_int32), _ptr(vals),
                                         ctypes.byref(n)), "sscf_get_C_tiles")
        return nt, tiles, vals

    def set_C_tiles(self, nt, tiles, vals):
        nt = np.ascontiguousarray(nt, dtype=np.int32)
        tiles = np.ascontiguousarray(tiles, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        _check(self.lib.sscf_set_C_tiles(self.h, _ptr(nt, ctypes.c_int32), _ptr(tiles, ctypes.c_int32), _ptr(vals)),
               "sscf_set_C_tiles")

    def get_C_cols(self, cols) -> np.ndarray:
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.empty((self.n_ao, cols.size))
        _check(self.lib.sscf_get_C_cols(self.h, int(cols.size), _ptr(cols, ctypes.c_int), _ptr(out)),
               "sscf_get_C_cols")
        return out

    def get_F_entries(self, i, j) -> np.ndarray:
        i = np.ascontiguousarray(i, dtype=np.int32)
        j = np.ascontiguousarray(j, dtype=np.int32)
        out = np.empty(i.size)
        _check(self.lib.sscf_get_F_entries(self.h, int(i.size), _ptr(i, ctypes.c_int), _ptr(j, ctypes.c_int),
                                           _ptr(out)), "sscf_get_F_entries")
        return out

    def get_blocks(self):
        """(pairs (n_mp, 2), H, H0, S as (n_mp, 6, 6)) on the molecule-pair pattern."""
        n = ctypes.c_int64()
        _check(self.lib.sscf_get_blocks(self.h, None, None, None, None, ctypes.byref(n)), "sscf_get_blocks")
        mn = np.empty((n.value, 2), dtype=np.int32)
        H, H0, S = (np.empty((n.value, 6, 6)) for _ in range(3))
        _check(self.lib.sscf_get_blocks(self.h, _ptr(mn, ctypes.c_int), _ptr(H), _ptr(H0), _ptr(S), None),
               "sscf_get_blocks")
        return mn, H, H0, S

    def set_fock_blocks(self, X):
        """Caller-built Fock matrix: (n_mp, 6, 6) blocks in the pair order of get_blocks()."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        _check(self.lib.sscf_set_fock_blocks(self.h, _ptr(X)), "sscf_set_fock_blocks")

    def density_blocks(self) -> np.ndarray:
        """P = 2 C_occ C_occ^T on the molecule-pair pattern, (n_mp, 6, 6) in the pair order of get_blocks()."""
        n = ctypes.c_int64()
        _check(self.lib.sscf_get_blocks(self.h, None, None, None, None, ctypes.byref(n)), "sscf_get_blocks")
        P = np.empty((n.value, 6, 6))
        _check(self.lib.sscf_get_density_blocks(self.h, _ptr(P)), "sscf_get_density_blocks")
        return P

    def get_H(self):
        H, H0, S = (np.empty((self.n_ao, self.n_ao)) for _ in range(3))
        _check(self.lib.sscf_get_H_dense(self.h, _ptr(H), _ptr(H0), _ptr(S)), "sscf_get_H_dense")
        return H, H0, S

    def get_F(self):
        F = np.empty((self.n_occ, self.n_mo - self.n_occ))
        d = np.empty(self.n_mo)
        _check(self.lib.sscf_get_F_dense(self.h, _ptr(F), _ptr(d)), "sscf_get_F_dense")
        return F, d

    def get_overlap(self) -> np.ndarray:
        """sigma = C^T S C of the last orthonormalisation pass (dense over the pass's MOs)."""
        n = ctypes.c_int()
        _check(self.lib.sscf_get_overlap_dense(self.h, None, ctypes.byref(n)), "sscf_get_overlap_dense")
        sig = np.empty((n.value, n.value))
        _check(self.lib.sscf_get_overlap_dense(self.h, _ptr(sig), None), "sscf_get_overlap_dense")
        return sig

    def get_charges(self, out=None):
        q, dq, Q = out if out is not None else (np.empty(self.n_atoms) for _ in range(3))
        _check(self.lib.sscf_get_charges(self.h, _ptr(q), _ptr(dq), _ptr(Q)), "sscf_get_charges")
        return q, dq, Q

    def set_charges(self, q_prev=None, dq_in=None, Q_in=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (q_prev, dq_in, Q_in)]
        _check(self.lib.sscf_set_charges(self.h, *[_ptr(a) for a in arrs]), "sscf_set_charges")

    def colouring(self) -> np.ndarray:
        C = np.empty((self.n_groups, self.n_groups), dtype=np.int32)
        _check(self.lib.sscf_get_colouring(self.h, _ptr(C, ctypes.c_int)), "sscf_get_colouring")
        return C

    def profile(self, enable: bool = True):
        _check(self.lib.sscf_profile(self.h, 1 if enable else 0), "sscf_profile")

    def profile_read(self) -> dict:
        """{launcher name: (milliseconds, calls)} since the last read (then reset)."""
        cap = 128
        n = ctypes.c_int()
        names = ctypes.create_string_buffer(32 * cap)
        ms = np.zeros(cap)
        calls = np.zeros(cap, dtype=np.int64)
        _check(self.lib.sscf_profile_read(self.h, cap, names, _ptr(ms), _ptr(calls, ctypes.c_int64),
                                          ctypes.byref(n)), "sscf_profile_read")
        raw = names.raw
        return {raw[32 * i:32 * i + 32].split(b"\0")[0].decode(): (float(ms[i]), int(calls[i]))
                for i in range(min(n.value, cap))}

    def pairs(self):
        n = ctypes.c_int64()
        _check(self.lib.sscf_get_pairs(self.h, 0, None, None, None, None, ctypes.byref(n)), "sscf_get_pairs")
        out = [np.empty(n.value, dtype=np.int32) for _ in range(4)]
        _check(self.lib.sscf_get_pairs(self.h, n.value, *[_ptr(a, ctypes.c_int32) for a in out],
                                       ctypes.byref(n)), "sscf_get_pairs")
        return tuple(out)
