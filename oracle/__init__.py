"""FP64 CPU oracle of Projective Affine Body Dynamics (Algorithm 1) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import this package. It shares nothing with the CUDA path; both consume the same
seeded inputs from ``scenes``.

The arithmetic lives in ``pabd_oracle.c`` (plain C, double precision, single thread);
this module only compiles it with gcc and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pabd_oracle.c")
_LIB = os.path.join(_HERE, "libpabd_oracle.so")
_lib = None

STATE_COLS = 22  # c(3) A(9) Q(4) v(3) w(3)
CONTACT = 5
GROUND = 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: collision decisions are IEEE single)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        L.po_create.restype = P
        L.po_create.argtypes = [D]
        L.po_destroy.argtypes = [P]
        L.po_add_body.argtypes = [P, D]
        L.po_add_body.restype = ctypes.c_int
        L.po_add_bond.argtypes = [P, D]
        L.po_add_bond.restype = ctypes.c_int
        L.po_step.argtypes = [P, ctypes.c_int]
        L.po_step.restype = ctypes.c_int
        L.po_detect.argtypes = [P]
        L.po_n_bodies.argtypes = [P]
        L.po_n_static_bonds.argtypes = [P]
        L.po_step_index.argtypes = [P]
        L.po_step_index.restype = ctypes.c_int64
        L.po_set_step_index.argtypes = [P, ctypes.c_int64]
        L.po_get_state.argtypes = [P, D]
        L.po_set_state.argtypes = [P, D]
        L.po_get_pairs.argtypes = [P, I, ctypes.c_int]
        L.po_get_pairs.restype = ctypes.c_int
        L.po_get_contacts.argtypes = [P, I, D, ctypes.c_int]
        L.po_get_contacts.restype = ctypes.c_int
        L.po_get_residual.argtypes = [P, D, ctypes.c_int]
        L.po_get_residual.restype = ctypes.c_int
        L.po_body_system.argtypes = [P, ctypes.c_int, D, D]
        L.po_get_static_bonds.argtypes = [P, I, D, ctypes.c_int]
        L.po_get_static_bonds.restype = ctypes.c_int
        L.po_polar_rotation.argtypes = [D, D, D]
        L.po_quat_to_mat.argtypes = [D, D]
        L.po_mat_to_quat.argtypes = [D, D]
        L.po_cholesky_solve.argtypes = [ctypes.c_int, D, D, D]
        L.po_cholesky_solve.restype = ctypes.c_int
        L.po_contact_rule.argtypes = [D, ctypes.c_double, ctypes.c_double, ctypes.c_double, D, D, D, D, D]
        L.po_get_al_state.argtypes = [P, D]
        L.po_get_activation_margin.argtypes = [P, D]
        L.po_set_activation_shift.argtypes = [P, ctypes.c_double]
        L.po_set_round_iterates.argtypes = [P, ctypes.c_int]
        L.po_last_sweeps.argtypes = [P]
        L.po_last_sweeps.restype = ctypes.c_int
        L.po_set_al_state.argtypes = [P, D]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def pack_params(p: dict) -> np.ndarray:
    return np.array([
        p["h"], *p["gravity"], p["n_iter"], p["has_ground"], *p["ground_n"], p["ground_d"],
        p["mu"], p["c_kappa"], p["d_hat_rel"], p["margin"], p["project"], p["body_contacts"],
        p["large_he"], p.get("resid_tol", 0.0),
    ], dtype=np.float64)


class OracleScene:
    """One oracle scene built from a ``scenes.Scene``."""

    def __init__(self, scene):
        self.L = lib()
        self.scene = scene
        pr = pack_params(scene.params)
        self.h = self.L.po_create(_dp(pr))
        for b in scene.bodies:
            row = np.array([*b["he"], b["mass"], *b["c"], *b["quat"], *b["v"], *b["omega"],
                            b["pinned"], b["group"]], dtype=np.float64)
            self.L.po_add_body(self.h, _dp(row))
        for bo in scene.bonds:
            row = np.array([bo["type"], bo["i"], bo["j"], *bo["xi"], *bo["xj"], *bo["axis"],
                            bo["kappa"], bo["rest"], bo["arm"], bo["amp"], bo["period"], bo["phase"],
                            bo["beta"], bo["alpha"], bo["gamma"]], dtype=np.float64)
            if self.L.po_add_bond(self.h, _dp(row)) < 0:
                raise ValueError("oracle rejected bond")
        self.n = scene.n_bodies

    def __del__(self):
        if getattr(self, "h", None):
            self.L.po_destroy(self.h)
            self.h = None

    def step(self, nsteps: int = 1) -> int:
        return self.L.po_step(self.h, nsteps)

    def detect(self):
        self.L.po_detect(self.h)

    @property
    def step_index(self) -> int:
        return self.L.po_step_index(self.h)

    @step_index.setter
    def step_index(self, k: int):
        self.L.po_set_step_index(self.h, k)

    def state(self) -> np.ndarray:
        out = np.zeros((self.n, STATE_COLS))
        self.L.po_get_state(self.h, _dp(out))
        return out

    def set_state(self, st: np.ndarray):
        st = np.ascontiguousarray(st, dtype=np.float64)
        assert st.shape == (self.n, STATE_COLS)
        self.L.po_set_state(self.h, _dp(st))

    def pairs(self) -> np.ndarray:
        n = self.L.po_get_pairs(self.h, None, 0)
        out = np.zeros((max(n, 1), 2), dtype=np.int32)
        self.L.po_get_pairs(self.h, _ip(out), n)
        return out[:n]

    def contacts(self):
        n = self.L.po_get_contacts(self.h, None, None, 0)
        meta = np.zeros((max(n, 1), 3), dtype=np.int32)
        data = np.zeros((max(n, 1), 11))
        self.L.po_get_contacts(self.h, _ip(meta), _dp(data), n)
        return meta[:n], data[:n]

    def residual(self) -> np.ndarray:
        n = self.L.po_get_residual(self.h, None, 0)
        out = np.zeros(max(n, 1))
        self.L.po_get_residual(self.h, _dp(out), n)
        return out[:n]

    def al_state(self) -> np.ndarray:
        """(kappa, lambda) of every static bond after expansion (zeros for non-AL bonds)."""
        n = self.L.po_n_static_bonds(self.h)
        out = np.zeros((max(n, 1), 2))
        self.L.po_get_al_state(self.h, _dp(out))
        return out[:n]

    def activation_margin(self) -> np.ndarray:
        """Per body, min over the last step's sweeps of |g - dhat| over its contacts (inf if none)."""
        out = np.zeros(max(self.n, 1))
        self.L.po_get_activation_margin(self.h, _dp(out))
        return out[:self.n]

    def last_sweeps(self) -> int:
        """Sweeps the last step ran (n_iter unless a residual threshold ended it sooner)."""
        return self.L.po_last_sweeps(self.h)

    def set_activation_shift(self, shift: float):
        """Test probe: contacts switch on at g < dhat + shift in the following steps (0 = the method)."""
        self.L.po_set_activation_shift(self.h, float(shift))

    def set_round_iterates(self, on: bool):
        """Test probe: every sweep's iterate rounded to single precision before the next sweep
        reads it, in the following steps (False = the method)."""
        self.L.po_set_round_iterates(self.h, 1 if on else 0)

    def set_al_state(self, st: np.ndarray):
        st = np.ascontiguousarray(st, dtype=np.float64)
        self.L.po_set_al_state(self.h, _dp(st))

    def body_system(self, body: int):
        H = np.zeros((12, 12))
        r = np.zeros(12)
        self.L.po_body_system(self.h, body, _dp(H), _dp(r))
        return H, r

    def static_bonds(self):
        n = self.L.po_get_static_bonds(self.h, None, None, 0)
        meta = np.zeros((max(n, 1), 3), dtype=np.int32)
        data = np.zeros((max(n, 1), 6))
        self.L.po_get_static_bonds(self.h, _ip(meta), _dp(data), n)
        return meta[:n], data[:n]


def polar_rotation(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    R = np.zeros(9)
    s = np.zeros(3)
    lib().po_polar_rotation(_dp(A), _dp(R), _dp(s))
    return R.reshape(3, 3), s


def quat_to_mat(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9)
    lib().po_quat_to_mat(_dp(q), _dp(R))
    return R.reshape(3, 3)


def mat_to_quat(R) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    q = np.zeros(4)
    lib().po_mat_to_quat(_dp(R), _dp(q))
    return q


def cholesky_solve(H, b) -> np.ndarray:
    H = np.ascontiguousarray(H, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    rc = lib().po_cholesky_solve(n, _dp(H), _dp(b), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError("oracle Cholesky failed")
    return x


def contact_rule(N, dhat, w, mu, yi, yj):
    """The contact/friction bond rule for one contact: returns (w, f_i, f_j)."""
    N, yi, yj = (np.ascontiguousarray(a, dtype=np.float64) for a in (N, yi, yj))
    wo = np.zeros(1)
    fi = np.zeros(3)
    fj = np.zeros(3)
    lib().po_contact_rule(_dp(N), dhat, w, mu, _dp(yi), _dp(yj), _dp(wo), _dp(fi), _dp(fj))
    return wo[0], fi, fj
