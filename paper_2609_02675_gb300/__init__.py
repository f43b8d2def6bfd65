"""Python binding of the GB300 Projective Affine Body Dynamics library (``libpabd.so``).

Argument marshalling only: every stage of a step runs in the library's CUDA kernels.
The module-level functions carry the C-ABI's names (``pabd_create_scene``,
``pabd_add_body``, ``pabd_add_bond``, ``pabd_step``, ``pabd_read_state`` ...); ``Scene``
builds a library scene from a ``scenes.Scene`` description.  PyTorch is used only to
provide the device memory (its caching allocator) and the CUDA stream.

Importing this package raises ImportError when ``libpabd.so`` has not been built (run
``__graft_entry__.build()``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpabd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (python -c "
                      "'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

STATE_COLS = 22
WORLD = 0xFFFFFFFF
OK, ERR_ARG, ERR_OOM, ERR_CAPACITY, ERR_DIVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_STATE = range(8)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
D3 = ctypes.c_double * 3


class pabd_scene_desc(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_double), ("gravity", D3), ("n_iter", ctypes.c_int),
        ("has_ground", ctypes.c_int), ("ground_n", D3), ("ground_d", ctypes.c_double),
        ("mu", ctypes.c_double), ("c_kappa", ctypes.c_double), ("d_hat_rel", ctypes.c_double),
        ("margin", ctypes.c_double), ("project", ctypes.c_int), ("body_contacts", ctypes.c_int),
        ("large_he", ctypes.c_double), ("precision_policy", ctypes.c_int),
        ("sweep_mode", ctypes.c_int), ("sweep_lanes", ctypes.c_int), ("max_pairs", ctypes.c_size_t), ("max_contacts", ctypes.c_size_t),
        ("resid_tol", ctypes.c_double), ("broadphase", ctypes.c_int), ("light_order", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class pabd_body_desc(ctypes.Structure):
    _fields_ = [
        ("he", D3), ("mass", ctypes.c_double), ("c", D3), ("quat", ctypes.c_double * 4),
        ("v", D3), ("omega", D3), ("pinned", ctypes.c_int), ("group", ctypes.c_int),
    ]


class pabd_bond_desc(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int), ("body_i", ctypes.c_uint32), ("body_j", ctypes.c_uint32),
        ("x_i", D3), ("x_j", D3), ("axis", D3), ("kappa", ctypes.c_double), ("rest_len", ctypes.c_double),
        ("arm", ctypes.c_double), ("drive_amp", ctypes.c_double), ("drive_period", ctypes.c_double),
        ("drive_phase", ctypes.c_double), ("al_beta", ctypes.c_double), ("al_alpha", ctypes.c_double),
        ("al_gamma", ctypes.c_double),
    ]


class pabd_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_bodies", "n_groups", "n_static_bonds", "n_bonds", "n_pairs", "n_contacts", "step_index",
        "max_pairs", "max_contacts", "graph_nodes", "launches", "fp64_bodies", "device_bytes",
        "sweep_mode", "sweep_lanes", "sweep_block", "sweep_grid", "coop_fallbacks", "heavy_bodies",
        "fp64_dynamic", "last_sweeps", "offgrid_bodies", "light_order", "tuned",
        "tune_sweep_ns0", "tune_sweep_ns1", "tune_sweep_ns2", "tune_sweep_ns3")]


_P = ctypes.c_void_p
_PD = ctypes.POINTER(ctypes.c_double)
_PF = ctypes.POINTER(ctypes.c_float)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PU32 = ctypes.POINTER(ctypes.c_uint32)
_PSZ = ctypes.POINTER(ctypes.c_size_t)

_SIGS = {
    "pabd_create_scene": [ctypes.POINTER(pabd_scene_desc), ctypes.POINTER(_P)],
    "pabd_add_body": [_P, ctypes.POINTER(pabd_body_desc), _PU32],
    "pabd_add_bond": [_P, ctypes.POINTER(pabd_bond_desc), _PU32, ctypes.POINTER(ctypes.c_int)],
    "pabd_add_bodies": [_P, _P, ctypes.c_size_t, _PU32, _PSZ],
    "pabd_add_bonds": [_P, _P, ctypes.c_size_t, _PSZ],
    "pabd_step": [_P, ctypes.c_int],
    "pabd_step_eager": [_P, ctypes.c_int],
    "pabd_step_many": [_P, ctypes.c_int, _PI32],
    "pabd_set_wait_limit": [_P, ctypes.c_uint32],
    "pabd_tune": [_P],
    "pabd_set_group_hold": [_P, _P, ctypes.c_size_t],
    "pabd_detect": [_P],
    "pabd_sync": [_P],
    "pabd_read_state": [_P, _PD, ctypes.c_size_t],
    "pabd_write_state": [_P, _PD, ctypes.c_size_t],
    "pabd_read_state_f32": [_P, _P, ctypes.c_size_t],
    "pabd_write_state_f32": [_P, _P, ctypes.c_size_t],
    "pabd_read_bond_state": [_P, _PD, ctypes.c_size_t],
    "pabd_write_bond_state": [_P, _PD, ctypes.c_size_t],
    "pabd_set_step_index": [_P, ctypes.c_int64],
    "pabd_set_profiling": [_P, ctypes.c_int],
    "pabd_read_profile": [_P, _PD, ctypes.c_size_t, ctypes.c_int],
    "pabd_read_pairs": [_P, _PI32, ctypes.c_size_t, _PSZ],
    "pabd_read_contacts": [_P, _PI32, _PF, ctypes.c_size_t, _PSZ],
    "pabd_read_residual": [_P, _PD, ctypes.c_size_t],
    "pabd_get_info": [_P, ctypes.POINTER(pabd_info)],
    "pabd_destroy_scene": [_P],
    "pabd_broadphase_noalloc": [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, _P, ctypes.c_int32, _P, _P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.pabd_status_str.argtypes = [ctypes.c_int]
_lib.pabd_status_str.restype = ctypes.c_char_p
_lib.pabd_last_cuda_error.argtypes = []
_lib.pabd_last_cuda_error.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["pabd_status_str", "pabd_last_cuda_error"])


class PabdError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.pabd_status_str(code).decode()
        if code == ERR_CUDA:
            msg += ": " + _lib.pabd_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}")
        self.code = code


def _check(code: int, where: str, allow=()):
    if code != OK and code not in allow:
        raise PabdError(code, where)
    return code


# ---- C-ABI, same names, argument marshalling only ----

def pabd_create_scene(desc: pabd_scene_desc):
    h = _P()
    _check(_lib.pabd_create_scene(ctypes.byref(desc), ctypes.byref(h)), "pabd_create_scene")
    return h


def pabd_add_body(s, body: pabd_body_desc) -> int:
    out = ctypes.c_uint32()
    _check(_lib.pabd_add_body(s, ctypes.byref(body), ctypes.byref(out)), "pabd_add_body")
    return out.value


def pabd_add_bond(s, bond: pabd_bond_desc):
    ids = (ctypes.c_uint32 * 2)()
    n = ctypes.c_int()
    _check(_lib.pabd_add_bond(s, ctypes.byref(bond), ids, ctypes.byref(n)), "pabd_add_bond")
    return list(ids[: n.value])


# numpy views with the C layout of pabd_body_desc / pabd_bond_desc
BODY_C_DTYPE = np.dtype([("he", "f8", 3), ("mass", "f8"), ("c", "f8", 3), ("quat", "f8", 4), ("v", "f8", 3),
                         ("omega", "f8", 3), ("pinned", "i4"), ("group", "i4")], align=True)
BOND_C_DTYPE = np.dtype([("type", "i4"), ("body_i", "u4"), ("body_j", "u4"), ("x_i", "f8", 3), ("x_j", "f8", 3),
                         ("axis", "f8", 3), ("kappa", "f8"), ("rest_len", "f8"), ("arm", "f8"),
                         ("drive_amp", "f8"), ("drive_period", "f8"), ("drive_phase", "f8"),
                         ("al_beta", "f8"), ("al_alpha", "f8"), ("al_gamma", "f8")], align=True)
assert BODY_C_DTYPE.itemsize == ctypes.sizeof(pabd_body_desc)
assert BOND_C_DTYPE.itemsize == ctypes.sizeof(pabd_bond_desc)


def pabd_add_bodies(s, rows: np.ndarray):
    rows = np.ascontiguousarray(rows, dtype=BODY_C_DTYPE)
    done = ctypes.c_size_t()
    _check(_lib.pabd_add_bodies(s, rows.ctypes.data, rows.shape[0], None, ctypes.byref(done)), "pabd_add_bodies")
    return done.value


def pabd_add_bonds(s, rows: np.ndarray):
    rows = np.ascontiguousarray(rows, dtype=BOND_C_DTYPE)
    done = ctypes.c_size_t()
    _check(_lib.pabd_add_bonds(s, rows.ctypes.data, rows.shape[0], ctypes.byref(done)), "pabd_add_bonds")
    return done.value


def pabd_step(s, nsteps: int = 1):
    return _check(_lib.pabd_step(s, nsteps), "pabd_step")


def pabd_step_eager(s, nsteps: int = 1):
    return _check(_lib.pabd_step_eager(s, nsteps), "pabd_step_eager")


def pabd_step_many(scenes, nsteps):
    """Scene k of `scenes` (handles) advances nsteps[k] steps on its own stream."""
    n = len(scenes)
    arr = (_P * max(n, 1))(*scenes)
    cnt = np.ascontiguousarray(nsteps, dtype=np.int32)
    return _check(_lib.pabd_step_many(ctypes.cast(arr, _P), n, cnt.ctypes.data_as(_PI32)), "pabd_step_many")


def pabd_set_group_hold(s, hold, n_groups: int):
    """hold: None (release all) or n_groups bytes, nonzero = group held still."""
    if hold is None:
        return _check(_lib.pabd_set_group_hold(s, None, n_groups), "pabd_set_group_hold")
    h = np.ascontiguousarray(hold, dtype=np.uint8)
    assert h.shape == (n_groups,)
    return _check(_lib.pabd_set_group_hold(s, h.ctypes.data, n_groups), "pabd_set_group_hold")


def pabd_tune(s):
    return _check(_lib.pabd_tune(s), "pabd_tune")


def pabd_set_wait_limit(s, polls: int):
    return _check(_lib.pabd_set_wait_limit(s, polls), "pabd_set_wait_limit")


def pabd_detect(s):
    return _check(_lib.pabd_detect(s), "pabd_detect")


def pabd_sync(s, allow=()):
    return _check(_lib.pabd_sync(s), "pabd_sync", allow)


def pabd_read_state(s, n_bodies: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((n_bodies, STATE_COLS), dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (n_bodies, STATE_COLS)
    _check(_lib.pabd_read_state(s, out.ctypes.data_as(_PD), n_bodies), "pabd_read_state")
    return out


def pabd_write_state(s, rows: np.ndarray):
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    _check(_lib.pabd_write_state(s, rows.ctypes.data_as(_PD), rows.shape[0]), "pabd_write_state")


def pabd_read_bond_state(s, n_static_bonds: int) -> np.ndarray:
    out = np.zeros((max(n_static_bonds, 1), 2), dtype=np.float64)
    _check(_lib.pabd_read_bond_state(s, out.ctypes.data_as(_PD), n_static_bonds), "pabd_read_bond_state")
    return out[:n_static_bonds]


def pabd_write_bond_state(s, st: np.ndarray):
    st = np.ascontiguousarray(st, dtype=np.float64).reshape(-1, 2)
    _check(_lib.pabd_write_bond_state(s, st.ctypes.data_as(_PD), st.shape[0]), "pabd_write_bond_state")


def pabd_read_state_f32(s, host: int, n_bodies: int):
    """Enqueue the device-layout state (24 floats per body) into the host buffer at address
    `host` (see include/pabd.h); the buffer is valid after pabd_sync."""
    return _check(_lib.pabd_read_state_f32(s, host, n_bodies), "pabd_read_state_f32")


def pabd_write_state_f32(s, host: int, n_bodies: int):
    """Enqueue the device-layout state from the host buffer at address `host`."""
    return _check(_lib.pabd_write_state_f32(s, host, n_bodies), "pabd_write_state_f32")


def pabd_set_step_index(s, k: int):
    _check(_lib.pabd_set_step_index(s, int(k)), "pabd_set_step_index")


PROFILE_KEYS = ("steps", "collision_ms", "csr_ms", "predict_ms", "sweep_ms", "unused_ms", "finalize_ms",
                "sweep_launches", "sweeps", "step_ms", "bonds_sum")


def pabd_set_profiling(s, on: bool):
    _check(_lib.pabd_set_profiling(s, int(bool(on))), "pabd_set_profiling")


def pabd_read_profile(s, reset: bool = False) -> dict:
    out = np.zeros(len(PROFILE_KEYS))
    _check(_lib.pabd_read_profile(s, out.ctypes.data_as(_PD), len(PROFILE_KEYS), int(bool(reset))),
           "pabd_read_profile")
    return dict(zip(PROFILE_KEYS, out.tolist()))


def pabd_read_pairs(s) -> np.ndarray:
    n = ctypes.c_size_t()
    _check(_lib.pabd_read_pairs(s, None, 0, ctypes.byref(n)), "pabd_read_pairs", (ERR_CAPACITY,))
    out = np.zeros((max(n.value, 1), 2), dtype=np.int32)
    _check(_lib.pabd_read_pairs(s, out.ctypes.data_as(_PI32), n.value, ctypes.byref(n)), "pabd_read_pairs",
           (ERR_CAPACITY,))
    return out[: n.value]


def pabd_read_contacts(s):
    n = ctypes.c_size_t()
    _check(_lib.pabd_read_contacts(s, None, None, 0, ctypes.byref(n)), "pabd_read_contacts", (ERR_CAPACITY,))
    meta = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    data = np.zeros((max(n.value, 1), 11), dtype=np.float32)
    _check(_lib.pabd_read_contacts(s, meta.ctypes.data_as(_PI32), data.ctypes.data_as(_PF), n.value,
                                   ctypes.byref(n)), "pabd_read_contacts", (ERR_CAPACITY,))
    return meta[: n.value], data[: n.value]


def pabd_read_residual(s, n_groups: int) -> np.ndarray:
    out = np.zeros(max(n_groups, 1))
    _check(_lib.pabd_read_residual(s, out.ctypes.data_as(_PD), n_groups), "pabd_read_residual")
    return out[:n_groups]


def pabd_get_info(s) -> dict:
    info = pabd_info()
    _check(_lib.pabd_get_info(s, ctypes.byref(info)), "pabd_get_info")
    return {n: getattr(info, n) for n, _ in pabd_info._fields_}


def pabd_destroy_scene(s):
    return _check(_lib.pabd_destroy_scene(s), "pabd_destroy_scene")


NOALLOC_MAX_BODIES = 16384


def pabd_broadphase_noalloc(q: int, vel: int, he: int, group: int, flags: int, n_bodies: int, h: float,
                            margin: float, d_hat_rel: float, pairs_out: int, max_pairs: int, n_pairs_out: int,
                            stream: int = 0):
    """Allocation-free broad phase on device pointers (see include/pabd.h)."""
    return _check(_lib.pabd_broadphase_noalloc(q, vel, he, group, flags, n_bodies, h, margin, d_hat_rel,
                                                pairs_out, max_pairs, n_pairs_out, stream or None),
                  "pabd_broadphase_noalloc")


# ---- torch plumbing: device memory and stream ----

class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


def scene_desc(params: dict, stream=0, allocator: _TorchAllocator | None = None, precision_policy=1,
               max_pairs=0, max_contacts=0, sweep_mode=0, sweep_lanes=0, broadphase=0,
               light_order=0) -> pabd_scene_desc:
    d = pabd_scene_desc()
    d.h = params["h"]
    d.gravity = D3(*params["gravity"])
    d.n_iter = int(params["n_iter"])
    d.has_ground = int(params["has_ground"])
    d.ground_n = D3(*params["ground_n"])
    d.ground_d = params["ground_d"]
    d.mu = params["mu"]
    d.c_kappa = params["c_kappa"]
    d.d_hat_rel = params["d_hat_rel"]
    d.margin = params["margin"]
    d.project = int(params["project"])
    d.body_contacts = int(params["body_contacts"])
    d.large_he = params["large_he"]
    d.precision_policy = int(precision_policy)
    d.sweep_mode = int(sweep_mode)
    d.sweep_lanes = int(sweep_lanes)
    d.max_pairs = int(max_pairs)
    d.max_contacts = int(max_contacts)
    d.resid_tol = float(params.get("resid_tol", 0.0))
    d.broadphase = int(broadphase)
    d.light_order = int(light_order)
    d.stream = stream or None
    if allocator is not None:
        d.alloc = allocator.alloc_cb
        d.free = allocator.free_cb
    else:
        d.alloc = ALLOC_FN()
        d.free = FREE_FN()
    return d


class Scene:
    """A library scene built from a ``scenes.Scene`` (bodies and user bonds)."""

    def __init__(self, scene, device: int = 0, stream=None, torch_memory: bool = True, precision_policy: int = 1,
                 max_pairs: int = 0, max_contacts: int = 0, sweep_mode: int = 0, sweep_lanes: int = 0,
                 broadphase: int = 0, light_order: int = 0):
        import torch
        torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.torch_stream = stream
        self._alloc = _TorchAllocator(device, stream.cuda_stream) if torch_memory else None
        self.desc = scene_desc(scene.params, stream.cuda_stream, self._alloc, precision_policy, max_pairs,
                               max_contacts, sweep_mode, sweep_lanes, broadphase, light_order)
        self.h = pabd_create_scene(self.desc)
        self.n = scene.n_bodies
        self.n_groups = scene.n_groups
        bodies = np.zeros(scene.n_bodies, dtype=BODY_C_DTYPE)
        for f in ("he", "mass", "c", "quat", "v", "omega", "pinned", "group"):
            bodies[f] = scene.bodies[f]
        pabd_add_bodies(self.h, bodies)
        nb = len(scene.bonds)
        if nb:
            bonds = np.zeros(nb, dtype=BOND_C_DTYPE)
            bonds["type"] = scene.bonds["type"]
            bonds["body_i"] = scene.bonds["i"].astype(np.int64).astype(np.uint32)
            j = scene.bonds["j"].astype(np.int64)
            bonds["body_j"] = np.where(j < 0, np.int64(WORLD), j).astype(np.uint32)
            bonds["x_i"], bonds["x_j"], bonds["axis"] = scene.bonds["xi"], scene.bonds["xj"], scene.bonds["axis"]
            bonds["kappa"], bonds["rest_len"], bonds["arm"] = scene.bonds["kappa"], scene.bonds["rest"], scene.bonds["arm"]
            bonds["drive_amp"], bonds["drive_period"] = scene.bonds["amp"], scene.bonds["period"]
            bonds["drive_phase"] = scene.bonds["phase"]
            bonds["al_beta"], bonds["al_alpha"] = scene.bonds["beta"], scene.bonds["alpha"]
            bonds["al_gamma"] = scene.bonds["gamma"]
            pabd_add_bonds(self.h, bonds)

    def close(self):
        if getattr(self, "h", None):
            pabd_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        pabd_step(self.h, n)

    def step_eager(self, n: int = 1):
        pabd_step_eager(self.h, n)

    def set_wait_limit(self, polls: int):
        pabd_set_wait_limit(self.h, polls)

    def set_group_hold(self, hold):
        """Hold the groups with hold[g] != 0 still from the next step on (None: release all)."""
        pabd_set_group_hold(self.h, hold, self.n_groups)

    def tune(self):
        """Re-run the sweep autotuner on the current state (see pabd_tune)."""
        pabd_tune(self.h)

    def detect(self):
        pabd_detect(self.h)

    def sync(self, allow=()):
        return pabd_sync(self.h, allow)

    def state(self, out=None) -> np.ndarray:
        return pabd_read_state(self.h, self.n, out)

    def set_state(self, rows: np.ndarray):
        pabd_write_state(self.h, rows)

    def read_state_f32(self, host_ptr: int):
        pabd_read_state_f32(self.h, host_ptr, self.n)

    def write_state_f32(self, host_ptr: int):
        pabd_write_state_f32(self.h, host_ptr, self.n)

    def set_step_index(self, k: int):
        pabd_set_step_index(self.h, k)

    def bond_state(self) -> np.ndarray:
        """(kappa, lambda) of every static bond (zeros for bonds other than AL_DISTANCE)."""
        return pabd_read_bond_state(self.h, pabd_get_info(self.h)["n_static_bonds"])

    def set_bond_state(self, st: np.ndarray):
        pabd_write_bond_state(self.h, st)

    def set_profiling(self, on: bool):
        pabd_set_profiling(self.h, on)

    def profile(self, reset: bool = False) -> dict:
        return pabd_read_profile(self.h, reset)

    def pairs(self) -> np.ndarray:
        return pabd_read_pairs(self.h)

    def contacts(self):
        return pabd_read_contacts(self.h)

    def residual(self) -> np.ndarray:
        return pabd_read_residual(self.h, self.n_groups)

    def info(self) -> dict:
        return pabd_get_info(self.h)
