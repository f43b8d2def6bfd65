"""Helpers shared by the GPU parity tests: the per-step error measure and teacher forcing."""
from __future__ import annotations

import numpy as np

SIGNS = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64)

# relative per-step position tolerance of the FP32 path against the FP64 oracle
REL_TOL = 1e-5


def corners(st: np.ndarray, he: np.ndarray) -> np.ndarray:
    """World positions y = A x + c of the 8 box corners of every body (N, 8, 3)."""
    x = SIGNS[None, :, :] * he[:, None, :]
    A = st[:, 3:12].reshape(-1, 3, 3)
    return st[:, None, 0:3] + np.einsum("nij,nkj->nki", A, x)


def scene_scale(st_ref: np.ndarray, he: np.ndarray) -> float:
    """Diagonal of the scene's bounding box (at least 1)."""
    y = corners(st_ref, he).reshape(-1, 3)
    return max(float(np.linalg.norm(y.max(0) - y.min(0))), 1.0)


def rel_err(st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray) -> float:
    """max over bodies and corners |y_gpu - y_ref| / scene diagonal."""
    if st_ref.shape[0] == 0:
        return 0.0
    d = np.linalg.norm(corners(st_gpu, he) - corners(st_ref, he), axis=-1)
    return float(d.max()) / scene_scale(st_ref, he)


def worst_body(st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray):
    """(body index, its corner error / scene diagonal) of the worst body."""
    d = np.linalg.norm(corners(st_gpu, he) - corners(st_ref, he), axis=-1).max(axis=1)
    k = int(np.argmax(d))
    return k, float(d[k]) / scene_scale(st_ref, he)


def teacher_forced_step(gpu, ref, n: int = 1):
    """Start the GPU from the oracle's state (rounded to FP32 on upload), step both n steps."""
    st0 = ref.state()
    gpu.set_state(st0)
    gpu.set_step_index(ref.step_index)
    ref.step(n)
    gpu.step(n)
    return gpu.state(), ref.state()


def activation_envelope_err(sc, st0, k0, st_gpu, st_ref, he, oracle_mod, ulps: float = 8.0):
    """Per-step error that allows for contacts at their activation threshold.

    A contact is active in a sweep iff g < dhat, decided from that sweep's iterate; the
    single-precision path decides it from an iterate that differs from the oracle's by
    rounding, so a contact within rounding of the threshold may switch the other way, and the
    Jacobi step is not continuous there.  The oracle is re-run from the same start with the
    threshold moved by +-delta, delta = `ulps` units of single-precision rounding at the
    scene's scale; each body is compared with the closest of the three oracle results.
    Returns (max error, worst body, its error against the unshifted oracle)."""
    scale = scene_scale(st_ref, he)
    delta = ulps * 2.0 ** -24 * scale
    d = np.linalg.norm(corners(st_gpu, he) - corners(st_ref, he), axis=-1).max(axis=1)
    best = d.copy()
    for sh in (delta, -delta):
        r = oracle_mod.OracleScene(sc)
        r.set_state(st0)
        r.step_index = k0
        r.set_activation_shift(sh)
        r.step(1)
        dv = np.linalg.norm(corners(st_gpu, he) - corners(r.state(), he), axis=-1).max(axis=1)
        best = np.minimum(best, dv)
    k = int(np.argmax(best))
    return float(best[k]) / scale, k, float(d[k]) / scale


def same_contacts(gpu_c, ref_c):
    """Bit-exact contact lists: same (type, i, j) rows in the same order and the same
    single-precision geometry; dhat and w agree to single-precision rounding."""
    gm, gd = gpu_c
    rm, rd = ref_c
    assert gm.shape == rm.shape, f"contact count {gm.shape[0]} vs {rm.shape[0]}"
    assert np.array_equal(gm, rm)
    assert np.array_equal(gd[:, :9], rd[:, :9].astype(np.float32))
    np.testing.assert_allclose(gd[:, 9:11], rd[:, 9:11], rtol=2e-7, atol=0)
