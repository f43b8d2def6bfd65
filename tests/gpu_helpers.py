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


def rounding_sensitivity(make_scene, st0, k0, st_ref, he, oracle_mod, mask=None, seeds=(0, 1, 2, 3)):
    """How far the oracle's own step moves under perturbations of single-precision size: the
    largest corner deviation (over the bodies in `mask`, as a fraction of the scene diagonal)
    of the oracle step from st0 against st_ref, over these probes:
      - the start state rounded to single precision;
      - the same, and every sweep's iterate rounded to single precision (the storage rounding
        that a single-precision path applies at every sweep);
      - for each seed, every start coordinate moved by one unit of single-precision rounding up
        or down (signs drawn from the seed), with the iterates rounded as above.
    Where the sweeps converge this is at the level of the rounding itself; where they do not, it
    is the map's amplification of rounding, which bounds how closely any single-precision path
    can follow the oracle there."""
    scale = scene_scale(st_ref, he)
    sel = np.ones(st_ref.shape[0], bool) if mask is None else np.asarray(mask, bool)
    starts = [(st0.astype(np.float32).astype(np.float64), False), (st0.astype(np.float32).astype(np.float64), True)]
    for seed in seeds:
        rng = np.random.default_rng(1000 + seed)
        starts.append((st0 * (1.0 + np.ldexp(rng.choice([-1.0, 1.0], st0.shape), -24)), True))
    worst = 0.0
    for st, rnd in starts:
        r = oracle_mod.OracleScene(make_scene())
        r.set_round_iterates(rnd)
        r.set_state(st)
        r.step_index = k0
        r.step(1)
        d = np.linalg.norm(corners(r.state(), he) - corners(st_ref, he), axis=-1).max(axis=1)
        worst = max(worst, float(d[sel].max()) / scale if sel.any() else 0.0)
    return worst


def same_contacts(gpu_c, ref_c):
    """Bit-exact contact lists: same (type, i, j) rows in the same order and the same
    single-precision geometry; dhat and w agree to single-precision rounding."""
    gm, gd = gpu_c
    rm, rd = ref_c
    assert gm.shape == rm.shape, f"contact count {gm.shape[0]} vs {rm.shape[0]}"
    assert np.array_equal(gm, rm)
    assert np.array_equal(gd[:, :9], rd[:, :9].astype(np.float32))
    np.testing.assert_allclose(gd[:, 9:11], rd[:, 9:11], rtol=2e-7, atol=0)


def body_corner_err(st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray) -> np.ndarray:
    """Per body: max over its box corners of |y_gpu - y_ref| (absolute)."""
    return np.linalg.norm(corners(st_gpu, he) - corners(st_ref, he), axis=-1).max(axis=1)


def velocity_ratios(st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray, h: float) -> dict:
    """v, omega and Q of a teacher-forced step against the oracle's (a9, Sec. 4.4), each as
    the worst ratio of its error to what the body's own position error e and single-precision
    rounding allow through the velocity recovery: v = (c1 - c0)/h moves by at most
    (2 e + 2^-23 |c|)/h; A1 by e/he_min per entry (plus its rounding 2^-22), so
    omega = vee(skew((A1 - A0) A0^T))/h by 4 (e/he_min + 2^-21)/h and Q = quat(A1) by
    4 (e/he_min + 2^-21).  Every ratio must stay below 1."""
    e = body_corner_err(st_gpu, st_ref, he)
    hmin = he.min(axis=1)
    cnorm = np.abs(st_ref[:, 0:3]).max(axis=1)
    dv = np.linalg.norm(st_gpu[:, 16:19] - st_ref[:, 16:19], axis=1)
    dw = np.linalg.norm(st_gpu[:, 19:22] - st_ref[:, 19:22], axis=1)
    qg, qr = st_gpu[:, 12:16], st_ref[:, 12:16]
    dq = np.minimum(np.linalg.norm(qg - qr, axis=1), np.linalg.norm(qg + qr, axis=1))
    rot = e / hmin + 2.0 ** -21
    return {"v": float((dv / ((2 * e + 2.0 ** -23 * cnorm) / h)).max()),
            "omega": float((dw / (4 * rot / h)).max()),
            "quat": float((dq / (4 * rot)).max())}


def residual_ratio(r_gpu: np.ndarray, r_ref: np.ndarray, st_gpu: np.ndarray, st_ref: np.ndarray, he: np.ndarray,
                   group: np.ndarray) -> float:
    """Per-group residual sqrt(sum |q^{k+1} - q^k|^2) of the last sweep (a8, Sec. 4.2) against
    the oracle's: each of the two iterates it differences is off by about the body's final
    error (e on c, e/he_min on A) plus its single-precision rounding, so the residual may move
    by twice that summed over the group's 12 coordinates per body; 1% of the residual on top
    covers iterates whose errors exceed the final one.  Returns the worst ratio (< 1)."""
    e = body_corner_err(st_gpu, st_ref, he)
    hmin = he.min(axis=1)
    cnorm = np.abs(st_ref[:, 0:3]).max(axis=1)
    per = 3 * (e + 2.0 ** -23 * cnorm) ** 2 + 9 * (e / hmin + 2.0 ** -22) ** 2
    ng = len(r_ref)
    allow = 2 * np.sqrt(np.bincount(group, weights=per, minlength=ng)) + 0.01 * np.abs(r_ref)
    return float((np.abs(r_gpu - r_ref) / allow).max()) if ng else 0.0


def threshold_rule_err(sc, st0, k0, st_gpu, he, oracle_mod, ulps: float = 8.0):
    """Per-step error under the activation reading (R22) for scenes where many contacts land.

    Each body is compared with the closest of the oracle's results at the activation
    thresholds dhat and dhat +- delta (delta = `ulps` units of single-precision rounding at the
    scene's scale).  A body still beyond the tolerance is accepted only if a body at most two
    links away -- links being this step's contacts and the scene's user bonds -- had a contact
    within delta of the threshold during the step (the oracle's activation margin): several
    such contacts switching in different sweeps are reproduced by no single shift, and the
    sweeps carry a switch through contacts and stiff joints to the neighbours.  Returns (max
    error over the other bodies, [(body, error)] of the accepted ones)."""
    ref = oracle_mod.OracleScene(sc)
    ref.set_state(st0)
    ref.step_index = k0
    ref.step(1)
    st_ref = ref.state()
    scale = scene_scale(st_ref, he)
    delta = ulps * 2.0 ** -24 * scale
    best = body_corner_err(st_gpu, st_ref, he) / scale
    for sh in (delta, -delta):
        r = oracle_mod.OracleScene(sc)
        r.set_state(st0)
        r.step_index = k0
        r.set_activation_shift(sh)
        r.step(1)
        best = np.minimum(best, body_corner_err(st_gpu, r.state(), he) / scale)
    bad = np.nonzero(best >= REL_TOL)[0]
    if not len(bad):
        return float(best.max()) if best.size else 0.0, []
    margin = ref.activation_margin()
    cm = ref.contacts()[0]
    links = {}
    pairs = list(zip(cm[:, 1], cm[:, 2])) + (list(zip(sc.bonds["i"], sc.bonds["j"])) if len(sc.bonds) else [])
    for i, j in pairs:
        if j >= 0:
            links.setdefault(int(i), set()).add(int(j))
            links.setdefault(int(j), set()).add(int(i))
    accepted = []
    keep = np.ones(best.shape, dtype=bool)
    for x in bad:
        ring = {int(x)} | links.get(int(x), set())
        ring = ring.union(*[links.get(y, set()) for y in list(ring)])
        near = min(margin[y] for y in ring)
        if near < delta:
            accepted.append((int(x), float(best[x])))
            keep[x] = False
    return float(best[keep].max()) if keep.any() else 0.0, accepted
