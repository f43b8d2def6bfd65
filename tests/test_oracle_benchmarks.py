"""The paper's convergence and stability examples (Sec. 6), re-created as synthetic scenes,
pinned on the oracle: the two-box spring (its first step's sweeps as a closed-form linear
iteration), the 11 x 11 spring net (linear convergence; the fixed point of the unprojected
sweeps is the dense-Newton minimiser on a small net) and the extreme-mass-ratio stack
(stays upright and comes to rest)."""
import numpy as np
import pytest

import oracle as O
import scenes as S
from tests.dense_newton import minimise


def _centre_gap_after(k, **kw):
    o = O.OracleScene(S.two_box_spring(n_iter=k, **kw))
    o.step(1)
    st = o.state()
    return st[1, 0] - st[0, 0]


def test_two_box_spring_first_step_closed_form():
    """Each body's system (Eq. 19) about its centre: G = [[m + w, w x], [w x, Pi + w x^2]]
    (x = +-1/2 the face centre, w = h^2 kappa), right-hand side [m (s - c) + f', x f'] with
    f' = +-w (gap - l).  The projection discards the stretch, so the centre distance u obeys
    u <- u + G^-1_00 m (s_u - u) - 2 w (G^-1_00 + x G^-1_01) (u - 1 - l): a linear iteration
    with ratio rho = 1 - m G^-1_00 - 2 w (G^-1_00 + G^-1_01 / 2) and fixed point
    u* = (s_u m G^-1_00 + 2 w a (1 + l)) / (m G^-1_00 + 2 w a), a = G^-1_00 + G^-1_01 / 2."""
    h, m, kappa, l, he = 1.0 / 60.0, 1.0, 1e4, 1.0, 0.5
    w = h * h * kappa
    Pi = m * he * he / 3.0
    Gi = np.linalg.inv(np.array([[m + w, 0.5 * w], [0.5 * w, Pi + 0.25 * w]]))
    a = Gi[0, 0] + 0.5 * Gi[0, 1]
    rho = 1.0 - m * Gi[0, 0] - 2.0 * w * a
    s_u = 3.0                                   # v = 0, no gravity: s = q^n
    u_star = (s_u * m * Gi[0, 0] + 2.0 * w * a * (1.0 + l)) / (m * Gi[0, 0] + 2.0 * w * a)
    u = [3.0] + [_centre_gap_after(k) for k in range(1, 9)]
    e = np.array(u) - u_star
    np.testing.assert_allclose(e[1:] / e[:-1], rho, rtol=1e-8)
    assert rho < 0                              # the error alternates in sign
    assert abs(_centre_gap_after(400) - u_star) < 1e-12


def test_spring_net_converges_linearly():
    """The 11 x 11 net's first step: the sweeps' error ratio settles to a constant below 1
    (linear convergence of the successive substitution, Sec. 6)."""
    ref = O.OracleScene(S.spring_net(n_iter=600))
    ref.step(1)
    q_star = ref.state()[:, :12]
    errs = []
    for k in (10, 20, 40, 80):
        o = O.OracleScene(S.spring_net(n_iter=k))
        o.step(1)
        errs.append(np.abs(o.state()[:, :12] - q_star).max())
    r = [errs[i + 1] / errs[i] for i in range(3)]
    assert all(x < 1.0 for x in r), r
    assert abs(np.log(r[2]) / np.log(r[1]) - 2.0) < 0.2    # doubling k squares the ratio: geometric


def test_small_net_fixed_point_is_dense_newton_minimiser():
    """A 3 x 3 net of affine bodies (no projection, nothing pinned, no gravity): the sweeps
    iterated to convergence reach the minimiser of Eq. 13 found by dense Newton."""
    sc = S.spring_net(n=3, n_iter=3000)
    sc.params = dict(sc.params, project=0, gravity=(0.0, 0.0, 0.0))
    sc.bodies["pinned"] = 0
    o = O.OracleScene(sc)
    st0 = o.state()
    s_q = np.concatenate([st0[:, 0:3], st0[:, 3:12]], axis=1)
    o.step(1)
    st = o.state()
    q_or = np.concatenate([st[:, 0:3], st[:, 3:12]], axis=1)
    q_nt = minimise(sc, s_q)
    assert np.abs(q_or - q_nt).max() < 1e-9
    assert np.abs(q_or - s_q).max() > 1e-3


def test_mass_ratio_stack_stays_upright_and_settles():
    """Six cubes, each ten times heavier than the one below (1 kg to 100 t): over ten seconds
    the stack stands -- no sideways drift, the order kept, each box above the one below it,
    heights bounded -- and its bouncing dies down (stable, as the paper reports)."""
    sc = S.mass_ratio_stack(n_steps=600)
    o = O.OracleScene(sc)
    vmax = []
    for k in range(600):
        o.step(1)
        st = o.state()
        assert np.isfinite(st).all()
        assert np.abs(st[:, [0, 2]]).max() < 1e-9
        assert np.all(np.diff(st[:, 1]) > 0.5) and st[:, 1].max() < 6.0
        vmax.append(np.abs(st[:, 16:19]).max())
    vmax = np.array(vmax)
    assert vmax[500:].max() < 0.25 * vmax[100:200].max()


def _trees_two(resid_tol=0.0, n_iter=40):
    sc = S.batched_trees(n_scenes=2, n_min=4, n_max=12, n_steps=10)
    sc.params = dict(sc.params, n_iter=n_iter, resid_tol=resid_tol)
    return sc


def test_residual_threshold_stops_each_scene_at_its_first_converged_sweep():
    """Sec. 4.2's stopping rule per scene: with a threshold, each independent scene (group)
    keeps the iterate of the first sweep whose residual is at most the threshold.  Pinned
    against the definition: the same scene alone with a fixed count k, the smallest k whose
    residual is at most the threshold."""
    tol = 1e-4
    sc = _trees_two(resid_tol=tol)
    o = O.OracleScene(sc)
    o.step(3)
    st0, k0 = o.state(), o.step_index
    o.step(1)
    st_tol = o.state()
    sizes = sc.meta["sizes"]
    off = np.concatenate([[0], np.cumsum(sizes)])
    for g in range(2):
        sl = slice(off[g], off[g + 1])
        for k in range(1, 41):
            sub = _trees_two(n_iter=k)
            r = O.OracleScene(sub)
            r.set_state(st0)
            r.step_index = k0
            r.step(1)
            if r.residual()[g] <= tol or k == 40:
                assert np.array_equal(r.state()[sl], st_tol[sl]), (g, k)
                break
    assert o.last_sweeps() < 40


def test_zero_threshold_changes_nothing():
    a = O.OracleScene(_trees_two())
    b = O.OracleScene(_trees_two(resid_tol=0.0))
    a.step(5)
    b.step(5)
    assert np.array_equal(a.state(), b.state()) and a.last_sweeps() == 40


def _corner_dev(a, b, he):
    """max corner distance between two states / scene diagonal (no GPU helpers here)."""
    signs = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=float)

    def corners(st):
        x = signs[None, :, :] * he[:, None, :]
        A = st[:, 3:12].reshape(-1, 3, 3)
        return st[:, None, 0:3] + np.einsum("nij,nkj->nki", A, x)

    ca, cb = corners(a), corners(b)
    y = cb.reshape(-1, 3)
    diag = max(float(np.linalg.norm(y.max(0) - y.min(0))), 1.0)
    return float(np.linalg.norm(ca - cb, axis=-1).max()) / diag


def test_unconverged_sweeps_amplify_input_rounding():
    """Where a scene's sweeps do not converge, the step amplifies a perturbation of its input:
    on the batched trees at step 17, a group runs all 40 sweeps without reaching the 1e-3
    threshold, and rounding the start state to single precision moves the result about 30
    times more after 40 sweeps than after 10 (1.0e-5 against 3.1e-7 of the scene diagonal).  This is the map's own sensitivity (the oracle
    against itself), which bounds how closely any single-precision path can follow it there."""
    def mk(n_iter, tol):
        sc = S.batched_trees(n_scenes=24, n_steps=30)
        sc.params = dict(sc.params, n_iter=n_iter, resid_tol=tol)
        return sc

    sc = mk(40, 1e-3)
    he = np.asarray(sc.bodies["he"], dtype=float)
    ref = O.OracleScene(sc)
    ref.step(17)
    st0, k0 = ref.state(), ref.step_index
    sens = {}
    for n_iter in (10, 40):
        a = O.OracleScene(mk(n_iter, 0.0))
        a.set_state(st0)
        a.step_index = k0
        a.step(1)
        b = O.OracleScene(mk(n_iter, 0.0))
        b.set_state(st0.astype(np.float32).astype(np.float64))
        b.step_index = k0
        b.step(1)
        sens[n_iter] = _corner_dev(b.state(), a.state(), he)
    ref.step(1)
    assert ref.last_sweeps() == 40  # some group never reached the threshold
    assert sens[10] < 1e-6
    assert sens[40] > 3e-6 and sens[40] > 10.0 * sens[10], sens


def test_iterate_rounding_probe():
    """The oracle's iterate-rounding probe and the sensitivity measure built on it.  Off, a step
    is the method's bit for bit.  On the 7-joint chain (10 sweeps, converging) it moves the step
    by about the rounding itself.  On the batched trees at step 17, where one group's 40 sweeps
    do not converge, perturbations of single-precision size move that group by more than the
    1e-5 tolerance while the converged groups stay at the rounding level: the tolerance cannot
    be met there by any single-precision path, only the map's own sensitivity."""
    from tests.gpu_helpers import rounding_sensitivity

    sc = S.chain_pendulum(n_steps=10)
    he = np.asarray(sc.bodies["he"], dtype=float)
    a, b, c = O.OracleScene(sc), O.OracleScene(sc), O.OracleScene(sc)
    b.set_round_iterates(False)
    c.set_round_iterates(True)
    for o in (a, b, c):
        o.step(5)
    assert np.array_equal(a.state(), b.state())
    dev = _corner_dev(c.state(), a.state(), he)
    assert 0.0 < dev < 1e-6, dev

    def mk():
        t = S.batched_trees(n_scenes=24, n_steps=30)
        t.params = dict(t.params, n_iter=40, resid_tol=1e-3)
        return t

    sc = mk()
    he = np.asarray(sc.bodies["he"], dtype=float)
    ref = O.OracleScene(sc)
    ref.step(17)
    st0, k0 = ref.state(), ref.step_index
    ref.step(1)
    assert ref.last_sweeps() == 40
    open_groups = np.nonzero(ref.residual() > 1e-3)[0]
    loose = np.isin(np.asarray(sc.bodies["group"]), open_groups)
    assert 0 < loose.sum() < len(loose)
    s_open = rounding_sensitivity(mk, st0, k0, ref.state(), he, O, mask=loose)
    s_closed = rounding_sensitivity(mk, st0, k0, ref.state(), he, O, mask=~loose)
    assert s_open > 1e-5 and s_closed < 1e-6, (s_open, s_closed)
