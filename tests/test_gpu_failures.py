"""Failure statuses the C-ABI promises, caused on the host or by a short bounded wait (no
GPU fault): a device-side wait that runs out (PABD_ERR_TIMEOUT), a state that overflows
single precision (PABD_ERR_DIVERGED), adding to a scene after its first step
(PABD_ERR_STATE); and the batched pabd_step_many."""
import numpy as np
import pytest

import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2609_02675_gb300 as mod
    return mod


def _small_pile():
    return S.box_pile(nx=4, ny=3, nz=4, spacing=2.3, stacked=True, n_iter=8)


def test_wait_that_runs_out_is_reported_and_the_context_survives(P):
    """The fused persistent sweep waits at a grid barrier between its sweeps; with the bound
    shortened to one poll the early blocks give up, the step ends, and the next synchronising
    call returns PABD_ERR_TIMEOUT.  The device stays usable for other scenes."""
    g = P.Scene(_small_pile(), sweep_mode=3)
    if g.info()["sweep_mode"] != 3:
        g.close()
        pytest.skip("cooperative launch not available: no grid barrier to time out")
    g.set_wait_limit(1)
    g.step(2)
    assert g.sync(allow=(P.ERR_TIMEOUT,)) == P.ERR_TIMEOUT
    g.close()
    # a fresh scene on the same device steps normally, through the same barrier
    ok = P.Scene(_small_pile(), sweep_mode=3)
    ok.step(3)
    assert ok.sync() == P.OK
    assert np.isfinite(ok.state()).all()
    ok.close()


def test_overflowing_state_is_reported_as_diverged(P):
    """Two boxes joined by a spring, one placed at 3e38 (finite in single precision): the
    bond's length overflows, the solve turns non-finite and the step latches
    PABD_ERR_DIVERGED, returned by the next synchronising call."""
    sc = S.two_box_spring()
    sc.params = dict(sc.params, has_ground=0, body_contacts=0)
    g = P.Scene(sc)
    st = g.state()
    st[1, 0] = 3e38
    g.set_state(st)
    g.step(1)
    assert g.sync(allow=(P.ERR_DIVERGED,)) == P.ERR_DIVERGED
    g.close()


def test_adding_after_the_first_step_is_a_state_error(P):
    sc = S.chain_pendulum(n_steps=2)
    g = P.Scene(sc)
    g.step(1)
    g.sync()
    body = P.pabd_body_desc()
    body.he[:] = (0.5, 0.5, 0.5)
    body.mass = 1.0
    body.quat[:] = (0.0, 0.0, 0.0, 1.0)
    body.group = 0
    with pytest.raises(P.PabdError) as e:
        P.pabd_add_body(g.h, body)
    assert e.value.code == P.ERR_STATE
    bond = P.pabd_bond_desc()
    bond.type = S.SPHERICAL
    bond.body_i, bond.body_j = 0, 1
    bond.kappa = 1.0
    with pytest.raises(P.PabdError) as e:
        P.pabd_add_bond(g.h, bond)
    assert e.value.code == P.ERR_STATE
    g.close()


def test_step_many_equals_stepping_each_scene(P):
    """pabd_step_many over scenes of different kinds and step counts gives each scene the
    state it reaches when stepped alone, bit for bit."""
    import torch
    makes = [(_small_pile, 4), (lambda: S.chain_pendulum(n_steps=10), 7), (lambda: S.batched_trees(n_scenes=6), 0),
             (lambda: S.batched_trees(n_scenes=5, seed=S.SEED_BASE + 40), 3)]
    many = [P.Scene(m(), stream=torch.cuda.Stream()) for m, _ in makes]
    P.pabd_step_many([g.h for g in many], [n for _, n in makes])
    for (m, n), g in zip(makes, many):
        alone = P.Scene(m())
        alone.step(n)
        assert g.sync() == P.OK
        assert np.array_equal(g.state(), alone.state())
        alone.close()
        g.close()
    with pytest.raises(P.PabdError) as e:
        P.pabd_step_many([None], [1])
    assert e.value.code == P.ERR_ARG


def test_state_f32_round_trip_and_step_identical(P):
    """pabd_read_state_f32 / pabd_write_state_f32 move the device-layout state (q, Q, v, omega
    as 24 floats per body) without conversion: the values equal pabd_read_state's, and a step
    from a state written either way is the same bit for bit."""
    import torch
    sc = S.batched_trees(n_scenes=5, n_steps=10)
    g = P.Scene(sc)
    g.step(4)
    n = sc.n_bodies
    host = torch.empty(24 * n, dtype=torch.float32, pin_memory=True)
    g.read_state_f32(host.data_ptr())
    g.sync()
    f = host.numpy().astype(np.float64)
    rows = g.state()
    assert np.array_equal(f[:12 * n].reshape(n, 12), rows[:, 0:12])
    assert np.array_equal(f[12 * n:16 * n].reshape(n, 4), rows[:, 12:16])
    assert np.array_equal(f[16 * n:20 * n].reshape(n, 4)[:, :3], rows[:, 16:19])
    assert np.array_equal(f[20 * n:24 * n].reshape(n, 4)[:, :3], rows[:, 19:22])
    g.step(3)
    after_a = g.state()
    g.write_state_f32(host.data_ptr())
    g.set_step_index(4)
    g.step(3)
    assert np.array_equal(g.state(), after_a)
    g.set_state(rows)
    g.set_step_index(4)
    g.step(3)
    assert np.array_equal(g.state(), after_a)
    g.close()
