"""The serving loop: every scene's result is the same alone and in the mix -- packed with other
small scenes as the groups of one library scene, or across an eviction to the host and back
-- and the server reports latency and throughput."""
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


def _scene(sid):
    return S.box_pile_n([40, 300, 1200, 90, 700][sid % 5], seed=S.SEED_BASE + 100 + sid, n_iter=10)


@pytest.mark.parametrize("budget_mb", [4096, 8])
def test_served_results_equal_alone(P, budget_mb):
    from paper_2609_02675_gb300.serve import Server, replay
    rng = np.random.default_rng(3)
    reqs = []
    t = 0.0
    for k in range(40):
        t += rng.exponential(0.002)
        reqs.append((t, int(rng.integers(0, 5)), int(rng.integers(1, 8))))
    srv = Server(_scene, hbm_budget=budget_mb << 20)
    t0, t1 = replay(srv, reqs, drain_timeout=120.0)
    st = srv.stats(t0, t1)
    assert st["requests_done"] == len(reqs)
    assert st["steps"] == sum(n for _, _, n in reqs)
    assert st["step_latency_ms"]["p99"] >= st["step_latency_ms"]["p50"] > 0
    if budget_mb < 100:
        assert srv.evictions > 0
    totals = {}
    for _, sid, n in reqs:
        totals[sid] = totals.get(sid, 0) + n
    if budget_mb > 100:
        assert st["packed_scenes"] > 0 and st["pool_launches"] > 0
    for sid, n in totals.items():
        mixed = srv.state(sid)
        alone = P.Scene(_scene(sid))
        alone.step(n)
        assert np.array_equal(alone.state(), mixed), sid
        alone.close()
    srv.close()


def test_group_hold_keeps_held_groups_and_steps_the_rest_as_alone(P):
    """pabd_set_group_hold: a held group keeps its whole state through the step; the other
    groups step exactly as they do alone (same lane count), bit for bit; a scene with drives
    refuses holds."""
    sc = S.batched_trees(n_scenes=6, n_steps=10)
    g = P.Scene(sc)
    lanes = g.info()["sweep_lanes"]
    st0 = g.state()
    hold = np.array([0, 1, 0, 1, 0, 0], dtype=np.uint8)
    g.set_group_hold(hold)
    g.step(5)
    st1 = g.state()
    g.set_group_hold(None)
    g.step(3)
    st2 = g.state()
    for k in range(6):
        rows = S.group_rows(sc, [k])
        if hold[k]:
            assert np.array_equal(st1[rows], st0[rows])
        alone = P.Scene(S.select_groups(sc, [k]), sweep_lanes=lanes)
        alone.step(3 if hold[k] else 8)
        assert np.array_equal(alone.state(), st2[rows]), k
        alone.close()
    g.close()
    q = P.Scene(S.quadruped_bed_rod(bed=(4, 1, 4), n_rod=4, n_steps=2))
    with pytest.raises(P.PabdError) as e:
        q.set_group_hold(np.zeros(q.n_groups, dtype=np.uint8))
    assert e.value.code == P.ERR_ARG
    q.close()


def test_packed_server_throughput_beats_one_scene_per_launch(P):
    """Many small resident scenes: the packed server (one launch steps every scene with work)
    completes the same request stream in less time than one launch per scene, with identical
    results."""
    from paper_2609_02675_gb300.serve import Server, replay

    def make(sid):
        return S.box_pile_n(20 + 7 * sid, seed=S.SEED_BASE + 300 + sid, stacked=True, n_iter=10)

    n_sc = 48
    reqs = [(0.0, sid, 40) for sid in range(n_sc)]
    out = {}
    for pack in (False, True):
        srv = Server(make, hbm_budget=8 << 30, pack=pack, rebuild_interval=0.0)
        t0, t1 = replay(srv, reqs, drain_timeout=120.0)
        st = srv.stats(t0, t1)
        assert st["requests_done"] == len(reqs)
        out[pack] = (t1 - t0, {sid: srv.state(sid) for sid in range(n_sc)}, st)
        srv.close()
    assert out[True][2]["pool_launches"] > 0
    for sid in range(n_sc):
        assert np.array_equal(out[True][1][sid], out[False][1][sid]), sid
    assert out[True][0] < out[False][0], (out[True][0], out[False][0])
