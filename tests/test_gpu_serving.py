"""The serving loop: every scene's result is the same alone and in the mix (also across an
eviction to the host and back), and the server reports latency and throughput."""
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
    for sid, n in totals.items():
        r = srv.resident.get(sid)
        mixed = r.scene.state() if r is not None else srv.evicted[sid][0]
        alone = P.Scene(_scene(sid))
        alone.step(n)
        assert np.array_equal(alone.state(), mixed), sid
        alone.close()
    srv.close()
