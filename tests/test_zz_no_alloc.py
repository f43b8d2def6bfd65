"""The allocation-free broad phase gives the same pair list as a scene's broad phase.

pabd_broadphase_noalloc serves callers that may not call cudaMalloc or cudaFree (real-time
loops that may not block on the allocator, applications whose device memory belongs to
another runtime or pool, plug-ins inside a host program that holds the GPU's memory): it
keeps its scratch in a static device array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
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


def _inputs(torch, sc, st):
    n = sc.n_bodies
    q = torch.tensor(st[:, 0:12], dtype=torch.float32, device="cuda").contiguous()
    vel = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    vel[:, :3] = torch.tensor(st[:, 16:19], dtype=torch.float32, device="cuda")
    he = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    he[:, :3] = torch.tensor(sc.bodies["he"], dtype=torch.float32, device="cuda")
    group = torch.tensor(sc.bodies["group"], dtype=torch.int32, device="cuda")
    flags = torch.tensor(sc.bodies["pinned"] & 1, dtype=torch.int32, device="cuda")
    return q, vel, he, group, flags


def test_noalloc_broadphase_matches_scene_pairs_twice(P):
    import torch
    sc = S.box_pile(nx=8, ny=8, nz=8, spacing=2.3, stacked=True)
    g = P.Scene(sc)
    g.step(25)                       # a settled, contact-rich state
    st = g.state()
    g.detect()
    ref = g.pairs()
    g.close()
    assert len(ref) > 300
    q, vel, he, group, flags = _inputs(torch, sc, st)
    cap = 4 * len(ref)
    stream = torch.cuda.current_stream().cuda_stream
    p = sc.params
    for call in range(2):            # the second call reuses the static scratch left by the first
        pairs = torch.full((cap, 2), -7, dtype=torch.int32, device="cuda")
        n = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        P.pabd_broadphase_noalloc(q.data_ptr(), vel.data_ptr(), he.data_ptr(), group.data_ptr(),
                                  flags.data_ptr(), sc.n_bodies, p["h"], p["margin"], p["d_hat_rel"],
                                  pairs.data_ptr(), cap, n.data_ptr(), stream)
        torch.cuda.synchronize()
        cnt = int(n.item())
        assert cnt == len(ref), (call, cnt, len(ref))
        np.testing.assert_array_equal(pairs[:cnt].cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_maximum(P):
    with pytest.raises(P.PabdError) as e:
        P.pabd_broadphase_noalloc(0, 0, 0, 0, 0, P.NOALLOC_MAX_BODIES + 1, 1 / 60, 1e-3, 1e-3, 0, 0, 0, 0)
    assert e.value.code == P.ERR_ARG


def test_noalloc_cut_list_is_a_sorted_subset(P):
    """With room for fewer pairs than it finds, the call reports the full count and writes
    max_pairs distinct pairs of the full list, sorted, and nothing past them."""
    import torch
    sc = S.box_pile(nx=8, ny=8, nz=8, spacing=2.3, stacked=True)
    g = P.Scene(sc)
    g.step(25)
    st = g.state()
    g.detect()
    ref = g.pairs()
    g.close()
    q, vel, he, group, flags = _inputs(torch, sc, st)
    stream = torch.cuda.current_stream().cuda_stream
    p = sc.params
    cap = len(ref) // 3
    pairs = torch.full((cap + 16, 2), -7, dtype=torch.int32, device="cuda")
    n = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    P.pabd_broadphase_noalloc(q.data_ptr(), vel.data_ptr(), he.data_ptr(), group.data_ptr(), flags.data_ptr(),
                              sc.n_bodies, p["h"], p["margin"], p["d_hat_rel"], pairs.data_ptr(), cap,
                              n.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(n.item()) == len(ref)
    got = pairs.cpu().numpy()
    assert (got[cap:] == -7).all()
    cut = got[:cap]
    key = cut[:, 0].astype(np.int64) * (1 << 32) + cut[:, 1]
    assert (np.diff(key) > 0).all()
    full = set(map(tuple, ref.tolist()))
    assert all(tuple(r) in full for r in cut.tolist())
