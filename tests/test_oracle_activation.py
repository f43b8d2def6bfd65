"""The contact activation threshold of the oracle (the reading of the cited contact rule:
a contact acts in a sweep iff g < dhat at that sweep's iterate) and the two test probes
around it: the per-body activation margin and the threshold shift."""
import numpy as np

import oracle as O
import scenes as S
from tests.gpu_helpers import corners, scene_scale


def test_margin_and_zero_shift():
    """A body without contacts has an infinite margin; a resting cube's margin is at most the
    distance |g - dhat| of its bottom face at the final iterate (the margin is the minimum over
    the sweeps); a zero shift leaves the step unchanged bit for bit."""
    sc = S.single_body(c=(0, 0.5 + 1e-4, 0), n_iter=10)
    a = O.OracleScene(sc)
    b = O.OracleScene(sc)
    b.set_activation_shift(0.0)
    a.step(60)
    b.step(60)
    assert np.array_equal(a.state(), b.state())
    m = a.activation_margin()
    gap = a.state()[0, 1] - 0.5          # the cube stays axis-aligned: g of its bottom corners
    assert m.shape == (1,) and 0 <= m[0] <= abs(gap - 1e-3) + 1e-12
    free = S.single_body(c=(0, 5.0, 0), n_iter=5)
    f = O.OracleScene(free)
    f.step(1)
    assert np.isinf(f.activation_margin()[0])


def test_activation_threshold_discontinuity():
    """The Jacobi step is not continuous at the activation threshold: in the reduced
    quadruped-on-bed scene, step 28 has a contact whose gap sits 1e-8 from dhat (far below
    single-precision resolution at the scene's 4 m scale), and moving the threshold by 1e-8
    moves a neighbouring light grain by more than 1e-4 of the scene diagonal -- so the
    single-precision path may legitimately land on either side."""
    sc = S.quadruped_bed_rod(bed=(12, 2, 12), n_rod=16, n_steps=40)
    ref = O.OracleScene(sc)
    ref.step(27)
    st0, k0 = ref.state(), ref.step_index
    he = np.ascontiguousarray(sc.bodies["he"])
    out = {}
    for sh in (0.0, 1e-8, -1e-8):
        r = O.OracleScene(sc)
        r.set_state(st0)
        r.step_index = k0
        r.set_activation_shift(sh)
        r.step(1)
        out[sh] = (r.state(), r.activation_margin())
    margin = out[0.0][1]
    assert margin.min() < 1e-8
    scale = scene_scale(out[0.0][0], he)
    d_up = np.linalg.norm(corners(out[1e-8][0], he) - corners(out[0.0][0], he), axis=-1).max() / scale
    d_dn = np.linalg.norm(corners(out[-1e-8][0], he) - corners(out[0.0][0], he), axis=-1).max() / scale
    assert max(d_up, d_dn) > 1e-4
    assert min(d_up, d_dn) == 0.0
