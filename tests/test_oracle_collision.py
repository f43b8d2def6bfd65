"""Pins of the oracle's collision detection (Alg. 1, first line) on hand-built layouts whose
pair lists and contact manifolds are known from the geometry alone (CPU only)."""
import numpy as np

import oracle as O
import scenes as S


def _scene(cs, he=0.5, quats=None, v=None, groups=None, pinned=None, bonds=None, **kw):
    n = len(cs)
    b = S._bodies(n)
    b["he"] = he
    b["mass"] = 1.0
    b["c"] = cs
    if quats is not None:
        b["quat"] = quats
    if v is not None:
        b["v"] = v
    if groups is not None:
        b["group"] = groups
    if pinned is not None:
        b["pinned"] = pinned
    bo = S._bonds(0) if bonds is None else bonds
    p = dict(has_ground=0)
    p.update(kw)
    return S.Scene("t", S.default_params(**p), b, bo, 1)


def _pairs(sc):
    o = O.OracleScene(sc)
    o.detect()
    return [tuple(p) for p in o.pairs()], o


def test_pairs_axis_aligned_row():
    # unit cubes at rest: inflation = dhat (1e-3 * edge 1) + margin 1e-3 = 2e-3 per body,
    # so two cubes overlap on x iff |dx| <= 1 + 4e-3
    cs = [(0, 0, 0), (1.0039, 0, 0), (2.5, 0, 0), (3.0, 0, 0), (10, 0, 0), (11.0041, 0, 0)]
    pairs, _ = _pairs(_scene(cs))
    assert pairs == [(0, 1), (2, 3)]


def test_pairs_rotated_box_uses_world_aabb():
    q45 = S._quat_axis_angle((0, 0, 1), np.pi / 4)
    quats = np.array([q45, (0, 0, 0, 1.0)])
    # rotated cube AABB half-width 0.5*sqrt(2); overlap iff dx <= 0.70711 + 0.5 + 0.004
    pairs, _ = _pairs(_scene([(0, 0, 0), (1.2100, 0, 0)], quats=quats))
    assert pairs == [(0, 1)]
    pairs, _ = _pairs(_scene([(0, 0, 0), (1.2122, 0, 0)], quats=quats))
    assert pairs == []


def test_pairs_velocity_inflation():
    # a body moving at 6 m/s is inflated by h*6 = 0.1 (h = 1/60)
    cs = [(0, 0, 0), (1.08, 0, 0)]
    assert _pairs(_scene(cs))[0] == []
    assert _pairs(_scene(cs, v=[(6.0, 0, 0), (0, 0, 0)]))[0] == [(0, 1)]


def test_pairs_filters_group_pinned_and_bonded():
    cs = [(0, 0, 0), (1.0, 0, 0), (2.0, 0, 0), (3.0, 0, 0)]
    assert _pairs(_scene(cs))[0] == [(0, 1), (1, 2), (2, 3)]
    assert _pairs(_scene(cs, groups=[0, 0, 1, 1]))[0] == [(0, 1), (2, 3)]
    assert _pairs(_scene(cs, pinned=[1, 1, 0, 0]))[0] == [(1, 2), (2, 3)]
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"], bo["kappa"] = S.SPHERICAL, 2, 1, 1.0
    assert _pairs(_scene(cs, bonds=bo))[0] == [(0, 1), (2, 3)]
    assert _pairs(_scene(cs, body_contacts=0))[0] == []


def test_pairs_brute_force_random():
    """The pair list equals the set of all (i < j) whose inflated boxes overlap on every axis
    (checked with numpy on random axis-aligned layouts where no gap is near zero)."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        n = 60
        cs = rng.uniform(0, 6, (n, 3))
        he = rng.uniform(0.2, 0.6, (n, 3))
        sc = _scene(cs)
        sc.bodies["he"] = he
        infl = 1e-3 * 2 * he.min(1) + 1e-3
        e = he + infl[:, None]
        gap = np.abs(cs[:, None, :] - cs[None, :, :]) - (e[:, None, :] + e[None, :, :])
        ov = (gap <= 0).all(-1)
        exp = [(i, j) for i in range(n) for j in range(i + 1, n) if ov[i, j]]
        near = np.abs(gap).min() < 1e-5
        pairs, _ = _pairs(sc)
        if not near:
            assert pairs == exp


def test_manifold_box_on_box_offset():
    """A unit cube resting 1 mm above another, offset by (0.2, 0.1): four contacts at the
    corners of the overlap rectangle, normal +y from the lower box's top face, anchors on
    that face, material points on the upper box's bottom face."""
    sc = _scene([(0, 0, 0), (0.2, 1.001, 0.1)])
    o = O.OracleScene(sc)
    o.detect()
    meta, data = o.contacts()
    assert len(meta) == 4
    # reference = the box whose face normal separates best (ties: b's axes first)
    i, j = meta[0, 1], meta[0, 2]
    assert {i, j} == {0, 1}
    xi, xj, N = data[:, 0:3], data[:, 3:6], data[:, 6:9]
    if j == 0:   # reference is the lower box: anchors on its top face y = +0.5, N = +y
        np.testing.assert_allclose(N, np.tile([0, 1, 0], (4, 1)), atol=1e-7)
        np.testing.assert_allclose(xj[:, 1], 0.5, atol=1e-7)
        np.testing.assert_allclose(xi[:, 1], -0.5, atol=1e-6)
        world_xz = np.sort(np.round(xj[:, [0, 2]], 5), axis=0)
    else:        # reference is the upper box: anchors on its bottom face, N = -y
        np.testing.assert_allclose(N, np.tile([0, -1, 0], (4, 1)), atol=1e-7)
        np.testing.assert_allclose(xj[:, 1], -0.5, atol=1e-7)
        world_xz = np.sort(np.round(xj[:, [0, 2]] + [0.2, 0.1], 5), axis=0)
    exp = np.sort(np.array([(-0.3, -0.4), (0.5, -0.4), (-0.3, 0.5), (0.5, 0.5)]), axis=0)
    np.testing.assert_allclose(world_xz, exp, atol=1e-5)


def test_manifold_side_contact_and_separation():
    # side by side along x with a 1 mm gap: normal along x
    sc = _scene([(0, 0, 0), (1.001, 0.3, 0.0)])
    o = O.OracleScene(sc)
    o.detect()
    meta, data = o.contacts()
    assert len(meta) == 4
    assert np.allclose(np.abs(data[:, 6:9]), [1, 0, 0], atol=1e-7)
    # 1 cm gap (more than the 4 mm inflation): the pair overlaps in AABB only if inflated more
    sc = _scene([(0, 0, 0), (1.01, 0.0, 0.0)], v=[(1.0, 0, 0), (0, 0, 0)])  # h*v inflates 1/60
    o = O.OracleScene(sc)
    o.detect()
    meta, _ = o.contacts()
    assert len(meta) == 4
    sc = _scene([(0, 0, 0), (1.01, 0.0, 0.0)])
    o = O.OracleScene(sc)
    o.detect()
    assert len(o.contacts()[0]) == 0


def test_ground_contacts_tilted_box():
    """A cube tilted 30 deg about z just above y = 0: its two lowest corners (both z signs)
    are within the inflation, anchored at their vertical projections."""
    th = np.deg2rad(30)
    q = S._quat_axis_angle((0, 0, 1), th)
    R = O.quat_to_mat(q)
    corners = np.array([[sx, sy, sz] for sz in (-0.5, 0.5) for sy in (-0.5, 0.5) for sx in (-0.5, 0.5)])
    low = (corners @ R.T)[:, 1].min()
    c = np.array([0.0, -low + 1e-3, 0.0])
    sc = _scene([c], quats=np.array([q]), has_ground=1)
    o = O.OracleScene(sc)
    o.detect()
    meta, data = o.contacts()
    assert len(meta) == 2 and (meta[:, 0] == O.GROUND).all() and (meta[:, 2] == -1).all()
    y = c + data[:, 0:3] @ R.T
    np.testing.assert_allclose(y[:, 1], 1e-3, atol=1e-6)
    np.testing.assert_allclose(data[:, 3:6], y * [1, 0, 1], atol=1e-6)
    np.testing.assert_allclose(data[:, 6:9], np.tile([0, 1, 0], (2, 1)))
