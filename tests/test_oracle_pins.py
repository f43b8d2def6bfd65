"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against a closed form, an identity printed in the paper, a
library routine on a special case, an independent brute-force minimiser, or a conservation
law -- never against the oracle itself.
"""
import math

import numpy as np
import pytest

import oracle as O
import scenes as S
from tests.dense_newton import minimise, quadrature_pi

H60 = 1.0 / 60.0
G = 9.81


def _rand_rot(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# --------------------------------------------------------------------------------------
# free bodies: Alg. 1 with no bonds gives H = M, so q^{n+1} = s exactly
# --------------------------------------------------------------------------------------

def test_ballistic_free_body_closed_form():
    """v_n = v_0 + n h g, c_n = c_0 + n h v_0 + h^2 g n(n+1)/2 (predictor of Alg. 1)."""
    v0 = np.array([1.3, 4.0, -0.7])
    c0 = np.array([0.2, 50.0, -1.0])
    n = 37
    o = O.OracleScene(S.single_body(c=c0, v=v0, has_ground=0))
    o.step(n)
    st = o.state()[0]
    g = np.array([0.0, -G, 0.0])
    # v = (c^{n+1} - c^n)/h: rounding of |c| ~ 50 divided by h, accumulated over n steps
    tol_v = 4 * n * 50.0 * np.finfo(float).eps / H60
    np.testing.assert_allclose(st[16:19], v0 + n * H60 * g, rtol=0, atol=tol_v)
    np.testing.assert_allclose(st[0:3], c0 + n * H60 * v0 + H60 ** 2 * g * n * (n + 1) / 2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(st[3:12].reshape(3, 3), np.eye(3), atol=1e-15)


@pytest.mark.parametrize("axis", [(0, 0, 1), (1, 2, -0.5)])
def test_free_spin_closed_form(axis):
    """Fixed-axis spin: tan(dtheta/2) = h|w|/2 per step and |w_{n+1}| = |w_n| / (1 + h^2|w_n|^2/4)
    (quaternion predictor of Alg. 1, skew part of (A^{n+1} - A^n)(A^n)^T / h)."""
    u = np.array(axis, dtype=float)
    u /= np.linalg.norm(u)
    w = 4.0
    o = O.OracleScene(S.single_body(omega=w * u, has_ground=0, gravity=(0, 0, 0)))
    th = 0.0
    for _ in range(60):
        o.step(1)
        th += 2.0 * math.atan(H60 * w / 2.0)
        w = w / (1.0 + H60 * H60 * w * w / 4.0)
    st = o.state()[0]
    np.testing.assert_allclose(st[19:22], w * u, atol=1e-12)
    q = st[12:16]
    ang = 2.0 * math.atan2(np.linalg.norm(q[:3]), q[3])
    assert abs(ang - th) < 1e-12
    np.testing.assert_allclose(q[:3] / np.linalg.norm(q[:3]), u, atol=1e-12)


# --------------------------------------------------------------------------------------
# pendulum, momentum, dense Newton
# --------------------------------------------------------------------------------------

def test_small_angle_pendulum_period():
    """Unit cube on a spherical bond at its top-face centre: T = 2 pi sqrt(I_p / (m g L)),
    I_p = m/6 + m/4, L = 1/2; implicit Euler period T_h = 2 pi h / atan(w0 h). Within 1%."""
    th0 = 0.05
    sc = S.single_body(quat=S._quat_axis_angle((0, 0, 1), th0), n_iter=200, has_ground=0)
    R = O.quat_to_mat(sc.bodies["quat"][0])
    sc.bodies["c"][0] = -R @ np.array([0.0, 0.5, 0.0])
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"] = S.SPHERICAL, 0, S.WORLD
    bo["xi"] = (0.0, 0.5, 0.0)
    bo["kappa"] = 1e4 / H60 ** 2
    sc.bonds = bo
    o = O.OracleScene(sc)
    ang = []
    for _ in range(560):
        o.step(1)
        A = o.state()[0, 3:12].reshape(3, 3)
        ang.append(math.atan2(A[1, 0], A[0, 0]))
    ang = np.array(ang)
    zc = np.where(np.diff(np.sign(ang)) != 0)[0]
    # linear interpolation of the zero crossings
    tz = np.array([(k + ang[k] / (ang[k] - ang[k + 1])) * H60 for k in zc])
    period = 2.0 * np.diff(tz).mean()
    w0 = math.sqrt(G * 0.5 / (1.0 / 6.0 + 0.25))
    Th = 2.0 * math.pi * H60 / math.atan(w0 * H60)
    assert abs(period / Th - 1.0) < 0.01
    assert abs(ang).max() <= th0 + 1e-9  # implicit Euler never gains amplitude


@pytest.mark.parametrize("btype", [S.SPRING, S.ELASTIC_NL])
@pytest.mark.parametrize("project", [0, 1])
def test_linear_momentum_isolated_pair(btype, project):
    """Two free bodies joined by one bond, no gravity: at convergence of the iteration the
    bond forces are equal and opposite, so sum m v is conserved.  Affine bodies (no
    projection) with off-centre attachment points; rigid bodies with the bond at the centres
    (with the projection, off-centre ends see the other body projected and themselves not,
    so their forces are not opposite at the alternation's fixed point)."""
    b = S._bodies(2)
    b["he"] = [(0.3, 0.4, 0.5), (0.5, 0.2, 0.3)]
    b["mass"] = [1.0, 2.5]
    b["c"] = [(0, 0, 0), (1.5, 0.2, -0.1)]
    b["v"] = [(0.5, -0.2, 0.1), (-0.3, 0.4, 0.2)]
    b["omega"] = [(0.3, 0.1, -0.2), (0.0, 0.5, 0.1)] if project else [(0, 0, 0), (0, 0, 0)]
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"] = btype, 0, 1
    if not project:
        bo["xi"] = (0.3, 0.1, 0.0)
        bo["xj"] = (-0.5, 0.0, 0.1)
    bo["kappa"] = 5.0 / H60 ** 2
    bo["rest"] = 1.1
    sc = S.Scene("pair", S.default_params(n_iter=600, gravity=(0, 0, 0), has_ground=0, body_contacts=0,
                                          project=project), b, bo, 1)
    o = O.OracleScene(sc)
    P0 = (b["mass"][:, None] * b["v"]).sum(0)
    for _ in range(5):
        o.step(1)
        assert o.residual()[0] < 1e-9
    st = o.state()
    P = (b["mass"][:, None] * st[:, 16:19]).sum(0)
    assert np.abs(P - P0).max() < 1e-9 * np.abs(b["mass"][:, None] * b["v"]).max()
    assert np.abs(st[:, 16:19] - b["v"]).max() > 1e-3   # the bond did act


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sissm_fixed_point_is_dense_newton_minimiser(seed):
    """Without the local projection, Eq. (19) iterated to convergence must be the minimiser of
    the incremental potential Eq. (13) (affine bodies, spherical/spring/NL-elastic bonds),
    found independently by dense Newton with line search."""
    sc = S.random_small(seed, n_bodies=3 + seed % 2, n_bonds=4, project=0, n_iter=4000)
    o = O.OracleScene(sc)
    st0 = o.state()
    s_q = np.concatenate([st0[:, 0:3], st0[:, 3:12]], axis=1)   # v = w = 0, g = 0: s = q^n
    o.step(1)
    st = o.state()
    q_or = np.concatenate([st[:, 0:3], st[:, 3:12]], axis=1)
    q_nt = minimise(sc, s_q)
    assert np.abs(q_or - q_nt).max() < 1e-9
    assert np.abs(q_or - s_q).max() > 1e-3   # the bonds did move the bodies


# --------------------------------------------------------------------------------------
# algebra of the per-body system (Eq. 20, 23, 24, 25), polar and quaternions
# --------------------------------------------------------------------------------------

def _bonded_scene():
    sc = S.random_small(7, n_bodies=3, n_bonds=5, n_iter=3)
    return sc, O.OracleScene(sc)


def test_dense_H_has_sparse_structure_of_eq24():
    """H_i = [[a I, e_x b^T, e_y b^T, e_z b^T], [b e_x^T, D, 0, 0], ...] with
    a = m + h^2 sum w~, b = h^2 sum w~ x, D = Pi + h^2 sum w~ x x^T, w~ = phi+/d (Eq. 24)."""
    sc, o = _bonded_scene()
    h = sc.params["h"]
    st = o.state()
    for body in range(sc.n_bodies):
        H, _ = o.body_system(body)
        m = sc.bodies["mass"][body]
        Pi = quadrature_pi(sc.bodies["he"][body], m)
        a = m
        bvec = np.zeros(3)
        D = Pi.copy()
        for bo in sc.bonds:
            for end, (bb, x, xo, other) in enumerate([(bo["i"], bo["xi"], bo["xj"], bo["j"]),
                                                      (bo["j"], bo["xj"], bo["xi"], bo["i"])]):
                if bb != body:
                    continue
                yi = st[bb, 0:3] + st[bb, 3:12].reshape(3, 3) @ x
                yo = st[other, 0:3] + st[other, 3:12].reshape(3, 3) @ xo
                d = np.linalg.norm(yo - yi)
                k, l = bo["kappa"], bo["rest"]
                # phi+ of each bond: spherical kappa d, spring kappa d, nonlinear elastic
                # phi'(d) d = kappa d^3 / l^2 (tangent split)
                phip = {S.SPHERICAL: k * d, S.SPRING: k * d, S.ELASTIC_NL: k * d ** 3 / (l * l)}[int(bo["type"])]
                wt = phip / d
                a += h * h * wt
                bvec += h * h * wt * x
                D += h * h * wt * np.outer(x, x)
        Hs = np.zeros((12, 12))
        Hs[:3, :3] = a * np.eye(3)
        for k in range(3):
            Hs[k, 3 + 3 * k:6 + 3 * k] = bvec
            Hs[3 + 3 * k:6 + 3 * k, k] = bvec
            Hs[3 + 3 * k:6 + 3 * k, 3 + 3 * k:6 + 3 * k] = D
        np.testing.assert_allclose(H, Hs, rtol=1e-12, atol=1e-9 * np.abs(Hs).max())


def test_eq25_block_inverse():
    """H^-1 from Eq. (25): [(1/a + a~) I, -e b~^T D~^-1; -D~^-1 b~ e^T, D~^-1 blocks],
    a~ = b~^T D~^-1 b~, b~ = b/a, D~ = D - b b^T / a; times H gives I."""
    sc, o = _bonded_scene()
    for body in range(sc.n_bodies):
        H, _ = o.body_system(body)
        a = H[0, 0]
        b = H[0, 3:6]
        D = H[3:6, 3:6]
        bt = b / a
        Dt = D - np.outer(b, b) / a
        Di = np.linalg.inv(Dt)
        at = bt @ Di @ bt
        Hi = np.zeros((12, 12))
        Hi[:3, :3] = (1.0 / a + at) * np.eye(3)
        for k in range(3):
            Hi[k, 3 + 3 * k:6 + 3 * k] = -(bt @ Di)
            Hi[3 + 3 * k:6 + 3 * k, k] = -(Di @ bt)
            Hi[3 + 3 * k:6 + 3 * k, 3 + 3 * k:6 + 3 * k] = Di
        np.testing.assert_allclose(Hi @ H, np.eye(12), atol=1e-9)


def test_cholesky_matches_library_solve():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((12, 12))
    H = X @ X.T + 12 * np.eye(12)
    b = rng.standard_normal(12)
    np.testing.assert_allclose(O.cholesky_solve(H, b), np.linalg.solve(H, b), rtol=1e-12, atol=1e-13)


def test_polar_rotation_special_cases():
    """The local solve returns R of A = R S (S symmetric positive definite); for det A < 0 it
    returns the proper rotation maximising tr(R^T A) (the smallest singular direction flips)."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        R = _rand_rot(rng)
        X = rng.standard_normal((3, 3))
        Sm = X @ X.T + 0.1 * np.eye(3)
        Rp, _ = O.polar_rotation(R @ Sm)
        np.testing.assert_allclose(Rp, R, atol=1e-10)
        # reflection: A = R diag(s1, s2, -s3) with s3 the smallest
        s = np.sort(rng.uniform(0.5, 2.0, 3))[::-1]
        Rp2, sig = O.polar_rotation(R @ np.diag([s[0], s[1], -s[2]]))
        np.testing.assert_allclose(Rp2, R, atol=1e-10)
        np.testing.assert_allclose(sig, s, rtol=1e-12)
    # rank-deficient input still yields a rotation
    for A in (np.outer([1.0, 2, 3], [0.5, -1, 2]), np.zeros((3, 3)), np.diag([1.0, 1.0, 0.0])):
        Rp, _ = O.polar_rotation(A)
        np.testing.assert_allclose(Rp.T @ Rp, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(Rp) - 1.0) < 1e-12


def test_quaternion_conversions_roundtrip():
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        R = O.quat_to_mat(q)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        q2 = O.mat_to_quat(R)
        assert min(np.abs(q2 - q).max(), np.abs(q2 + q).max()) < 1e-13
        # axis-angle definition: rotating the axis leaves it fixed, rotation angle from w
        ax = q[:3] / np.linalg.norm(q[:3])
        np.testing.assert_allclose(R @ ax, ax, atol=1e-13)
        ang = 2 * math.atan2(np.linalg.norm(q[:3]), q[3])
        assert abs(math.acos(np.clip((np.trace(R) - 1) / 2, -1, 1)) - min(ang, 2 * math.pi - ang)) < 1e-7


def test_mass_matrix_pi_is_box_second_moment():
    """Thm 4.1: Pi_0 = int rho x x^T dV; the oracle's H with no bonds is exactly M."""
    he = (0.3, 0.7, 1.1)
    sc = S.single_body(he=he, mass=2.3, has_ground=0)
    o = O.OracleScene(sc)
    H, _ = o.body_system(0)
    M = np.zeros((12, 12))
    M[:3, :3] = 2.3 * np.eye(3)
    P = quadrature_pi(np.array(he), 2.3)
    for k in range(3):
        M[3 + 3 * k:6 + 3 * k, 3 + 3 * k:6 + 3 * k] = P
    np.testing.assert_allclose(H, M, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------------------
# bond readings: closed forms of their equilibria
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("btype", [S.SPRING, S.ELASTIC_NL])
def test_hanging_body_equilibrium(btype):
    """A body hung from a world point by one bond at its centre settles where phi(d) = m g:
    spring kappa (d - l) = m g; nonlinear elastic (kappa/3)(d^3/l^2 - l) = m g."""
    m, kappa, l = 2.0, 400.0, 0.5
    sc = S.single_body(mass=m, c=(0, -0.6, 0), n_iter=60, has_ground=0)
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"] = btype, 0, S.WORLD
    bo["kappa"], bo["rest"] = kappa, l
    sc.bonds = bo
    o = O.OracleScene(sc)
    o.step(1500)
    d = -o.state()[0, 1]
    if btype == S.SPRING:
        d_ref = l + m * G / kappa
    else:
        d_ref = np.roots([1.0 / (l * l), 0.0, 0.0, -(l + 3 * m * G / kappa)]).real.max()
    assert abs(d - d_ref) < 1e-9


def test_resting_box_compression_closed_form():
    """Reading of contact (ground bonds pull corners to height dhat, w = c_kappa m) with the
    local projection: at rest the bottom corners sit e = h^2 g (1 + 12 c_kappa)/(4 c_kappa)
    below dhat (the global step spends 3/4 of each corner correction on the affine scaling
    that the projection removes: c moves m, a corner moves via A at cost Pi/he^2 = m/3)."""
    for he, ck in (((0.5, 0.5, 0.5), 1.0), ((0.3, 0.7, 1.1), 2.0), ((1.0, 0.4, 0.6), 4.0)):
        he = np.array(he)
        sc = S.single_body(he=he, c=(0, he[1] + 5e-4, 0), n_iter=20, c_kappa=ck)
        o = O.OracleScene(sc)
        o.step(800)
        y = o.state()[0, 1]
        dhat = 1e-3 * 2 * he.min()
        e = H60 ** 2 * G * (1 + 12 * ck) / (4 * ck)
        assert abs(y - (he[1] + dhat - e)) < 1e-7


def test_frictionless_slide_keeps_velocity_and_friction_stops():
    sc = S.single_body(c=(0, 0.4921, 0), v=(2.0, 0, 0), n_iter=20, mu=0.0)
    o = O.OracleScene(sc)
    o.step(150)
    st = o.state()[0]
    assert abs(st[16] - 2.0) < 1e-9 and abs(st[18]) < 1e-12
    sc = S.single_body(c=(0, 0.4921, 0), v=(2.0, 0, 0), n_iter=20, mu=0.5)
    o = O.OracleScene(sc)
    vs = []
    for _ in range(120):
        o.step(1)
        vs.append(o.state()[0, 16])
    vs = np.array(vs)
    assert np.all(np.diff(vs[:20]) < 0)
    assert abs(vs[-1]) < 1e-6


def test_contact_rule_coulomb_cone():
    """Force on end i = w (target - y_i)/h^2: normal part w (dhat - g)/h^2 >= 0; tangential
    part bounded by mu times the normal part, with equality while slipping; inactive for
    g >= dhat; equal and opposite on the two ends."""
    rng = np.random.default_rng(2)
    N = np.array([0.0, 0.0, 1.0])
    for _ in range(300):
        yj = rng.standard_normal(3)
        rr = rng.standard_normal(3) * np.array([0.02, 0.02, 0.01])
        yi = yj + rr
        dhat, w, mu = 1e-3, rng.uniform(0.5, 3), rng.uniform(0, 1)
        wo, fi, fj = O.contact_rule(N, dhat, w, mu, yi, yj)
        g = rr @ N
        if g >= dhat:
            assert wo == 0 and not fi.any()
            continue
        Fi = fi - w * yi
        Fj = fj - w * yj
        np.testing.assert_allclose(Fi, -Fj, atol=1e-13)
        Fn = Fi @ N
        Ft = np.linalg.norm(Fi - Fn * N)
        assert abs(Fn - w * (dhat - g)) < 1e-13
        assert Ft <= mu * Fn + 1e-13
        t = np.linalg.norm(rr - g * N)
        if t > mu * (dhat - g):
            assert abs(Ft - mu * Fn) < 1e-12


def test_revolute_hinge_keeps_axis():
    """A box hinged to the world about z (two zero-length bonds at pivot +- arm z) swings in
    the x-y plane: its z axis stays z and the hinge points stay on the axis."""
    sc = S.single_body(he=(0.5, 0.1, 0.2), c=(0.5, 0.0, 0.0), n_iter=40, has_ground=0)
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"] = S.REVOLUTE, 0, S.WORLD
    bo["xi"] = (-0.5, 0.0, 0.0)
    bo["axis"] = (0.0, 0.0, 1.0)
    bo["arm"] = 0.15
    bo["kappa"] = 1e4 * 0.5 / H60 ** 2  # mass 1 (default)
    sc.bonds = bo
    o = O.OracleScene(sc)
    for _ in range(60):
        o.step(1)
        st = o.state()[0]
        A = st[3:12].reshape(3, 3)
        assert np.abs(A @ np.array([0, 0, 1.0]) - np.array([0, 0, 1.0])).max() < 1e-6
        assert abs(st[2]) < 1e-6
    assert st[1] < -0.1  # it fell


def test_drive_tracks_target_angle():
    """A pinned parent drives a hinged child (no gravity, stiff joint and drive, slow period):
    the child's rotation about the hinge axis follows theta(t) = amp sin(2 pi t / T)."""
    b = S._bodies(2)
    b["he"] = [(0.2, 0.2, 0.2), (0.5, 0.1, 0.1)]
    b["mass"] = [1.0, 1.0]
    b["c"] = [(0, 0, 0), (0.7, 0, 0)]
    b["pinned"][0] = 1
    bo = np.zeros(2, dtype=S.BOND_DTYPE)
    for k, t in enumerate((S.REVOLUTE, S.DRIVE)):
        bo["type"][k], bo["i"][k], bo["j"][k] = t, 0, 1
        bo["xi"][k] = (0.2, 0, 0)
        bo["xj"][k] = (-0.5, 0, 0)
        bo["axis"][k] = (0, 0, 1)
        bo["arm"][k] = 0.1
    bo["kappa"] = [1e4 / H60 ** 2, 1e3 / H60 ** 2]
    bo["amp"][1], bo["period"][1] = 0.3, 4.0
    sc = S.Scene("drive", S.default_params(n_iter=80, gravity=(0, 0, 0), has_ground=0, body_contacts=0), b, bo, 1)
    o = O.OracleScene(sc)
    errs = []
    for n in range(1, 241):
        o.step(1)
        A = o.state()[1, 3:12].reshape(3, 3)
        th = math.atan2(A[1, 0], A[0, 0])
        errs.append(abs(th - 0.3 * math.sin(2 * math.pi * n * H60 / 4.0)))
    assert max(errs[60:]) < 0.02


# --------------------------------------------------------------------------------------
# augmented Lagrangian distance bond (Eq. 27-29)
# --------------------------------------------------------------------------------------

def test_al_bond_hanging_equilibrium():
    """Eq. 27-29: at the static equilibrium of a body hung by an augmented Lagrangian
    distance bond the constraint is exact (C = 0) and the multiplier is the tension m g;
    a plain spring of the same starting stiffness stretches by m g / kappa."""
    m, l, k0 = 2.0, 0.5, 1e4
    res = {}
    for kind in (S.AL_DISTANCE, S.SPRING):
        sc = S.single_body(mass=m, c=(0, -l, 0), n_iter=20, has_ground=0)
        bo = np.zeros(1, dtype=S.BOND_DTYPE)
        bo["type"], bo["i"], bo["j"] = kind, 0, S.WORLD
        bo["kappa"], bo["rest"] = k0, l
        bo["beta"], bo["alpha"], bo["gamma"] = 1e4, 0.99, 0.999
        sc.bonds = bo
        o = O.OracleScene(sc)
        o.step(600)
        res[kind] = (-o.state()[0, 1] - l, o.al_state()[0])
    c_al, (kap, lam) = res[S.AL_DISTANCE]
    assert abs(c_al) < 1e-9
    assert abs(lam - m * G) < 1e-9 * m * G
    assert kap >= k0
    assert abs(res[S.SPRING][0] - m * G / k0) < 1e-9


def test_al_warm_start_rule():
    """Between steps kappa^0 = max(gamma kappa^n, kappa_start) (Eq. 29): with the constraint
    satisfied, no multiplier and no gravity nothing moves, so the sweeps leave kappa as the
    warm start set it; it decays by gamma per step down to kappa_start."""
    sc = S.single_body(c=(0, -0.5, 0), n_iter=5, has_ground=0, gravity=(0, 0, 0))
    bo = np.zeros(1, dtype=S.BOND_DTYPE)
    bo["type"], bo["i"], bo["j"] = S.AL_DISTANCE, 0, S.WORLD
    bo["kappa"], bo["rest"] = 1e4, 0.5
    bo["beta"], bo["alpha"], bo["gamma"] = 1e4, 0.99, 0.999
    sc.bonds = bo
    o = O.OracleScene(sc)
    o.set_al_state(np.array([[5e4, 0.0]]))
    o.step(3)
    kap, lam = o.al_state()[0]
    assert abs(kap - 0.999 ** 3 * 5e4) < 1e-6 and abs(lam) < 1e-9
    o.set_al_state(np.array([[5e3, 0.0]]))
    o.step(1)
    assert o.al_state()[0][0] == 1e4
