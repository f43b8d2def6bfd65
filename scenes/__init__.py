"""Seeded synthetic scene generators: the inputs shared by the FP64 oracle and the CUDA path.

This module holds no arithmetic of the method (no mass matrices, no bonds' forces, no
integration): it only draws body sizes, masses, poses, velocities and bond attachment
points from a seeded NumPy generator and lays them out as two structured arrays.

Conventions (the paper's notation, Section 4):
  * a body is a box with half extents ``he`` whose material frame has its origin at the
    centre of mass, placed at translation ``c`` with orientation quaternion ``quat``
    stored as (x, y, z, w);
  * ``v`` and ``omega`` are the translational and world-frame angular velocities;
  * a bond joins the material point ``xi`` of body ``i`` to the material point ``xj`` of
    body ``j``; ``j == WORLD`` means ``xj`` is a fixed world point;
  * y is up, gravity is (0, -9.81, 0) unless a scene says otherwise.

Scene recipes follow the workloads the paper reports (Table 2, Section 5): a pinned chain
pendulum, a pile of boxes dropped on the ground, a driven quadruped on a granular bed with
a flexible rod, batches of small articulated trees, and a served request stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 260902675
WORLD = -1

# user-facing bond types (the C-ABI's pabd_bond_type has the same values)
SPHERICAL = 0
SPRING = 1
ELASTIC_NL = 2
REVOLUTE = 3
DRIVE = 4
AL_DISTANCE = 5   # augmented Lagrangian distance bond (hard constraint), kappa = kappa_start

BODY_DTYPE = np.dtype([
    ("he", "f8", 3), ("mass", "f8"), ("c", "f8", 3), ("quat", "f8", 4),
    ("v", "f8", 3), ("omega", "f8", 3), ("pinned", "i4"), ("group", "i4"),
])
BOND_DTYPE = np.dtype([
    ("type", "i4"), ("i", "i4"), ("j", "i4"), ("xi", "f8", 3), ("xj", "f8", 3),
    ("axis", "f8", 3), ("kappa", "f8"), ("rest", "f8"), ("arm", "f8"),
    ("amp", "f8"), ("period", "f8"), ("phase", "f8"),
    ("beta", "f8"), ("alpha", "f8"), ("gamma", "f8"),
])


def default_params(**kw) -> dict:
    """Scene-level parameters; every key is consumed by both the oracle and the library."""
    p = dict(
        h=1.0 / 60.0, gravity=(0.0, -9.81, 0.0), n_iter=20,
        has_ground=1, ground_n=(0.0, 1.0, 0.0), ground_d=0.0,
        mu=0.5, c_kappa=1.0, d_hat_rel=1e-3, margin=1e-3,
        project=1, body_contacts=1, large_he=1e30, resid_tol=0.0,
    )
    p.update(kw)
    return p


@dataclass
class Scene:
    name: str
    params: dict
    bodies: np.ndarray
    bonds: np.ndarray
    n_steps: int
    meta: dict = field(default_factory=dict)

    @property
    def n_bodies(self) -> int:
        return int(self.bodies.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.bodies["group"].max()) + 1 if self.n_bodies else 0


def _bodies(n: int) -> np.ndarray:
    b = np.zeros(n, dtype=BODY_DTYPE)
    b["quat"][:, 3] = 1.0
    return b


def _bonds(n: int) -> np.ndarray:
    return np.zeros(n, dtype=BOND_DTYPE)


def _quat_axis_angle(axis, angle) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    s = math.sin(0.5 * angle)
    return np.array([a[0] * s, a[1] * s, a[2] * s, math.cos(0.5 * angle)])


def _random_unit_quats(rng, n) -> np.ndarray:
    """Uniform random orientations (normalised 4-D Gaussian samples)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 3] < 0] *= -1.0
    return q


def _rot_z(theta) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# ---------------------------------------------------------------------------------------
# Small scenes used by the pins and unit tests
# ---------------------------------------------------------------------------------------

def single_body(he=(0.5, 0.5, 0.5), mass=1.0, c=(0, 0, 0), quat=(0, 0, 0, 1), v=(0, 0, 0),
                omega=(0, 0, 0), n_steps=10, **params) -> Scene:
    b = _bodies(1)
    b["he"][0] = he
    b["mass"][0] = mass
    b["c"][0] = c
    b["quat"][0] = quat
    b["v"][0] = v
    b["omega"][0] = omega
    return Scene("single_body", default_params(**params), b, _bonds(0), n_steps)


def random_small(seed: int, n_bodies=4, n_bonds=4, types=(SPHERICAL, SPRING, ELASTIC_NL),
                 stretch=0.3, kappa_scale=5.0, **params) -> Scene:
    """A few free boxes joined by pre-stretched bonds; zero initial velocity, no gravity."""
    rng = np.random.default_rng(seed)
    b = _bodies(n_bodies)
    b["he"] = rng.uniform(0.2, 0.6, (n_bodies, 3))
    b["mass"] = rng.uniform(0.5, 2.0, n_bodies)
    b["c"] = rng.uniform(-1.5, 1.5, (n_bodies, 3))
    b["quat"] = _random_unit_quats(rng, n_bodies)
    h = params.get("h", 1.0 / 60.0)
    bo = _bonds(n_bonds)
    for k in range(n_bonds):
        i = k % n_bodies
        j = (k + 1 + rng.integers(0, n_bodies - 1)) % n_bodies
        if j == i:
            j = (i + 1) % n_bodies
        bo["type"][k] = types[k % len(types)]
        bo["i"][k], bo["j"][k] = i, j
        bo["xi"][k] = rng.uniform(-1, 1, 3) * b["he"][i]
        bo["xj"][k] = rng.uniform(-1, 1, 3) * b["he"][j]
        bo["kappa"][k] = kappa_scale * min(b["mass"][i], b["mass"][j]) / h ** 2 * rng.uniform(0.5, 1.5)
        bo["rest"][k] = 0.5 + stretch * rng.uniform(0, 1)
    p = dict(gravity=(0.0, 0.0, 0.0), has_ground=0, body_contacts=0)
    p.update(params)
    return Scene("random_small", default_params(**p), b, bo, 1)


# ---------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------

def chain_pendulum(seed: int = SEED_BASE + 1, n_bodies=8, n_steps=100, diagonal=False) -> Scene:
    """Chain of unit cubes (mass 1) hung from a pinned body 0 by spherical joints that join
    the bottom corner (+1/2, -1/2, +1/2) of body i to the top corner (+1/2, +1/2, +1/2) of
    body i+1; initial angles about z uniform in [-0.5, 0.5] rad; joints start satisfied.
    diagonal=True joins diagonally opposite corners (-1/2, -1/2, -1/2) and (+1/2, +1/2, +1/2)
    instead: each inner body's two joints lie on its body diagonal, so its rotation about that
    diagonal is held only by its inertia (an ill-conditioned per-body system)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / 60.0
    b = _bodies(n_bodies)
    b["he"] = 0.5
    b["mass"] = 1.0
    b["pinned"][0] = 1
    bot = np.array([-0.5, -0.5, -0.5]) if diagonal else np.array([0.5, -0.5, 0.5])
    top = np.array([0.5, 0.5, 0.5])
    Rs = [np.eye(3)]
    cs = [np.zeros(3)]
    for i in range(1, n_bodies):
        th = rng.uniform(-0.5, 0.5)
        R = _rot_z(th)
        b["quat"][i] = _quat_axis_angle((0, 0, 1), th)
        c = cs[-1] + Rs[-1] @ bot - R @ top
        b["c"][i] = c
        Rs.append(R)
        cs.append(c)
    bo = _bonds(n_bodies - 1)
    kappa = 1e4 * 1.0 / h ** 2
    for k in range(n_bodies - 1):
        bo["type"][k] = SPHERICAL
        bo["i"][k], bo["j"][k] = k, k + 1
        bo["xi"][k] = bot
        bo["xj"][k] = top
        bo["kappa"][k] = kappa
    params = default_params(h=h, n_iter=20, ground_d=-(float(n_bodies)) - 0.05, mu=0.5)
    return Scene("chain_pendulum", params, b, bo, n_steps, dict(seed=seed, diagonal=diagonal))


def box_pile(seed: int = SEED_BASE + 2, nx=16, ny=16, nz=16, spacing=3.5, jitter=0.1,
             n_steps=300, n_iter=30, stacked=False) -> Scene:
    """Boxes with edges U[0.5, 2] per axis and density U[500, 2000], axis-aligned, on an
    nx*ny*nz grid (spacing 3.5, bottom layer centres at y = 2, jitter +-0.1 per axis),
    dropped on the ground plane y = 0; mu = 0.5, h = 1/60.  With stacked=True each column
    starts as a stack: every box rests 2 mm above the one below (contacts from step 0)."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    b = _bodies(n)
    edges = rng.uniform(0.5, 2.0, (n, 3))
    dens = rng.uniform(500.0, 2000.0, n)
    b["he"] = 0.5 * edges
    b["mass"] = dens * edges[:, 0] * edges[:, 1] * edges[:, 2]
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # body order: x fastest is irrelevant to the method; use (iy, iz, ix) so layers are contiguous
    order = np.lexsort((ix.ravel(), iz.ravel(), iy.ravel()))
    gx = ix.ravel()[order]; gy = iy.ravel()[order]; gz = iz.ravel()[order]
    b["c"][:, 0] = (gx - 0.5 * (nx - 1)) * spacing
    b["c"][:, 1] = 2.0 + gy * spacing
    b["c"][:, 2] = (gz - 0.5 * (nz - 1)) * spacing
    b["c"] += rng.uniform(-jitter, jitter, (n, 3))
    if stacked:
        col = gx * nz + gz
        order = np.lexsort((gy, col))                 # by column, bottom to top
        hgt = 2.0 * b["he"][order, 1] + 0.002         # each box plus the 2 mm gap below it
        top = np.cumsum(hgt)
        first = np.r_[True, col[order][1:] != col[order][:-1]]
        base = np.maximum.accumulate(np.where(first, top - hgt, 0.0))
        b["c"][order, 1] = top - base - b["he"][order, 1]
    params = default_params(h=1.0 / 60.0, n_iter=n_iter, mu=0.5)
    return Scene("box_pile", params, b, _bonds(0), n_steps, dict(seed=seed, grid=(nx, ny, nz)))


def slab_pile(n_side: int = 10, seed: int = SEED_BASE + 5, n_steps: int = 60, n_iter: int = 20) -> Scene:
    """A dynamic slab (mass 50, half-height 0.1) resting 1 mm above the ground, carrying an
    n_side x n_side grid of unit-mass cubes of edge 0.2 at spacing 0.4 (2 mm above it, yaw
    jitter +-0.2 rad, position jitter +-0.02): the slab's four contacts per cube make it a
    body with about 4 n_side^2 bond ends (a large body under a pile).  The slab is a large
    body (it bypasses the grid); h = 1/60."""
    rng = np.random.default_rng(seed)
    n = n_side * n_side + 1
    b = _bodies(n)
    half = 0.2 * n_side + 0.1
    b["he"][0] = (half, 0.1, half)
    b["mass"][0] = 50.0
    b["c"][0] = (0.0, 0.101, 0.0)
    ii, kk = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    x = (ii.ravel() - 0.5 * (n_side - 1)) * 0.4 + rng.uniform(-0.02, 0.02, n - 1)
    z = (kk.ravel() - 0.5 * (n_side - 1)) * 0.4 + rng.uniform(-0.02, 0.02, n - 1)
    b["he"][1:] = 0.1
    b["mass"][1:] = 1.0
    b["c"][1:, 0], b["c"][1:, 1], b["c"][1:, 2] = x, 0.202 + 0.1 + 0.002, z
    yaw = rng.uniform(-0.2, 0.2, n - 1)
    b["quat"][1:] = np.stack([np.zeros(n - 1), np.sin(yaw / 2), np.zeros(n - 1), np.cos(yaw / 2)], axis=1)
    params = default_params(h=1.0 / 60.0, n_iter=n_iter, large_he=1.0)
    return Scene("slab_pile", params, b, _bonds(0), n_steps, dict(seed=seed, n_side=n_side))


def box_pile_n(n: int, seed: int = SEED_BASE + 2, **kw) -> Scene:
    """A box pile with about n bodies on a near-cubic grid (scale sweeps, served scenes)."""
    side = max(1, int(round(n ** (1.0 / 3.0))))
    nx = nz = side
    ny = max(1, int(math.ceil(n / (side * side))))
    s = box_pile(seed=seed, nx=nx, ny=ny, nz=nz, **kw)
    s.bodies = s.bodies[:n].copy()
    s.meta["n"] = n
    return s


def quadruped_bed_rod(seed: int = SEED_BASE + 3, bed=(100, 5, 100), n_rod=64, n_steps=300) -> Scene:
    """A 13-body quadruped (torso 1 x 0.4 x 0.3, four legs of three 0.3 x 0.08 x 0.08 links,
    revolute joints about z driven sinusoidally: amplitude 0.4 rad, period 1 s, phase step
    pi/2 per leg) standing on a bed of small cubes (edge 0.03, density 1500, random
    orientations on a jittered lattice), plus a 64-segment flexible rod joined by nonlinear
    elastic bonds (stiffness log-uniform in [1e4, 1e6]) with segment 0 pinned; h = 1/60,
    20 iterations.  Bed lattice spacing is 0.056 so that randomly rotated cubes (extent up
    to 0.03*sqrt(3)) start separated."""
    rng = np.random.default_rng(seed)
    h = 1.0 / 60.0
    bx, by, bz = bed
    n_bed = bx * by * bz
    sp = 0.056
    n_dog = 13
    n = n_dog + n_bed + n_rod
    b = _bodies(n)
    bonds = []

    # -- quadruped ------------------------------------------------------------------
    bed_top = by * sp
    leg_len = 3 * 0.3
    torso_y = bed_top + leg_len + 0.15 + 0.02
    b["he"][0] = (0.5, 0.15, 0.2)
    b["mass"][0] = 1000.0 * 1.0 * 0.3 * 0.4
    b["c"][0] = (0.0, torso_y, 0.0)
    link_he = np.array([0.04, 0.15, 0.04])
    link_m = 1000.0 * 0.08 * 0.3 * 0.08
    hips = [(0.42, -0.15, 0.15), (0.42, -0.15, -0.15), (-0.42, -0.15, 0.15), (-0.42, -0.15, -0.15)]
    k_joint = 1e3 * link_m / h ** 2
    idx = 1
    for leg, hip in enumerate(hips):
        parent = 0
        p_anchor = np.array(hip)
        top = np.array([0.0, 0.15, 0.0])
        for _ in range(3):
            b["he"][idx] = link_he
            b["mass"][idx] = link_m
            pc = b["c"][parent] + p_anchor
            b["c"][idx] = pc - top
            for kind, kap in ((REVOLUTE, k_joint), (DRIVE, 0.1 * k_joint)):
                r = np.zeros(1, dtype=BOND_DTYPE)[0]
                r["type"] = kind
                r["i"], r["j"] = parent, idx
                r["xi"] = p_anchor
                r["xj"] = top
                r["axis"] = (0.0, 0.0, 1.0)
                r["kappa"] = kap
                r["arm"] = 0.04
                if kind == DRIVE:
                    r["amp"], r["period"], r["phase"] = 0.4, 1.0, 0.5 * math.pi * leg
                bonds.append(r)
            parent = idx
            p_anchor = np.array([0.0, -0.15, 0.0])
            idx += 1

    # -- granular bed ----------------------------------------------------------------
    i0 = n_dog
    gx, gy, gz = np.meshgrid(np.arange(bx), np.arange(by), np.arange(bz), indexing="ij")
    order = np.lexsort((gx.ravel(), gz.ravel(), gy.ravel()))
    gx = gx.ravel()[order]; gy = gy.ravel()[order]; gz = gz.ravel()[order]
    sl = slice(i0, i0 + n_bed)
    b["he"][sl] = 0.015
    b["mass"][sl] = 1500.0 * 0.03 ** 3
    b["c"][sl, 0] = (gx - 0.5 * (bx - 1)) * sp
    b["c"][sl, 1] = 0.5 * sp + gy * sp
    b["c"][sl, 2] = (gz - 0.5 * (bz - 1)) * sp
    b["c"][sl] += rng.uniform(-0.002, 0.002, (n_bed, 3))
    b["quat"][sl] = _random_unit_quats(rng, n_bed)

    # -- flexible rod (cantilever along +x from a pinned root) -------------------------
    r0 = n_dog + n_bed
    seg_he = np.array([0.05, 0.01, 0.01])
    gap = 0.01
    rod_y = torso_y + 0.6
    x0 = -0.5 * n_rod * (0.1 + gap)
    for s in range(n_rod):
        k = r0 + s
        b["he"][k] = seg_he
        b["mass"][k] = 1000.0 * 0.1 * 0.02 * 0.02
        b["c"][k] = (x0 + s * (0.1 + gap), rod_y, 1.0)
    b["pinned"][r0] = 1
    for s in range(n_rod - 1):
        kap = 10.0 ** rng.uniform(4.0, 6.0)
        for cy in (-0.01, 0.01):
            for cz in (-0.01, 0.01):
                r = np.zeros(1, dtype=BOND_DTYPE)[0]
                r["type"] = ELASTIC_NL
                r["i"], r["j"] = r0 + s, r0 + s + 1
                r["xi"] = (0.05, cy, cz)
                r["xj"] = (-0.05, cy, cz)
                r["kappa"] = kap
                r["rest"] = gap
                bonds.append(r)
    bo = np.array(bonds, dtype=BOND_DTYPE)
    params = default_params(h=h, n_iter=20, mu=0.5, large_he=0.1)
    return Scene("quadruped_bed_rod", params, b, bo, n_steps,
                 dict(seed=seed, n_dog=n_dog, n_bed=n_bed, n_rod=n_rod))


def mass_ratio_chain(n=6, ratio=100.0, al=True, n_iter=10, n_steps=300, kappa_start=1e4) -> Scene:
    """A chain of n unit boxes hanging from a pinned anchor box by distance bonds of rest
    length 0.2 between face centres; the last box is `ratio` times heavier (the paper's
    large-mass-ratio chain).  al=True: augmented Lagrangian bonds (kappa_start 1e4, beta
    1e4, alpha 0.99, gamma 0.999); al=False: plain springs of stiffness kappa_start."""
    b = _bodies(n + 1)
    b["he"] = 0.25
    b["mass"] = 1.0
    b["mass"][-1] = ratio
    b["pinned"][0] = 1
    gap = 0.2
    for k in range(n + 1):
        b["c"][k] = (0.0, -k * (0.5 + gap), 0.0)
    bo = _bonds(n)
    for k in range(n):
        bo["type"][k] = AL_DISTANCE if al else SPRING
        bo["i"][k], bo["j"][k] = k, k + 1
        bo["xi"][k] = (0.0, -0.25, 0.0)
        bo["xj"][k] = (0.0, 0.25, 0.0)
        bo["kappa"][k] = kappa_start
        bo["rest"][k] = gap
        bo["beta"][k], bo["alpha"][k], bo["gamma"][k] = 1e4, 0.99, 0.999
    params = default_params(n_iter=n_iter, has_ground=0, body_contacts=0)
    return Scene("mass_ratio_chain", params, b, bo, n_steps, dict(al=al, ratio=ratio))


def mass_ratio_stack(n=6, ratio=10.0, n_iter=20, n_steps=300) -> Scene:
    """A stack of n unit cubes on the ground, each `ratio` times heavier than the one below it
    (1, 10, 100, ... kg from the bottom up), 2 mm apart; h = 1/60, mu = 0.5 -- the paper's
    extreme-mass-ratio stack (Sec. 6, comparison with sequential impulses)."""
    b = _bodies(n)
    b["he"] = 0.5
    b["mass"] = ratio ** np.arange(n)
    b["c"][:, 1] = 0.5 + 0.002 + np.arange(n) * 1.002
    params = default_params(h=1.0 / 60.0, n_iter=n_iter, mu=0.5)
    return Scene("mass_ratio_stack", params, b, _bonds(0), n_steps, dict(ratio=ratio))


def two_box_spring(n_iter=20, n_steps=60, kappa=1e4) -> Scene:
    """Two unit cubes (1 kg) joined by a spring (Eq. 26 split) of rest length 1 between the
    centres of their facing faces, stretched to twice its rest length; no gravity, no ground --
    the paper's two-box convergence example (Sec. 6, comparison with AVBD)."""
    b = _bodies(2)
    b["he"] = 0.5
    b["mass"] = 1.0
    b["c"][0] = (-1.5, 0.0, 0.0)
    b["c"][1] = (1.5, 0.0, 0.0)
    bo = _bonds(1)
    bo["type"], bo["i"], bo["j"] = SPRING, 0, 1
    bo["xi"], bo["xj"] = (0.5, 0.0, 0.0), (-0.5, 0.0, 0.0)
    bo["kappa"], bo["rest"] = kappa, 1.0
    params = default_params(h=1.0 / 60.0, n_iter=n_iter, gravity=(0.0, 0.0, 0.0), has_ground=0, body_contacts=0)
    return Scene("two_box_spring", params, b, bo, n_steps, dict(kappa=kappa))


def spring_net(n=11, n_iter=20, n_steps=120, kappa=2e3, stretch=0.6) -> Scene:
    """An n x n net of cubes (edge 0.2, 0.5 kg) in the x-y plane at spacing 0.5, each joined
    to its four neighbours by springs between facing face centres (2 n (n - 1) springs: 220
    for n = 11) whose rest length is `stretch` times the initial face gap, so the net starts
    stretched; the two top corners are pinned and gravity pulls it down, so it contracts
    toward the middle and sags -- the paper's 11 x 11 net (Sec. 6, comparison with VBD)."""
    b = _bodies(n * n)
    b["he"] = 0.1
    b["mass"] = 0.5
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # ii: column (x), jj: row (y)
    b["c"][:, 0] = (ii.ravel() - 0.5 * (n - 1)) * 0.5
    b["c"][:, 1] = 1.0 + jj.ravel() * 0.5
    top = [k for k in range(n * n) if jj.ravel()[k] == n - 1 and ii.ravel()[k] in (0, n - 1)]
    b["pinned"][top] = 1
    gap = 0.5 - 0.2
    rows = []
    for k in range(n * n):
        x, y = ii.ravel()[k], jj.ravel()[k]
        for dx, dy, ax in ((1, 0, 0), (0, 1, 1)):
            if x + dx < n and y + dy < n:
                m = (x + dx) * n + (y + dy)
                r = np.zeros(1, dtype=BOND_DTYPE)[0]
                r["type"], r["i"], r["j"] = SPRING, k, m
                e = np.eye(3)[ax] * 0.1
                r["xi"], r["xj"] = e, -e
                r["kappa"], r["rest"] = kappa, stretch * gap
                rows.append(r)
    bo = np.array(rows, dtype=BOND_DTYPE)
    params = default_params(h=1.0 / 60.0, n_iter=n_iter, has_ground=0, body_contacts=0)
    return Scene("spring_net", params, b, bo, n_steps, dict(n=n, stretch=stretch))


def batched_trees(seed: int = SEED_BASE + 4, n_scenes=4096, n_min=4, n_max=64, n_steps=1000) -> Scene:
    """n_scenes independent articulated trees (one group each) of U{4..64} boxes with edges
    U[0.1, 0.5]; parent(i) ~ U{0..i-1} restricted to parents with a free face; the child is
    attached across a 0.02 gap at the centre of a random free face of its parent; bond type
    uniform over {spherical, revolute, nonlinear elastic}; ground contact only; h = 1/120,
    10 iterations."""
    rng = np.random.default_rng(seed)
    h = 1.0 / 120.0
    sizes = rng.integers(n_min, n_max + 1, n_scenes)
    n = int(sizes.sum())
    b = _bodies(n)
    bonds = []
    faces = [(0, 1.0), (0, -1.0), (1, 1.0), (1, -1.0), (2, 1.0), (2, -1.0)]
    gap = 0.02
    base = 0
    for g, m in enumerate(sizes):
        m = int(m)
        he = rng.uniform(0.05, 0.25, (m, 3))
        mass = 1000.0 * 8.0 * he.prod(axis=1)
        cs = np.zeros((m, 3))
        free = [set(range(6)) for _ in range(m)]
        for i in range(1, m):
            cand = [p for p in range(i) if free[p]]
            p = int(cand[rng.integers(0, len(cand))])
            f = sorted(free[p])[rng.integers(0, len(free[p]))]
            free[p].discard(f)
            ax, sg = faces[f]
            free[i].discard(f ^ 1)  # the child's face that looks back at its parent
            xi = np.zeros(3); xi[ax] = sg * he[p, ax]
            xj = np.zeros(3); xj[ax] = -sg * he[i, ax]
            cs[i] = cs[p] + xi - xj
            cs[i, ax] += sg * gap
            kind = (SPHERICAL, REVOLUTE, ELASTIC_NL)[int(rng.integers(0, 3))]
            r = np.zeros(1, dtype=BOND_DTYPE)[0]
            r["type"] = kind
            r["i"], r["j"] = base + p, base + i
            r["xi"], r["xj"] = xi, xj
            k_j = 1e3 * min(mass[p], mass[i]) / h ** 2
            if kind == SPHERICAL:
                r["kappa"] = k_j
                r["xj"] = xj - np.eye(3)[ax] * sg * gap  # zero-length joint at the parent's face
            elif kind == REVOLUTE:
                r["kappa"] = k_j
                r["xj"] = xj - np.eye(3)[ax] * sg * gap
                tang = [a for a in range(3) if a != ax]
                r["axis"] = np.eye(3)[tang[int(rng.integers(0, 2))]]
                r["arm"] = 0.5 * min(he[i, tang[0]], he[i, tang[1]])
            else:
                r["kappa"] = 0.1 * k_j
                r["rest"] = gap
            bonds.append(r)
        # lift the tree so its lowest point (axis-aligned boxes) sits 0.05 above the ground
        lo = (cs[:, 1] - he[:, 1]).min()
        cs[:, 1] += 0.05 - lo
        sl = slice(base, base + m)
        b["he"][sl] = he
        b["mass"][sl] = mass
        b["c"][sl] = cs
        b["group"][sl] = g
        base += m
    bo = np.array(bonds, dtype=BOND_DTYPE)
    params = default_params(h=h, n_iter=10, mu=0.5, body_contacts=0)
    return Scene("batched_trees", params, b, bo, n_steps, dict(seed=seed, sizes=sizes))


def request_stream(seed: int = SEED_BASE + 5, rate=1000.0, duration=1.0, p_new=0.2,
                   n_min=10, n_max=100_000, steps_max=60, max_scenes=None):
    """Poisson arrivals of step requests (scene_id, n_steps ~ U{1..60}); with probability
    p_new a request opens a new scene whose size is log-uniform in [n_min, n_max] (a box
    pile of that size), until max_scenes exist; otherwise it targets a uniformly chosen
    existing scene."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    sizes = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if not sizes or (rng.uniform() < p_new and (max_scenes is None or len(sizes) < max_scenes)):
            sizes.append(int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))))
            sid = len(sizes) - 1
        else:
            sid = int(rng.integers(0, len(sizes)))
        reqs.append((t, sid, int(rng.integers(1, steps_max + 1))))
    return reqs, sizes


def group_rows(sc: Scene, groups) -> np.ndarray:
    """Body indices of the given groups (independent scenes of a batch), in body order."""
    g = np.asarray(sc.bodies["group"])
    return np.nonzero(np.isin(g, np.asarray(groups)))[0]


def select_groups(sc: Scene, groups) -> Scene:
    """The sub-batch made of the given groups (ascending), renumbered 0..len-1, with their
    bonds; bodies keep their order.  Groups interact only through their own bonds, so the
    sub-batch steps exactly as those groups do inside the full batch."""
    groups = np.unique(np.asarray(groups))
    rows = group_rows(sc, groups)
    new_id = np.full(sc.n_bodies, -1, dtype=np.int64)
    new_id[rows] = np.arange(rows.size)
    b = sc.bodies[rows].copy()
    b["group"] = np.searchsorted(groups, b["group"])
    keep = new_id[sc.bonds["i"]] >= 0
    bo = sc.bonds[keep].copy()
    bo["i"] = new_id[bo["i"]]
    bo["j"] = np.where(bo["j"] >= 0, new_id[np.maximum(bo["j"], 0)], -1)
    meta = dict(sc.meta, groups=groups)
    if "sizes" in sc.meta:
        meta["sizes"] = np.asarray(sc.meta["sizes"])[groups]
    return Scene(sc.name + "_subset", dict(sc.params), b, bo, sc.n_steps, meta)
