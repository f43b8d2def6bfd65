"""Brute-force dense Newton minimiser of the incremental potential of Eq. (13), used to pin
the oracle's semi-implicit successive substitution (Eq. 15-19) on tiny systems.

Independent of the oracle: the affine moment of inertia is integrated by Gauss-Legendre
quadrature (Thm 4.1), the gradient and Hessian come from the bond energies Psi(d)
themselves, and the minimiser is found by Newton's method with a backtracking line search.
Only affine bodies (no rigidity projection) and distance bonds are handled.
"""
from __future__ import annotations

import numpy as np

import scenes as S


def quadrature_pi(he, mass, n=3) -> np.ndarray:
    """Pi = int rho x x^T dV over the box [-he, he] with uniform density."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    rho = mass / (8.0 * he[0] * he[1] * he[2])
    P = np.zeros((3, 3))
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            for c, wc in zip(xg, wg):
                x = np.array([a * he[0], b * he[1], c * he[2]])
                P += rho * wa * wb * wc * he[0] * he[1] * he[2] * np.outer(x, x)
    return P


def _jac(x):
    J = np.zeros((3, 12))
    J[:, :3] = np.eye(3)
    for k in range(3):
        J[k, 3 + 3 * k:6 + 3 * k] = x
    return J


def _psi(t, kappa, l, d):
    if t == S.SPRING:
        return 0.5 * kappa * (d - l) ** 2, kappa * (d - l), kappa
    if t == S.ELASTIC_NL:
        return ((kappa / 3.0) * (d ** 4 / (4 * l * l) - l * d),
                (kappa / 3.0) * (d ** 3 / (l * l) - l),
                kappa * d * d / (l * l))
    return 0.5 * kappa * d * d, kappa * d, kappa   # spherical (zero rest length)


def minimise(scene, s_q: np.ndarray, tol=1e-13, max_it=200):
    """argmin_q sum_b (q_b - s_b)^T M_b (q_b - s_b) / (2 h^2) + sum Psi(d), q of shape (nb, 12)."""
    h = scene.params["h"]
    nb = scene.n_bodies
    Ms = []
    for b in scene.bodies:
        P = quadrature_pi(b["he"], b["mass"])
        M = np.zeros((12, 12))
        M[:3, :3] = b["mass"] * np.eye(3)
        for k in range(3):
            M[3 + 3 * k:6 + 3 * k, 3 + 3 * k:6 + 3 * k] = P
        Ms.append(M)

    def energy_grad_hess(qf):
        q = qf.reshape(nb, 12)
        E = 0.0
        g = np.zeros(nb * 12)
        H = np.zeros((nb * 12, nb * 12))
        for b in range(nb):
            dq = q[b] - s_q[b]
            E += 0.5 * dq @ Ms[b] @ dq / h ** 2
            g[12 * b:12 * b + 12] += Ms[b] @ dq / h ** 2
            H[12 * b:12 * b + 12, 12 * b:12 * b + 12] += Ms[b] / h ** 2
        for bo in scene.bonds:
            i, j = int(bo["i"]), int(bo["j"])
            Ji = _jac(bo["xi"])
            yi = Ji @ q[i]
            if j == S.WORLD:
                yj, Jj = np.array(bo["xj"], dtype=float), None
            else:
                Jj = _jac(bo["xj"])
                yj = Jj @ q[j]
            r = yj - yi
            d = np.linalg.norm(r)
            n = r / d
            psi, phi, dphi = _psi(int(bo["type"]), bo["kappa"], bo["rest"], d)
            E += psi
            gy = phi * n                                    # dPsi / d y_j
            Hy = dphi * np.outer(n, n) + (phi / d) * (np.eye(3) - np.outer(n, n))
            blocks = [(i, -Ji)] + ([(j, Jj)] if Jj is not None else [])
            for (a, Ja) in blocks:
                g[12 * a:12 * a + 12] += Ja.T @ gy
                for (c, Jc) in blocks:
                    H[12 * a:12 * a + 12, 12 * c:12 * c + 12] += Ja.T @ Hy @ Jc
        return E, g, H

    q = s_q.reshape(-1).copy()
    for _ in range(max_it):
        E, g, H = energy_grad_hess(q)
        if np.linalg.norm(g) * h * h < tol:
            break
        w, V = np.linalg.eigh(H)
        w = np.maximum(np.abs(w), 1e-9 * np.abs(w).max())
        step = -(V @ ((V.T @ g) / w))
        t = 1.0
        while t > 1e-12:
            E1, _, _ = energy_grad_hess(q + t * step)
            if E1 <= E + 1e-4 * t * (g @ step):
                break
            t *= 0.5
        q = q + t * step
    return q.reshape(nb, 12)
