/*
 * pabd_oracle.c -- plain, slow, FP64 CPU oracle of Projective Affine Body Dynamics.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load this library. It shares no code, header, table or helper with the CUDA path.
 *
 * One time step follows Algorithm 1 of the paper in its order:
 *   collision detection on q^n  ->  predictor (c*, Q*, s = q^0)  ->
 *   n_iter x [ global solve of Eq. (19) for every body (Jacobi: all read q^k),
 *              local solve: c^{k+1} = c^{k+1/2}, A^{k+1} = rotation of A^{k+1/2} ]  ->
 *   v = (c^{n+1} - c^n)/h, [w]x from (A^{n+1} - A^n)(A^n)^-1 / h (skew part, Sec. 4.4).
 *
 * Everything is double precision except the integer decisions of collision detection
 * (which pair overlaps, which corner touches, which face is chosen), which are taken in
 * IEEE single precision with a fixed operation order on the single-precision rounding of
 * the state, exactly like the GPU path takes them; build with -ffp-contract=off.
 *
 * The global system of one body is assembled densely as the 12x12 H of Eq. (20) and the
 * right-hand side of Eq. (19) with J of Eq. (23); it is solved with a dense Cholesky
 * factorisation. No block (Eq. 24/25) or Kronecker structure is used.
 * The rotation of A^{k+1/2} comes from a one-sided Jacobi SVD (Hestenes), with the sign
 * of the last singular direction chosen so that the result is a proper rotation.
 *
 * Readings where the paper is silent (contact, friction, nonlinear elastic bond, joint
 * expansion) are written at the bond rules below.  Parity unpinned against the paper:
 * the contact/friction bond and the nonlinear elastic bond forms (the paper defers them
 * to a supplement that is not available); their implementation is pinned by closed-form
 * tests of the reading (resting/sliding box, hanging body equilibrium).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PO_WORLD (-1)

enum { PO_SPHERICAL = 0, PO_SPRING = 1, PO_ELASTIC_NL = 2, PO_REVOLUTE = 3, PO_DRIVE = 4,
       PO_CONTACT = 5, PO_GROUND = 6, PO_AL = 7 };

typedef struct {
    double he[3];
    double m;
    double Pi[9];      /* affine moment of inertia Pi_0 (material frame), Thm 4.1 */
    int pinned, group;
} po_static;

typedef struct {
    double c[3], A[9], Q[4], v[3], w[3];
} po_state;

typedef struct {
    int type, i, j;
    double xi[3], xj[3];
    double kappa, rest;
    /* drive: parent anchor rotates about u_i; child anchor is fixed */
    double ui[3], ri[3], arm, amp, period, phase;
    /* contact */
    double N[3], dhat, w, mu;
    /* augmented Lagrangian distance bond (Eq. 27-29): stiffness and multiplier, parameters */
    double al_k, al_lam, al_kstart, al_beta, al_alpha, al_gamma;
} po_bond;

typedef struct {
    double h, g[3];
    int n_iter;
    int has_ground;
    double gn[3], gd;
    double mu, c_kappa, d_hat_rel, margin;
    int project, body_contacts;
    double large_he;
    double resid_tol;       /* 0: n_iter sweeps; else a scene stops when its residual <= resid_tol */
} po_params;

typedef struct {
    po_params p;
    int nb, cap_b;
    po_static* bs;
    po_state* st;
    int nc, cap_c;          /* static (user) bonds after expansion */
    po_bond* cb;
    int nk, cap_k;          /* contact bonds of the current step */
    po_bond* kb;
    int np, cap_p;          /* broad-phase pairs of the current step */
    int* pairs;
    int64_t step;
    int n_groups;
    double* resid;          /* per group, last iteration of the last step */
    double* amargin;        /* per body: min over the last step's sweeps of |g - dhat| of its contacts */
    double act_shift;       /* test probe of the contact activation threshold, 0 in the method */
    int round_iterates;     /* test probe: each sweep's iterate rounded to single precision (0 in the method) */
    int last_sweeps;        /* sweeps the last step ran (n_iter unless a residual threshold ended it) */
    /* adjacency of static bonds (pairs excluded from contact) */
    int n_excl, cap_excl;
    int* excl;              /* sorted (min, max) pairs */
} po_scene;

/* ------------------------------------------------------------------------------------ */
/* small dense helpers                                                                    */
/* ------------------------------------------------------------------------------------ */

static void mat3_mul(const double* a, const double* b, double* o) {
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * r + k] * b[3 * k + c];
            t[3 * r + c] = s;
        }
    memcpy(o, t, sizeof t);
}

static void mat3_vec(const double* a, const double* x, double* o) {
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = a[3 * r] * x[0] + a[3 * r + 1] * x[1] + a[3 * r + 2] * x[2];
    memcpy(o, t, sizeof t);
}

static void mat3_tvec(const double* a, const double* x, double* o) {
    double t[3];
    for (int c = 0; c < 3; ++c) t[c] = a[c] * x[0] + a[3 + c] * x[1] + a[6 + c] * x[2];
    memcpy(o, t, sizeof t);
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void cross3(const double* a, const double* b, double* o) {
    double t[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    memcpy(o, t, sizeof t);
}

static double det3(const double* a) {
    return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
           a[2] * (a[3] * a[7] - a[4] * a[6]);
}

/* Unit quaternion (x, y, z, w) -> rotation matrix (the standard conversion, Shoemake 1985). */
void po_quat_to_mat(const double* q, double* R) {
    double x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rotation matrix -> unit quaternion (x, y, z, w), Shepperd's method: pick the largest of
   4w^2-1 = trace, 4x^2-1 = 2R00 - trace, ... to divide by. */
void po_mat_to_quat(const double* R, double* q) {
    double tr = R[0] + R[4] + R[8];
    double cand[4] = {tr, R[0], R[4], R[8]};
    int k = 0;
    for (int i = 1; i < 4; ++i) if (cand[i] > cand[k]) k = i;
    double x, y, z, w;
    if (k == 0) {
        double s = sqrt(1.0 + tr) * 2.0;  /* s = 4w */
        w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
    } else if (k == 1) {
        double s = sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;  /* s = 4x */
        x = 0.25 * s; w = (R[7] - R[5]) / s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
    } else if (k == 2) {
        double s = sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;  /* s = 4y */
        y = 0.25 * s; w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; z = (R[5] + R[7]) / s;
    } else {
        double s = sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;  /* s = 4z */
        z = 0.25 * s; w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s;
    }
    double n = sqrt(x * x + y * y + z * z + w * w);
    q[0] = x / n; q[1] = y / n; q[2] = z / n; q[3] = w / n;
}

/* Rotation closest to A in the Frobenius norm over SO(3) (local solve, Sec. 4.3):
   A = U S V^T by one-sided Jacobi (Hestenes) on the columns of A V, then
   R = U diag(1, 1, det(U V^T)) V^T.  If A has rank < 3 the missing columns of U are
   completed by cross products. Returns the singular values in sig (descending). */
void po_polar_rotation(const double* A, double* R, double* sig) {
    double B[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(B, A, sizeof B);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double alpha = 0, beta = 0, gamma = 0;
                for (int r = 0; r < 3; ++r) {
                    alpha += B[3 * r + p] * B[3 * r + p];
                    beta += B[3 * r + q] * B[3 * r + q];
                    gamma += B[3 * r + p] * B[3 * r + q];
                }
                if (fabs(gamma) <= 1e-300 || fabs(gamma) <= 1e-17 * sqrt(alpha * beta)) continue;
                double cur = fabs(gamma) / sqrt(alpha * beta);
                if (cur > off) off = cur;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int r = 0; r < 3; ++r) {
                    double bp = B[3 * r + p], bq = B[3 * r + q];
                    B[3 * r + p] = c * bp - s * bq;
                    B[3 * r + q] = s * bp + c * bq;
                    double vp = V[3 * r + p], vq = V[3 * r + q];
                    V[3 * r + p] = c * vp - s * vq;
                    V[3 * r + q] = s * vp + c * vq;
                }
            }
        if (off < 1e-15) break;
    }
    /* singular values = column norms; sort descending */
    double s[3];
    int idx[3] = {0, 1, 2};
    for (int c = 0; c < 3; ++c) s[c] = sqrt(B[c] * B[c] + B[3 + c] * B[3 + c] + B[6 + c] * B[6 + c]);
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (s[idx[b]] > s[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    double U[9], Vs[9];
    double scale = s[idx[0]] > 0 ? s[idx[0]] : 1.0;
    int rank = 0;
    for (int c = 0; c < 3; ++c) {
        int k = idx[c];
        for (int r = 0; r < 3; ++r) Vs[3 * r + c] = V[3 * r + k];
        if (s[k] > 1e-14 * scale) {
            for (int r = 0; r < 3; ++r) U[3 * r + c] = B[3 * r + k] / s[k];
            rank = c + 1;
        }
        if (sig) sig[c] = s[k];
    }
    /* complete U for rank-deficient A */
    if (rank == 0) { memcpy(R, (double[9]){1, 0, 0, 0, 1, 0, 0, 0, 1}, 9 * sizeof(double)); return; }
    if (rank == 1) {
        double u0[3] = {U[0], U[3], U[6]}, e[3] = {0, 0, 0};
        int m = 0;
        for (int k = 1; k < 3; ++k) if (fabs(u0[k]) < fabs(u0[m])) m = k;
        e[m] = 1.0;
        double u1[3];
        cross3(u0, e, u1);
        double n = norm3(u1);
        for (int r = 0; r < 3; ++r) U[3 * r + 1] = u1[r] / n;
    }
    if (rank <= 2) {
        double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]}, u2[3];
        cross3(u0, u1, u2);
        for (int r = 0; r < 3; ++r) U[3 * r + 2] = u2[r];
    }
    double dU = det3(U), dV = det3(Vs);
    double sgn = (dU * dV < 0) ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = U[3 * r + 0] * Vs[3 * c + 0] + U[3 * r + 1] * Vs[3 * c + 1] +
                           sgn * U[3 * r + 2] * Vs[3 * c + 2];
}

/* Dense Cholesky solve of the SPD n x n system H x = b (row-major), in place on copies. */
int po_cholesky_solve(int n, const double* H, const double* b, double* x) {
    double L[144];
    double y[12];
    if (n > 12) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[n * i + j];
            for (int k = 0; k < j; ++k) s -= L[n * i + k] * L[n * j + k];
            if (i == j) {
                if (!(s > 0)) return -2;
                L[n * i + i] = sqrt(s);
            } else {
                L[n * i + j] = s / L[n * j + j];
            }
        }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[n * i + k] * y[k];
        y[i] = s / L[n * i + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[n * k + i] * x[k];
        x[i] = s / L[n * i + i];
    }
    return 0;
}

/* J(x) of Eq. (23): 3 x 12, q = (c, a1, a2, a3), a_k the k-th row of A. */
static void jacobian(const double* x, double* J) {
    memset(J, 0, 36 * sizeof(double));
    for (int k = 0; k < 3; ++k) {
        J[12 * k + k] = 1.0;
        for (int l = 0; l < 3; ++l) J[12 * k + 3 + 3 * k + l] = x[l];
    }
}

static void state_to_q(const po_state* s, double* q) {
    for (int k = 0; k < 3; ++k) q[k] = s->c[k];
    for (int k = 0; k < 9; ++k) q[3 + k] = s->A[k];
}

/* y = J q = A x + c (Eq. 1) */
static void world_point(const double* q, const double* x, double* y) {
    for (int k = 0; k < 3; ++k) y[k] = q[k] + q[3 + 3 * k] * x[0] + q[3 + 3 * k + 1] * x[1] + q[3 + 3 * k + 2] * x[2];
}

/* ------------------------------------------------------------------------------------ */
/* scene construction                                                                     */
/* ------------------------------------------------------------------------------------ */

/* params: h, gx, gy, gz, n_iter, has_ground, nx, ny, nz, gd, mu, c_kappa, d_hat_rel,
           margin, project, body_contacts, large_he */
void* po_create(const double* pr) {
    po_scene* s = (po_scene*)calloc(1, sizeof(po_scene));
    po_params* p = &s->p;
    p->h = pr[0]; p->g[0] = pr[1]; p->g[1] = pr[2]; p->g[2] = pr[3];
    p->n_iter = (int)pr[4]; p->has_ground = (int)pr[5];
    p->gn[0] = pr[6]; p->gn[1] = pr[7]; p->gn[2] = pr[8]; p->gd = pr[9];
    p->mu = pr[10]; p->c_kappa = pr[11]; p->d_hat_rel = pr[12]; p->margin = pr[13];
    p->project = (int)pr[14]; p->body_contacts = (int)pr[15]; p->large_he = pr[16];
    p->resid_tol = pr[17];
    double n = norm3(p->gn);
    if (n > 0) for (int k = 0; k < 3; ++k) p->gn[k] /= n;
    return s;
}

void po_destroy(void* h) {
    po_scene* s = (po_scene*)h;
    if (!s) return;
    free(s->bs); free(s->st); free(s->cb); free(s->kb); free(s->pairs); free(s->resid); free(s->amargin); free(s->excl);
    free(s);
}

/* grow a heap array so that it holds at least `need` elements */
static void* grow(void* ptr, int* cap, int need, size_t elem) {
    if (need <= *cap) return ptr;
    int c = *cap ? *cap : 64;
    while (c < need) c *= 2;
    *cap = c;
    return realloc(ptr, (size_t)c * elem);
}

/* body: hx, hy, hz, mass, cx, cy, cz, qx, qy, qz, qw, vx, vy, vz, wx, wy, wz, pinned, group */
int po_add_body(void* h, const double* d) {
    po_scene* s = (po_scene*)h;
    int cap_st = s->cap_b;
    s->bs = (po_static*)grow(s->bs, &s->cap_b, s->nb + 1, sizeof(po_static));
    s->st = (po_state*)grow(s->st, &cap_st, s->nb + 1, sizeof(po_state));
    po_static* b = &s->bs[s->nb];
    po_state* x = &s->st[s->nb];
    memset(b, 0, sizeof *b);
    memset(x, 0, sizeof *x);
    for (int k = 0; k < 3; ++k) b->he[k] = d[k];
    b->m = d[3];
    /* Thm 4.1: Pi_0 = int rho x x^T dV; for a uniform box centred at its COM this is
       diag(m hx^2/3, m hy^2/3, m hz^2/3) with half extents h. */
    for (int k = 0; k < 3; ++k) b->Pi[4 * k] = b->m * b->he[k] * b->he[k] / 3.0;
    for (int k = 0; k < 3; ++k) x->c[k] = d[4 + k];
    double qn = sqrt(d[7] * d[7] + d[8] * d[8] + d[9] * d[9] + d[10] * d[10]);
    for (int k = 0; k < 4; ++k) x->Q[k] = d[7 + k] / qn;
    po_quat_to_mat(x->Q, x->A);
    for (int k = 0; k < 3; ++k) { x->v[k] = d[11 + k]; x->w[k] = d[14 + k]; }
    b->pinned = (int)d[17];
    b->group = (int)d[18];
    if (b->pinned) { memset(x->v, 0, sizeof x->v); memset(x->w, 0, sizeof x->w); }
    if (b->group + 1 > s->n_groups) s->n_groups = b->group + 1;
    return s->nb++;
}

static void push_static(po_scene* s, const po_bond* b) {
    s->cb = (po_bond*)grow(s->cb, &s->cap_c, s->nc + 1, sizeof(po_bond));
    s->cb[s->nc++] = *b;
}

static void add_excl(po_scene* s, int a, int b) {
    if (a < 0 || b < 0) return;
    s->excl = (int*)grow(s->excl, &s->cap_excl, 2 * s->n_excl + 2, sizeof(int));
    s->excl[2 * s->n_excl] = a < b ? a : b;
    s->excl[2 * s->n_excl + 1] = a < b ? b : a;
    s->n_excl++;
}

/* A unit vector orthogonal to u: normalize(u x e_k), e_k the axis least aligned with u
   (lowest index on ties). */
static void perp_unit(const double* u, double* r) {
    int m = 0;
    for (int k = 1; k < 3; ++k) if (fabs(u[k]) < fabs(u[m])) m = k;
    double e[3] = {0, 0, 0};
    e[m] = 1.0;
    cross3(u, e, r);
    double n = norm3(r);
    for (int k = 0; k < 3; ++k) r[k] /= n;
}

/* direction given in body i's material frame, expressed in body j's material frame
   through the initial orientations (world frame when j is WORLD) */
static void carry_dir(const po_scene* s, int i, int j, const double* di, double* dj) {
    double w[3];
    mat3_vec(s->st[i].A, di, w);
    if (j == PO_WORLD) { memcpy(dj, w, sizeof w); return; }
    mat3_tvec(s->st[j].A, w, dj);
}

/* bond: type, i, j, xi[3], xj[3], axis[3], kappa, rest, arm, amp, period, phase
   [, beta, alpha, gamma for the augmented Lagrangian distance bond, user type 5]
   Returns the number of internal bonds created (REVOLUTE expands to two). */
int po_add_bond(void* h, const double* d) {
    po_scene* s = (po_scene*)h;
    int type = (int)d[0], i = (int)d[1], j = (int)d[2];
    double xi[3] = {d[3], d[4], d[5]}, xj[3] = {d[6], d[7], d[8]}, ax[3] = {d[9], d[10], d[11]};
    double kappa = d[12], rest = d[13], arm = d[14], amp = d[15], period = d[16], phase = d[17];
    if (i == PO_WORLD) return -1;
    po_bond b;
    memset(&b, 0, sizeof b);
    b.i = i; b.j = j; b.kappa = kappa; b.rest = rest;
    add_excl(s, i, j);
    if (type == PO_SPHERICAL || type == PO_SPRING || type == PO_ELASTIC_NL) {
        b.type = type;
        memcpy(b.xi, xi, sizeof xi); memcpy(b.xj, xj, sizeof xj);
        push_static(s, &b);
        return 1;
    }
    if (type == 5) {  /* augmented Lagrangian distance bond: kappa = kappa_start */
        b.type = PO_AL;
        memcpy(b.xi, xi, sizeof xi); memcpy(b.xj, xj, sizeof xj);
        b.al_kstart = kappa; b.al_beta = d[18]; b.al_alpha = d[19]; b.al_gamma = d[20];
        b.al_k = kappa; b.al_lam = 0.0;
        push_static(s, &b);
        return 1;
    }
    double n = norm3(ax);
    double ui[3] = {ax[0] / n, ax[1] / n, ax[2] / n}, uj[3];
    carry_dir(s, i, j, ui, uj);
    if (type == PO_REVOLUTE) {
        /* hinge about u through the pivot: two zero-length bonds at pivot +- arm*u */
        for (int sg = 1; sg >= -1; sg -= 2) {
            b.type = PO_SPHERICAL;
            for (int k = 0; k < 3; ++k) {
                b.xi[k] = xi[k] + sg * arm * ui[k];
                b.xj[k] = xj[k] + sg * arm * uj[k];
            }
            push_static(s, &b);
        }
        return 2;
    }
    if (type == PO_DRIVE) {
        /* the child point pivot_j + arm*r_j is pulled to the parent point
           pivot_i + arm*Rot(u_i, theta(t)) r_i, theta(t) = amp sin(2 pi t / period + phase) */
        double ri[3], rj[3];
        perp_unit(ui, ri);
        carry_dir(s, i, j, ri, rj);
        b.type = PO_DRIVE;
        memcpy(b.ui, ui, sizeof ui);
        memcpy(b.ri, ri, sizeof ri);
        memcpy(b.xi, xi, sizeof xi);
        for (int k = 0; k < 3; ++k) b.xj[k] = xj[k] + arm * rj[k];
        b.arm = arm; b.amp = amp; b.period = period; b.phase = phase;
        push_static(s, &b);
        return 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------ */
/* collision detection (Alg. 1, first line), decisions in single precision                */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    float c[3], A[9], he[3], infl, lo[3], hi[3];
} po_fbox;

static void fbox_of(const po_scene* s, int b, po_fbox* f) {
    const po_state* x = &s->st[b];
    const po_static* bs = &s->bs[b];
    float dt = (float)s->p.h, mg = (float)s->p.margin, dr = (float)s->p.d_hat_rel;
    for (int k = 0; k < 3; ++k) f->c[k] = (float)x->c[k];
    for (int k = 0; k < 9; ++k) f->A[k] = (float)x->A[k];
    for (int k = 0; k < 3; ++k) f->he[k] = (float)bs->he[k];
    float v0 = (float)x->v[0], v1 = (float)x->v[1], v2 = (float)x->v[2];
    float dhat = dr * (2.0f * fminf(fminf(f->he[0], f->he[1]), f->he[2]));
    float speed = sqrtf((v0 * v0 + v1 * v1) + v2 * v2);
    f->infl = (dhat + dt * speed) + mg;
    for (int k = 0; k < 3; ++k) {
        float e = ((fabsf(f->A[3 * k]) * f->he[0] + fabsf(f->A[3 * k + 1]) * f->he[1]) +
                   fabsf(f->A[3 * k + 2]) * f->he[2]) + f->infl;
        f->lo[k] = f->c[k] - e;
        f->hi[k] = f->c[k] + e;
    }
}

static int is_excluded(const po_scene* s, int a, int b) {
    for (int k = 0; k < s->n_excl; ++k)
        if (s->excl[2 * k] == a && s->excl[2 * k + 1] == b) return 1;
    return 0;
}

/* corner index bits: bit0 -> x sign, bit1 -> y sign, bit2 -> z sign (1 = +) */
static void corner_f(const float* he, int k, float* x) {
    x[0] = (k & 1) ? he[0] : -he[0];
    x[1] = (k & 2) ? he[1] : -he[1];
    x[2] = (k & 4) ? he[2] : -he[2];
}

static double dhat_of(const po_scene* s, int b) {
    const double* he = s->bs[b].he;
    double m = he[0] < he[1] ? he[0] : he[1];
    if (he[2] < m) m = he[2];
    return s->p.d_hat_rel * 2.0 * m;
}

static void push_contact(po_scene* s, const po_bond* b) {
    s->kb = (po_bond*)grow(s->kb, &s->cap_k, s->nk + 1, sizeof(po_bond));
    s->kb[s->nk++] = *b;
}

/* Contact manifold of two boxes (reading; the paper's narrow phase is not given).
   All of it in IEEE single precision with a fixed operation order, on the single-precision
   rounding of the state, so that the CUDA path produces the same contact list bit for bit:
     1. reference face: separating-axis test over the six face normals of the two boxes,
        largest separation wins (b's axes 0..2 first, then a's, lowest index on ties);
        no contact if that separation exceeds the pair's inflation delta;
     2. incident face: the face of the other box whose normal is most anti-parallel to the
        reference normal N (largest |N . axis|, lowest axis on ties);
     3. the incident face's four vertices, taken in the reference frame, are clipped
        (Sutherland-Hodgman) against the four side planes of the reference face in the
        order (m1,+), (m1,-), (m2,+), (m2,-) with m1 = (l+1)%3, m2 = (l+2)%3;
     4. each clipped point whose height above the reference face is below delta becomes a
        contact bond: i = incident body, x_i its material point (carried through the
        clipping), j = reference body, x_j the point projected onto the reference face in
        j's frame, N = the reference face's outward normal in the world. */
typedef struct { float u[3], x[3]; } po_cpt;

static float fdot_col(const float* A, int l, const float* r) {
    return (A[l] * r[0] + A[3 + l] * r[1]) + A[6 + l] * r[2];
}

static void box_box(po_scene* s, int a, int b, const po_fbox* fa, const po_fbox* fb) {
    float delta = fa->infl + fb->infl;
    float d[3], dab[3], dba[3], R[9];
    for (int k = 0; k < 3; ++k) d[k] = fa->c[k] - fb->c[k];
    for (int l = 0; l < 3; ++l) dab[l] = fdot_col(fb->A, l, d);           /* c_a in b's frame */
    float dn[3] = {-d[0], -d[1], -d[2]};
    for (int k = 0; k < 3; ++k) dba[k] = fdot_col(fa->A, k, dn);          /* c_b in a's frame */
    for (int l = 0; l < 3; ++l)                                           /* R = A_b^T A_a */
        for (int k = 0; k < 3; ++k)
            R[3 * l + k] = (fb->A[l] * fa->A[k] + fb->A[3 + l] * fa->A[3 + k]) + fb->A[6 + l] * fa->A[6 + k];
    float best = 0.0f;
    int ref_b = 1, l = 0;
    for (int ax = 0; ax < 3; ++ax) {
        float ext = (fabsf(R[3 * ax]) * fa->he[0] + fabsf(R[3 * ax + 1]) * fa->he[1]) + fabsf(R[3 * ax + 2]) * fa->he[2];
        float sep = fabsf(dab[ax]) - (fb->he[ax] + ext);
        if (ax == 0 || sep > best) { best = sep; ref_b = 1; l = ax; }
    }
    for (int ax = 0; ax < 3; ++ax) {
        float ext = (fabsf(R[ax]) * fb->he[0] + fabsf(R[3 + ax]) * fb->he[1]) + fabsf(R[6 + ax]) * fb->he[2];
        float sep = fabsf(dba[ax]) - (fa->he[ax] + ext);
        if (sep > best) { best = sep; ref_b = 0; l = ax; }
    }
    if (!(best <= delta)) return;
    const po_fbox* fr = ref_b ? fb : fa;   /* reference box */
    const po_fbox* fi = ref_b ? fa : fb;   /* incident box */
    int ir = ref_b ? b : a, ii = ref_b ? a : b;
    float sg = ref_b ? (dab[l] >= 0.0f ? 1.0f : -1.0f) : (dba[l] >= 0.0f ? 1.0f : -1.0f);
    float N[3];
    for (int k = 0; k < 3; ++k) N[k] = sg * fr->A[3 * k + l];
    /* incident face */
    int ki = 0;
    float bestd = 0.0f, dsel = 0.0f;
    for (int k = 0; k < 3; ++k) {
        float dk = fdot_col(fi->A, k, N);
        if (k == 0 || fabsf(dk) > bestd) { bestd = fabsf(dk); ki = k; dsel = dk; }
    }
    float si = dsel > 0.0f ? -1.0f : 1.0f;
    int k1 = (ki + 1) % 3, k2 = (ki + 2) % 3;
    static const float sgn1[4] = {1.0f, -1.0f, -1.0f, 1.0f}, sgn2[4] = {1.0f, 1.0f, -1.0f, -1.0f};
    po_cpt poly[8], tmp[8];
    int np = 4;
    for (int v = 0; v < 4; ++v) {
        float x[3], y[3], r[3];
        x[ki] = si * fi->he[ki];
        x[k1] = sgn1[v] * fi->he[k1];
        x[k2] = sgn2[v] * fi->he[k2];
        for (int dd = 0; dd < 3; ++dd) {
            y[dd] = ((fi->c[dd] + fi->A[3 * dd] * x[0]) + fi->A[3 * dd + 1] * x[1]) + fi->A[3 * dd + 2] * x[2];
            r[dd] = y[dd] - fr->c[dd];
        }
        for (int m = 0; m < 3; ++m) { poly[v].u[m] = fdot_col(fr->A, m, r); poly[v].x[m] = x[m]; }
    }
    int m1 = (l + 1) % 3, m2 = (l + 2) % 3;
    int planes[4] = {m1, m1, m2, m2};
    float psg[4] = {1.0f, -1.0f, 1.0f, -1.0f};
    for (int pl = 0; pl < 4 && np > 0; ++pl) {
        int m = planes[pl];
        float ps = psg[pl], lim = fr->he[m];
        int nt = 0;
        for (int v = 0; v < np; ++v) {
            const po_cpt* P = &poly[v];
            const po_cpt* Q = &poly[(v + 1) % np];
            float dp = ps * P->u[m] - lim, dq = ps * Q->u[m] - lim;
            int pin = dp <= 0.0f, qin = dq <= 0.0f;
            if (pin) tmp[nt++] = *P;
            if (pin != qin) {
                float t = dp / (dp - dq);
                po_cpt X;
                for (int c = 0; c < 3; ++c) {
                    X.u[c] = P->u[c] + t * (Q->u[c] - P->u[c]);
                    X.x[c] = P->x[c] + t * (Q->x[c] - P->x[c]);
                }
                tmp[nt++] = X;
            }
        }
        np = nt;
        memcpy(poly, tmp, (size_t)nt * sizeof(po_cpt));
    }
    double da = dhat_of(s, a), db = dhat_of(s, b);
    double ma = s->bs[a].m, mb = s->bs[b].m;
    double mmin = s->bs[b].pinned ? ma : (s->bs[a].pinned ? mb : (ma < mb ? ma : mb));
    for (int v = 0; v < np; ++v) {
        float hgt = sg * poly[v].u[l] - fr->he[l];
        if (!(hgt < delta)) continue;
        po_bond c;
        memset(&c, 0, sizeof c);
        c.type = PO_CONTACT; c.i = ii; c.j = ir;
        for (int k = 0; k < 3; ++k) {
            c.xi[k] = (double)poly[v].x[k];
            c.xj[k] = (double)poly[v].u[k];
            c.N[k] = (double)N[k];
        }
        c.xj[l] = (double)(sg * fr->he[l]);
        c.dhat = da < db ? da : db;
        c.w = s->p.c_kappa * mmin;  /* = h^2 kappa_c with kappa_c = c_kappa min(m_i, m_j) / h^2 */
        c.mu = s->p.mu;
        push_contact(s, &c);
    }
}

/* Ground plane n.y = d: every corner of a dynamic body whose height (single precision) is
   below its inflation becomes a contact bond with j = WORLD, the anchor being the corner
   projected on the plane. */
static void ground_corners(po_scene* s, int a, const po_fbox* fa) {
    float n[3] = {(float)s->p.gn[0], (float)s->p.gn[1], (float)s->p.gn[2]}, gd = (float)s->p.gd;
    for (int k = 0; k < 8; ++k) {
        float x[3], y[3];
        corner_f(fa->he, k, x);
        for (int d = 0; d < 3; ++d)
            y[d] = ((fa->c[d] + fa->A[3 * d] * x[0]) + fa->A[3 * d + 1] * x[1]) + fa->A[3 * d + 2] * x[2];
        float g = ((n[0] * y[0] + n[1] * y[1]) + n[2] * y[2]) - gd;
        if (!(g < fa->infl)) continue;
        po_bond c;
        memset(&c, 0, sizeof c);
        c.type = PO_GROUND; c.i = a; c.j = PO_WORLD;
        for (int d = 0; d < 3; ++d) {
            c.xi[d] = (double)x[d];
            c.xj[d] = (double)(y[d] - g * n[d]);
            c.N[d] = (double)n[d];
        }
        c.dhat = dhat_of(s, a);
        c.w = s->p.c_kappa * s->bs[a].m;
        c.mu = s->p.mu;
        push_contact(s, &c);
    }
}

/* Broad phase by its definition: every pair (a < b) of the same group, not both pinned,
   not joined by a user bond, whose inflated single-precision AABBs overlap on all three
   axes; then narrow phase per pair (box-box manifold), then the ground (per body, corners in index
   order). */
void po_detect(void* h) {
    po_scene* s = (po_scene*)h;
    s->np = 0;
    s->nk = 0;
    po_fbox* fb = (po_fbox*)malloc((size_t)(s->nb > 0 ? s->nb : 1) * sizeof(po_fbox));
    for (int b = 0; b < s->nb; ++b) fbox_of(s, b, &fb[b]);
    if (s->p.body_contacts) {
        for (int a = 0; a < s->nb; ++a)
            for (int b = a + 1; b < s->nb; ++b) {
                if (s->bs[a].group != s->bs[b].group) continue;
                if (s->bs[a].pinned && s->bs[b].pinned) continue;
                int ov = 1;
                for (int k = 0; k < 3; ++k)
                    if (!(fb[a].lo[k] <= fb[b].hi[k] && fb[b].lo[k] <= fb[a].hi[k])) ov = 0;
                if (!ov) continue;
                if (is_excluded(s, a, b)) continue;
                s->pairs = (int*)grow(s->pairs, &s->cap_p, 2 * s->np + 2, sizeof(int));
                s->pairs[2 * s->np] = a;
                s->pairs[2 * s->np + 1] = b;
                s->np++;
            }
        for (int p = 0; p < s->np; ++p) {
            int a = s->pairs[2 * p], b = s->pairs[2 * p + 1];
            box_box(s, a, b, &fb[a], &fb[b]);
        }
    }
    if (s->p.has_ground)
        for (int a = 0; a < s->nb; ++a)
            if (!s->bs[a].pinned) ground_corners(s, a, &fb[a]);
    free(fb);
}

/* ------------------------------------------------------------------------------------ */
/* bond rules: per end (w, f) with the end's generalised force J^T f and H term w J^T J   */
/* ------------------------------------------------------------------------------------ */

/* Contact + Coulomb friction bond rule (reading) for end points yi (body i) and yj (body j
   or the world anchor), frozen normal N, contact distance dhat, weight w = h^2 kappa_c and
   friction coefficient mu. Writes w (0 when inactive) and the two ends' f. */
/* `shift` moves only the activation threshold (active iff g < dhat + shift); it is 0 in the
   method and set only by tests that probe how a step depends on a contact sitting at the
   threshold (a decision the single-precision path may take the other way). */
static void contact_rule_at(const double* N, double dhat, double shift, double w, double mu, const double* yi,
                            const double* yj, double* wout, double* fi, double* fj) {
    double rr[3], t[3];
    for (int k = 0; k < 3; ++k) rr[k] = yi[k] - yj[k];
    double g = dot3(N, rr);
    if (!(g < dhat + shift)) {
        *wout = 0;
        memset(fi, 0, 3 * sizeof(double));
        memset(fj, 0, 3 * sizeof(double));
        return;
    }
    for (int k = 0; k < 3; ++k) t[k] = rr[k] - g * N[k];
    double tn = norm3(t), tau = mu * (dhat - g);
    double sc = (tn > tau) ? tau / tn : 1.0;
    *wout = w;
    for (int k = 0; k < 3; ++k) {
        double rs = dhat * N[k] + (t[k] - t[k] * sc);   /* r* = dhat N + (t - t_c) */
        fi[k] = w * (yj[k] + rs);
        fj[k] = w * (yi[k] - rs);
    }
}

void po_contact_rule(const double* N, double dhat, double w, double mu, const double* yi,
                     const double* yj, double* wout, double* fi, double* fj) {
    contact_rule_at(N, dhat, 0.0, w, mu, yi, yj, wout, fi, fj);
}

/* Evaluate bond b from the iterate q (12 per body).  Outputs for end i (wi, fi) and end j
   (wj, fj); an end on WORLD is ignored by the caller.
   Distance bonds (Eq. 15-19): r = y_j - y_i, d = |r|, n = r/d, phi = dPsi/dd split into
   phi+ >= 0 (implicit) and phi- <= 0 (explicit):  w = h^2 phi+(d)/d,
   f_i = w y_j + h^2 phi-(d) n,  f_j = w y_i - h^2 phi-(d) n.
     spherical / revolute sub-bond / drive: Psi = kappa d^2/2   -> phi+ = kappa d, phi- = 0
     spring (Eq. 26):        Psi = kappa (d - l)^2 / 2         -> phi+ = kappa d, phi- = -kappa l
     nonlinear elastic:      phi = (kappa/3)(d^3/l^2 - l)      -> phi+ = phi'(d) d, phi- = phi(d) - phi'(d) d
   Contact (reading): rr = y_i - y_j, g = N.rr; active iff g < dhat; t = rr - g N,
   tau = mu (dhat - g), t_c = t clamped to |t_c| <= tau, r* = dhat N + (t - t_c);
   w = h^2 kappa_c on both ends, f_i = w (y_j + r*), f_j = w (y_i - r*). */
/* material point of end i; a drive bond's parent anchor turns with theta(t) about u_i */
static void bond_xi(const po_bond* b, double t_next, double* xi) {
    memcpy(xi, b->xi, 3 * sizeof(double));
    if (b->type != PO_DRIVE) return;
    double th = b->amp * sin(2.0 * M_PI * t_next / b->period + b->phase);
    double uxr[3];
    cross3(b->ui, b->ri, uxr);
    for (int k = 0; k < 3; ++k) xi[k] = b->xi[k] + b->arm * (cos(th) * b->ri[k] + sin(th) * uxr[k]);
}

static void eval_bond(const po_scene* s, const po_bond* b, const double* q, double t_next,
                      double* wi, double* fi, double* wj, double* fj) {
    const double h2 = s->p.h * s->p.h;
    double yi[3], yj[3], xi[3];
    bond_xi(b, t_next, xi);
    world_point(q + 12 * b->i, xi, yi);
    if (b->j == PO_WORLD) memcpy(yj, b->xj, sizeof yj);
    else world_point(q + 12 * b->j, b->xj, yj);

    if (b->type == PO_CONTACT || b->type == PO_GROUND) {
        contact_rule_at(b->N, b->dhat, s->act_shift, b->w, b->mu, yi, yj, wi, fi, fj);
        *wj = *wi;
        return;
    }
    double r[3], n[3];
    for (int k = 0; k < 3; ++k) r[k] = yj[k] - yi[k];
    double d = norm3(r);
    if (d > 1e-300) for (int k = 0; k < 3; ++k) n[k] = r[k] / d;
    else { n[0] = 0; n[1] = 1; n[2] = 0; }
    double w, phim;
    switch (b->type) {
        case PO_SPRING:
            w = h2 * b->kappa; phim = -b->kappa * b->rest; break;
        case PO_AL: {
            /* phi = kappa C + lambda, C = d - l (Eq. 27): phi+ = kappa d + max(lambda - kappa l, 0),
               phi- = min(lambda - kappa l, 0); d clamped away from 0 for the implicit part */
            double cst = b->al_lam - b->al_k * b->rest;
            double dd = d > 1e-9 ? d : 1e-9;
            w = h2 * (b->al_k + (cst > 0 ? cst / dd : 0.0));
            phim = cst < 0 ? cst : 0.0;
            break;
        }
        case PO_ELASTIC_NL:
            /* tangent split of phi(d) = (kappa/3)(d^3/l^2 - l): phi+ = phi'(d) d = kappa d^3/l^2,
               phi- = phi(d) - phi'(d) d = -(2 kappa d^3)/(3 l^2) - kappa l/3 <= 0 */
            w = h2 * b->kappa * d * d / (b->rest * b->rest);
            phim = -(2.0 * b->kappa * d * d * d) / (3.0 * b->rest * b->rest) - b->kappa * b->rest / 3.0;
            break;
        default: /* spherical, revolute sub-bond, drive */
            w = h2 * b->kappa; phim = 0.0; break;
    }
    *wi = *wj = w;
    for (int k = 0; k < 3; ++k) {
        fi[k] = w * yj[k] + h2 * phim * n[k];
        fj[k] = w * yi[k] - h2 * phim * n[k];
    }
}

/* Dense 12x12 H of Eq. (20) and right-hand side of Eq. (19) for body bi at iterate q. */
static void add_end(double* H, double* rhs, const double* x, double w, const double* f) {
    double J[36];
    jacobian(x, J);
    for (int a = 0; a < 12; ++a) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += J[12 * k + a] * f[k];
        rhs[a] += s;
        for (int c = 0; c < 12; ++c) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += J[12 * k + a] * J[12 * k + c];
            H[12 * a + c] += w * t;
        }
    }
}

static void mass_terms(const po_scene* s, int bi, const double* sq, double* H, double* rhs) {
    const po_static* b = &s->bs[bi];
    memset(H, 0, 144 * sizeof(double));
    memset(rhs, 0, 12 * sizeof(double));
    for (int k = 0; k < 3; ++k) H[12 * k + k] = b->m;
    for (int blk = 0; blk < 3; ++blk)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) H[12 * (3 + 3 * blk + r) + 3 + 3 * blk + c] = b->Pi[3 * r + c];
    for (int a = 0; a < 12; ++a) {
        double t = 0;
        for (int c = 0; c < 12; ++c) t += H[12 * a + c] * sq[c];
        rhs[a] = t;
    }
}

/* Augmented Lagrangian update of one bond after a sweep (Eq. 28), from the constraint of
   the new iterate q^{k+1} (the primal result of that sweep): lambda <- kappa C + lambda,
   kappa <- kappa + beta |C|, C = d - l, lambda taking the old kappa. */
static void al_update(po_bond* b, const double* q) {
    double yi[3], yj[3];
    world_point(q + 12 * b->i, b->xi, yi);
    if (b->j == PO_WORLD) memcpy(yj, b->xj, sizeof yj);
    else world_point(q + 12 * b->j, b->xj, yj);
    double r[3] = {yj[0] - yi[0], yj[1] - yi[1], yj[2] - yi[2]};
    double c = norm3(r) - b->rest;
    b->al_lam = b->al_k * c + b->al_lam;
    b->al_k = b->al_k + b->al_beta * fabs(c);
}

/* Assemble every dynamic body's H and rhs for the iterate q and predictor sq. */
/* Diagnostic, not part of the step: distance |g - dhat| of a contact from its activation
   threshold at iterate q, folded into the per-body minimum `margin`. */
static void note_margin(const po_bond* b, const double* q, double* margin) {
    double yi[3], yj[3];
    world_point(q + 12 * b->i, b->xi, yi);
    if (b->j == PO_WORLD) memcpy(yj, b->xj, sizeof yj);
    else world_point(q + 12 * b->j, b->xj, yj);
    double rr[3] = {yi[0] - yj[0], yi[1] - yj[1], yi[2] - yj[2]};
    double m = fabs(dot3(b->N, rr) - b->dhat);
    if (m < margin[b->i]) margin[b->i] = m;
    if (b->j != PO_WORLD && m < margin[b->j]) margin[b->j] = m;
}

static void assemble_all(const po_scene* s, const double* q, const double* sq, double t_next,
                         double* H, double* rhs, double* margin) {
    for (int b = 0; b < s->nb; ++b) mass_terms(s, b, sq + 12 * b, H + 144 * b, rhs + 12 * b);
    for (int pass = 0; pass < 2; ++pass) {
        int n = pass ? s->nk : s->nc;
        const po_bond* arr = pass ? s->kb : s->cb;
        for (int e = 0; e < n; ++e) {
            const po_bond* b = &arr[e];
            double wi, wj, fi[3], fj[3];
            if (margin && (b->type == PO_CONTACT || b->type == PO_GROUND)) note_margin(b, q, margin);
            eval_bond(s, b, q, t_next, &wi, fi, &wj, fj);
            double xi[3];
            bond_xi(b, t_next, xi);
            if (!s->bs[b->i].pinned) add_end(H + 144 * b->i, rhs + 12 * b->i, xi, wi, fi);
            if (b->j != PO_WORLD && !s->bs[b->j].pinned) add_end(H + 144 * b->j, rhs + 12 * b->j, b->xj, wj, fj);
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* one step (Algorithm 1)                                                                */
/* ------------------------------------------------------------------------------------ */

static int step_once(po_scene* s) {
    const double h = s->p.h;
    const int nb = s->nb;
    po_detect(s);                                                 /* collision detection */
    double* qn = (double*)malloc(sizeof(double) * 12 * (nb ? nb : 1));
    double* sq = (double*)malloc(sizeof(double) * 12 * (nb ? nb : 1));
    double* q = (double*)malloc(sizeof(double) * 12 * (nb ? nb : 1));
    double* q1 = (double*)malloc(sizeof(double) * 12 * (nb ? nb : 1));
    double* H = (double*)malloc(sizeof(double) * 144 * (nb ? nb : 1));
    double* rhs = (double*)malloc(sizeof(double) * 12 * (nb ? nb : 1));
    double* Qs = (double*)malloc(sizeof(double) * 4 * (nb ? nb : 1));
    int err = 0;
    for (int b = 0; b < nb; ++b) {
        po_state* x = &s->st[b];
        state_to_q(x, qn + 12 * b);
        if (s->bs[b].pinned) { memcpy(sq + 12 * b, qn + 12 * b, 12 * sizeof(double)); continue; }
        /* predictor: v* = v + h g; c* = c + h v*; Q* = Q + h/2 [w, 0] Q (then normalised);
           A* = R(Q*); s = q^0 = (c*, A*) */
        double vs[3], cs[3];
        for (int k = 0; k < 3; ++k) { vs[k] = x->v[k] + h * s->p.g[k]; cs[k] = x->c[k] + h * vs[k]; }
        const double* Q = x->Q;
        const double* w = x->w;
        double wq[4] = {  /* (w, 0) (x) Q, vector part first */
            w[0] * Q[3] + (w[1] * Q[2] - w[2] * Q[1]),
            w[1] * Q[3] + (w[2] * Q[0] - w[0] * Q[2]),
            w[2] * Q[3] + (w[0] * Q[1] - w[1] * Q[0]),
            -(w[0] * Q[0] + w[1] * Q[1] + w[2] * Q[2])};
        double Qn[4], nn = 0;
        for (int k = 0; k < 4; ++k) { Qn[k] = Q[k] + 0.5 * h * wq[k]; nn += Qn[k] * Qn[k]; }
        nn = sqrt(nn);
        for (int k = 0; k < 4; ++k) Qn[k] /= nn;
        memcpy(Qs + 4 * b, Qn, sizeof Qn);
        double As[9];
        po_quat_to_mat(Qn, As);
        for (int k = 0; k < 3; ++k) sq[12 * b + k] = cs[k];
        for (int k = 0; k < 9; ++k) sq[12 * b + 3 + k] = As[k];
    }
    memcpy(q, sq, sizeof(double) * 12 * nb);
    double t_next = (double)(s->step + 1) * h;
    /* augmented Lagrangian warm start (Eq. 29): kappa^0 = max(gamma kappa^n, kappa_start),
       lambda^0 = alpha gamma lambda^n */
    for (int e = 0; e < s->nc; ++e) {
        po_bond* b = &s->cb[e];
        if (b->type != PO_AL) continue;
        double k = b->al_gamma * b->al_k;
        b->al_k = k > b->al_kstart ? k : b->al_kstart;
        b->al_lam = b->al_alpha * b->al_gamma * b->al_lam;
    }
    if (!s->resid) s->resid = (double*)calloc((size_t)(s->n_groups > 0 ? s->n_groups : 1), sizeof(double));
    if (!s->amargin) s->amargin = (double*)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    for (int b = 0; b < nb; ++b) s->amargin[b] = INFINITY;
    /* Sec. 4.2: the sweeps stop at n_iter, or -- with a residual threshold -- a scene (group)
       stops after the first sweep whose residual is at most resid_tol; its bodies then keep
       that sweep's iterate while the other scenes go on */
    const int ng = s->n_groups > 0 ? s->n_groups : 1;
    char* done = (char*)calloc((size_t)ng, 1);
    double* r2g = (double*)calloc((size_t)ng, sizeof(double));
    s->last_sweeps = 0;
    for (int it = 0; it < s->p.n_iter; ++it) {
        assemble_all(s, q, sq, t_next, H, rhs, s->amargin);      /* Jacobi: all read q^k */
        for (int g = 0; g < ng; ++g) r2g[g] = 0;
        for (int b = 0; b < nb; ++b) {
            double* out = q1 + 12 * b;
            if (s->bs[b].pinned) { memcpy(out, qn + 12 * b, 12 * sizeof(double)); continue; }
            if (done[s->bs[b].group]) { memcpy(out, q + 12 * b, 12 * sizeof(double)); continue; }
            if (po_cholesky_solve(12, H + 144 * b, rhs + 12 * b, out) != 0) { err = 1; memcpy(out, q + 12 * b, 12 * sizeof(double)); }
            if (s->p.project) {                                   /* local solve */
                double R[9];
                po_polar_rotation(out + 3, R, NULL);
                memcpy(out + 3, R, sizeof R);
            }
            double r2 = 0;
            for (int k = 0; k < 12; ++k) { double dd = out[k] - q[12 * b + k]; r2 += dd * dd; }
            r2g[s->bs[b].group] += r2;
        }
        memcpy(q, q1, sizeof(double) * 12 * nb);
        if (s->round_iterates)
            for (int k = 0; k < 12 * nb; ++k) q[k] = (double)(float)q[k];
        for (int e = 0; e < s->nc; ++e)
            if (s->cb[e].type == PO_AL) al_update(&s->cb[e], q);
        s->last_sweeps = it + 1;
        int active = 0;
        for (int g = 0; g < s->n_groups; ++g) {
            if (done[g]) continue;
            s->resid[g] = sqrt(r2g[g]);
            if (s->p.resid_tol > 0 && s->resid[g] <= s->p.resid_tol) done[g] = 1;
            else ++active;
        }
        if (s->p.resid_tol > 0 && active == 0) break;
    }
    free(done);
    free(r2g);
    /* velocity recovery */
    for (int b = 0; b < nb; ++b) {
        po_state* x = &s->st[b];
        if (s->bs[b].pinned) continue;
        double* qb = q + 12 * b;
        double W[9], dA[9], At[9];
        for (int k = 0; k < 3; ++k) x->v[k] = (qb[k] - x->c[k]) / h;
        for (int k = 0; k < 9; ++k) dA[k] = (qb[3 + k] - x->A[k]) / h;
        for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) At[3 * r + c] = x->A[3 * c + r];
        mat3_mul(dA, At, W);  /* (A^{n+1} - A^n) (A^n)^{-1} / h with (A^n)^{-1} = (A^n)^T */
        x->w[0] = 0.5 * (W[7] - W[5]);
        x->w[1] = 0.5 * (W[2] - W[6]);
        x->w[2] = 0.5 * (W[3] - W[1]);
        for (int k = 0; k < 3; ++k) x->c[k] = qb[k];
        for (int k = 0; k < 9; ++k) x->A[k] = qb[3 + k];
        if (s->p.project) {
            double Qn[4];
            po_mat_to_quat(x->A, Qn);
            double dp = Qn[0] * x->Q[0] + Qn[1] * x->Q[1] + Qn[2] * x->Q[2] + Qn[3] * x->Q[3];
            if (dp < 0) for (int k = 0; k < 4; ++k) Qn[k] = -Qn[k];
            memcpy(x->Q, Qn, sizeof Qn);
        } else {
            memcpy(x->Q, Qs + 4 * b, 4 * sizeof(double));
        }
    }
    s->step++;
    free(qn); free(sq); free(q); free(q1); free(H); free(rhs); free(Qs);
    return err;
}

int po_step(void* h, int nsteps) {
    po_scene* s = (po_scene*)h;
    int err = 0;
    for (int k = 0; k < nsteps; ++k) err |= step_once(s);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* accessors                                                                              */
/* ------------------------------------------------------------------------------------ */

int po_n_bodies(void* h) { return ((po_scene*)h)->nb; }
int po_n_static_bonds(void* h) { return ((po_scene*)h)->nc; }
int64_t po_step_index(void* h) { return ((po_scene*)h)->step; }
void po_set_step_index(void* h, int64_t k) { ((po_scene*)h)->step = k; }

/* state rows: c(3), A(9, row-major), Q(4: x, y, z, w), v(3), w(3) = 22 doubles per body */
void po_get_state(void* h, double* out) {
    po_scene* s = (po_scene*)h;
    for (int b = 0; b < s->nb; ++b) {
        po_state* x = &s->st[b];
        double* o = out + 22 * b;
        memcpy(o, x->c, 3 * sizeof(double));
        memcpy(o + 3, x->A, 9 * sizeof(double));
        memcpy(o + 12, x->Q, 4 * sizeof(double));
        memcpy(o + 16, x->v, 3 * sizeof(double));
        memcpy(o + 19, x->w, 3 * sizeof(double));
    }
}

void po_set_state(void* h, const double* in) {
    po_scene* s = (po_scene*)h;
    for (int b = 0; b < s->nb; ++b) {
        po_state* x = &s->st[b];
        const double* o = in + 22 * b;
        memcpy(x->c, o, 3 * sizeof(double));
        memcpy(x->A, o + 3, 9 * sizeof(double));
        memcpy(x->Q, o + 12, 4 * sizeof(double));
        memcpy(x->v, o + 16, 3 * sizeof(double));
        memcpy(x->w, o + 19, 3 * sizeof(double));
    }
}

int po_get_pairs(void* h, int* out, int cap) {
    po_scene* s = (po_scene*)h;
    int n = s->np < cap ? s->np : cap;
    memcpy(out, s->pairs, 2 * (size_t)n * sizeof(int));
    return s->np;
}

/* contact rows: meta (type, i, j, corner-free) ints x3; data xi(3), xj(3), N(3), dhat, w */
int po_get_contacts(void* h, int* meta, double* data, int cap) {
    po_scene* s = (po_scene*)h;
    int n = s->nk < cap ? s->nk : cap;
    for (int k = 0; k < n; ++k) {
        const po_bond* b = &s->kb[k];
        meta[3 * k] = b->type; meta[3 * k + 1] = b->i; meta[3 * k + 2] = b->j;
        double* d = data + 11 * k;
        memcpy(d, b->xi, 3 * sizeof(double));
        memcpy(d + 3, b->xj, 3 * sizeof(double));
        memcpy(d + 6, b->N, 3 * sizeof(double));
        d[9] = b->dhat; d[10] = b->w;
    }
    return s->nk;
}

int po_get_residual(void* h, double* out, int cap) {
    po_scene* s = (po_scene*)h;
    int n = s->n_groups < cap ? s->n_groups : cap;
    if (s->resid) memcpy(out, s->resid, (size_t)n * sizeof(double));
    else memset(out, 0, (size_t)n * sizeof(double));
    return s->n_groups;
}

/* The dense per-body system (H of Eq. 20, rhs of Eq. 19) at the current state taken as
   the iterate, with the predictor s equal to the current state: exposes the assembly for
   the algebra pins (Eq. 24 structure, Eq. 25 inverse). Uses the contacts of the last
   detection. */
void po_body_system(void* h, int body, double* H, double* rhs) {
    po_scene* s = (po_scene*)h;
    int nb = s->nb;
    double* q = (double*)malloc(sizeof(double) * 12 * nb);
    double* HH = (double*)malloc(sizeof(double) * 144 * nb);
    double* rr = (double*)malloc(sizeof(double) * 12 * nb);
    for (int b = 0; b < nb; ++b) state_to_q(&s->st[b], q + 12 * b);
    assemble_all(s, q, q, (double)(s->step + 1) * s->p.h, HH, rr, NULL);
    memcpy(H, HH + 144 * body, 144 * sizeof(double));
    memcpy(rhs, rr + 12 * body, 12 * sizeof(double));
    free(q); free(HH); free(rr);
}

/* Sweeps the last step ran. */
int po_last_sweeps(void* h) { return ((po_scene*)h)->last_sweeps; }

/* Test probe: contacts of the following steps switch on at g < dhat + shift (0 restores the method). */
void po_set_activation_shift(void* h, double shift) { ((po_scene*)h)->act_shift = shift; }

/* Test probe: with on != 0, every sweep's iterate q^{k+1} of the following steps is rounded to
   single precision before the next sweep reads it -- the perturbation that a path storing its
   iterates in single precision applies at every sweep (0 restores the method). */
void po_set_round_iterates(void* h, int on) { ((po_scene*)h)->round_iterates = on; }

/* Per body, the smallest |g - dhat| of its contacts over the sweeps of the last step
   (infinity for a body without contacts): how close a contact came to switching on or off. */
void po_get_activation_margin(void* h, double* out) {
    po_scene* s = (po_scene*)h;
    for (int b = 0; b < s->nb; ++b) out[b] = s->amargin ? s->amargin[b] : INFINITY;
}

/* Augmented Lagrangian state (kappa, lambda) of every static bond (0, 0 for other types). */
void po_get_al_state(void* h, double* out) {
    po_scene* s = (po_scene*)h;
    for (int e = 0; e < s->nc; ++e) {
        out[2 * e] = s->cb[e].type == PO_AL ? s->cb[e].al_k : 0.0;
        out[2 * e + 1] = s->cb[e].type == PO_AL ? s->cb[e].al_lam : 0.0;
    }
}

void po_set_al_state(void* h, const double* in) {
    po_scene* s = (po_scene*)h;
    for (int e = 0; e < s->nc; ++e)
        if (s->cb[e].type == PO_AL) { s->cb[e].al_k = in[2 * e]; s->cb[e].al_lam = in[2 * e + 1]; }
}

/* Static internal bonds after expansion: type, i, j, xi(3), xj(3) (drive: xj child point) */
int po_get_static_bonds(void* h, int* meta, double* data, int cap) {
    po_scene* s = (po_scene*)h;
    int n = s->nc < cap ? s->nc : cap;
    for (int k = 0; k < n; ++k) {
        const po_bond* b = &s->cb[k];
        meta[3 * k] = b->type; meta[3 * k + 1] = b->i; meta[3 * k + 2] = b->j;
        memcpy(data + 6 * k, b->xi, 3 * sizeof(double));
        memcpy(data + 6 * k + 3, b->xj, 3 * sizeof(double));
    }
    return s->nc;
}
