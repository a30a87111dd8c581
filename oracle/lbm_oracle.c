/*
 * FP64 CPU oracle for the D3Q7 multiple-relaxation-time lattice Boltzmann
 * model with an off-diagonal (anisotropic) relaxation block, used to predict
 * effective thermal conductivity of heterogeneous anisotropic media
 * (Fang et al., arXiv 1503.08718, Sections 2.2-2.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product library never
 * links, calls or falls back to it, and the two share no source.
 *
 * It follows the paper's statement of the method step by step:
 *   - collision matrix Omega = M^-1 S M built literally (Eq. 8), with M from
 *     Eq. 11 and S the inverse of the block matrix of Eq. 12, tau from Eq. 13;
 *   - collision f^ = f - Omega (f - f^eq) with f^eq from Eq. 6 (Eq. 5);
 *   - push streaming (Eq. 5 left side, Eq. 21 across interfaces) with
 *     Dirichlet (Eq. 23), adiabatic Neumann (Eq. 24 with phi_n = 0) and
 *     periodic (Eq. 25) faces placed half a lattice spacing outside the nodes;
 *   - temperature T = sum f (Eq. 14), gradient from the 3x3 system of Eq. 15,
 *     flux q = -D grad T (Eq. 16 with rho c_p = 1 from Eq. 20, minus sign
 *     restored), effective conductivity from Eq. 22.
 *
 * Readings of the paper taken here (lattice units dx = dt = 1, c = 1):
 *   gamma = 1/8 (Section 2.2), eps = 2 gamma; tau_0 = tau_4 = tau_5 = tau_6 = 1;
 *   D = s * lambda for a lattice scale s chosen by the caller; hot wall
 *   (t_hot) on the axis-min face, cold wall on the axis-max face; initial
 *   field f^eq of a linear profile between the walls; state n is the
 *   pre-collision distribution after n full steps.
 *
 * Every parity claim is pinned by tests that do not reuse this code's
 * arithmetic: closed forms, conservation, a dense direct solve of the fixed
 * point and a mirror-symmetry identity for adiabatic faces.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 7
static const double GAMMA = 0.125;   /* Section 2.2: gamma = 1/8 */
static const double EPS = 0.25;      /* eps = 2 gamma */

/* D3Q7 discrete velocities of Eq. 7 (c = 1). */
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1};
static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5};

/* ------------------------------------------------------------------ */
/* Small dense linear algebra (Gauss-Jordan with partial pivoting)    */
/* ------------------------------------------------------------------ */

/* Inverts the n x n row-major matrix a into inv. Returns 0, or -1 if singular. */
static int invert(int n, const double *a, double *inv) {
    double w[Q * 2 * Q];
    int m = 2 * n;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            w[i * m + j] = a[i * n + j];
            w[i * m + n + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(w[r * m + c]) > fabs(w[p * m + c])) p = r;
        if (w[p * m + c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < m; ++j) {
                double t = w[c * m + j];
                w[c * m + j] = w[p * m + j];
                w[p * m + j] = t;
            }
        double d = w[c * m + c];
        for (int j = 0; j < m; ++j) w[c * m + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = w[r * m + c];
            if (f == 0.0) continue;
            for (int j = 0; j < m; ++j) w[r * m + j] -= f * w[c * m + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = w[i * m + n + j];
    return 0;
}

/* Solves the 3x3 system a x = b (a row-major) by Gaussian elimination. */
static int solve3(const double *a_in, const double *b_in, double *x) {
    double a[9], b[3];
    memcpy(a, a_in, sizeof a);
    memcpy(b, b_in, sizeof b);
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(a[r * 3 + c]) > fabs(a[p * 3 + c])) p = r;
        if (a[p * 3 + c] == 0.0) return -1;
        if (p != c) {
            for (int j = 0; j < 3; ++j) {
                double t = a[c * 3 + j];
                a[c * 3 + j] = a[p * 3 + j];
                a[p * 3 + j] = t;
            }
            double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            double f = a[r * 3 + c] / a[c * 3 + c];
            for (int j = c; j < 3; ++j) a[r * 3 + j] -= f * a[c * 3 + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < 3; ++j) s -= a[r * 3 + j] * x[j];
        x[r] = s / a[r * 3 + r];
    }
    return 0;
}

/* (xx, yy, zz, yz, xz, xy) -> row-major 3x3. */
static void full3(const double *t6, double *m) {
    m[0] = t6[0]; m[1] = t6[5]; m[2] = t6[4];
    m[3] = t6[5]; m[4] = t6[1]; m[5] = t6[3];
    m[6] = t6[4]; m[7] = t6[3]; m[8] = t6[2];
}

/* ------------------------------------------------------------------ */
/* Collision operator                                                 */
/* ------------------------------------------------------------------ */

/* Eq. 11 with c = 1: rows are 1, e_x, e_y, e_z, 6/-1, 2/2/-1.., 0/0/1/1/-1/-1. */
void orc_moment_matrix(double *M) {
    static const double m[Q * Q] = {
        1, 1, 1, 1, 1, 1, 1,
        0, 1, -1, 0, 0, 0, 0,
        0, 0, 0, 1, -1, 0, 0,
        0, 0, 0, 0, 0, 1, -1,
        6, -1, -1, -1, -1, -1, -1,
        0, 2, 2, -1, -1, -1, -1,
        0, 0, 0, 1, 1, -1, -1};
    memcpy(M, m, sizeof m);
}

/* Eq. 13 in lattice units: tau = I/2 + D/eps with D = s * lambda. */
void orc_tau(const double *lam6, double s, double *tau) {
    double lam[9];
    full3(lam6, lam);
    for (int i = 0; i < 9; ++i) tau[i] = s * lam[i] / EPS;
    tau[0] += 0.5;
    tau[4] += 0.5;
    tau[8] += 0.5;
}

/* Omega = M^-1 S M (Eq. 8); S is the inverse of the S^-1 of Eq. 12 with
 * tau_0 = tau_4 = tau_5 = tau_6 = 1 and the 3x3 block tau of Eq. 13.
 * M^-1 is computed numerically.  Returns 0, or -1 if a matrix is singular. */
int orc_collision_matrix(const double *lam6, double s, double *Omega) {
    double M[Q * Q], Minv[Q * Q], Sinv[Q * Q], S[Q * Q], tau[9], SM[Q * Q];
    orc_moment_matrix(M);
    orc_tau(lam6, s, tau);
    memset(Sinv, 0, sizeof Sinv);
    Sinv[0 * Q + 0] = 1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Sinv[(1 + a) * Q + (1 + b)] = tau[a * 3 + b];
    Sinv[4 * Q + 4] = 1.0;
    Sinv[5 * Q + 5] = 1.0;
    Sinv[6 * Q + 6] = 1.0;
    if (invert(Q, Sinv, S) || invert(Q, M, Minv)) return -1;
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += S[i * Q + k] * M[k * Q + j];
            SM[i * Q + j] = acc;
        }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += Minv[i * Q + k] * SM[k * Q + j];
            Omega[i * Q + j] = acc;
        }
    return 0;
}

/* Eq. 6: equilibrium of temperature T. */
static void equilibrium(double T, double *feq) {
    feq[0] = (1.0 - 6.0 * GAMMA) * T;
    for (int i = 1; i < Q; ++i) feq[i] = GAMMA * T;
}

/* Eq. 5 right side for one node: fhat = f - Omega (f - f^eq(sum f)). */
void orc_collide_node(const double *Omega, const double *f, double *fhat) {
    double T = 0.0, feq[Q], d[Q];
    for (int i = 0; i < Q; ++i) T += f[i];
    equilibrium(T, feq);
    for (int i = 0; i < Q; ++i) d[i] = f[i] - feq[i];
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += Omega[i * Q + k] * d[k];
        fhat[i] = f[i] - acc;
    }
}

/* Lattice scale putting the largest diagonal tau at tau_max. */
double orc_lattice_scale(const double *lam6, int n_phases, double tau_max) {
    double m = 0.0;
    for (int p = 0; p < n_phases; ++p)
        for (int a = 0; a < 3; ++a)
            if (lam6[p * 6 + a] > m) m = lam6[p * 6 + a];
    return EPS * (tau_max - 0.5) / m;
}

/* ------------------------------------------------------------------ */
/* Lattice state                                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n[3];          /* nx, ny, nz */
    int64_t N;
    uint8_t *phase;        /* [nz][ny][nx] */
    int n_phases;
    double *lam;           /* n_phases * 6 */
    double *tau;           /* n_phases * 9 */
    double *Omega;         /* n_phases * 49 */
    double s;
    int axis;              /* Dirichlet axis 0/1/2 */
    int lateral;           /* 0 periodic, 1 adiabatic */
    double t_hot, t_cold;
    double *f, *fn;        /* [7][N] pre-collision state and scratch */
    int64_t iter;
} orc_lbm;

void orc_destroy(orc_lbm *o) {
    if (!o) return;
    free(o->phase); free(o->lam); free(o->tau); free(o->Omega);
    free(o->f); free(o->fn);
    free(o);
}

orc_lbm *orc_create(int64_t nx, int64_t ny, int64_t nz, const uint8_t *phase,
                    int n_phases, const double *lam6, double s, int axis,
                    int lateral, double t_hot, double t_cold) {
    if (nx < 1 || ny < 1 || nz < 1 || n_phases < 1 || axis < 0 || axis > 2 ||
        lateral < 0 || lateral > 1 || !(s > 0.0))
        return NULL;
    orc_lbm *o = (orc_lbm *)calloc(1, sizeof *o);
    if (!o) return NULL;
    o->n[0] = nx; o->n[1] = ny; o->n[2] = nz;
    o->N = nx * ny * nz;
    o->n_phases = n_phases;
    o->s = s;
    o->axis = axis;
    o->lateral = lateral;
    o->t_hot = t_hot;
    o->t_cold = t_cold;
    o->phase = (uint8_t *)malloc((size_t)o->N);
    o->lam = (double *)malloc(sizeof(double) * 6 * n_phases);
    o->tau = (double *)malloc(sizeof(double) * 9 * n_phases);
    o->Omega = (double *)malloc(sizeof(double) * 49 * n_phases);
    o->f = (double *)malloc(sizeof(double) * Q * o->N);
    o->fn = (double *)malloc(sizeof(double) * Q * o->N);
    if (!o->phase || !o->lam || !o->tau || !o->Omega || !o->f || !o->fn) {
        orc_destroy(o);
        return NULL;
    }
    for (int64_t v = 0; v < o->N; ++v) {
        if (phase[v] >= n_phases) { orc_destroy(o); return NULL; }
        o->phase[v] = phase[v];
    }
    memcpy(o->lam, lam6, sizeof(double) * 6 * n_phases);
    for (int p = 0; p < n_phases; ++p) {
        orc_tau(lam6 + 6 * p, s, o->tau + 9 * p);
        if (orc_collision_matrix(lam6 + 6 * p, s, o->Omega + 49 * p)) {
            orc_destroy(o);
            return NULL;
        }
    }
    return o;
}

static inline int64_t node_index(const orc_lbm *o, int64_t x, int64_t y, int64_t z) {
    return (z * o->n[1] + y) * o->n[0] + x;
}

/* Initial state: f^eq of the linear profile between the walls,
 * T0(i) = t_hot + (t_cold - t_hot) (i + 1/2) / N_axis. */
void orc_init_linear(orc_lbm *o) {
    int64_t na = o->n[o->axis];
    for (int64_t z = 0; z < o->n[2]; ++z)
        for (int64_t y = 0; y < o->n[1]; ++y)
            for (int64_t x = 0; x < o->n[0]; ++x) {
                int64_t c[3] = {x, y, z};
                double T = o->t_hot + (o->t_cold - o->t_hot) * ((double)c[o->axis] + 0.5) / (double)na;
                double feq[Q];
                equilibrium(T, feq);
                int64_t v = node_index(o, x, y, z);
                for (int i = 0; i < Q; ++i) o->f[i * o->N + v] = feq[i];
            }
    o->iter = 0;
}

/* Initial state f^eq(T) of a given temperature field. */
void orc_init_field(orc_lbm *o, const double *T) {
    for (int64_t v = 0; v < o->N; ++v) {
        double feq[Q];
        equilibrium(T[v], feq);
        for (int i = 0; i < Q; ++i) o->f[i * o->N + v] = feq[i];
    }
    o->iter = 0;
}

void orc_set_f(orc_lbm *o, const double *f) { memcpy(o->f, f, sizeof(double) * Q * o->N); }
void orc_get_f(const orc_lbm *o, double *f) { memcpy(f, o->f, sizeof(double) * Q * o->N); }
int64_t orc_iter(const orc_lbm *o) { return o->iter; }

/* One full step: collide every node (Eq. 5), then push each post-collision
 * population to its neighbour x + e_i (Eq. 21), applying the face rule where
 * the neighbour lies outside the cell. */
static void step_once(orc_lbm *o) {
    const int64_t nx = o->n[0], ny = o->n[1], nz = o->n[2], N = o->N;
    double *f = o->f, *fn = o->fn;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z) {
        for (int64_t y = 0; y < ny; ++y) {
            for (int64_t x = 0; x < nx; ++x) {
                int64_t v = (z * ny + y) * nx + x;
                double fl[Q], fh[Q];
                for (int i = 0; i < Q; ++i) fl[i] = f[i * N + v];
                orc_collide_node(o->Omega + 49 * o->phase[v], fl, fh);
                fn[v] = fh[0];
                for (int i = 1; i < Q; ++i) {
                    int64_t c[3] = {x + EX[i], y + EY[i], z + EZ[i]};
                    int d = (i - 1) / 2;              /* axis the velocity runs along */
                    if (c[d] >= 0 && c[d] < o->n[d]) {
                        fn[i * N + node_index(o, c[0], c[1], c[2])] = fh[i];
                    } else if (d == o->axis) {
                        /* Eq. 23: the population leaving through a wall comes
                         * back reversed as -fhat + eps * T_wall. */
                        double tw = (c[d] < 0) ? o->t_hot : o->t_cold;
                        fn[OPP[i] * N + v] = -fh[i] + EPS * tw;
                    } else if (o->lateral == 0) {
                        /* Eq. 25: periodic wrap. */
                        c[d] = (c[d] < 0) ? o->n[d] - 1 : 0;
                        fn[i * N + node_index(o, c[0], c[1], c[2])] = fh[i];
                    } else {
                        /* Eq. 24 with phi_n = 0: plain bounce-back. */
                        fn[OPP[i] * N + v] = fh[i];
                    }
                }
            }
        }
    }
    o->f = fn;
    o->fn = f;
    o->iter += 1;
}

void orc_step(orc_lbm *o, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) step_once(o);
}

/* Eq. 14 on the current (pre-collision) state. */
void orc_temperature(const orc_lbm *o, double *T) {
    const int64_t N = o->N;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; ++v) {
        double t = 0.0;
        for (int i = 0; i < Q; ++i) t += o->f[i * N + v];
        T[v] = t;
    }
}

/* Eq. 15-16: per-node flux q (3 x N, component-major) from the current
 * pre-collision state: tau grad T = -j / eps, q = -D grad T. */
int orc_flux_field(const orc_lbm *o, double *q) {
    const int64_t N = o->N;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t v = 0; v < N; ++v) {
        const double *tau = o->tau + 9 * o->phase[v];
        double lam[9], rhs[3], g[3];
        full3(o->lam + 6 * o->phase[v], lam);
        rhs[0] = -(o->f[1 * N + v] - o->f[2 * N + v]) / EPS;
        rhs[1] = -(o->f[3 * N + v] - o->f[4 * N + v]) / EPS;
        rhs[2] = -(o->f[5 * N + v] - o->f[6 * N + v]) / EPS;
        if (solve3(tau, rhs, g)) { bad = 1; continue; }
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b) acc += o->s * lam[a * 3 + b] * g[b];
            q[a * N + v] = -acc;
        }
    }
    return bad ? -1 : 0;
}

/* Plane sums of the flux component along the Dirichlet axis: Q[k] over the
 * node plane with index k along that axis (length N_axis). */
int orc_plane_flux(const orc_lbm *o, double *Qk) {
    const int64_t N = o->N;
    double *q = (double *)malloc(sizeof(double) * 3 * N);
    if (!q) return -1;
    if (orc_flux_field(o, q)) { free(q); return -1; }
    int a = o->axis;
    for (int64_t k = 0; k < o->n[a]; ++k) Qk[k] = 0.0;
    for (int64_t z = 0; z < o->n[2]; ++z)
        for (int64_t y = 0; y < o->n[1]; ++y)
            for (int64_t x = 0; x < o->n[0]; ++x) {
                int64_t c[3] = {x, y, z};
                Qk[c[a]] += q[a * N + node_index(o, x, y, z)];
            }
    free(q);
    return 0;
}

/* Eq. 22 in lattice units: L = N_a, A = N_b N_c, and dividing by s turns the
 * lattice diffusivity back into conductivity.  Also returns the plane-flux
 * spread R_Q = (max Q - min Q) / |mean Q|. */
int orc_k_eff(const orc_lbm *o, double *k_eff, double *r_q) {
    int a = o->axis;
    int64_t na = o->n[a];
    double *Qk = (double *)malloc(sizeof(double) * na);
    if (!Qk) return -1;
    if (orc_plane_flux(o, Qk)) { free(Qk); return -1; }
    double sum = 0.0, mx = Qk[0], mn = Qk[0];
    for (int64_t k = 0; k < na; ++k) {
        sum += Qk[k];
        if (Qk[k] > mx) mx = Qk[k];
        if (Qk[k] < mn) mn = Qk[k];
    }
    double mean = sum / (double)na;
    double area = (double)(o->N / na);
    *k_eff = (double)na * mean / (o->s * (o->t_hot - o->t_cold) * area);
    if (r_q) *r_q = (mx - mn) / fabs(mean);
    free(Qk);
    return 0;
}

/* Iterates in check intervals of check_every steps (the last one shortened
 * by max_iters) until R_T <= tol at a check.  The paper states no stopping
 * rule; the reading taken here is the mean per-step temperature change over
 * the interval, relative to the field:
 *     R_T = sum|T^n - T^(n-m)| / (m * sum|T^n|),  m = steps in the interval.
 * Returns 0 when converged, 1 when max_iters was reached, -1 on a
 * non-finite residual or an error. */
int orc_solve(orc_lbm *o, double tol, int64_t check_every, int64_t max_iters,
              double *r_t_out) {
    const int64_t N = o->N;
    double *Tp = (double *)malloc(sizeof(double) * N);
    double *T = (double *)malloc(sizeof(double) * N);
    if (!Tp || !T) { free(Tp); free(T); return -1; }
    int rc = 1;
    double r_t = INFINITY;
    orc_temperature(o, Tp);
    while (o->iter < max_iters) {
        int64_t left = max_iters - o->iter;
        int64_t run = check_every < left ? check_every : left;
        orc_step(o, run);
        orc_temperature(o, T);
        double num = 0.0, den = 0.0;
        for (int64_t v = 0; v < N; ++v) {
            num += fabs(T[v] - Tp[v]);
            den += fabs(T[v]);
        }
        r_t = num / ((double)run * den);
        double *t = Tp; Tp = T; T = t;
        if (!isfinite(r_t)) { rc = -1; break; }
        if (r_t <= tol) { rc = 0; break; }
    }
    if (r_t_out) *r_t_out = r_t;
    free(Tp);
    free(T);
    return rc;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Synthetic braided-cell voxeliser (the oracle's own implementation)  */
/* ------------------------------------------------------------------ */
/*
 * Voxel-centre membership test for the synthetic four-directional braid
 * (the paper's step-wise approximation of curved yarn boundaries, Section
 * 3.2, with yarns at interior braiding angle g from z, Section 4.1).  All
 * arithmetic is FP64 evaluated left to right with no contraction (this file
 * is compiled with -ffp-contract=off) so that an independent implementation
 * following the same written recipe reproduces the phase map bit for bit.
 *
 * Family k of yarn i is i mod 4 with signs (+,+), (-,+), (-,-), (+,-).
 * anchors[2i], anchors[2i+1] are the yarn's axis point at z = 0.
 * Yarns are taken in order until the non-matrix fraction reaches phi; a voxel
 * belongs to the first yarn (lowest index) containing it.
 */
static int braid_inside(double cx, double cy, double cz, double x0, double y0,
                        const double *d, const double *u, const double *v,
                        double A, double B, double Nx, double Ny) {
    double t = cz / d[2];
    double px = x0 + d[0] * t;
    double py = y0 + d[1] * t;
    double rx = cx - px;
    double ry = cy - py;
    rx = rx - Nx * floor(rx / Nx + 0.5);      /* minimum image in x */
    ry = ry - Ny * floor(ry / Ny + 0.5);      /* minimum image in y */
    double rd = rx * d[0] + ry * d[1];
    double wx = rx - rd * d[0];
    double wy = ry - rd * d[1];
    double wz = -(rd * d[2]);
    double a = (wx * u[0] + wy * u[1]) / A;
    double b = (wx * v[0] + wy * v[1] + wz * v[2]) / B;
    return a * a + b * b <= 1.0;
}

int orc_braid_phase(int64_t nx, int64_t ny, int64_t nz, double g_rad, double A,
                    double B, const double *anchors, int n_max, double phi,
                    uint8_t *phase, int *n_used, double *fraction) {
    static const int SX[4] = {1, -1, -1, 1};
    static const int SY[4] = {1, 1, -1, -1};
    double dir[4][3], uu[4][3], vv[4][3];
    double h = sin(g_rad) / sqrt(2.0);
    double cg = cos(g_rad);
    for (int k = 0; k < 4; ++k) {
        double *d = dir[k], *u = uu[k], *v = vv[k];
        d[0] = SX[k] * h;
        d[1] = SY[k] * h;
        d[2] = cg;
        double nrm = sqrt(d[0] * d[0] + d[1] * d[1]);
        u[0] = -d[1] / nrm;
        u[1] = d[0] / nrm;
        u[2] = 0.0;
        v[0] = -(d[2] * u[1]);
        v[1] = d[2] * u[0];
        v[2] = d[0] * u[1] - d[1] * u[0];
    }
    int64_t N = nx * ny * nz;
    int *first = (int *)malloc(sizeof(int) * N);
    int64_t *hist = (int64_t *)calloc((size_t)n_max + 1, sizeof(int64_t));
    if (!first || !hist) { free(first); free(hist); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t vidx = (z * ny + y) * nx + x;
                int found = n_max;
                for (int i = 0; i < n_max; ++i) {
                    int k = i % 4;
                    if (braid_inside((double)x + 0.5, (double)y + 0.5, (double)z + 0.5,
                                     anchors[2 * i], anchors[2 * i + 1], dir[k], uu[k],
                                     vv[k], A, B, (double)nx, (double)ny)) {
                        found = i;
                        break;
                    }
                }
                first[vidx] = found;
            }
    for (int64_t v = 0; v < N; ++v) hist[first[v]] += 1;
    int used = -1;
    int64_t cum = 0;
    for (int i = 0; i < n_max; ++i) {
        cum += hist[i];
        if ((double)cum >= phi * (double)N) { used = i + 1; break; }
    }
    if (used < 0) { free(first); free(hist); return -2; }
    int64_t yarn = 0;
    for (int64_t v = 0; v < N; ++v) {
        if (first[v] < used) {
            phase[v] = (uint8_t)(1 + first[v] % 4);
            ++yarn;
        } else {
            phase[v] = 0;
        }
    }
    *n_used = used;
    *fraction = (double)yarn / (double)N;
    free(first);
    free(hist);
    return 0;
}
