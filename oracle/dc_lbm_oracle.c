/*
 * Plain FP64 CPU oracle of the direct-coupling multi-level H-RR lattice
 * Boltzmann method of arXiv 2004.14887.  TEST INFRASTRUCTURE ONLY: the
 * checker of the CUDA library, never part of the product path.  It shares no
 * code with the CUDA library.  It is written for clarity, not speed: every
 * level is a full box with a node-class array, every history slot is a full
 * copy of the level, every node does its own loops.
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against
 * closed forms, invariants and brute force (see the tests' docstrings).
 */
#include "dc_lbm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define CS2 (1.0 / 3.0)
#define QMAX 19

/* ------------------------------------------------------------------------ */
/* Lattices (Sec. 2, Eqs. xi_i and w_i).                                     */
/* D2Q9 numbering follows the labels of Fig. 1: 0 rest, 1 E, 2 NE, 3 N, 4 NW,
 * 5 W, 6 SW, 7 S, 8 SE.  D3Q19 follows the paper's groups (0 rest, 1-6 axes,
 * 7-18 face diagonals), opposite velocities adjacent inside each group.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int D, Q;
    int c[QMAX][3];
    double w[QMAX];
} lat_t;

static int lat_make(int lattice, lat_t *L)
{
    memset(L, 0, sizeof(*L));
    if (lattice == 9) {
        static const int c9[9][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}, {-1, 1},
                                     {-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
        L->D = 2;
        L->Q = 9;
        for (int i = 0; i < 9; i++) {
            L->c[i][0] = c9[i][0];
            L->c[i][1] = c9[i][1];
            L->c[i][2] = 0;
            int n2 = c9[i][0] * c9[i][0] + c9[i][1] * c9[i][1];
            L->w[i] = n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
        return 9;
    }
    if (lattice == 19) {
        static const int c19[19][3] = {
            {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
            {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
            {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
            {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        L->D = 3;
        L->Q = 19;
        for (int i = 0; i < 19; i++) {
            int n2 = 0;
            for (int a = 0; a < 3; a++) {
                L->c[i][a] = c19[i][a];
                n2 += c19[i][a] * c19[i][a];
            }
            L->w[i] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
        return 19;
    }
    return -1;
}

int orc_lattice(int lattice, int *c, double *w)
{
    lat_t L;
    if (lat_make(lattice, &L) < 0) return -1;
    for (int i = 0; i < L.Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
    }
    return L.Q;
}

/* Hermite polynomials (Sec. 2): H2_ab = c_a c_b - cs2 d_ab,
 * H3_aab = (c_a^2 - cs2) c_b for a != b. */
static double H2(const lat_t *L, int i, int a, int b)
{
    return (double)(L->c[i][a] * L->c[i][b]) - (a == b ? CS2 : 0.0);
}
static double H3aab(const lat_t *L, int i, int a, int b)
{
    return ((double)(L->c[i][a] * L->c[i][a]) - CS2) * (double)L->c[i][b];
}

/* symmetric 6-vector <-> 3x3 */
static const int SYM_A[6] = {0, 1, 2, 0, 0, 1};
static const int SYM_B[6] = {0, 1, 2, 1, 2, 2};
static void sym_to_mat(const double *s, double m[3][3])
{
    for (int k = 0; k < 6; k++) {
        m[SYM_A[k]][SYM_B[k]] = s[k];
        m[SYM_B[k]][SYM_A[k]] = s[k];
    }
}

/* Eq. (fEq_herm): f0_i = w_i rho [1 + c.u/cs2 + H2:uu/(2cs2^2)
 *                         + sum_{a!=b} H3_aab u_a^2 u_b/(2cs2^3)] */
static void feq_lat(const lat_t *L, double rho, const double *u, double *feq)
{
    for (int i = 0; i < L->Q; i++) {
        double cu = 0.0, h2 = 0.0, h3 = 0.0;
        for (int a = 0; a < L->D; a++) cu += L->c[i][a] * u[a];
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++) h2 += H2(L, i, a, b) * u[a] * u[b];
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++)
                if (a != b) h3 += H3aab(L, i, a, b) * u[a] * u[a] * u[b];
        feq[i] = L->w[i] * rho *
                 (1.0 + cu / CS2 + h2 / (2.0 * CS2 * CS2) + h3 / (2.0 * CS2 * CS2 * CS2));
    }
}

void orc_feq(int lattice, double rho, const double *u, double *feq)
{
    lat_t L;
    lat_make(lattice, &L);
    feq_lat(&L, rho, u, feq);
}

/* App. A, Eq. (Psi).  D3Q19: Psi_aaa = rho u_a^3, Psi_aab = rho u_b u_g^2 / 2
 * (g the third axis), Psi_xyz = rho ux uy uz.  D2Q9 represents the aab third
 * moments exactly, so only Psi_aaa remains (reading R3, pinned by the
 * third-moment test). */
static double Psi_comp(const lat_t *L, double rho, const double *u, int a, int b, int g)
{
    if (a == b && b == g) return rho * u[a] * u[a] * u[a];
    if (L->D == 2) return 0.0;
    if (a == b || a == g || b == g) {
        int al = (a == b || a == g) ? a : b;       /* the repeated axis */
        int be = (a == b) ? g : (a == g ? b : a);  /* the single axis */
        int ga = 3 - al - be;                      /* the third axis */
        return 0.5 * rho * u[be] * u[ga] * u[ga];
    }
    return rho * u[0] * u[1] * u[2];
}

void orc_Psi_tensor(int lattice, double rho, const double *u, double *out)
{
    lat_t L;
    lat_make(lattice, &L);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int g = 0; g < 3; g++)
                out[a * 9 + b * 3 + g] =
                    (a < L.D && b < L.D && g < L.D) ? Psi_comp(&L, rho, u, a, b, g) : 0.0;
}

/* App. A, Eq. (psi): psi_i = s * w_i/(2cs2^2) * sum_ab H2_ab C_ab */
static void psi_lat(const lat_t *L, const double *C6, int psi_sign, double *psi)
{
    double C[3][3];
    sym_to_mat(C6, C);
    for (int i = 0; i < L->Q; i++) {
        double s = 0.0;
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++) s += H2(L, i, a, b) * C[a][b];
        psi[i] = (double)psi_sign * L->w[i] / (2.0 * CS2 * CS2) * s;
    }
}

void orc_psi(int lattice, const double *C, int psi_sign, double *psi)
{
    lat_t L;
    lat_make(lattice, &L);
    psi_lat(&L, C, psi_sign, psi);
}

/* Eq. (a12_HRR) with Eq. (a1Proj) and Eq. (a1FD): a1 = sigma a1^PR + (1-sigma) a1^FD,
 * a1^PR = sum_i H2_i (f_i - f0_i + psi_i/2), a1^FD = -2 tau rho cs2 S. */
static void a1_lat(const lat_t *L, const double *f, double rho, const double *u,
                   const double *S6, const double *C6, double tau, double sigma,
                   int psi_sign, double a1[3][3], double *feq_out, double *psi_out)
{
    double feq[QMAX], psi[QMAX], S[3][3];
    feq_lat(L, rho, u, feq);
    psi_lat(L, C6, psi_sign, psi);
    sym_to_mat(S6, S);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) a1[a][b] = 0.0;
    for (int a = 0; a < L->D; a++)
        for (int b = 0; b < L->D; b++) {
            double pr = 0.0;
            for (int i = 0; i < L->Q; i++) pr += H2(L, i, a, b) * (f[i] - feq[i] + 0.5 * psi[i]);
            double fd = -2.0 * tau * rho * CS2 * S[a][b];
            a1[a][b] = sigma * pr + (1.0 - sigma) * fd;
        }
    if (feq_out) memcpy(feq_out, feq, sizeof(double) * L->Q);
    if (psi_out) memcpy(psi_out, psi, sizeof(double) * L->Q);
}

void orc_a1(int lattice, const double *f, double rho, const double *u, const double *S,
            const double *C, double tau, double sigma, int psi_sign, double *a1o)
{
    lat_t L;
    lat_make(lattice, &L);
    double a1[3][3];
    a1_lat(&L, f, rho, u, S, C, tau, sigma, psi_sign, a1, NULL, NULL);
    for (int k = 0; k < 6; k++) a1o[k] = a1[SYM_A[k]][SYM_B[k]];
}

/* Eq. (LBMscheme_reg): f_post = f0 + (1 - 1/tau) f1_reg + psi/2 with
 * f1_reg = w_i [H2:a1/(2cs2^2) + sum_{a!=b} H3_aab a1_aab/(2cs2^3)]  (reading R2)
 * and a1_aab = 2 u_a a1_ab + u_b a1_aa  (Eq. a13RR). */
static void collide_lat(const lat_t *L, const double *f, double rho, const double *u,
                        const double *S6, const double *C6, double tau, double sigma,
                        int psi_sign, double *fpost)
{
    double a1[3][3], feq[QMAX], psi[QMAX], a3[3][3];
    a1_lat(L, f, rho, u, S6, C6, tau, sigma, psi_sign, a1, feq, psi);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            a3[a][b] = (a != b && a < L->D && b < L->D) ? 2.0 * u[a] * a1[a][b] + u[b] * a1[a][a] : 0.0;
    for (int i = 0; i < L->Q; i++) {
        double h2 = 0.0, h3 = 0.0;
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++) h2 += H2(L, i, a, b) * a1[a][b];
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++)
                if (a != b) h3 += H3aab(L, i, a, b) * a3[a][b];
        double f1 = L->w[i] * (h2 / (2.0 * CS2 * CS2) + h3 / (2.0 * CS2 * CS2 * CS2));
        fpost[i] = feq[i] + (1.0 - 1.0 / tau) * f1 + 0.5 * psi[i];
    }
}

void orc_collide(int lattice, const double *f, double rho, const double *u, const double *S,
                 const double *C, double tau, double sigma, int psi_sign, double *fpost)
{
    lat_t L;
    lat_make(lattice, &L);
    collide_lat(&L, f, rho, u, S, C, tau, sigma, psi_sign, fpost);
}

/* ------------------------------------------------------------------------ */
/* Newton-Raphson of Sec. 3.2, Eqs. (system_fi) and (updated_macro).         */
/* ------------------------------------------------------------------------ */
/* d f0_i / d X, X = (rho, u_0..u_{D-1}) */
static void dfeq_lat(const lat_t *L, double rho, const double *u, int i, double *d)
{
    double feq[QMAX];
    feq_lat(L, rho, u, feq);
    d[0] = feq[i] / rho;
    for (int g = 0; g < L->D; g++) {
        double t1 = L->c[i][g] / CS2;
        double t2 = 0.0;
        for (int b = 0; b < L->D; b++) t2 += H2(L, i, g, b) * u[b];
        t2 /= CS2 * CS2;
        double t3 = 0.0;
        for (int a = 0; a < L->D; a++)
            for (int b = 0; b < L->D; b++) {
                if (a == b) continue;
                double dd = (a == g ? 2.0 * u[a] * u[b] : 0.0) + (b == g ? u[a] * u[a] : 0.0);
                t3 += H3aab(L, i, a, b) * dd;
            }
        t3 /= 2.0 * CS2 * CS2 * CS2;
        d[1 + g] = L->w[i] * rho * (t1 + t2 + t3);
    }
}

static void newton_system_lat(const lat_t *L, const double *fhat, const double *Gamma,
                              const double *X, double *F, double *J)
{
    int n = L->D + 1;
    double feq[QMAX];
    feq_lat(L, X[0], X + 1, feq);
    for (int r = 0; r < n; r++) {
        F[r] = 0.0;
        for (int k = 0; k < n; k++) J[r * n + k] = 0.0;
    }
    for (int i = 0; i < L->Q; i++) {
        double phi[4], d[4];
        phi[0] = 1.0;
        for (int a = 0; a < L->D; a++) phi[1 + a] = L->c[i][a];
        dfeq_lat(L, X[0], X + 1, i, d);
        for (int r = 0; r < n; r++) {
            F[r] += Gamma[i] * phi[r] * (fhat[i] - feq[i]);
            for (int k = 0; k < n; k++) J[r * n + k] -= Gamma[i] * phi[r] * d[k];
        }
    }
}

void orc_newton_system(int lattice, const double *fhat, const double *Gamma, const double *X,
                       double *F, double *J)
{
    lat_t L;
    lat_make(lattice, &L);
    newton_system_lat(&L, fhat, Gamma, X, F, J);
}

/* Gaussian elimination with partial pivoting: solve A x = b (n <= 4) */
static int gauss_solve(int n, double *A, double *b, double *x)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int r = k + 1; r < n; r++)
            if (fabs(A[r * n + k]) > fabs(A[p * n + k])) p = r;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; c++) {
                double t = A[k * n + c];
                A[k * n + c] = A[p * n + c];
                A[p * n + c] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int r = k + 1; r < n; r++) {
            double m = A[r * n + k] / A[k * n + k];
            for (int c = k; c < n; c++) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int c = k + 1; c < n; c++) s -= A[k * n + c] * x[c];
        x[k] = s / A[k * n + k];
    }
    return 0;
}

/* Start from the plain moments of fhat (reading R6); stop once max|dX| < 1e-12. */
static int newton_lat(const lat_t *L, const double *fhat, const double *Gamma, double *X)
{
    int n = L->D + 1;
    double rho = 0.0, m[3] = {0, 0, 0};
    for (int i = 0; i < L->Q; i++) {
        rho += fhat[i];
        for (int a = 0; a < L->D; a++) m[a] += L->c[i][a] * fhat[i];
    }
    X[0] = rho;
    for (int a = 0; a < 3; a++) X[1 + a] = a < L->D ? m[a] / rho : 0.0;
    for (int it = 1; it <= 10; it++) {
        double F[4], J[16], dX[4], negF[4];
        newton_system_lat(L, fhat, Gamma, X, F, J);
        for (int r = 0; r < n; r++) negF[r] = -F[r];
        if (gauss_solve(n, J, negF, dX) != 0) return -1;
        double mx = 0.0;
        for (int r = 0; r < n; r++) {
            X[r] += dX[r];
            if (fabs(dX[r]) > mx) mx = fabs(dX[r]);
        }
        if (mx < 1e-12) return it;
    }
    return -1;
}

int orc_newton(int lattice, const double *fhat, const double *Gamma, double *X)
{
    lat_t L;
    lat_make(lattice, &L);
    return newton_lat(&L, fhat, Gamma, X);
}

/* Eq. (TempInt), points t-dt^c, t, t+dt^c (reading R5): quadratic Lagrange at +1/2 coarse step */
void orc_tempint_weights(double *w3)
{
    double s = 0.5;
    w3[0] = s * (s - 1.0) / 2.0;
    w3[1] = (1.0 - s) * (1.0 + s);
    w3[2] = s * (s + 1.0) / 2.0;
}

/* 4-point Lagrange at x = 1/2 (in coarse spacing) through nodes xs[4] */
static void lagrange4_at_half(const double *xs, double *w)
{
    for (int k = 0; k < 4; k++) {
        double num = 1.0, den = 1.0;
        for (int j = 0; j < 4; j++) {
            if (j == k) continue;
            num *= 0.5 - xs[j];
            den *= xs[k] - xs[j];
        }
        w[k] = num / den;
    }
}

void orc_lagrange4_weights(int one_sided, double *w4)
{
    static const double centred[4] = {-1.0, 0.0, 1.0, 2.0};
    static const double onesided[4] = {0.0, 1.0, 2.0, 3.0};
    lagrange4_at_half(one_sided ? onesided : centred, w4);
}

/* Set rule (reading R4, reproducing Fig. 1 and App. B): population i is
 * fine-known at a node x if the fine node x - c_i exists, coarse-known if the
 * coarse node x/2 - c_i exists.  occ_f / occ_c give the existence of the
 * 3x3(x3) neighbours around x (fine units) and around x/2 (coarse units),
 * index (ox+1) + 3 (oy+1) + 9 (oz+1). */
void orc_known_from_occupancy(int lattice, const unsigned char *occ_f, const unsigned char *occ_c,
                              unsigned int *kf, unsigned int *kc)
{
    lat_t L;
    lat_make(lattice, &L);
    unsigned int f = 0, c = 0;
    for (int i = 0; i < L.Q; i++) {
        int k = (1 - L.c[i][0]) + 3 * (1 - L.c[i][1]) + 9 * (1 - L.c[i][2]);
        if (occ_f[k]) f |= 1u << i;
        if (occ_c[k]) c |= 1u << i;
    }
    *kf = f;
    *kc = c;
}

/* ------------------------------------------------------------------------ */
/* Hierarchy (Sec. 3.5 steps, recursive 2:1 sub-cycling)                     */
/* ------------------------------------------------------------------------ */
/* Every per-node loop of a step writes only its own node (and, in the coarse
 * rebuild, the one coarse node co-located with it), so the loops may run their
 * nodes in any order.  Built with -fopenmp they are shared out over threads; the
 * arithmetic of each node is unchanged, so both builds give identical bits.
 * Without -fopenmp the pragma is ignored and the loops run in index order. */
#ifdef _OPENMP
#define ORC_NODE_LOOP _Pragma("omp parallel for schedule(static)")
#else
#define ORC_NODE_LOOP
#endif
typedef struct {
    long n[3], off[3], N;
    int periodic[3];
    double tau;
    unsigned char *cls;
    unsigned int *kf, *kc;      /* fine-known / coarse-known masks */
    double *f, *g;              /* [Q][N] post-collision state, post-stream work */
    double *rho, *u;            /* macros, u [3][N] */
    double *S, *C;              /* supplied gradients [6][N] */
    double *hg[3];              /* history: full copies of g, [Q][N] */
    double *hrho[3], *hu[3];    /* history: moments of g */
    long nsteps;
} level_t;

struct orc_h {
    orc_desc d;
    lat_t L;
    int nl;
    level_t lev[ORC_MAX_LEVELS];
    int max_newton;
    long updates;
    int failed;
    char err[256];
};

static long mod_l(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* local index of the level-l node at global level-l coordinates p, or -1 */
static long node_at(const orc_h *h, int l, const long *p)
{
    const level_t *v = &h->lev[l];
    long q[3];
    for (int d = 0; d < 3; d++) {
        q[d] = p[d] - v->off[d];
        if (v->periodic[d]) q[d] = mod_l(q[d], v->n[d]);
        else if (q[d] < 0 || q[d] >= v->n[d]) return -1;
    }
    long idx = q[0] + v->n[0] * (q[1] + v->n[1] * q[2]);
    if (v->cls[idx] == ORC_HOLE) return -1;
    return idx;
}

/* Refined region of level l (l >= 1), in cells of its parent level l-1 given by their
 * lower corner c (global level-(l-1) coordinates): the cells of the box [lo, hi)
 * (level-0 cell units, times 2^(l-1)), all of them on an axis the level spans, and of
 * those the ones the mask marks. */
static int cell_refined(const orc_h *h, int l, const long *c)
{
    const orc_desc *d = &h->d;
    const level_t *pv = &h->lev[l - 1];
    long q[3];
    long ext[3] = {1, 1, 1};
    for (int a = 0; a < 3; a++) {
        if (a >= h->L.D) {
            q[a] = 0;
            continue;
        }
        long ca = c[a];
        if (pv->periodic[a]) ca = pv->off[a] + mod_l(ca - pv->off[a], pv->n[a]);
        if (h->lev[l].periodic[a]) { /* spans the axis */
            q[a] = 0;
            continue;
        }
        long psc = 1L << (l - 1);
        long lo = d->box_lo[l][a] * psc, hi = d->box_hi[l][a] * psc;
        if (ca < lo || ca >= hi) return 0;
        q[a] = ca - lo;
        ext[a] = hi - lo;
    }
    if (!d->mask[l]) return 1;
    return d->mask[l][q[0] + ext[0] * (q[1] + ext[1] * q[2])] != 0;
}

/* number of the 2^D cells around level-(l-1) node p that level l refines, and 2^D */
static int refined_cells_around(const orc_h *h, int l, const long *p, int *total)
{
    int D = h->L.D, cnt = 0, tot = 0;
    for (int k = 0; k < (1 << D); k++) {
        long c[3] = {p[0], p[1], p[2]};
        for (int a = 0; a < D; a++) c[a] -= (k >> a) & 1;
        cnt += cell_refined(h, l, c);
        tot++;
    }
    *total = tot;
    return cnt;
}

/* level-l node p (l >= 1): number of parent cells it touches (the node lies on their
 * closure) that level l refines, and how many it touches */
static int refined_parent_cells_of_fine(const orc_h *h, int l, const long *p, int *total)
{
    int D = h->L.D, cnt = 0, tot = 0;
    long opts[3][2];
    int no[3];
    for (int a = 0; a < 3; a++) {
        if (a >= D) {
            opts[a][0] = 0;
            no[a] = 1;
        } else if (mod_l(p[a], 2) == 0) {
            opts[a][0] = p[a] / 2 - 1;
            opts[a][1] = p[a] / 2;
            no[a] = 2;
        } else {
            opts[a][0] = (p[a] - 1) / 2;
            no[a] = 1;
        }
    }
    for (int i0 = 0; i0 < no[0]; i0++)
        for (int i1 = 0; i1 < no[1]; i1++)
            for (int i2 = 0; i2 < no[2]; i2++) {
                long c[3] = {opts[0][i0], opts[1][i1], opts[2][i2]};
                cnt += cell_refined(h, l, c);
                tot++;
            }
    *total = tot;
    return cnt;
}

static void coords_of(const level_t *v, long idx, long *p)
{
    long q0 = idx % v->n[0];
    long r = idx / v->n[0];
    long q1 = r % v->n[1];
    long q2 = r / v->n[1];
    p[0] = q0 + v->off[0];
    p[1] = q1 + v->off[1];
    p[2] = q2 + v->off[2];
}

static void set_err(orc_h *h, const char *m)
{
    snprintf(h->err, sizeof(h->err), "%s", m);
    h->failed = 1;
}

const char *orc_error(orc_h *h) { return h->err; }

static void *xcalloc(size_t n, size_t s)
{
    void *p = calloc(n, s);
    if (!p) {
        fprintf(stderr, "oracle: out of memory\n");
        abort();
    }
    return p;
}

orc_h *orc_create(const orc_desc *d, char *err, int errlen)
{
    orc_h *h = (orc_h *)xcalloc(1, sizeof(orc_h));
    h->d = *d;
#define FAIL(msg)                                       \
    do {                                                \
        if (err) snprintf(err, errlen, "%s", msg);      \
        orc_destroy(h);                                 \
        return NULL;                                    \
    } while (0)
    if (lat_make(d->lattice, &h->L) < 0) FAIL("lattice must be 9 or 19");
    if (d->n_levels < 1 || d->n_levels > ORC_MAX_LEVELS) FAIL("bad n_levels");
    h->nl = d->n_levels;
    int D = h->L.D;
    for (int a = 0; a < 3; a++) {
        if (d->coarse_n[a] < 1) FAIL("coarse_n must be positive");
        if (a >= D && d->coarse_n[a] != 1) FAIL("coarse_n[2] must be 1 in 2-D");
    }
    /* level geometry */
    for (int l = 0; l < h->nl; l++) {
        level_t *v = &h->lev[l];
        long sc = 1L << l;
        for (int a = 0; a < 3; a++) {
            if (a >= D) {
                v->n[a] = 1;
                v->off[a] = 0;
                v->periodic[a] = 1;
                continue;
            }
            if (l == 0) {
                v->n[a] = d->coarse_n[a];
                v->off[a] = 0;
                v->periodic[a] = 1;
                continue;
            }
            long lo = d->box_lo[l][a], hi = d->box_hi[l][a];
            if (lo == 0 && hi == d->coarse_n[a]) {
                if (!h->lev[l - 1].periodic[a]) FAIL("a spanning level needs a spanning parent");
                v->n[a] = d->coarse_n[a] * sc;
                v->off[a] = 0;
                v->periodic[a] = 1;
            } else {
                /* parent extent in level-0 cells */
                long plo = l == 1 ? 0 : d->box_lo[l - 1][a];
                long phi = l == 1 ? d->coarse_n[a] : d->box_hi[l - 1][a];
                int pper = h->lev[l - 1].periodic[a];
                long psc = 1L << (l - 1);
                /* margin of 4 parent cells between nested interfaces */
                if (!(lo < hi)) FAIL("empty patch");
                if ((hi - lo) * psc < 4) FAIL("patch faces need at least 4 parent cells");
                if (pper) {
                    if (lo * psc < 4 || (d->coarse_n[a] - hi) * psc < 4)
                        FAIL("patch too close to the periodic seam");
                } else if ((lo - plo) * psc < 4 || (phi - hi) * psc < 4) {
                    FAIL("patch needs 4 parent cells of margin inside its parent");
                }
                v->n[a] = (hi - lo) * sc + 1;
                v->off[a] = lo * sc;
                v->periodic[a] = 0;
            }
        }
        v->N = v->n[0] * v->n[1] * v->n[2];
        v->tau = l == 0 ? 0.5 + d->nu0 / CS2 : 2.0 * h->lev[l - 1].tau - 0.5; /* Eqs. linkTauNu, rescTau */
    }
    /* staircase regions (masks): 2-D, finest level, no spanned axis, and no two refined
     * cells that meet at a corner only (the interface stays a simple curve) */
    for (int l = 1; l < h->nl; l++) {
        if (!d->mask[l]) continue;
        if (D != 2) FAIL("refinement masks are 2-D only");
        if (l + 1 < h->nl) FAIL("a refinement mask is allowed on the finest level only");
        for (int a = 0; a < D; a++)
            if (h->lev[l].periodic[a]) FAIL("a masked level spans no axis");
        long psc = 1L << (l - 1);
        for (long cy = d->box_lo[l][1] * psc; cy <= d->box_hi[l][1] * psc; cy++)
            for (long cx = d->box_lo[l][0] * psc; cx <= d->box_hi[l][0] * psc; cx++) {
                long c00[3] = {cx - 1, cy - 1, 0}, c10[3] = {cx, cy - 1, 0}, c01[3] = {cx - 1, cy, 0},
                     c11[3] = {cx, cy, 0};
                int a00 = cell_refined(h, l, c00), a10 = cell_refined(h, l, c10), a01 = cell_refined(h, l, c01),
                    a11 = cell_refined(h, l, c11);
                if (a00 == a11 && a10 == a01 && a00 != a10) FAIL("two refined cells meet at a corner only");
            }
    }
    /* node classes */
    for (int l = 0; l < h->nl; l++) {
        level_t *v = &h->lev[l];
        v->cls = (unsigned char *)xcalloc(v->N, 1);
        for (long idx = 0; idx < v->N; idx++) {
            long p[3];
            coords_of(v, idx, p);
            /* classes from the refined cells around the node (Sec. 3.2; App. B for
             * staircase corners): a node whose cells the next level refines is a hole,
             * one with some refined cells is co-located with a TF node of the child; a
             * node of a refined level touching a cell its level does not refine lies on
             * the interface (TF if co-located with a parent node, else hanging), one
             * touching no refined cell is not a node of the level */
            unsigned char c = ORC_BULK;
            if (l + 1 < h->nl) {
                int tot, cnt = refined_cells_around(h, l + 1, p, &tot);
                if (cnt == tot) c = ORC_HOLE;
                else if (cnt > 0) c = ORC_TFC;
            }
            if (l > 0) {
                int tot, cnt = refined_parent_cells_of_fine(h, l, p, &tot);
                int all_even = 1;
                for (int a = 0; a < D; a++)
                    if (mod_l(p[a], 2) != 0) all_even = 0;
                if (cnt == 0) c = ORC_HOLE;
                else if (cnt < tot && c == ORC_BULK) c = all_even ? ORC_TFP : ORC_IE;
                else if (cnt < tot) FAIL("a level's interface meets its child's region");
            }
            v->cls[idx] = c;
        }
    }
    /* known masks (reading R4): fine-known if x - c_i is a node of the level,
     * coarse-known if x/2 - c_i is a node of the parent level */
    int Q = h->L.Q;
    for (int l = 0; l < h->nl; l++) {
        level_t *v = &h->lev[l];
        v->kf = (unsigned int *)xcalloc(v->N, sizeof(unsigned int));
        v->kc = (unsigned int *)xcalloc(v->N, sizeof(unsigned int));
        for (long idx = 0; idx < v->N; idx++) {
            if (v->cls[idx] == ORC_HOLE) continue;
            long p[3];
            coords_of(v, idx, p);
            unsigned char occ_f[27], occ_c[27];
            for (int k = 0; k < 27; k++) {
                long o[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
                long s[3] = {p[0] + o[0], p[1] + o[1], p[2] + o[2]};
                occ_f[k] = node_at(h, l, s) >= 0;
                occ_c[k] = 0;
                if (v->cls[idx] == ORC_TFP) {
                    long sc[3] = {p[0] / 2 + o[0], p[1] / 2 + o[1], p[2] / 2 + o[2]};
                    occ_c[k] = node_at(h, l - 1, sc) >= 0;
                }
            }
            orc_known_from_occupancy(d->lattice, occ_f, occ_c, &v->kf[idx], &v->kc[idx]);
            unsigned int kf = v->kf[idx], kc = v->kc[idx];
            unsigned int all = (1u << Q) - 1u;
            if ((v->cls[idx] == ORC_BULK) && kf != all) FAIL("bulk node with a missing population");
            if (v->cls[idx] == ORC_TFP && ((kf | kc) != all)) FAIL("TF node with a population unknown on both levels");
        }
    }
    /* arrays */
    for (int l = 0; l < h->nl; l++) {
        level_t *v = &h->lev[l];
        v->f = (double *)xcalloc((size_t)Q * v->N, sizeof(double));
        v->g = (double *)xcalloc((size_t)Q * v->N, sizeof(double));
        v->rho = (double *)xcalloc(v->N, sizeof(double));
        v->u = (double *)xcalloc(3 * v->N, sizeof(double));
        v->S = (double *)xcalloc(6 * v->N, sizeof(double));
        v->C = (double *)xcalloc(6 * v->N, sizeof(double));
        if (l + 1 < h->nl) {
            for (int k = 0; k < 3; k++) {
                v->hg[k] = (double *)xcalloc((size_t)Q * v->N, sizeof(double));
                v->hrho[k] = (double *)xcalloc(v->N, sizeof(double));
                v->hu[k] = (double *)xcalloc(3 * v->N, sizeof(double));
            }
        }
    }
#undef FAIL
    return h;
}

void orc_destroy(orc_h *h)
{
    if (!h) return;
    for (int l = 0; l < ORC_MAX_LEVELS; l++) {
        level_t *v = &h->lev[l];
        free(v->cls);
        free(v->kf);
        free(v->kc);
        free(v->f);
        free(v->g);
        free(v->rho);
        free(v->u);
        free(v->S);
        free(v->C);
        for (int k = 0; k < 3; k++) {
            free(v->hg[k]);
            free(v->hrho[k]);
            free(v->hu[k]);
        }
    }
    free(h);
}

int orc_level_info(orc_h *h, int l, long *n, long *off, int *periodic, double *tau)
{
    if (l < 0 || l >= h->nl) return -1;
    for (int a = 0; a < 3; a++) {
        n[a] = h->lev[l].n[a];
        off[a] = h->lev[l].off[a];
        periodic[a] = h->lev[l].periodic[a];
    }
    *tau = h->lev[l].tau;
    return 0;
}

int orc_node_class(orc_h *h, int l, unsigned char *cls)
{
    if (l < 0 || l >= h->nl) return -1;
    memcpy(cls, h->lev[l].cls, h->lev[l].N);
    return 0;
}

int orc_known_masks(orc_h *h, int l, unsigned int *kf, unsigned int *kc)
{
    if (l < 0 || l >= h->nl) return -1;
    memcpy(kf, h->lev[l].kf, h->lev[l].N * sizeof(unsigned int));
    memcpy(kc, h->lev[l].kc, h->lev[l].N * sizeof(unsigned int));
    return 0;
}

static void moments(const orc_h *h, const double *f, long N, long idx, double *rho, double *u)
{
    double r = 0.0, m[3] = {0, 0, 0};
    for (int i = 0; i < h->L.Q; i++) {
        double fi = f[(size_t)i * N + idx];
        r += fi;
        for (int a = 0; a < h->L.D; a++) m[a] += h->L.c[i][a] * fi;
    }
    *rho = r;
    for (int a = 0; a < 3; a++) u[a] = m[a] / r;
}

/* initial state: f = f0(rho, u) at every node (paper Sec. 4.1); history slot 0 holds it */
int orc_init(orc_h *h, int l, const double *rho, const double *u)
{
    if (l < 0 || l >= h->nl) return -1;
    level_t *v = &h->lev[l];
    int Q = h->L.Q;
    for (long idx = 0; idx < v->N; idx++) {
        double feq[QMAX], uu[3] = {0, 0, 0};
        if (v->cls[idx] == ORC_HOLE) {
            for (int i = 0; i < Q; i++) v->f[(size_t)i * v->N + idx] = 0.0;
            continue;
        }
        for (int a = 0; a < h->L.D; a++) uu[a] = u[(size_t)a * v->N + idx];
        feq_lat(&h->L, rho[idx], uu, feq);
        for (int i = 0; i < Q; i++) v->f[(size_t)i * v->N + idx] = feq[i];
    }
    v->nsteps = 0;
    if (l + 1 < h->nl) {
        memcpy(v->hg[0], v->f, sizeof(double) * Q * v->N);
        for (long idx = 0; idx < v->N; idx++) {
            if (v->cls[idx] == ORC_HOLE) continue;
            double r, uu[3];
            moments(h, v->f, v->N, idx, &r, uu);
            v->hrho[0][idx] = r;
            for (int a = 0; a < 3; a++) v->hu[0][(size_t)a * v->N + idx] = uu[a];
        }
    }
    h->failed = 0;
    return 0;
}

/* steps 2a-2c / 3a-3b: pull every population whose source is a node of this level */
static void stream_level(orc_h *h, int l)
{
    level_t *v = &h->lev[l];
    int Q = h->L.Q;
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] == ORC_HOLE) continue;
        long p[3];
        coords_of(v, idx, p);
        for (int i = 0; i < Q; i++) {
            long s[3] = {p[0] - h->L.c[i][0], p[1] - h->L.c[i][1], p[2] - h->L.c[i][2]};
            long src = node_at(h, l, s);
            v->g[(size_t)i * v->N + idx] = src >= 0 ? v->f[(size_t)i * v->N + src] : 0.0;
        }
    }
}

/* post-stream copies of a coarse level, kept for the child's Eq. (TempInt) */
static void push_history(orc_h *h, int l)
{
    level_t *v = &h->lev[l];
    int Q = h->L.Q;
    int slot = (int)((v->nsteps + 1) % 3);
    memcpy(v->hg[slot], v->g, sizeof(double) * Q * v->N);
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] != ORC_BULK) continue;
        double r, uu[3];
        moments(h, v->g, v->N, idx, &r, uu);
        v->hrho[slot][idx] = r;
        for (int a = 0; a < 3; a++) v->hu[slot][(size_t)a * v->N + idx] = uu[a];
    }
}

/* weights over the parent's history slots at this child sub-step */
static void parent_time_weights(const orc_h *h, int l, int phase, int *slot, double *w)
{
    const level_t *pv = &h->lev[l - 1];
    long n = pv->nsteps;
    slot[0] = (int)((n + 2) % 3); /* t - dt^c */
    slot[1] = (int)(n % 3);       /* t */
    slot[2] = (int)((n + 1) % 3); /* t + dt^c */
    if (phase == 1) {
        w[0] = 0.0;
        w[1] = 0.0;
        w[2] = 1.0;
    } else if (n == 0) {
        w[0] = 0.0;
        w[1] = 0.5;
        w[2] = 0.5;
    } else {
        orc_tempint_weights(w);
    }
}

/* steps 2d-2e / 3c and 3f: Newton at TF nodes, fine rebuild (Eq. rescff, applied
 * to every gamma=c population, reading R7) and, on sync sub-steps, coarse
 * rebuild of every population (Eq. rescfc). */
static void reconstruct_tf(orc_h *h, int l, int phase)
{
    level_t *v = &h->lev[l];
    level_t *pv = &h->lev[l - 1];
    int Q = h->L.Q, D = h->L.D;
    double R = 0.5 * v->tau / pv->tau; /* Eq. (fneqResc) */
    int slot[3];
    double wt[3];
    parent_time_weights(h, l, phase, slot, wt);
    int worst = 0; /* largest Newton count, -1 once a node did not converge */
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] != ORC_TFP) continue;
        long p[3], pc[3];
        coords_of(v, idx, p);
        for (int a = 0; a < 3; a++) pc[a] = p[a] / 2;
        long cidx = node_at(h, l - 1, pc);
        double fhat[QMAX], Gam[QMAX], X[4], feq[QMAX];
        int gam_c[QMAX];
        for (int i = 0; i < Q; i++) {
            int fk = (v->kf[idx] >> i) & 1u, ck = (v->kc[idx] >> i) & 1u;
            /* Table 1: DC2 takes coarse data on P and M^f, DC1 only on M^f */
            gam_c[i] = h->d.dc_variant == 1 ? !fk : ck;
            if (gam_c[i]) {
                double s = 0.0;
                for (int k = 0; k < 3; k++)
                    if (wt[k] != 0.0) s += wt[k] * pv->hg[slot[k]][(size_t)i * pv->N + cidx];
                fhat[i] = s;
                Gam[i] = R;
            } else {
                fhat[i] = v->g[(size_t)i * v->N + idx];
                Gam[i] = 1.0;
            }
        }
        int it = newton_lat(&h->L, fhat, Gam, X);
        if (it < 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            worst = -1;
            continue;
        }
#ifdef _OPENMP
#pragma omp critical(orc_newton_count)
#endif
        {
            if (worst >= 0 && it > worst) worst = it;
        }
        feq_lat(&h->L, X[0], X + 1, feq);
        for (int i = 0; i < Q; i++)
            if (gam_c[i]) v->g[(size_t)i * v->N + idx] = feq[i] + R * (fhat[i] - feq[i]);
        v->rho[idx] = X[0];
        for (int a = 0; a < 3; a++) v->u[(size_t)a * v->N + idx] = a < D ? X[1 + a] : 0.0;
        if (phase == 1) {
            for (int i = 0; i < Q; i++)
                pv->g[(size_t)i * pv->N + cidx] = feq[i] + (v->g[(size_t)i * v->N + idx] - feq[i]) / R;
            pv->rho[cidx] = X[0];
            for (int a = 0; a < 3; a++) pv->u[(size_t)a * pv->N + cidx] = a < D ? X[1 + a] : 0.0;
        }
    }
    if (worst < 0) {
        set_err(h, "Newton did not converge in 10 iterations");
        return;
    }
    if (worst > h->max_newton) h->max_newton = worst;
}

static void bulk_macros(orc_h *h, int l)
{
    level_t *v = &h->lev[l];
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] != ORC_BULK) continue;
        double r, uu[3];
        moments(h, v->g, v->N, idx, &r, uu);
        v->rho[idx] = r;
        for (int a = 0; a < 3; a++) v->u[(size_t)a * v->N + idx] = uu[a];
    }
}

/* centred differences (Eqs. a1FD_scheme, PSI_FD) from the macros of the two
 * neighbours along every axis; spacing is the stencil half-width in node units */
static void gradients_from(const orc_h *h, double mr[3][2], double mu[3][2][3], double spacing,
                           double *S6, double *C6)
{
    int D = h->L.D;
    double du[3][3] = {{0}}; /* du[b][a] = d_b u_a */
    double dPsi[3][27];      /* dPsi[g] = d_g Psi */
    memset(dPsi, 0, sizeof(dPsi));
    for (int b = 0; b < D; b++) {
        double Pp[27], Pm[27];
        orc_Psi_tensor(h->d.lattice, mr[b][0], mu[b][0], Pp);
        orc_Psi_tensor(h->d.lattice, mr[b][1], mu[b][1], Pm);
        for (int a = 0; a < D; a++) du[b][a] = (mu[b][0][a] - mu[b][1][a]) / (2.0 * spacing);
        for (int k = 0; k < 27; k++) dPsi[b][k] = (Pp[k] - Pm[k]) / (2.0 * spacing);
    }
    for (int k = 0; k < 6; k++) {
        int a = SYM_A[k], b = SYM_B[k];
        if (a >= D || b >= D) {
            S6[k] = 0.0;
            C6[k] = 0.0;
            continue;
        }
        S6[k] = 0.5 * (du[b][a] + du[a][b]);
        double c = 0.0;
        for (int g = 0; g < D; g++) c += dPsi[g][a * 9 + b * 3 + g];
        C6[k] = c;
    }
}

/* steps 2f / 3d (Sec. 3.3): coarse-stencil gradients at TF nodes, rescaled by 1/2
 * for the fine level (Eqs. PijResc, PSIResc); on sync sub-steps the unscaled
 * values go to the co-located coarse node (reading R8). */
static void tf_gradients(orc_h *h, int l, int phase)
{
    level_t *v = &h->lev[l];
    level_t *pv = &h->lev[l - 1];
    int D = h->L.D;
    int slot[3];
    double wt[3];
    parent_time_weights(h, l, phase, slot, wt);
    int bad = 0;
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] != ORC_TFP) continue;
        long p[3];
        coords_of(v, idx, p);
        double mr[3][2], mu[3][2][3];
        int ok = 1;
        for (int b = 0; b < D; b++)
            for (int s = 0; s < 2; s++) {
                long y[3] = {p[0], p[1], p[2]};
                y[b] += s == 0 ? 2 : -2;
                long j = node_at(h, l, y);
                if (j >= 0) {
                    mr[b][s] = v->rho[j];
                    for (int a = 0; a < 3; a++) mu[b][s][a] = v->u[(size_t)a * v->N + j];
                } else {
                    long yc[3] = {y[0] / 2, y[1] / 2, y[2] / 2};
                    long jc = node_at(h, l - 1, yc);
                    if (jc < 0 || pv->cls[jc] != ORC_BULK) {
                        ok = 0;
                        continue;
                    }
                    double r = 0.0, uu[3] = {0, 0, 0};
                    for (int k = 0; k < 3; k++) {
                        if (wt[k] == 0.0) continue;
                        r += wt[k] * pv->hrho[slot[k]][jc];
                        for (int a = 0; a < 3; a++) uu[a] += wt[k] * pv->hu[slot[k]][(size_t)a * pv->N + jc];
                    }
                    mr[b][s] = r;
                    for (int a = 0; a < 3; a++) mu[b][s][a] = uu[a];
                }
            }
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            bad = 1;
            continue;
        }
        double Sc[6], Cc[6];
        gradients_from(h, mr, mu, 1.0, Sc, Cc); /* coarse units: neighbours one coarse cell away */
        for (int k = 0; k < 6; k++) {
            v->S[(size_t)k * v->N + idx] = 0.5 * Sc[k];
            v->C[(size_t)k * v->N + idx] = 0.5 * Cc[k];
        }
        if (phase == 1) {
            long pc[3] = {p[0] / 2, p[1] / 2, p[2] / 2};
            long cidx = node_at(h, l - 1, pc);
            for (int k = 0; k < 6; k++) {
                pv->S[(size_t)k * pv->N + cidx] = Sc[k];
                pv->C[(size_t)k * pv->N + cidx] = Cc[k];
            }
        }
    }
    if (bad) set_err(h, "TF gradient stencil leaves the parent's bulk");
}

/* Stencil of the hanging node idx of level l (Sec. 3.2, 4-point 1-D Lagrange along the
 * interface; reading R10 for boxes and 3-D faces, R15 for 2-D staircases): the level-l
 * coordinates of its nodes in pts and their weights in w; returns their number (the
 * tensor product over the node's odd axes), -1 if a node of it is not a TF node. */
static int ie_stencil(const orc_h *h, int l, long idx, long (*pts)[3], double *w)
{
    const level_t *v = &h->lev[l];
    int D = h->L.D;
    double wc[4], wo[4];
    orc_lagrange4_weights(0, wc);
    orc_lagrange4_weights(1, wo);
    long p[3], q[3];
    coords_of(v, idx, p);
    for (int a = 0; a < 3; a++) q[a] = p[a] - v->off[a];
    long pos[3][4];
    double wts[3][4];
    int cnt[3];
    for (int a = 0; a < 3; a++) {
        if (a >= D || mod_l(p[a], 2) == 0) {
            cnt[a] = 1;
            pos[a][0] = p[a];
            wts[a][0] = 1.0;
            continue;
        }
        cnt[a] = 4;
        long s = q[a];
        if (D == 2) {
            /* 2-D (boxes and staircases, reading R15): along the hanging node's odd
             * axis, the first of the centred and the two one-sided 4-point sets whose
             * nodes are all TF nodes of the level; where the interface turns within
             * a coarse cell of the node and none is complete, the linear 2-point
             * set of the two TF nodes that end the node's edge */
            static const long cand[3][4] = {{-3, -1, 1, 3}, {-1, 1, 3, 5}, {1, -1, -3, -5}};
            int pick = -1;
            for (int k = 0; k < 3 && pick < 0; k++) {
                int all_tf = 1;
                for (int m = 0; m < 4; m++) {
                    long y[3] = {p[0], p[1], p[2]};
                    y[a] += cand[k][m];
                    long j = node_at(h, l, y);
                    if (j < 0 || v->cls[j] != ORC_TFP) all_tf = 0;
                }
                if (all_tf) pick = k;
            }
            if (pick < 0) {
                cnt[a] = 2;
                pos[a][0] = p[a] - 1;
                pos[a][1] = p[a] + 1;
                wts[a][0] = wts[a][1] = 0.5;
            } else {
                for (int m = 0; m < 4; m++) {
                    pos[a][m] = p[a] + cand[pick][m];
                    wts[a][m] = pick == 0 ? wc[m] : wo[m];
                }
            }
            continue;
        }
        if (v->periodic[a] || (s - 3 >= 0 && s + 3 <= v->n[a] - 1)) {
            long o[4] = {-3, -1, 1, 3};
            for (int k = 0; k < 4; k++) {
                pos[a][k] = p[a] + o[k];
                wts[a][k] = wc[k];
            }
        } else if (s - 3 < 0) {
            long o[4] = {-1, 1, 3, 5};
            for (int k = 0; k < 4; k++) {
                pos[a][k] = p[a] + o[k];
                wts[a][k] = wo[k];
            }
        } else {
            long o[4] = {1, -1, -3, -5};
            for (int k = 0; k < 4; k++) {
                pos[a][k] = p[a] + o[k];
                wts[a][k] = wo[k];
            }
        }
    }
    int m = 0;
    for (int i0 = 0; i0 < cnt[0]; i0++)
        for (int i1 = 0; i1 < cnt[1]; i1++)
            for (int i2 = 0; i2 < cnt[2]; i2++) {
                long y[3] = {pos[0][i0], pos[1][i1], pos[2][i2]};
                long j = node_at(h, l, y);
                if (j < 0 || v->cls[j] != ORC_TFP) return -1;
                for (int a = 0; a < 3; a++) pts[m][a] = y[a];
                w[m] = wts[0][i0] * wts[1][i1] * wts[2][i2];
                m++;
            }
    return m;
}

int orc_ie_stencil(orc_h *h, int l, long idx, long *pts, double *w)
{
    if (l < 1 || l >= h->nl || idx < 0 || idx >= h->lev[l].N || h->lev[l].cls[idx] != ORC_IE) return -1;
    return ie_stencil(h, l, idx, (long (*)[3])pts, w);
}

/* steps 2g / 3e: the missing populations (M^f), S and psi (through C) of hanging nodes
 * from their stencil of TF nodes (ie_stencil). */
static void ie_complete(orc_h *h, int l)
{
    level_t *v = &h->lev[l];
    int Q = h->L.Q;
    int bad = 0;
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] != ORC_IE) continue;
        long pts[16][3];
        double wts[16];
        int n = ie_stencil(h, l, idx, pts, wts);
        if (n < 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            bad = 1;
            continue;
        }
        double acc_f[QMAX], acc_S[6], acc_C[6];
        memset(acc_f, 0, sizeof(acc_f));
        memset(acc_S, 0, sizeof(acc_S));
        memset(acc_C, 0, sizeof(acc_C));
        for (int m = 0; m < n; m++) {
            long j = node_at(h, l, pts[m]);
            double wgt = wts[m];
            for (int i = 0; i < Q; i++) acc_f[i] += wgt * v->g[(size_t)i * v->N + j];
            for (int k = 0; k < 6; k++) {
                acc_S[k] += wgt * v->S[(size_t)k * v->N + j];
                acc_C[k] += wgt * v->C[(size_t)k * v->N + j];
            }
        }
        for (int i = 0; i < Q; i++)
            if (!((v->kf[idx] >> i) & 1u)) v->g[(size_t)i * v->N + idx] = acc_f[i];
        for (int k = 0; k < 6; k++) {
            v->S[(size_t)k * v->N + idx] = acc_S[k];
            v->C[(size_t)k * v->N + idx] = acc_C[k];
        }
        double r, uu[3];
        moments(h, v->g, v->N, idx, &r, uu);
        v->rho[idx] = r;
        for (int a = 0; a < 3; a++) v->u[(size_t)a * v->N + idx] = uu[a];
    }
    if (bad) set_err(h, "hanging-node stencil does not land on TF nodes");
}

/* steps 2h / 3g: collision of every node; bulk nodes use the centred
 * differences of Eqs. (a1FD_scheme) and (PSI_FD), interface nodes the supplied S, C */
static void collide_level(orc_h *h, int l)
{
    level_t *v = &h->lev[l];
    int Q = h->L.Q, D = h->L.D;
    long active = 0;
    for (long idx = 0; idx < v->N; idx++) active += v->cls[idx] != ORC_HOLE;
    ORC_NODE_LOOP
    for (long idx = 0; idx < v->N; idx++) {
        unsigned char c = v->cls[idx];
        if (c == ORC_HOLE) continue;
        double S6[6], C6[6];
        if (c == ORC_BULK) {
            long p[3];
            coords_of(v, idx, p);
            double mr[3][2], mu[3][2][3];
            for (int b = 0; b < D; b++)
                for (int s = 0; s < 2; s++) {
                    long y[3] = {p[0], p[1], p[2]};
                    y[b] += s == 0 ? 1 : -1;
                    long j = node_at(h, l, y);
                    mr[b][s] = v->rho[j];
                    for (int a = 0; a < 3; a++) mu[b][s][a] = v->u[(size_t)a * v->N + j];
                }
            gradients_from(h, mr, mu, 1.0, S6, C6);
        } else {
            for (int k = 0; k < 6; k++) {
                S6[k] = v->S[(size_t)k * v->N + idx];
                C6[k] = v->C[(size_t)k * v->N + idx];
            }
        }
        double fin[QMAX], fout[QMAX], uu[3];
        for (int i = 0; i < Q; i++) fin[i] = v->g[(size_t)i * v->N + idx];
        for (int a = 0; a < 3; a++) uu[a] = v->u[(size_t)a * v->N + idx];
        collide_lat(&h->L, fin, v->rho[idx], uu, S6, C6, v->tau, h->d.sigma, h->d.psi_sign, fout);
        for (int i = 0; i < Q; i++) v->f[(size_t)i * v->N + idx] = fout[i];
    }
    h->updates += active;
}

/* Sec. 3.5: one step of level l (async phase 0 / sync phase 1 for l > 0),
 * with two sub-steps of the next finer level inside it. */
static void advance_level(orc_h *h, int l, int phase)
{
    if (h->failed) return;
    stream_level(h, l);
    if (l + 1 < h->nl) push_history(h, l);
    if (l > 0) reconstruct_tf(h, l, phase);
    if (h->failed) return;
    if (l + 1 < h->nl) {
        advance_level(h, l + 1, 0);
        advance_level(h, l + 1, 1);
        if (h->failed) return;
    }
    bulk_macros(h, l);
    if (l > 0) {
        tf_gradients(h, l, phase);
        ie_complete(h, l);
        if (h->failed) return;
    }
    collide_level(h, l);
    h->lev[l].nsteps++;
}

int orc_advance(orc_h *h, long n)
{
    for (long s = 0; s < n; s++) {
        advance_level(h, 0, 1);
        if (h->failed) return -1;
    }
    return 0;
}

int orc_get_macros(orc_h *h, int l, double *rho, double *u)
{
    if (l < 0 || l >= h->nl) return -1;
    level_t *v = &h->lev[l];
    for (long idx = 0; idx < v->N; idx++) {
        if (v->cls[idx] == ORC_HOLE) {
            rho[idx] = 0.0;
            for (int a = 0; a < h->L.D; a++) u[(size_t)a * v->N + idx] = 0.0;
            continue;
        }
        double r, uu[3];
        moments(h, v->f, v->N, idx, &r, uu);
        rho[idx] = r;
        for (int a = 0; a < h->L.D; a++) u[(size_t)a * v->N + idx] = uu[a];
    }
    return 0;
}

int orc_get_pops(orc_h *h, int l, double *f)
{
    if (l < 0 || l >= h->nl) return -1;
    memcpy(f, h->lev[l].f, sizeof(double) * h->L.Q * h->lev[l].N);
    return 0;
}

int orc_get_gradients(orc_h *h, int l, double *S, double *C)
{
    if (l < 0 || l >= h->nl) return -1;
    memcpy(S, h->lev[l].S, sizeof(double) * 6 * h->lev[l].N);
    memcpy(C, h->lev[l].C, sizeof(double) * 6 * h->lev[l].N);
    return 0;
}

int orc_set_pops(orc_h *h, int l, const double *f)
{
    if (l < 0 || l >= h->nl) return -1;
    memcpy(h->lev[l].f, f, sizeof(double) * h->L.Q * h->lev[l].N);
    return 0;
}

int orc_max_newton_iters(orc_h *h) { return h->max_newton; }

/* Threads of the node loops: sets the count when n > 0 and returns the count in use
 * (1 in the build without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
long orc_node_updates(orc_h *h) { return h->updates; }
