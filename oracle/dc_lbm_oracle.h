/*
 * Plain FP64 CPU oracle of the direct-coupling (DC) multi-level H-RR lattice
 * Boltzmann method (Astoul, Wissocq, Boussuge, Sengissen, Sagaut,
 * "Lattice Boltzmann method for computational aeroacoustics on non-uniform
 * meshes: a direct grid coupling approach", arXiv 2004.14887).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the checker of the CUDA path: it
 * is slow on purpose (nested loops, full-level copies, no blocking or fusion)
 * and shares no code, header, table or constant with the GPU library.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the product path never does.
 *
 * Every function follows the paper's equations in the paper's order:
 *   equilibrium           Eq. (fEq_herm) with a0^(2)=rho uu, a0^(3)=rho uuu
 *   off-equilibrium       Eqs. (fNEq_herm), (a12_HRR), (a1Proj), (a1FD_scheme), (a13RR)
 *   collision             Eq. (LBMscheme_reg)
 *   cubic-Mach correction App. A, Eqs. (psi), (Psi), (PSI_FD)
 *   level rescaling       Sec. 3.1, Eqs. (rescNu), (rescTau), (fneqResc), (PijResc), (PSIResc)
 *   DC interface          Sec. 3.2-3.5, Eqs. (cond_fneq) ... (rescfc), Table 1, App. B
 * Where the paper is ambiguous, the reading taken is stated at the code that applies it.
 */
#ifndef DC_LBM_ORACLE_H
#define DC_LBM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LEVELS 4

enum { ORC_HOLE = 0, ORC_BULK = 1, ORC_TFP = 2, ORC_IE = 3, ORC_TFC = 4 };

typedef struct {
    int lattice;                         /* 9 (D2Q9) or 19 (D3Q19) */
    int n_levels;                        /* 1..ORC_MAX_LEVELS */
    long coarse_n[3];                    /* level-0 nodes per axis (periodic); coarse_n[2]=1 in 2-D */
    long box_lo[ORC_MAX_LEVELS][3];      /* level l>=1 patch, level-0 cell units, [lo,hi) */
    long box_hi[ORC_MAX_LEVELS][3];
    double nu0;                          /* kinematic viscosity, level-0 lattice units */
    double sigma;                        /* H-RR hybridisation, 0.98 in the paper */
    int dc_variant;                      /* 2 = DC2 (Table 1), 1 = DC1 */
    int psi_sign;                        /* +1 / -1 multiplier on psi_i */
    /* Refined region of level l >= 1 as a staircase of parent cells (Sec. 4.1.2, 4.2.2,
     * App. B): NULL refines every parent cell of the box; otherwise one byte per
     * parent (level l-1) cell of the box, x fastest, nonzero = refined.  2-D only, on
     * the finest level, on a box that spans no axis. */
    const unsigned char *mask[ORC_MAX_LEVELS];
} orc_desc;

/* lattice tables: c[Q][3], w[Q]; returns Q or -1 */
int orc_lattice(int lattice, int *c, double *w);

/* Eq. (fEq_herm): feq[Q] from rho, u[3] */
void orc_feq(int lattice, double rho, const double *u, double *feq);
/* App. A Eq. (psi): psi[Q] from C[6] = (xx,yy,zz,xy,xz,yz) of C_ab = sum_g d_g Psi_abg */
void orc_psi(int lattice, const double *C, int psi_sign, double *psi);
/* App. A Eq. (Psi): full symmetric Psi_abg of one node, out[27] indexed a*9+b*3+g */
void orc_Psi_tensor(int lattice, double rho, const double *u, double *out);
/* Eq. (LBMscheme_reg): one node's post-collision populations.
 * S[6] strain rate (xx,yy,zz,xy,xz,yz) feeding a1^FD, C[6] as above. */
void orc_collide(int lattice, const double *f, double rho, const double *u,
                 const double *S, const double *C, double tau, double sigma,
                 int psi_sign, double *fpost);
/* off-equilibrium Hermite coefficient a1^(2) (Eq. a12_HRR), out[6] */
void orc_a1(int lattice, const double *f, double rho, const double *u,
            const double *S, const double *C, double tau, double sigma,
            int psi_sign, double *a1);

/* Eq. (system_fi): F(X) and J_F(X) = dF/dX, X=(rho,ux,uy[,uz]) */
void orc_newton_system(int lattice, const double *fhat, const double *Gamma,
                       const double *X, double *F, double *J);
/* Newton-Raphson of Eq. (updated_macro); returns iterations, -1 if not converged in 10 */
int orc_newton(int lattice, const double *fhat, const double *Gamma, double *X);

/* Eq. (TempInt), read at t-dt^c, t, t+dt^c: weights for g(t+dt^f) */
void orc_tempint_weights(double *w3);
/* 4-point Lagrange weights at x=1/2 (centred: nodes -1,0,1,2) or one-sided (0,1,2,3) */
void orc_lagrange4_weights(int one_sided, double *w4);

/* set rule of reading R4 on a 3^3 occupancy neighbourhood (index (ox+1)+3(oy+1)+9(oz+1)) */
void orc_known_from_occupancy(int lattice, const unsigned char *occ_f, const unsigned char *occ_c,
                              unsigned int *kf, unsigned int *kc);

/* hierarchy */
typedef struct orc_h orc_h;
orc_h *orc_create(const orc_desc *d, char *err, int errlen);
void orc_destroy(orc_h *h);
int orc_level_info(orc_h *h, int l, long *n, long *off, int *periodic, double *tau);
int orc_node_class(orc_h *h, int l, unsigned char *cls);
/* fine-known / coarse-known bit masks of every node of level l (0 where not defined) */
int orc_known_masks(orc_h *h, int l, unsigned int *known_f, unsigned int *known_c);
int orc_init(orc_h *h, int l, const double *rho, const double *u);
int orc_advance(orc_h *h, long n_coarse_steps);
int orc_get_macros(orc_h *h, int l, double *rho, double *u);
int orc_get_pops(orc_h *h, int l, double *f);
int orc_set_pops(orc_h *h, int l, const double *f);
/* S_ab and C_ab = sum_g d_g Psi_abg last supplied to the interface nodes of level l
 * ([6][N], order xx yy zz xy xz yz; lattice units of level l; zero elsewhere): at a
 * TF node of a fine level the coarse-stencil values times 1/2, at the co-located
 * coarse node the unscaled values of the last sync sub-step, at hanging nodes the
 * interpolated ones. */
int orc_get_gradients(orc_h *h, int l, double *S, double *C);
/* Test accessor: the stencil of hanging node idx of level l, its nodes' level-l
 * coordinates pts[n][3] and weights w[n] (n <= 16 returned; -1 if idx is no hanging
 * node or its stencil misses a TF node). */
int orc_ie_stencil(orc_h *h, int l, long idx, long *pts, double *w);
int orc_max_newton_iters(orc_h *h);
long orc_node_updates(orc_h *h);
const char *orc_error(orc_h *h);
/* threads of the per-node loops (OpenMP build): sets the count when n > 0, returns
 * the count in use; 1 in the plain build.  Both builds compute identical bits. */
int orc_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
