/*
 * lqcd_oracle.h -- interface of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and oracle/lqcd_oracle.c are used
 * by the test-suite, by __graft_entry__.smoke() and by the cpu_baseline /
 * reference arm of bench.py.  The GPU library neither includes nor links
 * them, and they include nothing from the GPU library.
 *
 * Conventions (the same documented layouts as the GPU library's C-ABI,
 * restated here independently):
 *  - lattice sites x = (x0,x1,x2,x3), 0 <= x_mu < L_mu, x0 = time
 *    (Sec. 1, below eq. (1));
 *  - site order "checkerboard": all even sites, then all odd sites;
 *    inside one parity the lexicographic index
 *    lex = ((x0*L1 + x1)*L2 + x2)*L3 + x3 divided by two;
 *  - spinor fields: double[V][4 spin][3 colour][re,im];
 *  - gauge field:   double[4 mu][V][3][3][re,im], U_mu(x) row-major;
 *  - momenta/forces: double[4 mu][V][8], coefficients on T^a = lambda^a/2;
 *  - x0-slabs of thickness l0 (Sec. 1, one-dimensional decomposition),
 *    slab k = x0 / l0, colour k mod 2 (0 red, 1 black);
 *  - boundary (Schur) fields: double[nb/2][2 face][V3][2][3][re,im];
 *    black slab k = 2j+1 has ordinal j, face 0 is its first time slice
 *    (range of (1+gamma_0)/2), face 1 its last time slice (range of
 *    (1-gamma_0)/2); V3 spatial sites in lexicographic (x1,x2,x3) order.
 */
#ifndef LQCD_ORACLE_H
#define LQCD_ORACLE_H
#include <stdint.h>

typedef struct {
    int L[4];  /* L0 (time, slab direction), L1, L2, L3 */
    int l0;    /* slab thickness; L0 % (2*l0) == 0 */
    int bc_t;  /* +1 periodic / -1 antiperiodic fermion wrap in x0 */
    int l0s;   /* iterated decomposition (Sec. 1): sub-slabs of thickness
                  l0s = l0/2 (W2); 0 = none */
} lqo_geom;

enum { LQO_HOP_ALL = 0, LQO_HOP_INTRA = 1, LQO_HOP_CROSS = 2, LQO_HOP_INTRA2 = 3, LQO_HOP_CROSS2 = 4 };
enum { LQO_R = 0, LQO_RDAG = 1, LQO_RINV = 2, LQO_RINVDAG = 3 };
enum { LQO_LF = 0, LQO_SW = 1 };

typedef struct {
    double beta, kappa, tau, lambda;
    int nlevels;      /* 1..5 */
    int scheme[5];
    int nsteps[5];
    int level_gauge, level_w1, level_schur; /* -1: term left out */
    int pf_init;      /* 0: heatbath phi = W eta; 1: phi = eta directly */
    int roll;         /* 1: shift U along x0 after the trajectory */
    int schur_route;  /* 0: R^-1 by solving R itself; 1: through M^-1 */
    int metropolis;   /* 1: accept/reject; 0: always keep the new field */
    double tol;       /* relative residual of every linear solve */
    int maxit;
    const double* step_scale; /* NULL, or [2][L0] s(x0) for space-like / time-like links */
    int level_w2, level_schur2; /* iterated decomposition terms, -1: left out */
    double rho;                 /* mass preconditioning W3,eo = W2,eo + rho */
    int level_s2, level_s1;     /* |W3,eo W2,eo^-1 phi|^2 and |W3,eo^-1 phi|^2, -1: left out */
} lqo_hmc_params;

/* pseudo-fermion fields of the MD (NULL where the term is left out) */
typedef struct {
    const double* w1;     /* full spinor, |W1^-1 phi|^2 */
    const double* schur;  /* boundary field, |R^-1 phi|^2 */
    const double* w2;     /* full spinor, |W2^-1 phi|^2 */
    const double* schur2; /* second-level boundary field, |R2^-1 phi|^2 */
    const double* s2;     /* even sites, |W3,eo W2,eo^-1 phi|^2 */
    const double* s1;     /* even sites, |W3,eo^-1 phi|^2 */
} lqo_pf_fields;

typedef struct {
    double dH, H0, H1;
    double plaq;      /* average Re tr(plaquette)/3 after the trajectory */
    double u;         /* Metropolis uniform */
    int accepted;
    int shift;        /* x0 roll applied */
    int status;       /* 0 ok, <0 a solve did not converge */
} lqo_hmc_result;

int  lqo_geom_check(const lqo_geom* g);
void lqo_index_maps(const lqo_geom* g, int32_t* maps);
void lqo_gamma(double* g5x4x4x2);

void lqo_hop(const lqo_geom* g, const double* U, const double* in, double* out,
             int mode, int dagger);
void lqo_apply_M(const lqo_geom* g, const double* U, double kappa,
                 const double* in, double* out, int dagger);
void lqo_apply_W1(const lqo_geom* g, const double* U, double kappa,
                  const double* in, double* out, int dagger);
void lqo_dslash_eo(const lqo_geom* g, const double* U, const double* in_half,
                   double* out_half, int parity, int dagger);
void lqo_mhat(const lqo_geom* g, const double* U, double kappa,
              const double* in_e, double* out_e, int dagger);
void lqo_block_dslash(const lqo_geom* g, const double* U, double kappa,
                      const double* in, double* out, int colour, int dagger);
int  lqo_block_solve(const lqo_geom* g, const double* U, double kappa,
                     double* x, const double* b, int colour, int dagger,
                     double tol, int maxit, int* iters);
int  lqo_solve_M(const lqo_geom* g, const double* U, double kappa, double* x,
                 const double* b, int dagger, double tol, int maxit, int* iters);
int  lqo_nbnd(const lqo_geom* g);
void lqo_embed_boundary(const lqo_geom* g, const double* coords, double* full);
void lqo_project_boundary(const lqo_geom* g, const double* full, double* coords);
int  lqo_schur(const lqo_geom* g, const double* U, double kappa, double* out,
               const double* in, int op, int route, double tol, int maxit);
void lqo_bilinear(const lqo_geom* g, const double* U, const double* a,
                  const double* b, int mask, double coef, double* F);
int  lqo_pf_w1(const lqo_geom* g, const double* U, double kappa,
               const double* phi, double* F, double* S, double tol, int maxit);
int  lqo_pf_schur(const lqo_geom* g, const double* U, double kappa,
                  const double* phi, double* F, double* S, int route,
                  double tol, int maxit);
double lqo_gauge_action(const lqo_geom* g, const double* U, double beta);
void lqo_gauge_force(const lqo_geom* g, const double* U, double beta, double* F);
double lqo_plaquette(const lqo_geom* g, const double* U);
void lqo_su3_expi(const double* X, double* E);
void lqo_update_U(const lqo_geom* g, double* U, const double* P, double dt);
void lqo_update_U_scaled(const lqo_geom* g, double* U, const double* P, double dt, const double* scale);
int  lqo_step_scheme(int scheme, int L0, double* out);
void lqo_force_profile(const lqo_geom* g, const double* F, double* out);
void lqo_roll_x0(const lqo_geom* g, double* U, int shift);
void lqo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void lqo_normals(uint64_t seed, uint32_t stream, uint32_t traj, int64_t n, double* out);
void lqo_uniforms_metropolis(uint64_t seed, uint32_t traj, int L0, double* u, int* shift);
int  lqo_md(const lqo_geom* g, double* U, double* P, const lqo_pf_fields* pf,
            const lqo_hmc_params* prm);
void lqo_apply_w3eo(const lqo_geom* g, const double* U, double kappa, double rho,
                    const double* in_e, double* out_e, int dagger);
int  lqo_solve_w3eo(const lqo_geom* g, const double* U, double kappa, double rho, double* x_e,
                    const double* b_e, int dagger, double tol, int maxit, int* iters);
int  lqo_pf_s1(const lqo_geom* g, const double* U, double kappa, double rho, const double* phi_e,
               double* F, double* S, double tol, int maxit);
int  lqo_pf_s2(const lqo_geom* g, const double* U, double kappa, double rho, const double* phi_e,
               double* F, double* S, double tol, int maxit);
int  lqo_block_solve2(const lqo_geom* g, const double* U, double kappa, double* x,
                      const double* b, int colour, int dagger, double tol, int maxit, int* iters);
void lqo_apply_W2(const lqo_geom* g, const double* U, double kappa, const double* in,
                  double* out, int dagger);
int  lqo_nbnd2(const lqo_geom* g);
void lqo_embed_boundary2(const lqo_geom* g, const double* coords, double* full);
void lqo_project_boundary2(const lqo_geom* g, const double* full, double* coords);
int  lqo_schur2(const lqo_geom* g, const double* U, double kappa, double* out,
                const double* in, int op, int route, double tol, int maxit);
int  lqo_pf_w2(const lqo_geom* g, const double* U, double kappa, const double* phi,
               double* F, double* S, double tol, int maxit);
int  lqo_pf_schur2(const lqo_geom* g, const double* U, double kappa, const double* phi,
                   double* F, double* S, int route, double tol, int maxit);
int  lqo_hmc_trajectory(const lqo_geom* g, double* U, const lqo_hmc_params* prm,
                        uint64_t seed, uint32_t traj, const double* P0,
                        const double* eta1, const double* eta2,
                        lqo_hmc_result* res);
#endif
