/*
 * lqcd.h -- C-ABI of the GB300 (sm_103a) hot path of the Schwarz-
 * preconditioned two-flavour Wilson HMC with a one-dimensional (x0-slab)
 * domain decomposition (M. Hasenbusch, "HMC algorithm for two-flavour
 * lattice QCD: Schwarz-preconditioning with a one-dimensional domain
 * decomposition", Lattice 2007, arXiv:0710.0066).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status: every function returns LQCD_OK (0) or a negative LQCD_ERR_*;
 *   lqcd_last_error() gives a one-line description.  No function exits,
 *   traps or waits without bound: device-side waits are bounded and
 *   report LQCD_ERR_TIMEOUT.
 * Threads: a handle is not thread-safe; calls on one handle must not
 *   overlap (separate handles are independent).
 * Memory: every field pointer is a DEVICE pointer owned by the caller
 *   (16-byte aligned); the library reads/writes it on the handle's stream
 *   and owns only its internal workspace, allocated in lqcd_create.
 * Sites x = (x0,x1,x2,x3), 0 <= x_mu < L_mu, x0 is time (Sec. 1, text
 *   after eq. (1)).  All L_mu even; x0-slabs of thickness l0 with
 *   L0 % (2 l0) == 0 (Sec. 1, one-dimensional block decomposition:
 *   l_mu = L_mu for mu = 1,2,3); slab k = x0 / l0, colour k mod 2
 *   (0 = red, 1 = black).
 * Site order ("checkerboard"): all even sites (x0+x1+x2+x3 even), then all
 *   odd sites; within one parity the lexicographic index
 *   ((x0*L1 + x1)*L2 + x2)*L3 + x3, divided by two.
 * Layouts (double precision, interleaved re,im):
 *   spinor (full lattice)   double[V][4 spin][3 colour][2]
 *   spinor (one parity)     double[V/2][4][3][2]
 *   gauge field             double[4 mu][V][3][3][2], U_mu(x) row-major
 *   momenta / forces        double[4 mu][V][8]: coefficients p^a of
 *                           P = sum_a p^a T^a, T^a = lambda^a / 2
 *   boundary field (R)      double[L0/(2 l0)][2 face][V3][2][3][2]: black
 *                           slab k = 2j+1 has ordinal j; face 0 is its first
 *                           time slice with spin basis (e_i - e_{i+2})/sqrt2
 *                           of range (1+gamma_0)/2, face 1 its last slice
 *                           with basis (e_i + e_{i+2})/sqrt2 of range
 *                           (1-gamma_0)/2, i = 0,1; V3 spatial sites in
 *                           lexicographic (x1,x2,x3) order.
 *   second-level boundary   double[L0/(2 l0s)][V3][2][3][2] (iterated
 *   field (R2)              decomposition, lqcd_set_subslabs): black
 *                           sub-slab 2j+1 (sub-slab k = x0 / l0s) has
 *                           ordinal j; its first time slice with the face-0
 *                           spin basis above.
 * Gamma matrices: chiral basis, gamma_0 = [[0,-1],[-1,0]],
 *   gamma_k = [[0,-i sigma_k],[i sigma_k,0]], gamma_5 = diag(1,1,-1,-1).
 * Fermion phase bc_t (+1 / -1) on every x0 hop that wraps L0-1 <-> 0.
 * Precision argument: LQCD_PREC_F64 runs everything in double precision;
 *   LQCD_PREC_F32 / LQCD_PREC_F16 / LQCD_PREC_BF16 run stencils and inner
 *   Krylov iterations with single-, half- (IEEE fp16, each site scaled by
 *   its largest component) or bfloat16-precision storage (8 exponent bits,
 *   no scale; 8 significant bits) of spinors and links, FP32 arithmetic,
 *   and keep
 *   double-precision residuals, dot products and outer defect correction;
 *   there the double hopping sweeps of the outer residual and of the
 *   even-odd source / reconstruction read the double fields and links and
 *   compute in double-float arithmetic (pairs of floats, ~2^-46 relative),
 *   because GB300's FP64 rate would bound them.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqcd_ctx* lqcd_t;

enum {
    LQCD_OK = 0,
    LQCD_ERR_ARG = -1,        /* bad pointer, size or flag */
    LQCD_ERR_GEOM = -2,       /* invalid lattice / slab geometry */
    LQCD_ERR_NOCONVERGE = -3, /* a solve hit max_iter */
    LQCD_ERR_CUDA = -4,       /* a CUDA runtime call failed */
    LQCD_ERR_NAN = -5,        /* non-finite residual or energy */
    LQCD_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up */
    LQCD_ERR_STATE = -7       /* call order (e.g. no gauge field set) */
};

enum { LQCD_PREC_F64 = 0, LQCD_PREC_F32 = 1, LQCD_PREC_F16 = 2, LQCD_PREC_BF16 = 3 };
enum { LQCD_OP_HOP = 0, LQCD_OP_MHAT = 1 };
enum { LQCD_SCHUR_R = 0, LQCD_SCHUR_RDAG = 1, LQCD_SCHUR_RINV = 2, LQCD_SCHUR_RINVDAG = 3,
       LQCD_SCHUR2_R = 4, LQCD_SCHUR2_RDAG = 5, LQCD_SCHUR2_RINV = 6, LQCD_SCHUR2_RINVDAG = 7 };
enum { LQCD_TERM_W1 = 0, LQCD_TERM_SCHUR = 1, LQCD_TERM_W2 = 2, LQCD_TERM_SCHUR2 = 3,
       LQCD_TERM_S2 = 4, LQCD_TERM_S1 = 5 };
enum { LQCD_EO_APPLY = 0, LQCD_EO_SOLVE = 1 };
enum { LQCD_SOLVER_BICGSTAB = 0, LQCD_SOLVER_SERIES = 1, LQCD_SOLVER_SAP = 2, LQCD_SOLVER_SAP_BLOCKS = 3 };
enum { LQCD_MAX_LEVELS = 5 };
enum { LQCD_LF = 0, LQCD_SW = 1 };

/* Create a handle for the lattice L[4] with x0-slabs of thickness l0 and
 * fermion phase bc_t on the x0 wrap.  stream: a cudaStream_t (NULL = the
 * legacy default stream); every call of this handle is ordered on it.
 * Allocates the internal workspace on the current device.
 * Errors: LQCD_ERR_GEOM (odd extent, L0 % (2 l0) != 0, V >= 2^31),
 * LQCD_ERR_ARG, LQCD_ERR_CUDA.  (Sec. 1: lattice, blocks l_0 x L1 x L2 x L3.) */
int lqcd_create(lqcd_t* h, const int L[4], int l0, int bc_t, void* stream);
int lqcd_destroy(lqcd_t h);
const char* lqcd_last_error(lqcd_t h);
int lqcd_set_stream(lqcd_t h, void* stream);

/* Iterated decomposition (Sec. 1: the one-dimensional slabs can be
 * decomposed again, second step l0^(2) = l0^(1)/2): split
 * every slab once more into two sub-slabs of thickness l0s = l0 / 2,
 * sub-slab k = x0 / l0s with colour k mod 2.  W2 is eq. (2) with every hop
 * between different sub-slabs removed.  With the sites of W1 ordered
 * red|black by sub-slab colour, W1 = [[A2,B2],[C2,D2]], W2 = diag(A2,D2)
 * and det W1 = det W2 det R2 with R2 = E2 (1 - C2 A2^-1 B2 D2^-1) E2^dag on
 * the second-level boundary field (layout above): the range of C2 is the
 * first slice of each black sub-slab (its last slice borders the next slab,
 * which W1 does not reach).  Together det M = det R det R2 det W2.
 * Enables lqcd_subblock_*, LQCD_SCHUR2_*, LQCD_TERM_W2 / _SCHUR2 and the
 * level_w2 / level_schur2 trajectory terms.  l0s = 0 switches it off.
 * Errors: LQCD_ERR_GEOM (l0 odd or l0s != l0/2). */
int lqcd_set_subslabs(lqcd_t h, int l0s);

/* Load the gauge field U (device, gauge layout above, SU(3) links) into the
 * handle; builds the double, single (12-real, two rows) and half (12-real)
 * internal copies.  lqcd_get_gauge writes the handle's double-precision
 * field back in the same layout.  (Sec. 1: U_{x,mu} in SU(3).) */
int lqcd_set_gauge(lqcd_t h, const double* U);
int lqcd_get_gauge(lqcd_t h, double* U);

/* Fill maps (device int32[14][V]) with the integer index maps, site s in
 * checkerboard order: 0 lexicographic index, 1 parity, 2 slab, 3 colour,
 * 4..7 site of x+mu_hat, 8..11 site of x-mu_hat (periodic), 12 face flags
 * (1: first slice of its slab, 2: last slice), 13 boundary-field site
 * (j*2+f)*V3 + lex3 for black face sites (face 0 if both), else -1.
 * (Sec. 1: sites, slabs, red/black blocks.) */
int lqcd_index_maps(lqcd_t h, int32_t* maps);

/* Even-odd pieces of the Wilson matrix, eq. (2), M = 1 - kappa H with
 *   (H psi)(x) = sum_mu (1-gamma_mu) U_mu(x) psi(x+mu)
 *                     + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu).
 * op = LQCD_OP_HOP:  out_p = H_{p,1-p} in_{1-p}  (in: parity 1-p field,
 *                    out: parity p field); kappa unused.
 * op = LQCD_OP_MHAT: out_e = in_e - kappa^2 H_eo H_oe in_e (parity must be
 *                    0), the even-odd reduced matrix used for the global
 *                    solver (Sec. 3: BiCGstab with even-odd preconditioning).
 * dagger = 1 applies the adjoint (H^dag swaps the projectors).  precision
 * selects the internal storage (results returned in double).  Asynchronous. */
int lqcd_dslash_eo(lqcd_t h, double* out, const double* in, double kappa, int parity,
                   int dagger, int op, int precision);

/* W1: eq. (2) with every hop between different x0-slabs removed (Sec. 1:
 * the block operator keeps only the hops inside one block),
 * applied on the slabs of one colour (0 red, 1 black, -1 all); out is zero
 * on the other slabs.  Full-lattice fields.  Asynchronous. */
int lqcd_block_dslash(lqcd_t h, double* out, const double* in, double kappa, int colour,
                      int dagger, int precision);

/* Solve W1 x = b (dagger: W1^dag x = b) independently on every slab of the
 * given colour (-1: all slabs) in one persistent batched launch: even-odd
 * reduced BiCGstab per slab, inner iterations in `precision`, double
 * precision residuals and defect correction to |b - W1 x| <= tol |b| per
 * slab.  x is zero on the other slabs.  iters_out (host int[nb], may be
 * NULL) receives the inner iterations per slab, resid_out (host
 * double[nb], may be NULL) the final relative residual per slab (0 for
 * slabs not solved).  Synchronous.  Errors: LQCD_ERR_NOCONVERGE after
 * max_iter inner iterations, LQCD_ERR_TIMEOUT.  (Sec. 1 W1; Sec. 3 solver.) */
int lqcd_block_solve_batched(lqcd_t h, double* x, const double* b, double kappa, int colour,
                             int dagger, int precision, double tol, int max_iter,
                             int* iters_out, double* resid_out);

/* W2 (iterated decomposition, see lqcd_set_subslabs): the same as
 * lqcd_block_dslash / lqcd_block_solve_batched with the sub-slabs in place
 * of the slabs; colour is the sub-slab colour, iters_out / resid_out are
 * indexed by sub-slab (host arrays of L0/l0s entries).
 * Errors as there, and LQCD_ERR_STATE without sub-slabs. */
int lqcd_subblock_dslash(lqcd_t h, double* out, const double* in, double kappa, int colour,
                         int dagger, int precision);
int lqcd_subblock_solve_batched(lqcd_t h, double* x, const double* b, double kappa, int colour,
                                int dagger, int precision, double tol, int max_iter,
                                int* iters_out, double* resid_out);

/* Even-odd and mass preconditioning of W2 (Sec. 1): on the even sites of
 * the sub-slabs, W2,eo = 1 - kappa^2 H_eo H_oe (the Schur complement of
 * W2's odd-odd block, det W2 = det W2,eo) and W3,eo = W2,eo + rho.
 * op LQCD_EO_APPLY: out = W3,eo in (dagger: W3,eo^dag in);
 * op LQCD_EO_SOLVE: out = W3,eo^-1 in (dagger: W3,eo^-dag in), every
 * sub-slab in one batched launch, relative residual <= tol, inner
 * iteration `method`: LQCD_SOLVER_BICGSTAB, or LQCD_SOLVER_SERIES, the
 * geometric series sum_k (kappa^2 H_eo H_oe / (1+rho))^k / (1+rho) (Sec. 3,
 * the solver of the block terms; it converges only when that operator's
 * spectral radius is below one, else LQCD_ERR_NOCONVERGE); iters_out
 * (host int[L0/l0s], may be NULL) the inner iterations per sub-slab.
 * rho = 0 gives W2,eo.  in/out: even-site fields, the one-parity layout
 * above (double[V/2][4][3][2]).  Synchronous.  LQCD_ERR_STATE without
 * sub-slabs. */
int lqcd_subblock_eo(lqcd_t h, double* out, const double* in, double kappa, double rho,
                     int dagger, int op, int precision, int method, double tol, int max_iter,
                     int* iters_out);

/* Solve M x = b (dagger: M^dag x = b) on the full lattice: even-odd reduced
 * system, double precision defect correction to |b - M x| <= tol |b|, inner
 * iterations in `precision` by the handle's global solver
 * (lqcd_set_global_solver).  iters_out / resid_out: host scalars (may be
 * NULL).  Synchronous.  (Sec. 3: the S4 solver.) */
int lqcd_solve_wilson(lqcd_t h, double* x, const double* b, double kappa, int dagger,
                      int precision, double tol, int max_iter, int* iters_out,
                      double* resid_out);

/* Boundary operator of det^2(W1^-1 M) (Sec. 1, pseudo-fermions on the
 * boundaries of the black blocks, dimension halved).  With sites ordered
 * red|black, M = [[A,B],[C,D]], W1 = diag(A,D), block LU gives
 * det M = det W1 det R with
 *   R = E (1 - C A^-1 B D^-1) E^dag
 * on the boundary space (E: orthonormal spin-projected black-face
 * coordinates, layout above).  op: R, R^dag, R^-1 = E D (M^-1)_bb E^dag,
 * R^-dag.  in/out: boundary fields.
 * op LQCD_SCHUR2_*: the same four operators one level down (lqcd_set_subslabs):
 * R2 = E2 (1 - C2 A2^-1 B2 D2^-1) E2^dag with B2 = C2 = -kappa H between the
 * two sub-slabs of a slab, R2^-1 = E2 D2 (W1^-1)_bb E2^dag; in/out are
 * second-level boundary fields (LQCD_ERR_STATE without sub-slabs).
 * Synchronous. */
int lqcd_schur_apply(lqcd_t h, double* out, const double* in, double kappa, int op,
                     int precision, double tol, int max_iter);

/* Pseudo-fermion action and force (Sec. 1 eq. (3), Sec. 2 eq. (4)):
 * term W1:    S = |W1^-1 phi|^2, phi a full-lattice spinor;
 * term SCHUR: S = |R^-1 phi|^2, phi a boundary field;
 * term W2:    S = |W2^-1 phi|^2, phi a full-lattice spinor;
 * term SCHUR2: S = |R2^-1 phi|^2, phi a second-level boundary field
 * (W2 / SCHUR2: iterated decomposition, LQCD_ERR_STATE without sub-slabs).
 * F (device double[4][V][8]) += dS/dw^a for U_mu(x) -> exp(i w^a T^a) U_mu(x)
 * (not zeroed).  S_out (host, may be NULL) receives S.  F may be NULL to
 * compute S only.  Solutions are recomputed, never stored.  Synchronous. */
int lqcd_pf_force(lqcd_t h, double* F, const double* phi, double kappa, int term,
                  int precision, double tol, int max_iter, double* S_out);

/* The two mass-preconditioned parts of det^2 W2 in the four-part action
 * (Sec. 1, S2 and S1), phi an even-site field:
 * term LQCD_TERM_S2: S = |W3,eo W2,eo^-1 phi|^2  (det^2 of W2,eo W3,eo^-1);
 * term LQCD_TERM_S1: S = |W3,eo^-1 phi|^2        (det^2 of W3,eo);
 * W3,eo = W2,eo + rho.  F, S_out as in lqcd_pf_force.  Synchronous. */
int lqcd_pf_force_eo(lqcd_t h, double* F, const double* phi, double kappa, double rho, int term,
                     int precision, double tol, int max_iter, double* S_out);

/* Wilson gauge action (Sec. 1): S_G = -beta/3 sum_x sum_{mu>nu} Re tr P_{mu nu}(x).
 * F (device, may be NULL) += dS_G/dw^a; S_out / plaq_out (host, may be NULL)
 * receive S_G and the average Re tr P / 3.  Synchronous. */
int lqcd_gauge_force(lqcd_t h, double* F, double beta, double* S_out, double* plaq_out);

/* Average force per time slice, the diagnostic of Sec. 3 (Fig. 1 plots the
 * mean force on the space-like links against x0): out (device double[2][L0])
 * receives, for each x0, the mean over the slice's space-like links
 * (row 0) and time-like links (row 1) of |F| = (sum_a F_a^2)^(1/2).
 * F: device forces double[4][V][8] (e.g. from lqcd_pf_force).  Asynchronous. */
int lqcd_force_profile(lqcd_t h, const double* F, double* out);

/* T_U of Sec. 2 eq. (4) on its own: U_mu(x) <- exp(i dt P_mu(x)) U_mu(x)
 * with P = sum_a P^a T^a (momenta layout), exponential by Cayley-Hamilton
 * in double precision, then reunitarised.  U: device gauge field, updated
 * in place; it also becomes the handle's gauge field.  Used by the
 * autograd binding (actions as functions of Lie-algebra coordinates) and
 * its finite-difference tests.  Synchronous. */
int lqcd_link_update(lqcd_t h, double* U, const double* P, double dt);

/* Philox4x32-10 normal deviates (Salmon et al., SC'11) as used by the HMC
 * heatbath: out[k] (device double[n]) for counter (k/2 lo, k/2 hi, stream,
 * traj) and key (seed lo, seed hi); two 53-bit uniforms per counter and
 * Box-Muller (cos for even k, sin for odd k).  Asynchronous. */
int lqcd_rng_normals(lqcd_t h, double* out, int64_t n, uint64_t seed, uint32_t stream,
                     uint32_t traj);

typedef struct {
    double beta, kappa;
    double tau;         /* trajectory length */
    double lambda;      /* SW / Omelyan parameter, the paper uses 1/6 */
    int nlevels;        /* 1..LQCD_MAX_LEVELS integration levels */
    int scheme[LQCD_MAX_LEVELS];  /* LQCD_LF or LQCD_SW per level */
    int nsteps[LQCD_MAX_LEVELS];  /* n_j: steps of level j per step of level j+1;
                           nsteps[nlevels-1] = steps per trajectory */
    int level_gauge;    /* level of S_G, -1 to leave the term out */
    int level_w1;       /* level of |W1^-1 phi1|^2, or -1 */
    int level_schur;    /* level of |R^-1 phi2|^2, or -1 */
    int pf_init;        /* 0: heatbath phi = W eta; 1: phi = eta directly */
    int roll;           /* 1: shift U along x0 by a random amount after */
    int metropolis;     /* 1: accept/reject on dH; 0: always accept */
    int precision;      /* LQCD_PREC_* for every solve */
    double tol;         /* relative residual of every solve */
    int max_iter;
    /* position-dependent step size (Sec. 2): the step of link U_mu(x) is
     * dt * s(x0), one table for space-like and one for time-like links.
     * step_scheme: 0 none (s = 1), 1/2/3 the paper's schemes A (period 6),
     * B (period 8), C (period 16), repeated along x0 (L0 must be a multiple
     * of the period; scheme A's space-like s(5) is read as 0.2, the value
     * that gives the stated average 0.525).  step_scale: optional host
     * table double[2][L0] (row 0 space-like, row 1 time-like) overriding
     * step_scheme.  s = 0 freezes a link. */
    int step_scheme;
    const double* step_scale;
    /* iterated decomposition (lqcd_set_subslabs): levels of |W2^-1 phi3|^2
     * and |R2^-1 phi4|^2, or -1 (must be -1 without sub-slabs).  The action
     * S_G + |R^-1 phi2|^2 + |R2^-1 phi4|^2 + |W2^-1 phi3|^2 takes
     * level_w1 = -1.  phi3 = W2 eta3, phi4 = R2 eta4 are always drawn by the
     * heatbath (Philox streams 5 and 6; pf_init applies to phi1, phi2). */
    int level_w2;
    int level_schur2;
    /* mass preconditioning of W2 (Sec. 1, W3,eo = W2,eo + rho): levels of
     * S2 = |W3,eo W2,eo^-1 phi5|^2 and S1 = |W3,eo^-1 phi6|^2, or -1 (must be
     * -1 without sub-slabs).  The paper's four-part action is level_schur
     * (S4), level_schur2 (S3), level_s2 (S2), level_s1 (S1) with
     * level_w1 = level_w2 = -1.  phi5 = W2,eo W3,eo^-1 eta5 and
     * phi6 = W3,eo eta6 are drawn on Philox streams 7 and 8 (the even-site
     * half of a full-lattice draw). */
    double rho;
    int level_s2;
    int level_s1;
    int eo_solver;      /* inner iteration of the S2 / S1 solves (W3,eo, W2,eo):
                           LQCD_SOLVER_BICGSTAB or LQCD_SOLVER_SERIES */
    int block_solver;   /* inner iteration of the W1 / W2 block solves of the
                           |W1^-1 phi1|^2 and |W2^-1 phi3|^2 terms (the solves
                           inside R and R2 keep BiCGstab):
                           LQCD_SOLVER_BICGSTAB or LQCD_SOLVER_SERIES, the
                           geometric series of Sec. 3 (which needs its
                           spectral radius below one) */
    int use_graph;      /* 1: lqcd_hmc_trajectory runs the molecular dynamics
                           as a CUDA graph, recorded the first time for a
                           parameter set (not run then) and replayed; the
                           solves inside report failures once, after the
                           replay.  Same kernels in the same order: the
                           results equal the eager run's. */
    int chrono;         /* 1: each force solve of the molecular dynamics
                           starts from a chronological guess: the linear
                           extrapolation in MD time of its solutions at the
                           two previous force evaluations of its term (one
                           kept: that one; the first solve of a trajectory
                           starts from zero); 2: the quadratic extrapolation
                           through the three previous solutions (fewer kept:
                           the lower orders); 3: as 2, except that the whole-
                           lattice solves of the boundary term start from the
                           combination of their last (up to) six solutions
                           that minimises the residual under the current
                           links (minimal residual extrapolation: the
                           solutions' images under the even-odd matrix in
                           single precision, the small normal equations
                           solved on the device).  The solves still run to tol,
                           so the forces agree with chrono = 0 to the solver
                           tolerance, and reversibility holds to it.  Needs
                           12 (chrono + 1) extra even-site double fields on
                           the device (chrono = 3: 42, and six single-
                           precision ones; allocated on first use). */
} lqcd_hmc_params;

/* Pseudo-fermion fields of lqcd_md (device pointers, NULL where the term
 * is left out): w1, w2 full spinors; schur, schur2 first- / second-level
 * boundary fields; s2, s1 even-site fields. */
typedef struct {
    const double* w1;
    const double* schur;
    const double* w2;
    const double* schur2;
    const double* s2;
    const double* s1;
} lqcd_pf_fields;

typedef struct {
    double dH, H0, H1;
    double plaq;        /* average Re tr P / 3 of the field returned */
    double u;           /* Metropolis uniform */
    int accepted;
    int shift;          /* x0 roll applied */
    int64_t solver_iters; /* inner Krylov iterations, whole trajectory */
    int n_solves;
    int n_force;        /* force evaluations */
    int64_t site_iters; /* sum over solves of inner iterations x even sites
                           of the system */
    int64_t hop_sites;  /* half-lattice hopping site updates of those inner
                           iterations (four per BiCGstab iteration and site,
                           two per geometric-series iteration and site) */
} lqcd_hmc_result;

/* One HMC trajectory (Sec. 2): heatbath (momenta p^a ~ N(0,1), eta ~
 * exp(-|eta|^2)), phi1 = W1 eta1, phi2 = R eta2 (and phi3, phi4 of the
 * iterated decomposition), molecular dynamics
 * T_{X,top}(dt_top)^{n_top} with the recursive LF / SW levels of eqs.
 * (5)-(7), Metropolis on dH, then the x0 shift of the configuration.
 * U: device gauge field, overwritten with the field after the trajectory.
 * P0 / eta1 / eta2: optional device inputs (momenta, full spinor,
 * boundary field) replacing the Philox draws of (seed, traj); NULL draws
 * them.  res: host.  Synchronous. */
int lqcd_hmc_trajectory(lqcd_t h, double* U, const lqcd_hmc_params* prm, uint64_t seed,
                        uint32_t traj, const double* P0, const double* eta1,
                        const double* eta2, lqcd_hmc_result* res);

/* Molecular dynamics only: integrates (U, P) in place (device buffers, gauge
 * and momenta layouts) for the fixed pseudo-fermion fields f (host struct
 * of device pointers).  Synchronous. */
int lqcd_md(lqcd_t h, double* U, double* P, const lqcd_pf_fields* f, const lqcd_hmc_params* prm);

/* Kernel timing with CUDA events on the handle's stream.  kernel ids:
 * 0 hopping sweep, 1 persistent solver, 2 force, 3 gauge force / update,
 * 4 layout / BLAS-1.  enable: 0 off, 1 all ids, otherwise a bit mask
 * (1 << id) of the ids to time.  lqcd_profile_read returns, per id, the launches,
 * the summed device time (ms) and the summed algorithmic DRAM bytes of
 * the launches recorded since the last reset (synchronises the stream). */
int lqcd_profile_enable(lqcd_t h, int enable);
int lqcd_profile_reset(lqcd_t h);
int lqcd_profile_read(lqcd_t h, int kernel_id, int64_t* launches, double* ms, double* bytes);
/* The individual device times (ms) of the launches of kernel_id recorded
 * since the last reset, in launch order: up to cap of them into ms_out
 * (host float[cap]); *n_out (host) receives how many were recorded (at most
 * 65536 are kept).  Synchronises the stream. */
int lqcd_profile_times(lqcd_t h, int kernel_id, float* ms_out, int64_t cap, int64_t* n_out);

/* Launch schedules picked by measurement on this handle's lattice and
 * gauge field (the paper has no counterpart; its code ran on CPUs):
 * what & 1: threads per block of the hopping sweep (64 / 128 / 256), per
 * storage precision; what & 2: sites per thread of the persistent solver
 * (1 / 2, i.e. CTAs per system, or 0: every co-resident CTA with an equal
 * contiguous share of the sites), per precision, separately for the
 * batched slab solve and the global solve, each candidate timed on a
 * solve at `kappa` to 1e-10.  The choices stay with the handle; results
 * are the same up to rounding for every choice.  Synchronous.
 * lqcd_tune_read fills out (host int[12]) with hop block size [F64, F32,
 * F16, BF16], slab-solve sites per thread [F64, F32, F16, BF16], global-
 * solve sites per thread [F64, F32, F16, BF16]. */
int lqcd_autotune(lqcd_t h, int what, double kappa);
int lqcd_tune_read(lqcd_t h, int* out);
/* Sets the persistent solver's schedule of every precision and both solve
 * kinds to `spt` (1 or 2 sites per thread, 0 every co-resident CTA with an
 * equal share of the sites), as lqcd_autotune would pick it.  Results are
 * the same up to rounding.  Errors: LQCD_ERR_ARG (spt outside 0..2). */
int lqcd_set_solver_schedule(lqcd_t h, int spt);
/* enable = 1: single-precision geometric-series slab solves (the sub-slab
 * and W3,eo solves, and the trajectory's W1 / S1 / S2 terms with the
 * series) of at most 8192 sites per system run on thread-block clusters
 * where the device allows 16-CTA clusters: one cluster per slab, the
 * series' vectors in the cluster's distributed shared memory, the
 * system's CTAs meeting at a bounded mbarrier handshake (the paper has no
 * counterpart).  Results are the same up to rounding.  Default: disabled
 * (0), the grid-wide persistent solver, which measured 2.2x faster on the
 * 16^3x32 slabs (6.0 against 2.7 ms per series solve). */
int lqcd_set_cluster_series(lqcd_t h, int enable);

/* Inner iteration of every whole-lattice solve of the handle (the S4
 * solver of Sec. 3: lqcd_solve_wilson, R^-1 / R^-dag and the boundary-term
 * force, and the trajectory's), inside the same double defect correction:
 *   LQCD_SOLVER_BICGSTAB (default): BiCGstab on the even-odd reduced
 *     matrix 1 - kappa^2 H_eo H_oe;
 *   LQCD_SOLVER_SAP: the paper's "BiCGstab with even-odd and Schwarz
 *     preconditioning": BiCGstab on M with right preconditioner K^-1, one
 *     multiplicative Schwarz cycle over the x0-slabs (all red slabs, then
 *     all black slabs with the source corrected by the hops from the red
 *     faces), each slab solve the geometric series of its even-odd reduced
 *     operator truncated after sap_terms terms (0..64), so that K^-1 is a
 *     fixed linear map; the inner system M y = (r, 0) gives the even-odd
 *     reduced correction y_e.  The series needs the slab operator's
 *     spectral radius below one to precondition well (it always gives a
 *     valid, if weaker, preconditioner).
 *   LQCD_SOLVER_SAP_BLOCKS: the same Schwarz-preconditioned BiCGstab with
 *     the cycle taken over small 4-D blocks instead of the x0-slabs: block
 *     extent 4 in every direction whose L is a multiple of 4, else 2;
 *     blocks coloured by the parity of their block coordinates; each
 *     block's even-odd reduced operator inverted by sap_terms terms of its
 *     geometric series (the paper does not fix the blocks of its S4
 *     preconditioner).  Every block is solved by one CTA with the block's
 *     links and vectors in shared memory.
 * Selecting LQCD_SOLVER_SAP or LQCD_SOLVER_SAP_BLOCKS allocates their
 * workspace (11 full-lattice vectors, 2.1 KB per lattice site) on the
 * current device; it is kept until lqcd_destroy.
 * Errors: LQCD_ERR_ARG (other methods, sap_terms out of range),
 * LQCD_ERR_CUDA (allocation); a later solve returns LQCD_ERR_GEOM for an
 * odd extent with LQCD_SOLVER_SAP_BLOCKS. */
int lqcd_set_global_solver(lqcd_t h, int method, int sap_terms);

/* Limit of one barrier wait inside the persistent solver, in GPU clock
 * cycles (clock64): a CTA that has waited that long for the other CTAs of
 * its system gives up, the solve ends with LQCD_ERR_TIMEOUT and every CTA
 * returns at its next barrier; the handle stays usable.  cycles <= 0
 * restores the default, 4e9 cycles (about two seconds).  A diagnostic for
 * exercising the bounded-wait path (the paper has no counterpart); it
 * applies to solves launched after the call (a recorded MD graph is
 * recorded again).  Host only, never fails on a valid handle. */
int lqcd_set_wait_limit(lqcd_t h, int64_t cycles);

/* Number of kernels this handle has launched since lqcd_create (host
 * counter; *count is a host int64). */
int lqcd_launch_count(lqcd_t h, int64_t* count);

/* Wilson gauge action without a handle and without any device allocation,
 * for callers that cannot call cudaMalloc (for example code running while
 * another framework owns the whole device memory pool, or host threads that
 * must not trigger the device synchronisation an allocation implies); such
 * callers cannot create a handle either.  The paper has no counterpart: it
 * is a service entry point, not a step of the method.
 * U: device gauge field, C-ABI layout, lattice L[4] (all even).
 * out: device double[2], receives S_G = -beta/3 sum Re tr P and the average
 * Re tr P / 3.  stream: cudaStream_t (NULL = legacy default); asynchronous.
 * Per-block partial sums live in a fixed 128 KiB array compiled into the
 * library and kept by every GPU that loads it until the process exits; at
 * most 2,097,152 sites (32^3 x 64), larger lattices return LQCD_ERR_GEOM.
 * The first call on a device looks the array's address up with
 * cudaGetSymbolAddress (that device current); make it before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race.
 * Errors: LQCD_ERR_ARG (null pointer), LQCD_ERR_GEOM, LQCD_ERR_CUDA. */
int lqcd_gauge_action_static(const int L[4], const double* U, double beta, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
