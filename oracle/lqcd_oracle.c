/*
 * lqcd_oracle.c -- FP64 CPU oracle for the hot path of the Schwarz-
 * preconditioned two-flavour Wilson HMC with a one-dimensional (x0-slab)
 * domain decomposition (M. Hasenbusch, Lattice 2007, arXiv:0710.0066).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, by
 * __graft_entry__.smoke() and by bench.py's cpu_baseline / reference arm.
 * The GPU library neither links nor calls any of this; the two share no
 * source, header, table or helper.
 *
 * Plain, slow, double-precision C.  Every operator is the paper's
 * definition written out over explicit site loops with explicit 4x4 gamma
 * matrices and explicit Gell-Mann generators:
 *   S_G                   Sec. 1, text after eq. (1)
 *   M                     Sec. 1, eq. (2)
 *   |W^-1 phi|^2 actions  Sec. 1, eq. (3) ("factorpf")
 *   W1, slabs, red/black  Sec. 1, block decomposition in x0 only
 *   T_U, T_P, LF, SW      Sec. 2, eqs. (4)-(7)
 *   recursive levels      Sec. 2, eqs. (iterateLF), (iterateSW)
 *   x0 shift              end of Sec. 2
 * Readings where the paper is silent (each one restated at its function):
 *   chiral gamma basis; fermion phase bc_t on the x0 wrap; the boundary
 *   operator R = Pi (1 - C A^-1 B D^-1) Pi obtained by block LU of eq. (2)
 *   (the paper cites Luscher's eqs. (3.12)-(3.13) without restating them);
 *   momenta P = sum_a p^a T^a with H = 1/2 sum p^2; Philox4x32-10 streams.
 *
 * The hopping loops and the site loops of the bilinear force are
 * parallelised with OpenMP over independent output sites only; sums are
 * serial, so results do not depend on the thread count.
 */
#include "lqcd_oracle.h"
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int L[4];
    int l0, bc_t, nb;
    int V, Vh, V3;
    int l0s, nbs; /* iterated decomposition: sub-slabs of thickness l0s = l0/2 */
} G;

int lqo_geom_check(const lqo_geom* g)
{
    for (int mu = 0; mu < 4; ++mu)
        if (g->L[mu] < 2 || (g->L[mu] & 1)) return -2;
    if (g->l0 < 1 || g->L[0] % (2 * g->l0)) return -2;
    if (g->bc_t != 1 && g->bc_t != -1) return -1;
    if (g->l0s && (g->l0s < 1 || g->l0 != 2 * g->l0s)) return -2;
    return 0;
}

static G mkg(const lqo_geom* in)
{
    G g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = in->L[mu];
    g.l0 = in->l0;
    g.bc_t = in->bc_t;
    g.V3 = g.L[1] * g.L[2] * g.L[3];
    g.V = g.L[0] * g.V3;
    g.Vh = g.V / 2;
    g.nb = g.L[0] / g.l0;
    g.l0s = in->l0s;
    g.nbs = g.l0s ? g.L[0] / g.l0s : 0;
    return g;
}

static int lexi(const G* g, const int x[4])
{
    return ((x[0] * g->L[1] + x[1]) * g->L[2] + x[2]) * g->L[3] + x[3];
}

static int site_of(const G* g, const int x[4])
{
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    return p * g->Vh + lexi(g, x) / 2;
}

static void coords_of(const G* g, int s, int x[4])
{
    int p = s / g->Vh, h = s % g->Vh;
    for (int c = 0; c < 2; ++c) {
        int lex = 2 * h + c;
        x[3] = lex % g->L[3]; lex /= g->L[3];
        x[2] = lex % g->L[2]; lex /= g->L[2];
        x[1] = lex % g->L[1]; lex /= g->L[1];
        x[0] = lex;
        if (((x[0] + x[1] + x[2] + x[3]) & 1) == p) return;
    }
}

/* neighbour x + dir*mu_hat with periodic wrap; *ph is the fermion phase of
 * the hop (bc_t when the x0 hop wraps, 1 otherwise) */
static int shift_of(const G* g, int s, int mu, int dir, double* ph)
{
    int x[4];
    coords_of(g, s, x);
    *ph = 1.0;
    x[mu] += dir;
    if (x[mu] == g->L[mu]) { x[mu] = 0; if (mu == 0) *ph = g->bc_t; }
    if (x[mu] < 0) { x[mu] = g->L[mu] - 1; if (mu == 0) *ph = g->bc_t; }
    return site_of(g, x);
}

static int slab_of(const G* g, int s)
{
    int x[4];
    coords_of(g, s, x);
    return x[0] / g->l0;
}

/* neighbour / phase / slab tables of the last geometry used, filled from
 * shift_of and slab_of above (only a cache of their values) */
static int sub_of(const G* g, int s)
{
    int x[4];
    coords_of(g, s, x);
    return g->l0s ? x[0] / g->l0s : 0;
}

static struct {
    int L[4], l0, bc_t, V, l0s;
    int* nbr;     /* [s][mu][dir 0:+,1:-] */
    double* ph;
    int* slab;
    int* sub;
} TAB = {{0, 0, 0, 0}, 0, 0, 0, 0, NULL, NULL, NULL, NULL};

static void tables(const G* g)
{
    if (TAB.nbr && TAB.V == g->V && TAB.l0 == g->l0 && TAB.bc_t == g->bc_t && TAB.l0s == g->l0s &&
        !memcmp(TAB.L, g->L, sizeof(TAB.L)))
        return;
    free(TAB.nbr); free(TAB.ph); free(TAB.slab); free(TAB.sub);
    TAB.nbr = malloc(sizeof(int) * (size_t)g->V * 8);
    TAB.ph = malloc(sizeof(double) * (size_t)g->V * 8);
    TAB.slab = malloc(sizeof(int) * (size_t)g->V);
    TAB.sub = malloc(sizeof(int) * (size_t)g->V);
    for (int s = 0; s < g->V; ++s) {
        TAB.slab[s] = slab_of(g, s);
        TAB.sub[s] = sub_of(g, s);
        for (int mu = 0; mu < 4; ++mu)
            for (int d = 0; d < 2; ++d)
                TAB.nbr[(s * 4 + mu) * 2 + d] = shift_of(g, s, mu, d ? -1 : +1, &TAB.ph[(s * 4 + mu) * 2 + d]);
    }
    memcpy(TAB.L, g->L, sizeof(TAB.L));
    TAB.V = g->V; TAB.l0 = g->l0; TAB.bc_t = g->bc_t; TAB.l0s = g->l0s;
}

/* index maps, each of length V in checkerboard site order:
 *  0 lex, 1 parity, 2 slab, 3 colour, 4..7 forward neighbours (mu=0..3),
 *  8..11 backward neighbours, 12 face flags (1 first slice of its slab,
 *  2 last slice), 13 boundary-coordinate site index for black face sites
 *  ((j*2+f)*V3 + lex3 with f the first matching face) or -1 */
void lqo_index_maps(const lqo_geom* gi, int32_t* maps)
{
    G g = mkg(gi);
    for (int s = 0; s < g.V; ++s) {
        int x[4];
        coords_of(&g, s, x);
        int slab = x[0] / g.l0;
        maps[0 * g.V + s] = lexi(&g, x);
        maps[1 * g.V + s] = (x[0] + x[1] + x[2] + x[3]) & 1;
        maps[2 * g.V + s] = slab;
        maps[3 * g.V + s] = slab % 2;
        for (int mu = 0; mu < 4; ++mu) {
            double ph;
            maps[(4 + mu) * g.V + s] = shift_of(&g, s, mu, +1, &ph);
            maps[(8 + mu) * g.V + s] = shift_of(&g, s, mu, -1, &ph);
        }
        int first = (x[0] == slab * g.l0);
        int last = (x[0] == slab * g.l0 + g.l0 - 1);
        maps[12 * g.V + s] = first + 2 * last;
        int lex3 = (x[1] * g.L[2] + x[2]) * g.L[3] + x[3];
        int b = -1;
        if (slab % 2 == 1 && (first || last)) {
            int f = first ? 0 : 1;
            b = ((slab / 2) * 2 + f) * g.V3 + lex3;
        }
        maps[13 * g.V + s] = b;
    }
}

/* ------------------------------------------------------------------ */
/* gamma matrices (chiral basis, hermitian, Euclidean), 2x2 blocks:    */
/*   gamma_0 = [[0,-1],[-1,0]],  gamma_k = [[0,-i s_k],[i s_k,0]]      */
/* ------------------------------------------------------------------ */
static cplx GAM[5][4][4];   /* gamma_0..gamma_3, gamma_5 */
static cplx PM[4][4][4];    /* 1 - gamma_mu */
static cplx PP[4][4][4];    /* 1 + gamma_mu */
static int gam_ready = 0;

static void init_gamma(void)
{
    if (gam_ready) return;
    cplx sig[4][2][2] = {
        {{1, 0}, {0, 1}},
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAM, 0, sizeof(GAM));
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            GAM[0][a][2 + b] = -sig[0][a][b];
            GAM[0][2 + a][b] = -sig[0][a][b];
            for (int k = 1; k < 4; ++k) {
                GAM[k][a][2 + b] = -I * sig[k][a][b];
                GAM[k][2 + a][b] = I * sig[k][a][b];
            }
        }
    /* gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 */
    cplx t1[4][4], t2[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            t1[a][b] = 0;
            for (int c = 0; c < 4; ++c) t1[a][b] += GAM[0][a][c] * GAM[1][c][b];
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            t2[a][b] = 0;
            for (int c = 0; c < 4; ++c) t2[a][b] += t1[a][c] * GAM[2][c][b];
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            GAM[4][a][b] = 0;
            for (int c = 0; c < 4; ++c) GAM[4][a][b] += t2[a][c] * GAM[3][c][b];
        }
    for (int mu = 0; mu < 4; ++mu)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                PM[mu][a][b] = (a == b ? 1.0 : 0.0) - GAM[mu][a][b];
                PP[mu][a][b] = (a == b ? 1.0 : 0.0) + GAM[mu][a][b];
            }
    gam_ready = 1;
}

void lqo_gamma(double* out)
{
    init_gamma();
    memcpy(out, GAM, sizeof(GAM));
}

/* Gell-Mann generators T^a = lambda^a / 2 */
static cplx TG[8][3][3];
static int tg_ready = 0;

static void init_generators(void)
{
    if (tg_ready) return;
    memset(TG, 0, sizeof(TG));
    const double h = 0.5;
    TG[0][0][1] = h;  TG[0][1][0] = h;
    TG[1][0][1] = -I * h; TG[1][1][0] = I * h;
    TG[2][0][0] = h;  TG[2][1][1] = -h;
    TG[3][0][2] = h;  TG[3][2][0] = h;
    TG[4][0][2] = -I * h; TG[4][2][0] = I * h;
    TG[5][1][2] = h;  TG[5][2][1] = h;
    TG[6][1][2] = -I * h; TG[6][2][1] = I * h;
    TG[7][0][0] = h / sqrt(3.0); TG[7][1][1] = h / sqrt(3.0);
    TG[7][2][2] = -2.0 * h / sqrt(3.0);
    tg_ready = 1;
}

/* ------------------------------------------------------------------ */
/* small 3x3 helpers                                                   */
/* ------------------------------------------------------------------ */
static const cplx* link(const G* g, const cplx* U, int mu, int s)
{
    return U + ((size_t)mu * g->V + s) * 9;
}

static void mm(const cplx* a, const cplx* b, cplx* c) /* c = a b */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx t = 0;
            for (int k = 0; k < 3; ++k) t += a[i * 3 + k] * b[k * 3 + j];
            c[i * 3 + j] = t;
        }
}

static void dag(const cplx* a, cplx* b) /* b = a^dagger */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[i * 3 + j] = conj(a[j * 3 + i]);
}

/* ------------------------------------------------------------------ */
/* the hopping term of eq. (2)                                         */
/*  (H psi)(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu)                     */
/*                    + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)              */
/*  M = 1 - kappa H.  H^dag swaps the two projectors.                  */
/*  mode ALL: every hop; INTRA: hops inside one slab (W1);             */
/*  CROSS: hops between different slabs (the blocks B, C of M).        */
/* ------------------------------------------------------------------ */
/* which hops a mode keeps: ALL; INTRA / CROSS: inside one slab / between
 * slabs; INTRA2: inside one sub-slab (W2); CROSS2: between the two
 * sub-slabs of one slab (the blocks B2, C2 of W1) */
static int hop_in(const G* g, int s, int t, int mode)
{
    (void)g;
    if (mode == LQO_HOP_ALL) return 1;
    int same = TAB.slab[s] == TAB.slab[t];
    if (mode == LQO_HOP_INTRA) return same;
    if (mode == LQO_HOP_CROSS) return !same;
    int same2 = TAB.sub[s] == TAB.sub[t];
    if (mode == LQO_HOP_INTRA2) return same2;
    return same && !same2;
}

static void hop_c(const G* g, const cplx* U, const cplx* in, cplx* out, int mode, int dagger)
{
    init_gamma();
    tables(g);
#pragma omp parallel for schedule(static) if (g->V >= 4096)
    for (int s = 0; s < g->V; ++s) {
        cplx acc[4][3];
        memset(acc, 0, sizeof(acc));
        for (int mu = 0; mu < 4; ++mu) {
            for (int dir = +1; dir >= -1; dir -= 2) {
                int k = (s * 4 + mu) * 2 + (dir > 0 ? 0 : 1);
                double ph = TAB.ph[k];
                int t = TAB.nbr[k];
                if (!hop_in(g, s, t, mode)) continue;
                cplx u[9];
                if (dir > 0) memcpy(u, link(g, U, mu, s), sizeof(u));
                else dag(link(g, U, mu, t), u);
                const cplx* psi = in + (size_t)t * 12;
                cplx uv[4][3];
                for (int sp = 0; sp < 4; ++sp)
                    for (int i = 0; i < 3; ++i) {
                        cplx v = 0;
                        for (int j = 0; j < 3; ++j) v += u[i * 3 + j] * psi[sp * 3 + j];
                        uv[sp][i] = v;
                    }
                int minus = (dir > 0) != (dagger != 0); /* forward: 1-g, dagger flips */
                cplx (*P)[4] = minus ? PM[mu] : PP[mu];
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) {
                        if (P[a][b] == 0) continue;
                        for (int i = 0; i < 3; ++i) acc[a][i] += ph * P[a][b] * uv[b][i];
                    }
            }
        }
        memcpy(out + (size_t)s * 12, acc, sizeof(acc));
    }
}

void lqo_hop(const lqo_geom* gi, const double* U, const double* in, double* out, int mode, int dagger)
{
    G g = mkg(gi);
    hop_c(&g, (const cplx*)U, (const cplx*)in, (cplx*)out, mode, dagger);
}

static void apply_1mkH(const G* g, const cplx* U, double kappa, const cplx* in, cplx* out,
                       int mode, int dagger)
{
    hop_c(g, U, in, out, mode, dagger);
    for (size_t i = 0; i < (size_t)g->V * 12; ++i) out[i] = in[i] - kappa * out[i];
}

void lqo_apply_M(const lqo_geom* gi, const double* U, double kappa, const double* in,
                 double* out, int dagger)
{
    G g = mkg(gi);
    apply_1mkH(&g, (const cplx*)U, kappa, (const cplx*)in, (cplx*)out, LQO_HOP_ALL, dagger);
}

void lqo_apply_W1(const lqo_geom* gi, const double* U, double kappa, const double* in,
                  double* out, int dagger)
{
    G g = mkg(gi);
    apply_1mkH(&g, (const cplx*)U, kappa, (const cplx*)in, (cplx*)out, LQO_HOP_INTRA, dagger);
}

/* even-odd pieces: out_p = H_{p,1-p} in_{1-p} (full hop on a field that is
 * zero on parity p, restricted to parity p) */
void lqo_dslash_eo(const lqo_geom* gi, const double* U, const double* in_half,
                   double* out_half, int parity, int dagger)
{
    G g = mkg(gi);
    size_t n = (size_t)g.V * 12;
    cplx* full = calloc(n, sizeof(cplx));
    cplx* res = calloc(n, sizeof(cplx));
    memcpy(full + (size_t)(1 - parity) * g.Vh * 12, in_half, sizeof(cplx) * g.Vh * 12);
    hop_c(&g, (const cplx*)U, full, res, LQO_HOP_ALL, dagger);
    memcpy(out_half, res + (size_t)parity * g.Vh * 12, sizeof(cplx) * g.Vh * 12);
    free(full);
    free(res);
}

/* Mhat = 1 - kappa^2 H_eo H_oe on even sites (Sec. 1, even-odd form used
 * for W2 and for the global solver of S4) */
void lqo_mhat(const lqo_geom* gi, const double* U, double kappa, const double* in_e,
              double* out_e, int dagger)
{
    G g = mkg(gi);
    size_t nh = (size_t)g.Vh * 12;
    double* t_o = malloc(sizeof(cplx) * nh);
    double* t_e = malloc(sizeof(cplx) * nh);
    lqo_dslash_eo(gi, U, in_e, t_o, 1, dagger);
    lqo_dslash_eo(gi, U, t_o, t_e, 0, dagger);
    const cplx* a = (const cplx*)in_e;
    cplx* o = (cplx*)out_e;
    cplx* te = (cplx*)t_e;
    for (size_t i = 0; i < nh; ++i) o[i] = a[i] - kappa * kappa * te[i];
    free(t_o);
    free(t_e);
}

/* W1 applied on the slabs of one colour (-1: all slabs); zero elsewhere */
void lqo_block_dslash(const lqo_geom* gi, const double* U, double kappa, const double* in,
                      double* out, int colour, int dagger)
{
    G g = mkg(gi);
    apply_1mkH(&g, (const cplx*)U, kappa, (const cplx*)in, (cplx*)out, LQO_HOP_INTRA, dagger);
    cplx* o = (cplx*)out;
    for (int s = 0; s < g.V; ++s)
        if (colour >= 0 && slab_of(&g, s) % 2 != colour)
            memset(o + (size_t)s * 12, 0, sizeof(cplx) * 12);
}

/* ------------------------------------------------------------------ */
/* CG on the normal equations (textbook CGNR): solves A x = b          */
/* ------------------------------------------------------------------ */
typedef void (*opfn)(void* ctx, const cplx* in, cplx* out, int dagger);

static double nrm2(const cplx* a, size_t n)
{
    double s = 0;
    for (size_t i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static int cgnr(opfn A, void* ctx, size_t n, cplx* x, const cplx* b, double tol, int maxit,
                int* iters)
{
    cplx* r = malloc(sizeof(cplx) * n);
    cplx* z = malloc(sizeof(cplx) * n);
    cplx* p = malloc(sizeof(cplx) * n);
    cplx* w = malloc(sizeof(cplx) * n);
    double bb = nrm2(b, n);
    int k = 0, status = 0;
    memset(x, 0, sizeof(cplx) * n);
    if (bb == 0) goto done;
    memcpy(r, b, sizeof(cplx) * n);
    A(ctx, r, z, 1);
    memcpy(p, z, sizeof(cplx) * n);
    double zz = nrm2(z, n);
    for (k = 0; k < maxit; ++k) {
        if (nrm2(r, n) <= tol * tol * bb) break;
        A(ctx, p, w, 0);
        double ww = nrm2(w, n);
        double alpha = zz / ww;
        for (size_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
        A(ctx, r, z, 1);
        double zz2 = nrm2(z, n);
        double beta = zz2 / zz;
        zz = zz2;
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    /* true residual */
    A(ctx, x, w, 0);
    for (size_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    double lim = 10.0 * tol > 1e-13 ? 10.0 * tol : 1e-13;
    if (!(nrm2(r, n) <= lim * lim * bb)) status = -3;
done:
    if (iters) *iters = k;
    free(r); free(z); free(p); free(w);
    return status;
}


/* operator context: A = 1 - kappa H_mode, or its adjoint when adj = 1 */
typedef struct { const G* g; const cplx* U; double kappa; int mode; int adj; } opctx;

static void op_1mkH(void* c, const cplx* in, cplx* out, int dagger)
{
    opctx* o = (opctx*)c;
    apply_1mkH(o->g, o->U, o->kappa, in, out, o->mode, dagger ^ o->adj);
}

static void keep_colour(const G* g, cplx* f, int colour)
{
    if (colour < 0) return;
    for (int s = 0; s < g->V; ++s)
        if (slab_of(g, s) % 2 != colour) memset(f + (size_t)s * 12, 0, sizeof(cplx) * 12);
}

/* x = W1^-1 b on the slabs of one colour (-1: all).  W1 is block diagonal,
 * so the full-lattice solve with the source kept on those slabs yields the
 * block solutions there and zero elsewhere.  dagger: W1^dag x = b. */
static int block_solve_c(const G* g, const cplx* U, double kappa, cplx* x, const cplx* b,
                         int colour, int dagger, double tol, int maxit, int* iters)
{
    size_t n = (size_t)g->V * 12;
    cplx* bb = malloc(sizeof(cplx) * n);
    memcpy(bb, b, sizeof(cplx) * n);
    keep_colour(g, bb, colour);
    opctx o = {g, U, kappa, LQO_HOP_INTRA, dagger};
    int st = cgnr(op_1mkH, &o, n, x, bb, tol, maxit, iters);
    free(bb);
    return st;
}

int lqo_block_solve(const lqo_geom* gi, const double* U, double kappa, double* x,
                    const double* b, int colour, int dagger, double tol, int maxit, int* iters)
{
    G g = mkg(gi);
    return block_solve_c(&g, (const cplx*)U, kappa, (cplx*)x, (const cplx*)b, colour, dagger,
                         tol, maxit, iters);
}

static int solve_M_c(const G* g, const cplx* U, double kappa, cplx* x, const cplx* b,
                     int dagger, double tol, int maxit, int* iters)
{
    opctx o = {g, U, kappa, LQO_HOP_ALL, dagger};
    return cgnr(op_1mkH, &o, (size_t)g->V * 12, x, b, tol, maxit, iters);
}

int lqo_solve_M(const lqo_geom* gi, const double* U, double kappa, double* x, const double* b,
                int dagger, double tol, int maxit, int* iters)
{
    G g = mkg(gi);
    return solve_M_c(&g, (const cplx*)U, kappa, (cplx*)x, (const cplx*)b, dagger, tol, maxit, iters);
}

/* ------------------------------------------------------------------ */
/* boundary space of the black slabs (Sec. 1: the pseudo-fermion of    */
/* det^2(W1^-1 M) lives on the boundaries of the black blocks, with    */
/* half the spin components).  Orthonormal spin bases:                  */
/*   face 0 (first slice), range (1+g0)/2: (e_i - e_{i+2})/sqrt2        */
/*   face 1 (last slice),  range (1-g0)/2: (e_i + e_{i+2})/sqrt2        */
/* ------------------------------------------------------------------ */
static double BASIS[2][2][4]; /* [face][i][spin] */
static int basis_ready = 0;

static void init_basis(void)
{
    if (basis_ready) return;
    memset(BASIS, 0, sizeof(BASIS));
    const double r = 1.0 / sqrt(2.0);
    for (int i = 0; i < 2; ++i) {
        BASIS[0][i][i] = r; BASIS[0][i][i + 2] = -r;
        BASIS[1][i][i] = r; BASIS[1][i][i + 2] = r;
    }
    basis_ready = 1;
}

int lqo_nbnd(const lqo_geom* gi)
{
    G g = mkg(gi);
    return (g.nb / 2) * 2 * g.V3 * 6;
}

/* site of black slab ordinal j, face f, spatial lex index lex3 */
static int face_site(const G* g, int j, int f, int lex3)
{
    int k = 2 * j + 1;
    int x[4];
    x[0] = k * g->l0 + (f ? g->l0 - 1 : 0);
    x[3] = lex3 % g->L[3];
    x[2] = (lex3 / g->L[3]) % g->L[2];
    x[1] = lex3 / (g->L[3] * g->L[2]);
    return site_of(g, x);
}

/* full = E^dag coords (full-lattice spinor, zero off the black faces) */
static void embed_c(const G* g, const cplx* c, cplx* full)
{
    init_basis();
    memset(full, 0, sizeof(cplx) * (size_t)g->V * 12);
    for (int j = 0; j < g->nb / 2; ++j)
        for (int f = 0; f < 2; ++f)
            for (int l3 = 0; l3 < g->V3; ++l3) {
                int s = face_site(g, j, f, l3);
                const cplx* cc = c + ((size_t)(j * 2 + f) * g->V3 + l3) * 6;
                for (int sp = 0; sp < 4; ++sp)
                    for (int col = 0; col < 3; ++col)
                        for (int i = 0; i < 2; ++i)
                            full[(size_t)s * 12 + sp * 3 + col] += BASIS[f][i][sp] * cc[i * 3 + col];
            }
}

/* coords = E full (orthogonal projection onto the black-face subspace) */
static void project_c(const G* g, const cplx* full, cplx* c)
{
    init_basis();
    for (int j = 0; j < g->nb / 2; ++j)
        for (int f = 0; f < 2; ++f)
            for (int l3 = 0; l3 < g->V3; ++l3) {
                int s = face_site(g, j, f, l3);
                cplx* cc = c + ((size_t)(j * 2 + f) * g->V3 + l3) * 6;
                for (int i = 0; i < 2; ++i)
                    for (int col = 0; col < 3; ++col) {
                        cplx v = 0;
                        for (int sp = 0; sp < 4; ++sp)
                            v += BASIS[f][i][sp] * full[(size_t)s * 12 + sp * 3 + col];
                        cc[i * 3 + col] = v;
                    }
            }
}

void lqo_embed_boundary(const lqo_geom* gi, const double* coords, double* full)
{
    G g = mkg(gi);
    embed_c(&g, (const cplx*)coords, (cplx*)full);
}

void lqo_project_boundary(const lqo_geom* gi, const double* full, double* coords)
{
    G g = mkg(gi);
    project_c(&g, (const cplx*)full, (cplx*)coords);
}

/* ------------------------------------------------------------------ */
/* boundary operator from block LU of eq. (2), sites ordered red|black: */
/*   M = [[A, B], [C, D]],  W1 = diag(A, D),  B, C = -kappa H_cross     */
/*   det M = det W1 det(1 - C A^-1 B D^-1) = det W1 det R,              */
/*   R = E (1 - C A^-1 B D^-1) E^dag   on the black-face space.         */
/* R^-1 either by solving R itself (route 0) or, since                  */
/* (1 - C A^-1 B D^-1)^-1 = D (M^-1)_bb, as E D (M^-1)_bb E^dag (1).    */
/* ------------------------------------------------------------------ */
typedef struct { const G* g; const cplx* U; double kappa; double tol; int maxit; int status; } rctx;

static void schur_R_c(rctx* r, const cplx* in, cplx* out, int dagger)
{
    const G* g = r->g;
    size_t n = (size_t)g->V * 12;
    int nbnd = (g->nb / 2) * 2 * g->V3 * 6;
    cplx* e = malloc(sizeof(cplx) * n);
    cplx* y = malloc(sizeof(cplx) * n);
    cplx* z = malloc(sizeof(cplx) * n);
    embed_c(g, in, e);
    if (!dagger) {
        /* y = D^-1 e; z = B y; y = A^-1 z; z = C y */
        r->status |= block_solve_c(g, r->U, r->kappa, y, e, 1, 0, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS, 0);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve_c(g, r->U, r->kappa, y, z, 0, 0, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS, 0);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
    } else {
        /* R^dag = E (1 - D^-dag B^dag A^-dag C^dag) E^dag */
        hop_c(g, r->U, e, z, LQO_HOP_CROSS, 1);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve_c(g, r->U, r->kappa, y, z, 0, 1, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS, 1);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve_c(g, r->U, r->kappa, y, z, 1, 1, r->tol, r->maxit, NULL);
        memcpy(z, y, sizeof(cplx) * n);
    }
    cplx* pz = malloc(sizeof(cplx) * nbnd);
    project_c(g, z, pz);
    for (int i = 0; i < nbnd; ++i) out[i] = in[i] - pz[i];
    free(pz); free(e); free(y); free(z);
}

typedef struct { rctx* r; int adj; } rctx_adj;

static void op_R_adj(void* c, const cplx* in, cplx* out, int dagger)
{
    rctx_adj* ra = (rctx_adj*)c;
    schur_R_c(ra->r, in, out, dagger ^ ra->adj);
}

static int schur_c(const G* g, const cplx* U, double kappa, cplx* out, const cplx* in, int op,
                   int route, double tol, int maxit)
{
    size_t n = (size_t)g->V * 12;
    int nbnd = (g->nb / 2) * 2 * g->V3 * 6;
    /* the inner block solves are taken much tighter than the outer one */
    rctx r = {g, U, kappa, tol * 1e-3 > 1e-14 ? tol * 1e-3 : 1e-14, maxit, 0};
    if (op == LQO_R || op == LQO_RDAG) {
        schur_R_c(&r, in, out, op == LQO_RDAG);
        return r.status;
    }
    int dagger = (op == LQO_RINVDAG);
    if (route == 0) {
        rctx_adj ra = {&r, dagger};
        int st = cgnr(op_R_adj, &ra, nbnd, out, in, tol, maxit, NULL);
        return st | r.status;
    }
    cplx* e = malloc(sizeof(cplx) * n);
    cplx* psi = malloc(sizeof(cplx) * n);
    cplx* w = malloc(sizeof(cplx) * n);
    int st;
    embed_c(g, in, e);
    if (!dagger) {
        /* R^-1 = E D (M^-1)_bb E^dag */
        st = solve_M_c(g, U, kappa, psi, e, 0, tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14, maxit, NULL);
        keep_colour(g, psi, 1);
        apply_1mkH(g, U, kappa, psi, w, LQO_HOP_INTRA, 0);
        keep_colour(g, w, 1);
    } else {
        /* R^-dag = E (M^-dag)_bb D^dag E^dag */
        apply_1mkH(g, U, kappa, e, w, LQO_HOP_INTRA, 1);
        keep_colour(g, w, 1);
        st = solve_M_c(g, U, kappa, psi, w, 1, tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14, maxit, NULL);
        memcpy(w, psi, sizeof(cplx) * n);
        keep_colour(g, w, 1);
    }
    project_c(g, w, out);
    free(e); free(psi); free(w);
    return st;
}

int lqo_schur(const lqo_geom* gi, const double* U, double kappa, double* out, const double* in,
              int op, int route, double tol, int maxit)
{
    G g = mkg(gi);
    return schur_c(&g, (const cplx*)U, kappa, (cplx*)out, (const cplx*)in, op, route, tol, maxit);
}

/* ------------------------------------------------------------------ */
/* forces                                                              */
/* For a link U_mu(x) moved along T^a, delta U = i w T^a U.  The        */
/* derivative of 2 Re <a, H b> along that direction is                 */
/*  2 Re[ a(x)^dag (1-g_mu) (iT^a U) b(x+mu)                            */
/*      + a(x+mu)^dag (1+g_mu) (iT^a U)^dag b(x) ]   (times the phase). */
/* mask: ALL links, INTRA (both ends in one slab) or CROSS.            */
/* F[mu][x][a] += coef * derivative                                     */
/* ------------------------------------------------------------------ */
static void bilinear_c(const G* g, const cplx* U, const cplx* a, const cplx* b, int mask,
                       double coef, double* F)
{
    init_gamma();
    init_generators();
    tables(g);
#pragma omp parallel for schedule(static) if (g->V >= 4096)
    for (int s = 0; s < g->V; ++s) {
        for (int mu = 0; mu < 4; ++mu) {
            double ph = TAB.ph[(s * 4 + mu) * 2];
            int t = TAB.nbr[(s * 4 + mu) * 2];
            if (!hop_in(g, s, t, mask)) continue;
            const cplx* u = link(g, U, mu, s);
            for (int c = 0; c < 8; ++c) {
                cplx du[9], dd[9];
                mm(&TG[c][0][0], u, du);
                for (int i = 0; i < 9; ++i) du[i] *= I;
                dag(du, dd);
                cplx tot = 0;
                /* a(x)^dag (1-g) du b(x+mu) */
                for (int sa = 0; sa < 4; ++sa)
                    for (int sb = 0; sb < 4; ++sb) {
                        if (PM[mu][sa][sb] == 0 && PP[mu][sa][sb] == 0) continue;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) {
                                tot += conj(a[(size_t)s * 12 + sa * 3 + i]) * PM[mu][sa][sb] *
                                       du[i * 3 + j] * b[(size_t)t * 12 + sb * 3 + j];
                                tot += conj(a[(size_t)t * 12 + sa * 3 + i]) * PP[mu][sa][sb] *
                                       dd[i * 3 + j] * b[(size_t)s * 12 + sb * 3 + j];
                            }
                    }
                F[((size_t)mu * g->V + s) * 8 + c] += coef * 2.0 * creal(ph * tot);
            }
        }
    }
}

void lqo_bilinear(const lqo_geom* gi, const double* U, const double* a, const double* b,
                  int mask, double coef, double* F)
{
    G g = mkg(gi);
    bilinear_c(&g, (const cplx*)U, (const cplx*)a, (const cplx*)b, mask, coef, F);
}

/* S_W1 = |W1^-1 phi|^2.  dS = -2 Re <xi, dW1 eta>, eta = W1^-1 phi,
 * xi = W1^-dag eta, dW1 = -kappa dH on intra-slab links. */
int lqo_pf_w1(const lqo_geom* gi, const double* Ud, double kappa, const double* phi, double* F,
              double* S, double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    size_t n = (size_t)g.V * 12;
    cplx* eta = malloc(sizeof(cplx) * n);
    cplx* xi = malloc(sizeof(cplx) * n);
    int st = block_solve_c(&g, U, kappa, eta, (const cplx*)phi, -1, 0, tol, maxit, NULL);
    if (S) *S = nrm2(eta, n);
    if (F) {
        st |= block_solve_c(&g, U, kappa, xi, eta, -1, 1, tol, maxit, NULL);
        bilinear_c(&g, U, xi, eta, LQO_HOP_INTRA, kappa, F);
    }
    free(eta); free(xi);
    return st;
}

/* S_R = |R^-1 phi|^2.  dS = -2 Re <xi, dR eta> with eta = R^-1 phi,
 * xi = R^-dag eta and dR = -E d(C A^-1 B D^-1) E^dag:
 *  d(CA^-1BD^-1) = dC A^-1BD^-1 - CA^-1 dA A^-1BD^-1 + CA^-1 dB D^-1
 *                  - CA^-1BD^-1 dD D^-1,
 * every term one bilinear of dH between block-solved vectors. */
int lqo_pf_schur(const lqo_geom* gi, const double* Ud, double kappa, const double* phi,
                 double* F, double* S, int route, double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    size_t n = (size_t)g.V * 12;
    int nbnd = (g.nb / 2) * 2 * g.V3 * 6;
    cplx* eta = malloc(sizeof(cplx) * nbnd);
    cplx* xi = malloc(sizeof(cplx) * nbnd);
    int st = schur_c(&g, U, kappa, eta, (const cplx*)phi, LQO_RINV, route, tol, maxit);
    if (S) *S = nrm2(eta, nbnd);
    if (F) {
        double it = tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14;
        st |= schur_c(&g, U, kappa, xi, eta, LQO_RINVDAG, route, tol, maxit);
        cplx* et = malloc(sizeof(cplx) * n);
        cplx* xt = malloc(sizeof(cplx) * n);
        cplx* y1 = malloc(sizeof(cplx) * n);
        cplx* y2 = malloc(sizeof(cplx) * n);
        cplx* z1 = malloc(sizeof(cplx) * n);
        cplx* z2 = malloc(sizeof(cplx) * n);
        cplx* w = malloc(sizeof(cplx) * n);
        embed_c(&g, eta, et);
        embed_c(&g, xi, xt);
        /* y1 = D^-1 eta~ ; y2 = A^-1 B y1 */
        st |= block_solve_c(&g, U, kappa, y1, et, 1, 0, it, maxit, NULL);
        hop_c(&g, U, y1, w, LQO_HOP_CROSS, 0);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve_c(&g, U, kappa, y2, w, 0, 0, it, maxit, NULL);
        /* z1 = A^-dag C^dag xi~ ; z2 = D^-dag B^dag z1 */
        hop_c(&g, U, xt, w, LQO_HOP_CROSS, 1);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve_c(&g, U, kappa, z1, w, 0, 1, it, maxit, NULL);
        hop_c(&g, U, z1, w, LQO_HOP_CROSS, 1);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve_c(&g, U, kappa, z2, w, 1, 1, it, maxit, NULL);
        /* dS = 2 Re[<xi~, dC y2> - <z1, dA y2> + <z1, dB y1> - <z2, dD y1>],
         * dC = dB = -kappa dH (cross links), dA = dD = -kappa dH (intra) */
        bilinear_c(&g, U, xt, y2, LQO_HOP_CROSS, -kappa, F);
        bilinear_c(&g, U, z1, y2, LQO_HOP_INTRA, +kappa, F);
        bilinear_c(&g, U, z1, y1, LQO_HOP_CROSS, -kappa, F);
        bilinear_c(&g, U, z2, y1, LQO_HOP_INTRA, +kappa, F);
        free(et); free(xt); free(y1); free(y2); free(z1); free(z2); free(w);
    }
    free(eta); free(xi);
    return st;
}

/* ------------------------------------------------------------------ */
/* iterated decomposition (Sec. 1: l0^(2) = l0^(1)/2, W2 = M restricted */
/* to the sub-slabs).  With the sites of W1 ordered red|black by the     */
/* sub-slab colour, W1 = [[A2, B2], [C2, D2]], W2 = diag(A2, D2), and     */
/* B2, C2 = -kappa H on the hops between the two sub-slabs of one slab.  */
/* Block LU: det W1 = det W2 det R2 with                                  */
/*   R2 = E2 (1 - C2 A2^-1 B2 D2^-1) E2^dag                               */
/* on the range of C2: the first time slice of each black sub-slab,      */
/* spin projected with (1+g0)/2 (its last slice borders the next slab,   */
/* which W1 does not reach).  det M = det R1 det R2 det W2.               */
/* Boundary field layout: [nbs/2][V3][2][3] complex, same spin basis as  */
/* face 0 of the first level.                                             */
/* ------------------------------------------------------------------ */
static void keep_colour2(const G* g, cplx* f, int colour)
{
    if (colour < 0) return;
    for (int s = 0; s < g->V; ++s)
        if (sub_of(g, s) % 2 != colour) memset(f + (size_t)s * 12, 0, sizeof(cplx) * 12);
}

/* x = W2^-1 b on the sub-slabs of one colour (-1: all) */
static int block_solve2_c(const G* g, const cplx* U, double kappa, cplx* x, const cplx* b, int colour,
                          int dagger, double tol, int maxit, int* iters)
{
    size_t n = (size_t)g->V * 12;
    cplx* bb = malloc(sizeof(cplx) * n);
    memcpy(bb, b, sizeof(cplx) * n);
    keep_colour2(g, bb, colour);
    opctx o = {g, U, kappa, LQO_HOP_INTRA2, dagger};
    int st = cgnr(op_1mkH, &o, n, x, bb, tol, maxit, iters);
    free(bb);
    return st;
}

int lqo_block_solve2(const lqo_geom* gi, const double* U, double kappa, double* x, const double* b,
                     int colour, int dagger, double tol, int maxit, int* iters)
{
    G g = mkg(gi);
    if (!g.l0s) return -2;
    return block_solve2_c(&g, (const cplx*)U, kappa, (cplx*)x, (const cplx*)b, colour, dagger, tol, maxit,
                          iters);
}

void lqo_apply_W2(const lqo_geom* gi, const double* U, double kappa, const double* in, double* out,
                  int dagger)
{
    G g = mkg(gi);
    apply_1mkH(&g, (const cplx*)U, kappa, (const cplx*)in, (cplx*)out, LQO_HOP_INTRA2, dagger);
}

int lqo_nbnd2(const lqo_geom* gi)
{
    G g = mkg(gi);
    return (g.nbs / 2) * g.V3 * 6;
}

static int face2_site(const G* g, int j, int lex3)
{
    int x[4];
    x[0] = (2 * j + 1) * g->l0s;
    x[3] = lex3 % g->L[3];
    x[2] = (lex3 / g->L[3]) % g->L[2];
    x[1] = lex3 / (g->L[3] * g->L[2]);
    return site_of(g, x);
}

static void embed2_c(const G* g, const cplx* c, cplx* full)
{
    init_basis();
    memset(full, 0, sizeof(cplx) * (size_t)g->V * 12);
    for (int j = 0; j < g->nbs / 2; ++j)
        for (int l3 = 0; l3 < g->V3; ++l3) {
            int s = face2_site(g, j, l3);
            const cplx* cc = c + ((size_t)j * g->V3 + l3) * 6;
            for (int sp = 0; sp < 4; ++sp)
                for (int col = 0; col < 3; ++col)
                    for (int i = 0; i < 2; ++i)
                        full[(size_t)s * 12 + sp * 3 + col] += BASIS[0][i][sp] * cc[i * 3 + col];
        }
}

static void project2_c(const G* g, const cplx* full, cplx* c)
{
    init_basis();
    for (int j = 0; j < g->nbs / 2; ++j)
        for (int l3 = 0; l3 < g->V3; ++l3) {
            int s = face2_site(g, j, l3);
            cplx* cc = c + ((size_t)j * g->V3 + l3) * 6;
            for (int i = 0; i < 2; ++i)
                for (int col = 0; col < 3; ++col) {
                    cplx v = 0;
                    for (int sp = 0; sp < 4; ++sp) v += BASIS[0][i][sp] * full[(size_t)s * 12 + sp * 3 + col];
                    cc[i * 3 + col] = v;
                }
        }
}

void lqo_embed_boundary2(const lqo_geom* gi, const double* coords, double* full)
{
    G g = mkg(gi);
    embed2_c(&g, (const cplx*)coords, (cplx*)full);
}

void lqo_project_boundary2(const lqo_geom* gi, const double* full, double* coords)
{
    G g = mkg(gi);
    project2_c(&g, (const cplx*)full, (cplx*)coords);
}

static void schur2_R_c(rctx* r, const cplx* in, cplx* out, int dagger)
{
    const G* g = r->g;
    size_t n = (size_t)g->V * 12;
    int nb2 = (g->nbs / 2) * g->V3 * 6;
    cplx* e = malloc(sizeof(cplx) * n);
    cplx* y = malloc(sizeof(cplx) * n);
    cplx* z = malloc(sizeof(cplx) * n);
    embed2_c(g, in, e);
    if (!dagger) {
        /* y = D2^-1 e; z = B2 y; y = A2^-1 z; z = C2 y */
        r->status |= block_solve2_c(g, r->U, r->kappa, y, e, 1, 0, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS2, 0);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve2_c(g, r->U, r->kappa, y, z, 0, 0, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS2, 0);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
    } else {
        hop_c(g, r->U, e, z, LQO_HOP_CROSS2, 1);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve2_c(g, r->U, r->kappa, y, z, 0, 1, r->tol, r->maxit, NULL);
        hop_c(g, r->U, y, z, LQO_HOP_CROSS2, 1);
        for (size_t i = 0; i < n; ++i) z[i] *= -r->kappa;
        r->status |= block_solve2_c(g, r->U, r->kappa, y, z, 1, 1, r->tol, r->maxit, NULL);
        memcpy(z, y, sizeof(cplx) * n);
    }
    cplx* pz = malloc(sizeof(cplx) * nb2);
    project2_c(g, z, pz);
    for (int i = 0; i < nb2; ++i) out[i] = in[i] - pz[i];
    free(pz); free(e); free(y); free(z);
}

static void op_R2_adj(void* c, const cplx* in, cplx* out, int dagger)
{
    rctx_adj* ra = (rctx_adj*)c;
    schur2_R_c(ra->r, in, out, dagger ^ ra->adj);
}

static int schur2_c(const G* g, const cplx* U, double kappa, cplx* out, const cplx* in, int op, int route,
                    double tol, int maxit)
{
    size_t n = (size_t)g->V * 12;
    int nb2 = (g->nbs / 2) * g->V3 * 6;
    rctx r = {g, U, kappa, tol * 1e-3 > 1e-14 ? tol * 1e-3 : 1e-14, maxit, 0};
    if (op == LQO_R || op == LQO_RDAG) {
        schur2_R_c(&r, in, out, op == LQO_RDAG);
        return r.status;
    }
    int dagger = (op == LQO_RINVDAG);
    if (route == 0) {
        rctx_adj ra = {&r, dagger};
        int st = cgnr(op_R2_adj, &ra, nb2, out, in, tol, maxit, NULL);
        return st | r.status;
    }
    /* (1 - C2 A2^-1 B2 D2^-1)^-1 = D2 (W1^-1)_bb on the black sub-slabs */
    cplx* e = malloc(sizeof(cplx) * n);
    cplx* psi = malloc(sizeof(cplx) * n);
    cplx* w = malloc(sizeof(cplx) * n);
    double it = tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14;
    int st;
    embed2_c(g, in, e);
    if (!dagger) {
        st = block_solve_c(g, U, kappa, psi, e, -1, 0, it, maxit, NULL);
        keep_colour2(g, psi, 1);
        apply_1mkH(g, U, kappa, psi, w, LQO_HOP_INTRA2, 0);
        keep_colour2(g, w, 1);
    } else {
        apply_1mkH(g, U, kappa, e, w, LQO_HOP_INTRA2, 1);
        keep_colour2(g, w, 1);
        st = block_solve_c(g, U, kappa, psi, w, -1, 1, it, maxit, NULL);
        memcpy(w, psi, sizeof(cplx) * n);
        keep_colour2(g, w, 1);
    }
    project2_c(g, w, out);
    free(e); free(psi); free(w);
    return st;
}

int lqo_schur2(const lqo_geom* gi, const double* U, double kappa, double* out, const double* in, int op,
               int route, double tol, int maxit)
{
    G g = mkg(gi);
    if (!g.l0s) return -2;
    return schur2_c(&g, (const cplx*)U, kappa, (cplx*)out, (const cplx*)in, op, route, tol, maxit);
}

/* S_W2 = |W2^-1 phi|^2: dS = -2 Re <xi, dW2 eta>, dW2 = -kappa dH (intra sub-slab) */
int lqo_pf_w2(const lqo_geom* gi, const double* Ud, double kappa, const double* phi, double* F, double* S,
              double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    size_t n = (size_t)g.V * 12;
    if (!g.l0s) return -2;
    cplx* eta = malloc(sizeof(cplx) * n);
    cplx* xi = malloc(sizeof(cplx) * n);
    int st = block_solve2_c(&g, U, kappa, eta, (const cplx*)phi, -1, 0, tol, maxit, NULL);
    if (S) *S = nrm2(eta, n);
    if (F) {
        st |= block_solve2_c(&g, U, kappa, xi, eta, -1, 1, tol, maxit, NULL);
        bilinear_c(&g, U, xi, eta, LQO_HOP_INTRA2, kappa, F);
    }
    free(eta); free(xi);
    return st;
}

/* S_R2 = |R2^-1 phi|^2: the four block-LU terms of the first level with
 * (M, W1) replaced by (W1, W2): C2, B2 on the hops between the two
 * sub-slabs of a slab, A2, D2 on the hops inside sub-slabs */
int lqo_pf_schur2(const lqo_geom* gi, const double* Ud, double kappa, const double* phi, double* F,
                  double* S, int route, double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    size_t n = (size_t)g.V * 12;
    if (!g.l0s) return -2;
    int nb2 = (g.nbs / 2) * g.V3 * 6;
    cplx* eta = malloc(sizeof(cplx) * nb2);
    cplx* xi = malloc(sizeof(cplx) * nb2);
    int st = schur2_c(&g, U, kappa, eta, (const cplx*)phi, LQO_RINV, route, tol, maxit);
    if (S) *S = nrm2(eta, nb2);
    if (F) {
        double it = tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14;
        st |= schur2_c(&g, U, kappa, xi, eta, LQO_RINVDAG, route, tol, maxit);
        cplx* et = malloc(sizeof(cplx) * n);
        cplx* xt = malloc(sizeof(cplx) * n);
        cplx* y1 = malloc(sizeof(cplx) * n);
        cplx* y2 = malloc(sizeof(cplx) * n);
        cplx* z1 = malloc(sizeof(cplx) * n);
        cplx* z2 = malloc(sizeof(cplx) * n);
        cplx* w = malloc(sizeof(cplx) * n);
        embed2_c(&g, eta, et);
        embed2_c(&g, xi, xt);
        st |= block_solve2_c(&g, U, kappa, y1, et, 1, 0, it, maxit, NULL);
        hop_c(&g, U, y1, w, LQO_HOP_CROSS2, 0);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve2_c(&g, U, kappa, y2, w, 0, 0, it, maxit, NULL);
        hop_c(&g, U, xt, w, LQO_HOP_CROSS2, 1);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve2_c(&g, U, kappa, z1, w, 0, 1, it, maxit, NULL);
        hop_c(&g, U, z1, w, LQO_HOP_CROSS2, 1);
        for (size_t i = 0; i < n; ++i) w[i] *= -kappa;
        st |= block_solve2_c(&g, U, kappa, z2, w, 1, 1, it, maxit, NULL);
        bilinear_c(&g, U, xt, y2, LQO_HOP_CROSS2, -kappa, F);
        bilinear_c(&g, U, z1, y2, LQO_HOP_INTRA2, +kappa, F);
        bilinear_c(&g, U, z1, y1, LQO_HOP_CROSS2, -kappa, F);
        bilinear_c(&g, U, z2, y1, LQO_HOP_INTRA2, +kappa, F);
        free(et); free(xt); free(y1); free(y2); free(z1); free(z2); free(w);
    }
    free(eta); free(xi);
    return st;
}

/* ------------------------------------------------------------------ */
/* even-odd and mass preconditioning of W2 (Sec. 1).  On the even sites */
/*   W2,eo = 1 - kappa^2 H_eo H_oe   (hops inside the sub-slabs),        */
/*   W3,eo = W2,eo + rho,                                                 */
/* det W2 = det W2,eo (Schur complement of the odd-odd identity block).  */
/* The four-part action represents det^2 W2 by                           */
/*   S2 = |W3,eo W2,eo^-1 phi|^2   (det^2 of W2,eo W3,eo^-1),            */
/*   S1 = |W3,eo^-1 phi|^2         (det^2 of W3,eo),                     */
/* phi an even-site field double[V/2][4][3] complex.                      */
/* ------------------------------------------------------------------ */
/* out_e = (1 + rho) in_e - kappa^2 (H_eo H_oe) in_e; dagger: the adjoint,
 * (1 + rho) - kappa^2 (H^dag)_eo (H^dag)_oe */
static void w3eo_c(const G* g, const cplx* U, double kappa, double rho, const cplx* in, cplx* out, int dagger)
{
    size_t n = (size_t)g->V * 12, nh = (size_t)g->Vh * 12;
    cplx* f = calloc(n, sizeof(cplx));
    cplx* t = malloc(sizeof(cplx) * n);
    memcpy(f, in, sizeof(cplx) * nh);
    hop_c(g, U, f, t, LQO_HOP_INTRA2, dagger); /* odd part: H_oe in */
    memset(t, 0, sizeof(cplx) * nh);
    hop_c(g, U, t, f, LQO_HOP_INTRA2, dagger); /* even part: H_eo H_oe in */
    for (size_t i = 0; i < nh; ++i) out[i] = (1.0 + rho) * in[i] - kappa * kappa * f[i];
    free(f);
    free(t);
}

/* A = W3,eo (adj = 0) or its adjoint (adj = 1) */
typedef struct { const G* g; const cplx* U; double kappa, rho; int adj; } eoctx;

static void op_w3eo(void* c, const cplx* in, cplx* out, int dagger)
{
    eoctx* o = (eoctx*)c;
    w3eo_c(o->g, o->U, o->kappa, o->rho, in, out, dagger ^ o->adj);
}

/* x = W3,eo^-1 b (dagger: W3,eo^-dag b); rho = 0 gives W2,eo */
static int w3eo_solve(const G* g, const cplx* U, double kappa, double rho, cplx* x, const cplx* b, int dagger,
                      double tol, int maxit, int* iters)
{
    eoctx o = {g, U, kappa, rho, dagger};
    return cgnr(op_w3eo, &o, (size_t)g->Vh * 12, x, b, tol, maxit, iters);
}

void lqo_apply_w3eo(const lqo_geom* gi, const double* U, double kappa, double rho, const double* in,
                    double* out, int dagger)
{
    G g = mkg(gi);
    w3eo_c(&g, (const cplx*)U, kappa, rho, (const cplx*)in, (cplx*)out, dagger);
}

int lqo_solve_w3eo(const lqo_geom* gi, const double* U, double kappa, double rho, double* x, const double* b,
                   int dagger, double tol, int maxit, int* iters)
{
    G g = mkg(gi);
    if (!g.l0s) return -2;
    return w3eo_solve(&g, (const cplx*)U, kappa, rho, (cplx*)x, (const cplx*)b, dagger, tol, maxit, iters);
}

/* full-lattice fields for the force of <a, d(H_eo H_oe) b> on the even
 * sites: A = (a_e, (H^dag)_oe a_e), B = (b_e, H_oe b_e), so that
 * <a, dH_eo H_oe b> + <a, H_eo dH_oe b> = <A, dH B> over sub-slab hops */
static void eo_pair(const G* g, const cplx* U, const cplx* a_e, const cplx* b_e, cplx* A, cplx* B)
{
    size_t n = (size_t)g->V * 12, nh = (size_t)g->Vh * 12;
    cplx* t = malloc(sizeof(cplx) * n);
    memset(A, 0, sizeof(cplx) * n);
    memcpy(A, a_e, sizeof(cplx) * nh);
    hop_c(g, U, A, t, LQO_HOP_INTRA2, 1);
    memcpy(A + nh, t + nh, sizeof(cplx) * nh);
    memset(B, 0, sizeof(cplx) * n);
    memcpy(B, b_e, sizeof(cplx) * nh);
    hop_c(g, U, B, t, LQO_HOP_INTRA2, 0);
    memcpy(B + nh, t + nh, sizeof(cplx) * nh);
    free(t);
}

/* S1 = |W3,eo^-1 phi|^2: eta = W3^-1 phi, xi = W3^-dag eta,
 * dS1 = -2 Re <xi, dW3 eta> = 2 kappa^2 Re <xi, d(H_eo H_oe) eta> */
int lqo_pf_s1(const lqo_geom* gi, const double* Ud, double kappa, double rho, const double* phi, double* F,
              double* S, double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    if (!g.l0s) return -2;
    size_t n = (size_t)g.V * 12, nh = (size_t)g.Vh * 12;
    cplx* eta = malloc(sizeof(cplx) * nh);
    int st = w3eo_solve(&g, U, kappa, rho, eta, (const cplx*)phi, 0, tol, maxit, NULL);
    if (S) *S = nrm2(eta, nh);
    if (F) {
        cplx* xi = malloc(sizeof(cplx) * nh);
        cplx* A = malloc(sizeof(cplx) * n);
        cplx* B = malloc(sizeof(cplx) * n);
        st |= w3eo_solve(&g, U, kappa, rho, xi, eta, 1, tol, maxit, NULL);
        eo_pair(&g, U, xi, eta, A, B);
        bilinear_c(&g, U, A, B, LQO_HOP_INTRA2, kappa * kappa, F);
        free(xi); free(A); free(B);
    }
    free(eta);
    return st;
}

/* S2 = |W3,eo W2,eo^-1 phi|^2 = |chi|^2, zeta = W2^-1 phi, chi = phi + rho zeta;
 * d chi = -rho W2^-1 dW2 zeta, so dS2 = -2 rho Re <W2^-dag chi, dW2 zeta>
 *                                     = 2 rho kappa^2 Re <lambda, d(H_eo H_oe) zeta> */
int lqo_pf_s2(const lqo_geom* gi, const double* Ud, double kappa, double rho, const double* phi, double* F,
              double* S, double tol, int maxit)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    if (!g.l0s) return -2;
    size_t n = (size_t)g.V * 12, nh = (size_t)g.Vh * 12;
    const cplx* ph = (const cplx*)phi;
    cplx* zeta = malloc(sizeof(cplx) * nh);
    cplx* chi = malloc(sizeof(cplx) * nh);
    int st = w3eo_solve(&g, U, kappa, 0.0, zeta, ph, 0, tol, maxit, NULL);
    for (size_t i = 0; i < nh; ++i) chi[i] = ph[i] + rho * zeta[i];
    if (S) *S = nrm2(chi, nh);
    if (F) {
        cplx* lam = malloc(sizeof(cplx) * nh);
        cplx* A = malloc(sizeof(cplx) * n);
        cplx* B = malloc(sizeof(cplx) * n);
        st |= w3eo_solve(&g, U, kappa, 0.0, lam, chi, 1, tol, maxit, NULL);
        eo_pair(&g, U, lam, zeta, A, B);
        bilinear_c(&g, U, A, B, LQO_HOP_INTRA2, rho * kappa * kappa, F);
        free(lam); free(A); free(B);
    }
    free(zeta); free(chi);
    return st;
}

/* ------------------------------------------------------------------ */
/* gauge action S_G = -beta/3 sum_x sum_{mu>nu} Re tr(plaquette)        */
/* ------------------------------------------------------------------ */
static double plaq_re(const G* g, const cplx* U, int s, int mu, int nu)
{
    double ph;
    int smu = shift_of(g, s, mu, +1, &ph);
    int snu = shift_of(g, s, nu, +1, &ph);
    cplx a[9], b[9], c[9], d[9];
    mm(link(g, U, mu, s), link(g, U, nu, smu), a);
    dag(link(g, U, mu, snu), c);
    mm(a, c, b);
    dag(link(g, U, nu, s), c);
    mm(b, c, d);
    return creal(d[0] + d[4] + d[8]);
}

double lqo_gauge_action(const lqo_geom* gi, const double* Ud, double beta)
{
    G g = mkg(gi);
    double sum = 0;
    for (int s = 0; s < g.V; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < mu; ++nu) sum += plaq_re(&g, (const cplx*)Ud, s, mu, nu);
    return -beta / 3.0 * sum;
}

double lqo_plaquette(const lqo_geom* gi, const double* Ud)
{
    G g = mkg(gi);
    double sum = 0;
    for (int s = 0; s < g.V; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < mu; ++nu) sum += plaq_re(&g, (const cplx*)Ud, s, mu, nu);
    return sum / (6.0 * g.V * 3.0);
}

/* dS_G along T^a on U_mu(y): -beta/3 Re tr(i T^a U_mu(y) A), with A the
 * sum over nu != mu of the two staples closing a plaquette with U_mu(y):
 *   up:   U_nu(y+mu) U_mu(y+nu)^dag U_nu(y)^dag
 *   down: U_nu(y+mu-nu)^dag U_mu(y-nu)^dag U_nu(y-nu) */
void lqo_gauge_force(const lqo_geom* gi, const double* Ud, double beta, double* F)
{
    G g = mkg(gi);
    const cplx* U = (const cplx*)Ud;
    init_generators();
    for (int s = 0; s < g.V; ++s)
        for (int mu = 0; mu < 4; ++mu) {
            cplx A[9] = {0}, t1[9], t2[9], t3[9];
            double ph;
            int smu = shift_of(&g, s, mu, +1, &ph);
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                int snu = shift_of(&g, s, nu, +1, &ph);
                int smnu = shift_of(&g, s, nu, -1, &ph);
                int smumnu = shift_of(&g, smu, nu, -1, &ph);
                dag(link(&g, U, mu, snu), t1);
                mm(link(&g, U, nu, smu), t1, t2);
                dag(link(&g, U, nu, s), t1);
                mm(t2, t1, t3);
                for (int i = 0; i < 9; ++i) A[i] += t3[i];
                dag(link(&g, U, nu, smumnu), t1);
                dag(link(&g, U, mu, smnu), t2);
                mm(t1, t2, t3);
                mm(t3, link(&g, U, nu, smnu), t1);
                for (int i = 0; i < 9; ++i) A[i] += t1[i];
            }
            cplx UA[9];
            mm(link(&g, U, mu, s), A, UA);
            for (int c = 0; c < 8; ++c) {
                cplx tr = 0;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) tr += I * TG[c][i][k] * UA[k * 3 + i];
                F[((size_t)mu * g.V + s) * 8 + c] += -beta / 3.0 * creal(tr);
            }
        }
}

/* ------------------------------------------------------------------ */
/* T_U (eq. (3)): U -> exp(i dt P) U.  exp by Taylor series with        */
/* scaling and squaring, then re-unitarisation (Gram-Schmidt on rows 1  */
/* and 2, row 3 = conj(row1 x row2)).                                   */
/* ------------------------------------------------------------------ */
void lqo_su3_expi(const double* Xd, double* Ed)
{
    /* E = exp(i X) for a hermitian 3x3 X */
    const cplx* X = (const cplx*)Xd;
    cplx* E = (cplx*)Ed;
    double nrm = 0;
    for (int i = 0; i < 9; ++i) nrm += creal(X[i] * conj(X[i]));
    nrm = sqrt(nrm);
    int k = 0;
    while (nrm / ldexp(1.0, k) > 0.25) ++k;
    cplx Y[9], term[9], tmp[9];
    for (int i = 0; i < 9; ++i) Y[i] = I * X[i] / ldexp(1.0, k);
    for (int i = 0; i < 9; ++i) { E[i] = (i % 4 == 0) ? 1 : 0; term[i] = E[i]; }
    for (int m = 1; m <= 20; ++m) {
        mm(term, Y, tmp);
        for (int i = 0; i < 9; ++i) { term[i] = tmp[i] / m; E[i] += term[i]; }
    }
    for (int q = 0; q < k; ++q) {
        mm(E, E, tmp);
        memcpy(E, tmp, sizeof(tmp));
    }
}

static void reunit(cplx* u)
{
    double n0 = 0;
    for (int j = 0; j < 3; ++j) n0 += creal(u[j] * conj(u[j]));
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; ++j) u[j] *= n0;
    cplx d = 0;
    for (int j = 0; j < 3; ++j) d += conj(u[j]) * u[3 + j];
    for (int j = 0; j < 3; ++j) u[3 + j] -= d * u[j];
    double n1 = 0;
    for (int j = 0; j < 3; ++j) n1 += creal(u[3 + j] * conj(u[3 + j]));
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; ++j) u[3 + j] *= n1;
    u[6] = conj(u[1] * u[5] - u[2] * u[4]);
    u[7] = conj(u[2] * u[3] - u[0] * u[5]);
    u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

/* average force per time slice (Sec. 3, Fig. 1): out[x0] = mean over the
 * space-like links of slice x0 of |F| (Euclidean norm of the 8 coefficients),
 * out[L0 + x0] the same for the time-like links */
void lqo_force_profile(const lqo_geom* gi, const double* F, double* out)
{
    G g = mkg(gi);
    memset(out, 0, sizeof(double) * 2 * g.L[0]);
    for (int s = 0; s < g.V; ++s) {
        int x[4];
        coords_of(&g, s, x);
        for (int mu = 0; mu < 4; ++mu) {
            double n = 0;
            for (int a = 0; a < 8; ++a) n += F[((size_t)mu * g.V + s) * 8 + a] * F[((size_t)mu * g.V + s) * 8 + a];
            out[(mu == 0 ? g.L[0] : 0) + x[0]] += sqrt(n);
        }
    }
    for (int t = 0; t < g.L[0]; ++t) {
        out[t] /= 3.0 * g.V3;
        out[g.L[0] + t] /= g.V3;
    }
}

/* position-dependent step size (Sec. 2): the step of link U_mu(x) is
 * dt * s(x0) with one table for space-like and one for time-like links,
 * repeated with the scheme's period along x0.  scale: [2][L0] (row 0
 * space-like, row 1 time-like) or NULL for s = 1. */
static double link_scale(const G* g, const double* scale, size_t l)
{
    if (!scale) return 1.0;
    int mu = (int)(l / g->V), s = (int)(l % g->V), x[4];
    coords_of(g, s, x);
    return scale[(mu == 0 ? g->L[0] : 0) + x[0]];
}

/* the schemes of Sec. 2 as [2][L0] tables; returns -1 when L0 is not a
 * multiple of the period.  Scheme A's space-like value at x0 = 5 is printed
 * as "2"; 0.2 is the value that reproduces the stated average 0.525. */
int lqo_step_scheme(int scheme, int L0, double* out)
{
    static const double As[6] = {0.2, 0.5, 1, 1, 0.5, 0.2}, At[6] = {0.2, 0.5, 1, 0.5, 0.2, 0};
    static const double Bs[8] = {0, 0.5, 1, 1, 1, 1, 0.5, 0}, Bt[8] = {0, 0.5, 1, 1, 1, 0.5, 0, 0};
    static const double Cs[16] = {0, 0.25, 0.5, 1, 1, 1, 1, 0.25, 0.25, 1, 1, 1, 1, 0.5, 0.25, 0};
    static const double Ct[16] = {0, 0, 0.25, 0.5, 1, 1, 0.25, 0, 0.25, 1, 1, 1, 0.5, 0.25, 0, 0};
    const double *sp, *tm;
    int per;
    if (scheme == 1) { sp = As; tm = At; per = 6; }
    else if (scheme == 2) { sp = Bs; tm = Bt; per = 8; }
    else if (scheme == 3) { sp = Cs; tm = Ct; per = 16; }
    else return -1;
    if (L0 % per) return -1;
    for (int t = 0; t < L0; ++t) {
        out[t] = sp[t % per];
        out[L0 + t] = tm[t % per];
    }
    return 0;
}

void lqo_update_U_scaled(const lqo_geom* gi, double* Ud, const double* P, double dt, const double* scale)
{
    G g = mkg(gi);
    cplx* U = (cplx*)Ud;
    init_generators();
    for (size_t l = 0; l < (size_t)4 * g.V; ++l) {
        cplx X[9] = {0}, E[9], nu[9];
        const double dl = dt * link_scale(&g, scale, l);
        if (dl == 0.0) continue; /* a frozen link */
        for (int c = 0; c < 8; ++c)
            for (int i = 0; i < 9; ++i) X[i] += dl * P[l * 8 + c] * (&TG[c][0][0])[i];
        lqo_su3_expi((const double*)X, (double*)E);
        mm(E, U + l * 9, nu);
        reunit(nu);
        memcpy(U + l * 9, nu, sizeof(nu));
    }
}

void lqo_update_U(const lqo_geom* gi, double* Ud, const double* P, double dt)
{
    G g = mkg(gi);
    cplx* U = (cplx*)Ud;
    init_generators();
    for (size_t l = 0; l < (size_t)4 * g.V; ++l) {
        cplx X[9] = {0}, E[9], nu[9];
        for (int c = 0; c < 8; ++c)
            for (int i = 0; i < 9; ++i) X[i] += dt * P[l * 8 + c] * (&TG[c][0][0])[i];
        lqo_su3_expi((const double*)X, (double*)E);
        mm(E, U + l * 9, nu);
        reunit(nu);
        memcpy(U + l * 9, nu, sizeof(nu));
    }
}

/* U'_mu(x) = U_mu(x - shift * 0hat): the configuration moved forward in x0 */
void lqo_roll_x0(const lqo_geom* gi, double* Ud, int shift)
{
    G g = mkg(gi);
    cplx* U = (cplx*)Ud;
    size_t n = (size_t)4 * g.V * 9;
    cplx* t = malloc(sizeof(cplx) * n);
    for (int s = 0; s < g.V; ++s) {
        int x[4];
        coords_of(&g, s, x);
        x[0] = ((x[0] - shift) % g.L[0] + g.L[0]) % g.L[0];
        int src = site_of(&g, x);
        for (int mu = 0; mu < 4; ++mu)
            memcpy(t + ((size_t)mu * g.V + s) * 9, U + ((size_t)mu * g.V + src) * 9, sizeof(cplx) * 9);
    }
    memcpy(U, t, sizeof(cplx) * n);
    free(t);
}

/* ------------------------------------------------------------------ */
/* random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)    */
/* key = (seed lo, seed hi); counter = (i lo, i hi, stream, traj).      */
/* normal k: counter index i = k/2; the four words give two 53-bit      */
/* uniforms u1=(w0,w1), u2=(w2,w3) in (0,1) and Box-Muller gives        */
/* sqrt(-2 ln u1) cos(2 pi u2) (k even), ... sin(2 pi u2) (k odd).       */
/* ------------------------------------------------------------------ */
void lqo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) / 9007199254740992.0;
}

void lqo_normals(uint64_t seed, uint32_t stream, uint32_t traj, int64_t n, double* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < n; ++k) {
        uint64_t i = (uint64_t)k / 2;
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, traj}, w[4];
        lqo_philox4x32_10(ctr, key, w);
        double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
        double rad = sqrt(-2.0 * log(u1));
        out[k] = (k % 2 == 0) ? rad * cos(2.0 * M_PI * u2) : rad * sin(2.0 * M_PI * u2);
    }
}

/* stream 4, counter index 0: Metropolis uniform from (w0,w1), x0 shift
 * floor(w2 * L0 / 2^32) */
void lqo_uniforms_metropolis(uint64_t seed, uint32_t traj, int L0, double* u, int* shift)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {0, 0, 4, traj}, w[4];
    lqo_philox4x32_10(ctr, key, w);
    *u = u53(w[0], w[1]);
    *shift = (int)(((uint64_t)w[2] * (uint64_t)L0) >> 32);
}

/* ------------------------------------------------------------------ */
/* HMC trajectory (Sec. 2)                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    const G* g;
    const lqo_geom* gi;
    const lqo_hmc_params* prm;
    double* U;
    double* P;
    lqo_pf_fields pf;
    double* F;
    int status;
} md_t;

/* T_P,j(dt): P -> P - dt dS_j/dU for the action terms on level j */
static void T_P(md_t* m, int j, double dt)
{
    const lqo_hmc_params* p = m->prm;
    size_t nl = (size_t)4 * m->g->V * 8;
    int any = 0;
    memset(m->F, 0, sizeof(double) * nl);
    if (p->level_gauge == j) { lqo_gauge_force(m->gi, m->U, p->beta, m->F); any = 1; }
    if (p->level_w1 == j) {
        m->status |= lqo_pf_w1(m->gi, m->U, p->kappa, m->pf.w1, m->F, NULL, p->tol, p->maxit);
        any = 1;
    }
    if (p->level_schur == j) {
        m->status |= lqo_pf_schur(m->gi, m->U, p->kappa, m->pf.schur, m->F, NULL, p->schur_route,
                                  p->tol, p->maxit);
        any = 1;
    }
    if (p->level_w2 == j) {
        m->status |= lqo_pf_w2(m->gi, m->U, p->kappa, m->pf.w2, m->F, NULL, p->tol, p->maxit);
        any = 1;
    }
    if (p->level_schur2 == j) {
        m->status |= lqo_pf_schur2(m->gi, m->U, p->kappa, m->pf.schur2, m->F, NULL, p->schur_route, p->tol,
                                   p->maxit);
        any = 1;
    }
    if (p->level_s2 == j) {
        m->status |= lqo_pf_s2(m->gi, m->U, p->kappa, p->rho, m->pf.s2, m->F, NULL, p->tol, p->maxit);
        any = 1;
    }
    if (p->level_s1 == j) {
        m->status |= lqo_pf_s1(m->gi, m->U, p->kappa, p->rho, m->pf.s1, m->F, NULL, p->tol, p->maxit);
        any = 1;
    }
    if (!any) return;
    for (size_t i = 0; i < nl; ++i) m->P[i] -= dt * link_scale(m->g, p->step_scale, i / 8) * m->F[i];
}

static void T_U(md_t* m, double dt) { lqo_update_U_scaled(m->gi, m->U, m->P, dt, m->prm->step_scale); }

/* elementary step of level j with step size dt, eqs. (4)-(7) */
static void step(md_t* m, int j, double dt)
{
    const lqo_hmc_params* p = m->prm;
    double lam = p->lambda;
    if (j == 0) {
        if (p->scheme[0] == LQO_LF) {
            T_P(m, 0, dt / 2); T_U(m, dt); T_P(m, 0, dt / 2);
        } else {
            T_P(m, 0, lam * dt); T_U(m, dt / 2); T_P(m, 0, (1 - 2 * lam) * dt);
            T_U(m, dt / 2); T_P(m, 0, lam * dt);
        }
        return;
    }
    int n = p->nsteps[j - 1];
    double di = dt / n;
    if (p->scheme[j] == LQO_LF) {
        T_P(m, j, dt / 2);
        for (int i = 0; i < n; ++i) step(m, j - 1, di);
        T_P(m, j, dt / 2);
    } else {
        T_P(m, j, lam * dt);
        for (int i = 0; i < n / 2; ++i) step(m, j - 1, di);
        T_P(m, j, (1 - 2 * lam) * dt);
        for (int i = 0; i < n / 2; ++i) step(m, j - 1, di);
        T_P(m, j, lam * dt);
    }
}

/* the molecular-dynamics part of a trajectory, T_LF/SW,top(dt_top)^n_top,
 * on (U, P) in place for fixed pseudo-fermion fields */
int lqo_md(const lqo_geom* gi, double* U, double* P, const lqo_pf_fields* pf, const lqo_hmc_params* p)
{
    G g = mkg(gi);
    double* F = malloc(sizeof(double) * (size_t)4 * g.V * 8);
    md_t m = {&g, gi, p, U, P, *pf, F, 0};
    int top = p->nlevels - 1;
    double dt = p->tau / p->nsteps[top];
    for (int i = 0; i < p->nsteps[top]; ++i) step(&m, top, dt);
    free(F);
    return m.status;
}

static double kinetic(const double* P, size_t nl)
{
    double s = 0;
    for (size_t i = 0; i < nl; ++i) s += P[i] * P[i];
    return 0.5 * s;
}

int lqo_hmc_trajectory(const lqo_geom* gi, double* U, const lqo_hmc_params* p, uint64_t seed,
                       uint32_t traj, const double* P0, const double* eta1, const double* eta2,
                       lqo_hmc_result* res)
{
    G g = mkg(gi);
    size_t nl = (size_t)4 * g.V * 8, n = (size_t)g.V * 12, nu = (size_t)4 * g.V * 9;
    int nbnd = (g.nb / 2) * 2 * g.V3 * 6;
    int nb2 = (g.nbs / 2) * g.V3 * 6;
    double* P = malloc(sizeof(double) * nl);
    double* e1 = malloc(sizeof(cplx) * n);
    double* e2 = malloc(sizeof(cplx) * nbnd);
    double* phi1 = malloc(sizeof(cplx) * n);
    double* phi2 = malloc(sizeof(cplx) * nbnd);
    double* e3 = malloc(sizeof(cplx) * n);
    double* phi3 = malloc(sizeof(cplx) * n);
    double* e4 = malloc(sizeof(cplx) * (nb2 + 1));
    double* phi4 = malloc(sizeof(cplx) * (nb2 + 1));
    size_t nh = (size_t)g.Vh * 12;
    double* e5 = malloc(sizeof(cplx) * nh);
    double* phi5 = malloc(sizeof(cplx) * nh);
    double* e6 = malloc(sizeof(cplx) * nh);
    double* phi6 = malloc(sizeof(cplx) * nh);
    double* U0 = malloc(sizeof(cplx) * nu);
    memcpy(U0, U, sizeof(cplx) * nu);
    int st = 0;
    /* heatbath: p^a ~ N(0,1); eta ~ exp(-|eta|^2) (re, im of variance 1/2) */
    if (P0) memcpy(P, P0, sizeof(double) * nl);
    else lqo_normals(seed, 1, traj, (int64_t)nl, P);
    if (eta1) memcpy(e1, eta1, sizeof(cplx) * n);
    else {
        lqo_normals(seed, 2, traj, (int64_t)n * 2, e1);
        for (size_t i = 0; i < n * 2; ++i) e1[i] *= sqrt(0.5);
    }
    if (eta2) memcpy(e2, eta2, sizeof(cplx) * nbnd);
    else {
        lqo_normals(seed, 3, traj, (int64_t)nbnd * 2, e2);
        for (int i = 0; i < nbnd * 2; ++i) e2[i] *= sqrt(0.5);
    }
    double H0 = kinetic(P, nl);
    if (p->level_gauge >= 0) H0 += lqo_gauge_action(gi, U, p->beta);
    if (p->level_w1 >= 0) {
        if (p->pf_init == 0) {
            lqo_apply_W1(gi, U, p->kappa, e1, phi1, 0);
            H0 += nrm2((const cplx*)e1, n);
        } else {
            double S;
            memcpy(phi1, e1, sizeof(cplx) * n);
            st |= lqo_pf_w1(gi, U, p->kappa, phi1, NULL, &S, p->tol, p->maxit);
            H0 += S;
        }
    }
    if (p->level_schur >= 0) {
        if (p->pf_init == 0) {
            st |= lqo_schur(gi, U, p->kappa, phi2, e2, LQO_R, p->schur_route, p->tol, p->maxit);
            H0 += nrm2((const cplx*)e2, nbnd);
        } else {
            double S;
            memcpy(phi2, e2, sizeof(cplx) * nbnd);
            st |= lqo_pf_schur(gi, U, p->kappa, phi2, NULL, &S, p->schur_route, p->tol, p->maxit);
            H0 += S;
        }
    }
    /* iterated decomposition: phi3 = W2 eta3 (stream 5), phi4 = R2 eta4 (stream 6) */
    if (p->level_w2 >= 0) {
        lqo_normals(seed, 5, traj, (int64_t)n * 2, e3);
        for (size_t i = 0; i < n * 2; ++i) e3[i] *= sqrt(0.5);
        lqo_apply_W2(gi, U, p->kappa, e3, phi3, 0);
        H0 += nrm2((const cplx*)e3, n);
    }
    if (p->level_schur2 >= 0) {
        lqo_normals(seed, 6, traj, (int64_t)nb2 * 2, e4);
        for (int i = 0; i < nb2 * 2; ++i) e4[i] *= sqrt(0.5);
        st |= lqo_schur2(gi, U, p->kappa, phi4, e4, LQO_R, p->schur_route, p->tol, p->maxit);
        H0 += nrm2((const cplx*)e4, nb2);
    }
    /* mass preconditioning of W2: phi_S2 = W2,eo W3,eo^-1 eta (stream 7),
     * phi_S1 = W3,eo eta (stream 8), even-site fields */
    if (p->level_s2 >= 0) {
        lqo_normals(seed, 7, traj, (int64_t)nh * 2, e5);
        for (size_t i = 0; i < nh * 2; ++i) e5[i] *= sqrt(0.5);
        double* t = malloc(sizeof(cplx) * nh);
        st |= w3eo_solve(&g, (const cplx*)U, p->kappa, p->rho, (cplx*)t, (const cplx*)e5, 0, p->tol * 1e-2,
                         p->maxit, NULL);
        w3eo_c(&g, (const cplx*)U, p->kappa, 0.0, (const cplx*)t, (cplx*)phi5, 0);
        free(t);
        H0 += nrm2((const cplx*)e5, nh);
    }
    if (p->level_s1 >= 0) {
        lqo_normals(seed, 8, traj, (int64_t)nh * 2, e6);
        for (size_t i = 0; i < nh * 2; ++i) e6[i] *= sqrt(0.5);
        w3eo_c(&g, (const cplx*)U, p->kappa, p->rho, (const cplx*)e6, (cplx*)phi6, 0);
        H0 += nrm2((const cplx*)e6, nh);
    }
    lqo_pf_fields pf = {phi1, phi2, phi3, phi4, phi5, phi6};
    st |= lqo_md(gi, U, P, &pf, p);
    double H1 = kinetic(P, nl);
    if (p->level_s2 >= 0) {
        double S;
        st |= lqo_pf_s2(gi, U, p->kappa, p->rho, phi5, NULL, &S, p->tol, p->maxit);
        H1 += S;
    }
    if (p->level_s1 >= 0) {
        double S;
        st |= lqo_pf_s1(gi, U, p->kappa, p->rho, phi6, NULL, &S, p->tol, p->maxit);
        H1 += S;
    }
    if (p->level_w2 >= 0) {
        double S;
        st |= lqo_pf_w2(gi, U, p->kappa, phi3, NULL, &S, p->tol, p->maxit);
        H1 += S;
    }
    if (p->level_schur2 >= 0) {
        double S;
        st |= lqo_pf_schur2(gi, U, p->kappa, phi4, NULL, &S, p->schur_route, p->tol, p->maxit);
        H1 += S;
    }
    if (p->level_gauge >= 0) H1 += lqo_gauge_action(gi, U, p->beta);
    if (p->level_w1 >= 0) {
        double S;
        st |= lqo_pf_w1(gi, U, p->kappa, phi1, NULL, &S, p->tol, p->maxit);
        H1 += S;
    }
    if (p->level_schur >= 0) {
        double S;
        st |= lqo_pf_schur(gi, U, p->kappa, phi2, NULL, &S, p->schur_route, p->tol, p->maxit);
        H1 += S;
    }
    double u;
    int shift;
    lqo_uniforms_metropolis(seed, traj, g.L[0], &u, &shift);
    double dH = H1 - H0;
    int acc = 1;
    if (p->metropolis) acc = (dH <= 0) || (u < exp(-dH));
    if (!acc) memcpy(U, U0, sizeof(cplx) * nu);
    if (!p->roll) shift = 0;
    if (shift) lqo_roll_x0(gi, U, shift);
    if (res) {
        res->dH = dH; res->H0 = H0; res->H1 = H1; res->u = u;
        res->accepted = acc; res->shift = shift; res->status = st;
        res->plaq = lqo_plaquette(gi, U);
    }
    free(P); free(e1); free(e2); free(phi1); free(phi2); free(U0);
    free(e3); free(phi3); free(e4); free(phi4);
    free(e5); free(phi5); free(e6); free(phi6);
    return st;
}
