// lqcd_api.cu -- handle, composite operators and the extern "C" entry
// points declared in include/lqcd.h.
//
// Composite operators on internal double full-lattice fields:
//   W1^-1 / M^-1  : even-odd reduction around the persistent batched solver
//                   b_e' = b_e + kappa H_eo b_o,  solve (1 - k^2 H_eo H_oe) x_e = b_e',
//                   x_o = b_o + kappa H_oe x_e;  adjoints via gamma5 (W^dag = g5 W g5)
//   R      = E (1 - C A^-1 B D^-1) E^dag,  C, B = -kappa H_cross  (block LU of eq. (2))
//   R^-1   = E D (M^-1)_bb E^dag,          R^-dag = E (M^-dag)_bb D^dag E^dag
//   dS_R   = 2 Re <eta~, dD psi> - 2 Re <chi, dM psi> with psi = M^-1 E^dag phi,
//            eta~ = E^dag E D psi_b (so S_R = |eta~|^2), chi = M^-dag D^dag eta~
//   dS_W1  = -2 Re <xi, dW1 eta>, eta = W1^-1 phi, xi = W1^-dag eta
// Second level of the iterated decomposition (Sec. 1), the same formulas one
// level down: (M, W1, H_cross, H_intra) -> (W1, W2, H_cross2, H_intra2), the
// sub-slab operators run on the sub-slab geometry (GeoScope), the boundary
// is the first slice of every black sub-slab.
//   R2^-1 = E2 D2 (W1^-1)_bb E2^dag,  S_R2 = |R2^-1 phi|^2, S_W2 = |W2^-1 phi|^2
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lqcd_common.cuh"

int reduction_blocks();
int bnd_sub(lqcd_ctx* h, double* out, const double* in, int n);

namespace {

enum { F_T1 = 0, F_T2, F_A, F_B, F_C, F_D, F_E, F_G, F_PHI1, F_ETA1, F_PHI3, F_PHI5, F_PHI6, NFIELD };

inline double2* fld(lqcd_ctx* h, int k) { return h->f64[k]; }

int nbnd_of(const Geo& g) { return (g.nb / 2) * 2 * g.V3 * 6; }
// complex entries of a second-level boundary field (first slices only)
int nbnd2_of(const Geo& g1) { return g1.l0s ? (g1.L[0] / g1.l0s / 2) * g1.V3 * 6 : 0; }

bool prec_ok(int p)
{
    return p == LQCD_PREC_F64 || p == LQCD_PREC_F32 || p == LQCD_PREC_F16 || p == LQCD_PREC_BF16;
}

SpinorF none()
{
    SpinorF f;
    f.v = nullptr;
    f.nrm = nullptr;
    f.N = 0;
    return f;
}

// full-lattice out = a x + c H_mode in on the output slabs of `colour`
int hop_full(lqcd_ctx* h, int mode, int dag, int colour, double2* out, const double2* in, double a,
             const double2* x, double c)
{
    const int Vh = h->g.Vh;
    for (int p = 0; p < 2; ++p) {
        SpinorF xo = x ? sp64((double2*)x, p, Vh) : none();
        LQ_TRY(hop_sweep(h, PREC64, mode, dag, p, colour, sp64(out, p, Vh), sp64((double2*)in, 1 - p, Vh), a, xo, c));
    }
    if (colour >= 0) LQ_TRY(keep_colour(h, out, colour));
    return LQCD_OK;
}

// Chronological initial guess of slot k for a solve on the links at MD
// time h->md_time (even half of x): the Lagrange extrapolation in MD time of
// the solutions kept (Brower, Ivanenko, Levi, Orginos, Nucl. Phys. B 484
// (1997) 353: the chronological inverter): nothing kept, zero (*guess = 0);
// one, that solution; two, the straight line through them; three (chrono =
// 2), the parabola.  Solutions at coinciding times drop to the lower
// order.  dag: the unknown of the adjoint system is gamma5 x.
int chrono_guess(lqcd_ctx* h, int k, double2* x, int dag, int* guess)
{
    constexpr int D = lqcd_ctx::CHRONO_MAX;
    *guess = 0;
    if (k < 0 || !h->chrono_buf[D * k] || h->chrono_n[k] == 0) return LQCD_OK;
    const int depth = std::max(1, h->chrono_depth[k]);
    // newest first: buffers cur, cur - 1, cur - 2 (mod depth)
    const int j2 = h->chrono_cur[k], j1 = (j2 + depth - 1) % depth, j0 = (j2 + depth - 2) % depth;
    const double t = h->md_time, t2 = h->chrono_t[k][j2], t1 = h->chrono_t[k][j1], t0 = h->chrono_t[k][j0];
    const double2 *x2 = h->chrono_buf[D * k + j2], *x1 = h->chrono_buf[D * k + j1], *x0 = h->chrono_buf[D * k + j0];
    int n = std::min(h->chrono_n[k], 3);
    if (n >= 2 && t1 == t2) n = 1;
    if (n >= 3 && (t0 == t1 || t0 == t2)) n = 2;
    if (n == 3) {
        const double w2 = (t - t0) * (t - t1) / ((t2 - t0) * (t2 - t1));
        const double w1 = (t - t0) * (t - t2) / ((t1 - t0) * (t1 - t2));
        const double w0 = (t - t1) * (t - t2) / ((t0 - t1) * (t0 - t2));
        LQ_TRY(lincomb3_even(h, x, w2, x2, w1, x1, w0, x0, dag));
    } else if (n == 2) {
        const double s = (t - t2) / (t2 - t1);
        LQ_TRY(lincomb_even(h, x, 1.0 + s, x2, -s, x1, dag));
    } else {
        LQ_TRY(lincomb_even(h, x, 1.0, x2, 0.0, x2, dag));
    }
    *guess = 1;
    return LQCD_OK;
}

// keep the even half of the solution x of slot k (the oldest one is dropped)
int chrono_store(lqcd_ctx* h, int k, const double2* x)
{
    constexpr int D = lqcd_ctx::CHRONO_MAX;
    if (k < 0 || !h->chrono_buf[D * k] || h->chrono_frozen) return LQCD_OK;
    const int depth = std::max(1, h->chrono_depth[k]);
    h->chrono_cur[k] = (h->chrono_cur[k] + 1) % depth;
    LQ_CUDA(h, cudaMemcpyAsync(h->chrono_buf[D * k + h->chrono_cur[k]], x, sizeof(double2) * 12 * (size_t)h->g.Vh,
                               cudaMemcpyDeviceToDevice, h->stream));
    h->chrono_t[k][h->chrono_cur[k]] = h->md_time;
    h->chrono_n[k] = h->chrono_n[k] < depth ? h->chrono_n[k] + 1 : depth;
    return LQCD_OK;
}

// minimal-residual guess of slot k for the whole-lattice even-odd system
// with source b_e (the solve's b_e' = b_e + kappa H_eo b_o): over all kept
// solutions of the slot (chrono = 3, lqcd_chrono.cu)
int chrono_mre(lqcd_ctx* h, int k, double2* x, const double2* b_e, double kappa, int dag, int* guess)
{
    *guess = 0;
    constexpr int D = lqcd_ctx::CHRONO_MAX;
    if (k < 0 || !h->chrono_buf[D * k] || h->chrono_n[k] == 0) return LQCD_OK;
    const double2* sol[lqcd_ctx::NMRE];
    const int n = std::min(h->chrono_n[k], (int)lqcd_ctx::NMRE);
    for (int i = 0; i < n; ++i) sol[i] = h->chrono_buf[D * k + i];
    LQ_TRY(chrono_mre_guess(h, sol, n, x, b_e, kappa, dag));
    *guess = 1;
    return LQCD_OK;
}

// x = W^-1 b (block: W1 on the slabs of `colour`; global: M).  x, b full
// double fields, b is not modified, x must not alias b.  slot >= 0: the
// solve starts from the chronological guess of that slot and keeps its
// solution there.
int solve_full(lqcd_ctx* h, int mode, int colour, int dagger, int prec, double kappa, double2* x,
               const double2* b, double tol, int max_iter, int* iters, double* resid,
               int method = SOLVER_BICGSTAB, int slot = -1)
{
    const int Vh = h->g.Vh;
    const double2* bb = b;
    if (dagger) {
        LQ_TRY(gamma5_full(h, fld(h, F_T1), b));
        bb = fld(h, F_T1);
    }
    const int col = mode == MODE_ALL ? -1 : colour;
    // b_e' = b_e + kappa H_eo b_o (double fields; double-float arithmetic
    // around a mixed-precision solve)
    const int hp = prec == PREC64 ? PREC64 : PRECDF;
    LQ_TRY(hop_sweep(h, hp, mode, 0, 0, col, sp64(fld(h, F_T2), 0, Vh), sp64((double2*)bb, 1, Vh), 1.0,
                     sp64((double2*)bb, 0, Vh), kappa));
    int guess = 0;
    if (mode == MODE_ALL && h->chrono_mre && slot >= 0)
        LQ_TRY(chrono_mre(h, slot, x, fld(h, F_T2), kappa, dagger, &guess));
    else
        LQ_TRY(chrono_guess(h, slot, x, dagger, &guess));
    // whole-lattice solves take the handle's global solver (plain or
    // Schwarz-preconditioned BiCGstab), block solves the caller's method
    LQ_TRY(eo_solve(h, mode, col, prec, kappa, x, fld(h, F_T2), tol, max_iter, iters, resid, 1.0,
                    mode == MODE_ALL ? h->global_method : method, guess));
    // x_o = b_o + kappa H_oe x_e
    LQ_TRY(hop_sweep(h, hp, mode, 0, 1, col, sp64(x, 1, Vh), sp64(x, 0, Vh), 1.0, sp64((double2*)bb, 1, Vh),
                     kappa));
    if (col >= 0) LQ_TRY(keep_colour(h, x, col));
    if (dagger) LQ_TRY(gamma5_full(h, x, x));
    return chrono_store(h, slot, x);
}

struct SolveCfg {
    int prec;
    double tol;
    int max_iter;
    int method = SOLVER_BICGSTAB;  // inner iteration of the W3,eo / W2,eo solves
    int slot = -1;                 // first chronological slot of the term (force solves), or -1
};

// slot k + 1 for the second (adjoint) solve of a term, or -1
inline int next_slot(int k) { return k >= 0 ? k + 1 : -1; }

// R, R^dag, R^-1, R^-dag on boundary coordinates (device doubles)
int schur_op(lqcd_ctx* h, double* out, const double* in, double kappa, int op, const SolveCfg& c)
{
    double2 *A = fld(h, F_A), *B = fld(h, F_B), *C = fld(h, F_C), *D = fld(h, F_D), *E = fld(h, F_E);
    const int nb2 = 2 * nbnd_of(h->g);
    LQ_TRY(embed_boundary(h, A, in));
    if (op == LQCD_SCHUR_R) {
        LQ_TRY(solve_full(h, MODE_INTRA, 1, 0, c.prec, kappa, B, A, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(hop_full(h, MODE_CROSS, 0, 0, C, B, 0.0, nullptr, -kappa));
        LQ_TRY(solve_full(h, MODE_INTRA, 0, 0, c.prec, kappa, D, C, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(hop_full(h, MODE_CROSS, 0, 1, E, D, 0.0, nullptr, -kappa));
        LQ_TRY(project_boundary(h, out, E));
    } else if (op == LQCD_SCHUR_RDAG) {
        LQ_TRY(hop_full(h, MODE_CROSS, 1, 0, C, A, 0.0, nullptr, -kappa));
        LQ_TRY(solve_full(h, MODE_INTRA, 0, 1, c.prec, kappa, D, C, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(hop_full(h, MODE_CROSS, 1, 1, E, D, 0.0, nullptr, -kappa));
        LQ_TRY(solve_full(h, MODE_INTRA, 1, 1, c.prec, kappa, B, E, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(project_boundary(h, out, B));
    } else if (op == LQCD_SCHUR_RINV) {
        LQ_TRY(solve_full(h, MODE_ALL, -1, 0, c.prec, kappa, B, A, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(hop_full(h, MODE_INTRA, 0, 1, C, B, 1.0, B, -kappa));
        LQ_TRY(project_boundary(h, out, C));
        return LQCD_OK;
    } else {
        LQ_TRY(hop_full(h, MODE_INTRA, 1, 1, C, A, 1.0, A, -kappa));
        LQ_TRY(solve_full(h, MODE_ALL, -1, 1, c.prec, kappa, B, C, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(project_boundary(h, out, B));
        return LQCD_OK;
    }
    // out = in - E(...)
    return bnd_sub(h, out, in, nb2);
}

// F += coef * dS/dw for S = |W1^-1 phi|^2; *S_dev (device) receives S
int pf_w1(lqcd_ctx* h, double* F, const double2* phi, double kappa, double coef, const SolveCfg& c,
          double* S_dev, const double* ss = nullptr)
{
    double2 *eta = fld(h, F_A), *xi = fld(h, F_B);
    LQ_TRY(solve_full(h, MODE_INTRA, -1, 0, c.prec, kappa, eta, phi, c.tol, c.max_iter, nullptr, nullptr,
                      c.method, c.slot));
    if (S_dev) LQ_TRY(norm2_dev(h, (const double*)eta, (int64_t)48 * h->g.Vh, S_dev));
    if (!F) return LQCD_OK;
    LQ_TRY(solve_full(h, MODE_INTRA, -1, 1, c.prec, kappa, xi, eta, c.tol, c.max_iter, nullptr, nullptr,
                      c.method, next_slot(c.slot)));
    return force_bilinear(h, F, xi, eta, MODE_INTRA, kappa * coef, nullptr, nullptr, 0, 0.0, c.prec, ss);
}

// F += coef * dS/dw for S = |R^-1 phi|^2 (phi: device boundary coordinates)
int pf_schur(lqcd_ctx* h, double* F, const double* phi, double kappa, double coef, const SolveCfg& c,
             double* S_dev, const double* ss = nullptr)
{
    double2 *A = fld(h, F_A), *psi = fld(h, F_B), *C = fld(h, F_C), *et = fld(h, F_D), *E = fld(h, F_E),
            *chi = fld(h, F_G);
    const int nbd = 2 * nbnd_of(h->g);
    double* eta = h->bnd[1];
    LQ_TRY(embed_boundary(h, A, phi));
    LQ_TRY(solve_full(h, MODE_ALL, -1, 0, c.prec, kappa, psi, A, c.tol, c.max_iter, nullptr, nullptr,
                      SOLVER_BICGSTAB, c.slot));
    LQ_TRY(hop_full(h, MODE_INTRA, 0, 1, C, psi, 1.0, psi, -kappa));
    LQ_TRY(project_boundary(h, eta, C));
    if (S_dev) LQ_TRY(norm2_dev(h, eta, nbd, S_dev));
    if (!F) return LQCD_OK;
    LQ_TRY(embed_boundary(h, et, eta));
    LQ_TRY(hop_full(h, MODE_INTRA, 1, 1, E, et, 1.0, et, -kappa));
    LQ_TRY(solve_full(h, MODE_ALL, -1, 1, c.prec, kappa, chi, E, c.tol, c.max_iter, nullptr, nullptr,
                      SOLVER_BICGSTAB, next_slot(c.slot)));
    return force_bilinear(h, F, et, psi, MODE_INTRA, -kappa * coef, chi, psi, MODE_ALL, kappa * coef, c.prec, ss);
}

// ---------------------------------------------------------------------------
// second level (iterated decomposition); all called with h->g the level-1
// geometry and h->g1.l0s > 0
// ---------------------------------------------------------------------------
// x = W2^-1 b on the sub-slabs of `colour` (-1: all)
int sub_solve(lqcd_ctx* h, int colour, int dagger, const SolveCfg& c, double kappa, double2* x, const double2* b)
{
    GeoScope sc(h, sub_geo(h->g1));
    return solve_full(h, MODE_INTRA, colour, dagger, c.prec, kappa, x, b, c.tol, c.max_iter, nullptr, nullptr);
}

// out = a x + c H_intra2 in (dag: H^dag) on the sub-slabs of `colour`
int sub_hop(lqcd_ctx* h, int dag, int colour, double2* out, const double2* in, double a, const double2* x, double c)
{
    GeoScope sc(h, sub_geo(h->g1));
    return hop_full(h, MODE_INTRA, dag, colour, out, in, a, x, c);
}

int embed2(lqcd_ctx* h, double2* full, const double* coords)
{
    GeoScope sc(h, sub_geo(h->g1));
    return embed_boundary(h, full, coords, 1);
}

int project2(lqcd_ctx* h, double* coords, const double2* full)
{
    GeoScope sc(h, sub_geo(h->g1));
    return project_boundary(h, coords, full, 1);
}

// R2, R2^dag, R2^-1, R2^-dag (op 0..3) on second-level boundary fields
int schur2_op(lqcd_ctx* h, double* out, const double* in, double kappa, int op, const SolveCfg& c)
{
    double2 *A = fld(h, F_A), *B = fld(h, F_B), *C = fld(h, F_C), *D = fld(h, F_D), *E = fld(h, F_E);
    LQ_TRY(embed2(h, A, in));
    if (op == LQCD_SCHUR_R) {
        // (1 - C2 A2^-1 B2 D2^-1), B2 = C2 = -kappa H_cross2
        LQ_TRY(sub_solve(h, 1, 0, c, kappa, B, A));
        LQ_TRY(hop_full(h, MODE_CROSS2, 0, -1, C, B, 0.0, nullptr, -kappa));
        LQ_TRY(sub_solve(h, 0, 0, c, kappa, D, C));
        LQ_TRY(hop_full(h, MODE_CROSS2, 0, -1, E, D, 0.0, nullptr, -kappa));
        LQ_TRY(project2(h, out, E));
    } else if (op == LQCD_SCHUR_RDAG) {
        LQ_TRY(hop_full(h, MODE_CROSS2, 1, -1, C, A, 0.0, nullptr, -kappa));
        LQ_TRY(sub_solve(h, 0, 1, c, kappa, D, C));
        LQ_TRY(hop_full(h, MODE_CROSS2, 1, -1, E, D, 0.0, nullptr, -kappa));
        LQ_TRY(sub_solve(h, 1, 1, c, kappa, B, E));
        LQ_TRY(project2(h, out, B));
    } else if (op == LQCD_SCHUR_RINV) {
        LQ_TRY(solve_full(h, MODE_INTRA, -1, 0, c.prec, kappa, B, A, c.tol, c.max_iter, nullptr, nullptr));
        LQ_TRY(sub_hop(h, 0, 1, C, B, 1.0, B, -kappa));
        return project2(h, out, C);
    } else {
        LQ_TRY(sub_hop(h, 1, 1, C, A, 1.0, A, -kappa));
        LQ_TRY(solve_full(h, MODE_INTRA, -1, 1, c.prec, kappa, B, C, c.tol, c.max_iter, nullptr, nullptr));
        return project2(h, out, B);
    }
    return bnd_sub(h, out, in, 2 * nbnd2_of(h->g1));
}

// F += coef * dS/dw for S = |W2^-1 phi|^2
int pf_w2(lqcd_ctx* h, double* F, const double2* phi, double kappa, double coef, const SolveCfg& c,
          double* S_dev, const double* ss = nullptr)
{
    GeoScope sc(h, sub_geo(h->g1));
    return pf_w1(h, F, phi, kappa, coef, c, S_dev, ss);
}

// F += coef * dS/dw for S = |R2^-1 phi|^2 (phi: device second-level boundary field)
int pf_schur2(lqcd_ctx* h, double* F, const double* phi, double kappa, double coef, const SolveCfg& c,
              double* S_dev, const double* ss = nullptr)
{
    double2 *A = fld(h, F_A), *psi = fld(h, F_B), *C = fld(h, F_C), *et = fld(h, F_D), *E = fld(h, F_E),
            *chi = fld(h, F_G);
    double* eta = h->bnd[1];
    LQ_TRY(embed2(h, A, phi));
    LQ_TRY(solve_full(h, MODE_INTRA, -1, 0, c.prec, kappa, psi, A, c.tol, c.max_iter, nullptr, nullptr,
                      SOLVER_BICGSTAB, c.slot));
    LQ_TRY(sub_hop(h, 0, 1, C, psi, 1.0, psi, -kappa));
    LQ_TRY(project2(h, eta, C));
    if (S_dev) LQ_TRY(norm2_dev(h, eta, 2 * nbnd2_of(h->g1), S_dev));
    if (!F) return LQCD_OK;
    LQ_TRY(embed2(h, et, eta));
    LQ_TRY(sub_hop(h, 1, 1, E, et, 1.0, et, -kappa));
    LQ_TRY(solve_full(h, MODE_INTRA, -1, 1, c.prec, kappa, chi, E, c.tol, c.max_iter, nullptr, nullptr,
                      SOLVER_BICGSTAB, next_slot(c.slot)));
    return force_bilinear(h, F, et, psi, MODE_INTRA2, -kappa * coef, chi, psi, MODE_INTRA, kappa * coef, c.prec,
                          ss);
}

// ---------------------------------------------------------------------------
// even-odd + mass preconditioning of W2 (Sec. 1): W2,eo = 1 - kappa^2 H_eo H_oe
// on the even sites of the sub-slabs, W3,eo = W2,eo + rho.  Even-site fields
// live in the parity-0 half of full double fields.
//   S1 = |W3,eo^-1 phi|^2:  dS1 = 2 kappa^2 Re <xi, d(H_eo H_oe) eta>,
//        eta = W3^-1 phi, xi = W3^-dag eta
//   S2 = |W3,eo W2,eo^-1 phi|^2 = |phi + rho zeta|^2, zeta = W2^-1 phi:
//        dS2 = 2 rho kappa^2 Re <W2^-dag chi, d(H_eo H_oe) zeta>
// ---------------------------------------------------------------------------
// out_e = (1 + rho) in_e - kappa^2 H_eo H_oe in_e (dag: the adjoint); out != in
int w3eo_apply(lqcd_ctx* h, double2* out, const double2* in, double kappa, double rho, int dag)
{
    GeoScope sc(h, sub_geo(h->g1));
    const int Vh = h->g.Vh;
    double2* t = fld(h, F_T1);
    LQ_TRY(hop_sweep(h, PREC64, MODE_INTRA, dag, 1, -1, sp64(t, 1, Vh), sp64((double2*)in, 0, Vh), 0.0, none(),
                     1.0));
    return hop_sweep(h, PREC64, MODE_INTRA, dag, 0, -1, sp64(out, 0, Vh), sp64(t, 1, Vh), 1.0 + rho,
                     sp64((double2*)in, 0, Vh), -kappa * kappa);
}

// x_e = W3,eo^-1 b_e, all sub-slabs in one batched launch (dag: W3,eo^-dag =
// g5 W3,eo^-1 g5); x must not alias b
int w3eo_solve(lqcd_ctx* h, double2* x, const double2* b, double kappa, double rho, int dag, const SolveCfg& c,
               int* iters = nullptr, double* resid = nullptr, int slot = -1)
{
    GeoScope sc(h, sub_geo(h->g1));
    const double2* bb = b;
    if (dag) {
        LQ_TRY(gamma5_full(h, fld(h, F_T2), b));
        bb = fld(h, F_T2);
    }
    int guess = 0;
    LQ_TRY(chrono_guess(h, slot, x, dag, &guess));
    LQ_TRY(eo_solve(h, MODE_INTRA, -1, c.prec, kappa, x, bb, c.tol, c.max_iter, iters, resid, 1.0 + rho, c.method,
                    guess));
    if (dag) LQ_TRY(gamma5_full(h, x, x));
    return chrono_store(h, slot, x);
}

// F += coef * d/dw 2 Re <a, d(H_eo H_oe) b> for even-site a, b (parity-0
// halves); their odd halves are overwritten with (H^dag)_oe a and H_oe b
int eo_force(lqcd_ctx* h, double* F, double2* a, double2* b, double coef, int prec, const double* ss)
{
    GeoScope sc(h, sub_geo(h->g1));
    const int Vh = h->g.Vh;
    LQ_TRY(hop_sweep(h, PREC64, MODE_INTRA, 1, 1, -1, sp64(a, 1, Vh), sp64(a, 0, Vh), 0.0, none(), 1.0));
    LQ_TRY(hop_sweep(h, PREC64, MODE_INTRA, 0, 1, -1, sp64(b, 1, Vh), sp64(b, 0, Vh), 0.0, none(), 1.0));
    return force_bilinear(h, F, a, b, MODE_INTRA, coef, nullptr, nullptr, 0, 0.0, prec, ss);
}

int pf_s1(lqcd_ctx* h, double* F, const double2* phi, double kappa, double rho, double coef, const SolveCfg& c,
          double* S_dev, const double* ss = nullptr)
{
    double2 *eta = fld(h, F_A), *xi = fld(h, F_B);
    LQ_TRY(w3eo_solve(h, eta, phi, kappa, rho, 0, c, nullptr, nullptr, c.slot));
    if (S_dev) LQ_TRY(norm2_dev(h, (const double*)eta, (int64_t)24 * h->g.Vh, S_dev));
    if (!F) return LQCD_OK;
    LQ_TRY(w3eo_solve(h, xi, eta, kappa, rho, 1, c, nullptr, nullptr, next_slot(c.slot)));
    return eo_force(h, F, xi, eta, kappa * kappa * coef, c.prec, ss);
}

int pf_s2(lqcd_ctx* h, double* F, const double2* phi, double kappa, double rho, double coef, const SolveCfg& c,
          double* S_dev, const double* ss = nullptr)
{
    double2 *zeta = fld(h, F_A), *lam = fld(h, F_B), *chi = fld(h, F_C);
    LQ_TRY(w3eo_solve(h, zeta, phi, kappa, 0.0, 0, c, nullptr, nullptr, c.slot));
    LQ_TRY(axpby_full(h, chi, 1.0, phi, 0.0, -1));
    LQ_TRY(axpby_full(h, chi, rho, zeta, 1.0, -1));
    if (S_dev) LQ_TRY(norm2_dev(h, (const double*)chi, (int64_t)24 * h->g.Vh, S_dev));
    if (!F) return LQCD_OK;
    LQ_TRY(w3eo_solve(h, lam, chi, kappa, 0.0, 1, c, nullptr, nullptr, next_slot(c.slot)));
    return eo_force(h, F, lam, zeta, rho * kappa * kappa * coef, c.prec, ss);
}

// ---------------------------------------------------------------------------
// integrator schedule (Sec. 2, eqs. (5)-(7)); consecutive kicks of one level
// act on the same field and are merged
// ---------------------------------------------------------------------------
struct Op {
    int kind;  // 0: T_P(level), 1: T_U
    int level;
    double dt;
};

void push_p(std::vector<Op>& v, int level, double dt)
{
    if (!v.empty() && v.back().kind == 0 && v.back().level == level) {
        v.back().dt += dt;
        return;
    }
    v.push_back({0, level, dt});
}

void build_step(const lqcd_hmc_params& p, int j, double dt, std::vector<Op>& v)
{
    const double lam = p.lambda;
    if (j == 0) {
        if (p.scheme[0] == LQCD_LF) {
            push_p(v, 0, 0.5 * dt);
            v.push_back({1, 0, dt});
            push_p(v, 0, 0.5 * dt);
        } else {
            push_p(v, 0, lam * dt);
            v.push_back({1, 0, 0.5 * dt});
            push_p(v, 0, (1.0 - 2.0 * lam) * dt);
            v.push_back({1, 0, 0.5 * dt});
            push_p(v, 0, lam * dt);
        }
        return;
    }
    const int n = p.nsteps[j - 1];
    const double di = dt / n;
    if (p.scheme[j] == LQCD_LF) {
        push_p(v, j, 0.5 * dt);
        for (int i = 0; i < n; ++i) build_step(p, j - 1, di, v);
        push_p(v, j, 0.5 * dt);
    } else {
        push_p(v, j, lam * dt);
        for (int i = 0; i < n / 2; ++i) build_step(p, j - 1, di, v);
        push_p(v, j, (1.0 - 2.0 * lam) * dt);
        for (int i = 0; i < n / 2; ++i) build_step(p, j - 1, di, v);
        push_p(v, j, lam * dt);
    }
}

// chronological slots of the force solves: the solve of a term and its
// adjoint solve; the boundary term's are the whole-lattice solves
enum { SLOT_W1 = 0, SLOT_SCHUR = 2, SLOT_W2 = 4, SLOT_SCHUR2 = 6, SLOT_S2 = 8, SLOT_S1 = 10 };

// solutions kept per slot: chrono + 1 (polynomial extrapolation, at most
// three), all NMRE for the whole-lattice slots with chrono = 3
int chrono_slot_depth(const lqcd_hmc_params& p, int k)
{
    if (p.chrono == 3 && (k == SLOT_SCHUR || k == SLOT_SCHUR + 1)) return lqcd_ctx::NMRE;
    return std::min(p.chrono, 2) + 1;
}

void chrono_configure(lqcd_ctx* h, const lqcd_hmc_params& p)
{
    for (int k = 0; k < lqcd_ctx::NCHRONO; ++k) h->chrono_depth[k] = chrono_slot_depth(p, k);
    h->chrono_mre = p.chrono == 3;
}

// the chronological slots of the force solves (chrono_slot_depth even-half
// double fields each) and the minimal-residual workspace, allocated before
// any capture
int chrono_alloc(lqcd_ctx* h, const lqcd_hmc_params* p)
{
    if (!p->chrono) return LQCD_OK;
    if (p->chrono == 3) LQ_TRY(chrono_mre_alloc(h));
    constexpr int D = lqcd_ctx::CHRONO_MAX;
    const size_t bytes = sizeof(double2) * 12 * (size_t)h->g.Vh;
    for (int k = 0; k < lqcd_ctx::NCHRONO; ++k)
        for (int j = 0; j < chrono_slot_depth(*p, k); ++j) {
            double2*& b = h->chrono_buf[D * k + j];
            if (b) continue;
            LQ_CUDA(h, cudaMalloc(&b, bytes));
            LQ_CUDA(h, cudaMemsetAsync(b, 0, bytes, h->stream));
        }
    return LQCD_OK;
}

int check_params(lqcd_ctx* h, const lqcd_hmc_params* p)
{
    if (!p || p->nlevels < 1 || p->nlevels > LQCD_MAX_LEVELS || !(p->tau > 0) || !prec_ok(p->precision) || !(p->tol > 0)) {
        h->err = "hmc params: bad nlevels / tau / precision / tol";
        return LQCD_ERR_ARG;
    }
    for (int j = 0; j < p->nlevels; ++j) {
        if (p->nsteps[j] < 1 || (p->scheme[j] != LQCD_LF && p->scheme[j] != LQCD_SW)) {
            h->err = "hmc params: bad nsteps / scheme";
            return LQCD_ERR_ARG;
        }
        if (j >= 1 && p->scheme[j] == LQCD_SW && (p->nsteps[j - 1] % 2)) {
            h->err = "hmc params: an SW level needs an even number of inner steps";
            return LQCD_ERR_ARG;
        }
    }
    const int lv[7] = {p->level_gauge, p->level_w1, p->level_schur, p->level_w2, p->level_schur2,
                       p->level_s2, p->level_s1};
    for (int k = 0; k < 7; ++k)
        if (lv[k] < -1 || lv[k] >= p->nlevels) {
            h->err = "hmc params: term level out of range";
            return LQCD_ERR_ARG;
        }
    if ((p->level_w2 >= 0 || p->level_schur2 >= 0 || p->level_s2 >= 0 || p->level_s1 >= 0) && !h->g1.l0s) {
        h->err = "hmc params: the W2 / R2 / S2 / S1 terms need sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    if (p->use_graph != 0 && p->use_graph != 1) {
        h->err = "hmc params: use_graph must be 0 or 1";
        return LQCD_ERR_ARG;
    }
    if (p->chrono < 0 || p->chrono > 3) {
        h->err = "hmc params: chrono must be 0, 1, 2 or 3";
        return LQCD_ERR_ARG;
    }
    if ((p->eo_solver != LQCD_SOLVER_BICGSTAB && p->eo_solver != LQCD_SOLVER_SERIES) ||
        (p->block_solver != LQCD_SOLVER_BICGSTAB && p->block_solver != LQCD_SOLVER_SERIES)) {
        h->err = "hmc params: bad eo_solver / block_solver";
        return LQCD_ERR_ARG;
    }
    if (!p->step_scale && p->step_scheme) {
        const int per[4] = {0, 6, 8, 16};
        if (p->step_scheme < 0 || p->step_scheme > 3 || h->g.L[0] % per[p->step_scheme]) {
            h->err = "hmc params: step_scheme unknown or its period does not divide L0";
            return LQCD_ERR_ARG;
        }
    }
    return LQCD_OK;
}

// step-size schemes of Sec. 2 (space-like, time-like values over one period)
void scheme_table(int scheme, int L0, double* out)
{
    static const double a_sp[6] = {0.2, 0.5, 1.0, 1.0, 0.5, 0.2};  // s(5): printed "2", read 0.2
    static const double a_tm[6] = {0.2, 0.5, 1.0, 0.5, 0.2, 0.0};
    static const double b_sp[8] = {0.0, 0.5, 1.0, 1.0, 1.0, 1.0, 0.5, 0.0};
    static const double b_tm[8] = {0.0, 0.5, 1.0, 1.0, 1.0, 0.5, 0.0, 0.0};
    static const double c_sp[16] = {0.0, 0.25, 0.5, 1.0, 1.0, 1.0, 1.0, 0.25, 0.25, 1.0, 1.0, 1.0, 1.0, 0.5, 0.25, 0.0};
    static const double c_tm[16] = {0.0, 0.0, 0.25, 0.5, 1.0, 1.0, 0.25, 0.0, 0.25, 1.0, 1.0, 1.0, 0.5, 0.25, 0.0, 0.0};
    const double* sp = scheme == 1 ? a_sp : scheme == 2 ? b_sp : c_sp;
    const double* tm = scheme == 1 ? a_tm : scheme == 2 ? b_tm : c_tm;
    const int per = scheme == 1 ? 6 : scheme == 2 ? 8 : 16;
    for (int t = 0; t < L0; ++t) {
        out[t] = sp[t % per];
        out[L0 + t] = tm[t % per];
    }
}

// device step-size table of this MD, or null for s = 1
int md_scale_table(lqcd_ctx* h, const lqcd_hmc_params& p, const double** out)
{
    *out = nullptr;
    if (!p.step_scale && !p.step_scheme) return LQCD_OK;
    const int L0 = h->g.L[0];
    std::vector<double> tab(2 * L0);
    if (p.step_scale) std::copy(p.step_scale, p.step_scale + 2 * L0, tab.begin());
    else scheme_table(p.step_scheme, L0, tab.data());
    LQ_CUDA(h, cudaMemcpyAsync(h->d_sscale, tab.data(), sizeof(double) * 2 * L0, cudaMemcpyHostToDevice, h->stream));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    *out = h->d_sscale;
    return LQCD_OK;
}

// pseudo-fermion fields of the MD: phi1 (W1), phi2 (R), phi3 (W2), phi4 (R2),
// phi5 (S2, even sites), phi6 (S1, even sites)
struct PfFields {
    const double2* phi1;
    const double* phi2;
    const double2* phi3;
    const double* phi4;
    const double2* phi5;
    const double2* phi6;
};

// the molecular dynamics of eqs. (5)-(7); ss: device step-size table or null
int do_md(lqcd_ctx* h, const lqcd_hmc_params& p, double* P, const PfFields& pf, int* nforce, const double* ss)
{
    std::vector<Op> ops;
    const int top = p.nlevels - 1;
    const double dt = p.tau / p.nsteps[top];
    for (int i = 0; i < p.nsteps[top]; ++i) build_step(p, top, dt, ops);
    // chronological slots (two per term: the solve and its adjoint)
    const bool ch = p.chrono != 0;
    const SolveCfg cw1{p.precision, p.tol, p.max_iter, p.block_solver, ch ? SLOT_W1 : -1};
    const SolveCfg csch{p.precision, p.tol, p.max_iter, SOLVER_BICGSTAB, ch ? SLOT_SCHUR : -1};
    const SolveCfg cw2{p.precision, p.tol, p.max_iter, p.block_solver, ch ? SLOT_W2 : -1};
    const SolveCfg csch2{p.precision, p.tol, p.max_iter, SOLVER_BICGSTAB, ch ? SLOT_SCHUR2 : -1};
    const SolveCfg cs2{p.precision, p.tol, p.max_iter, p.eo_solver, ch ? SLOT_S2 : -1};
    const SolveCfg cs1{p.precision, p.tol, p.max_iter, p.eo_solver, ch ? SLOT_S1 : -1};
    for (int k = 0; k < lqcd_ctx::NCHRONO; ++k) h->chrono_n[k] = h->chrono_cur[k] = 0;
    chrono_configure(h, p);
    h->md_time = 0.0;
    for (const Op& o : ops) {
        if (o.kind == 1) {
            LQ_TRY(update_links(h, P, o.dt, ss));
            h->md_time += o.dt;
            continue;
        }
        if (p.level_gauge == o.level) LQ_TRY(gauge_force_kick(h, P, -o.dt * p.beta / 6.0, p.precision, ss));
        if (p.level_w1 == o.level) {
            LQ_TRY(pf_w1(h, P, pf.phi1, p.kappa, -o.dt, cw1, nullptr, ss));
            ++*nforce;
        }
        if (p.level_schur == o.level) {
            LQ_TRY(pf_schur(h, P, pf.phi2, p.kappa, -o.dt, csch, nullptr, ss));
            ++*nforce;
        }
        if (p.level_w2 == o.level) {
            LQ_TRY(pf_w2(h, P, pf.phi3, p.kappa, -o.dt, cw2, nullptr, ss));
            ++*nforce;
        }
        if (p.level_schur2 == o.level) {
            LQ_TRY(pf_schur2(h, P, pf.phi4, p.kappa, -o.dt, csch2, nullptr, ss));
            ++*nforce;
        }
        if (p.level_s2 == o.level) {
            LQ_TRY(pf_s2(h, P, pf.phi5, p.kappa, p.rho, -o.dt, cs2, nullptr, ss));
            ++*nforce;
        }
        if (p.level_s1 == o.level) {
            LQ_TRY(pf_s1(h, P, pf.phi6, p.kappa, p.rho, -o.dt, cs1, nullptr, ss));
            ++*nforce;
        }
    }
    return LQCD_OK;
}

// the parameters a recorded MD graph depends on (the step table by value)
std::vector<unsigned char> md_key(const lqcd_ctx* h, const lqcd_hmc_params& p)
{
    std::vector<double> k = {p.beta, p.kappa, p.tau, p.lambda, (double)p.nlevels, (double)p.level_gauge,
                             (double)p.level_w1, (double)p.level_schur, (double)p.level_w2, (double)p.level_schur2,
                             (double)p.level_s2, (double)p.level_s1, p.rho, (double)p.precision, p.tol,
                             (double)p.max_iter, (double)p.eo_solver, (double)p.block_solver,
                             (double)p.step_scheme, (double)p.chrono,
                             (double)h->prof.on, (double)h->g1.l0s, (double)h->wait_limit,
                             (double)h->global_method, (double)h->sap_terms};
    for (int q = 0; q < NPREC; ++q) {
        k.push_back((double)h->tune.hop_bs[q]);
        k.push_back((double)h->tune.solve_spt[q][0]);
        k.push_back((double)h->tune.solve_spt[q][1]);
        k.push_back((double)h->tune.cluster_series);
    }
    for (int j = 0; j < LQCD_MAX_LEVELS; ++j) {
        k.push_back((double)p.scheme[j]);
        k.push_back((double)p.nsteps[j]);
    }
    if (p.step_scale)
        for (int t = 0; t < 2 * h->g.L[0]; ++t) k.push_back(p.step_scale[t]);
    std::vector<unsigned char> out(k.size() * sizeof(double));
    memcpy(out.data(), k.data(), out.size());
    return out;
}

// the molecular dynamics as a CUDA graph: recorded (not run) the first time
// for a parameter set, then replayed; the solves inside report their status
// and iteration counts through device memory, read once after the replay
int md_graph(lqcd_ctx* h, const lqcd_hmc_params& p, const PfFields& pf, const double* ss, int* nforce)
{
    std::vector<unsigned char> key = md_key(h, p);
    if (!h->md_exec || key != h->md_key) {
        if (h->md_exec) {
            cudaGraphExecDestroy(h->md_exec);
            h->md_exec = nullptr;
        }
        for (auto& r : h->prof.graph_recs) {
            h->prof.pool.push_back(r.a);
            h->prof.pool.push_back(r.b);
        }
        h->prof.graph_recs.clear();
        if (!h->cap_stream) LQ_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = h->stream;
        const int64_t l0 = h->launches;
        const int s0 = h->solve_count;
        h->stream = h->cap_stream;
        h->deferred = true;
        h->capturing = true;
        cudaError_t eb = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        int nf = 0;
        int st = eb == cudaSuccess ? do_md(h, p, h->P, pf, &nf, ss) : LQCD_OK;
        cudaGraph_t graph = nullptr;
        cudaError_t ee = eb == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &graph) : eb;
        h->stream = user;
        h->deferred = false;
        h->capturing = false;
        const int64_t nl = h->launches - l0;
        const int ns = h->solve_count - s0;
        h->launches = l0;
        h->solve_count = s0;
        if (st != LQCD_OK || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st == LQCD_OK) {
                h->err = std::string("recording the MD graph: ") + cudaGetErrorString(ee);
                st = LQCD_ERR_CUDA;
            }
            return st;
        }
        cudaError_t ei = cudaGraphInstantiate(&h->md_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            h->md_exec = nullptr;
            h->err = std::string("instantiating the MD graph: ") + cudaGetErrorString(ei);
            return LQCD_ERR_CUDA;
        }
        h->md_key = key;
        h->md_launches = nl;
        h->md_nforce = nf;
        h->md_solves = ns;
    }
    {
        // clears what eager solves left in the sticky word; each of them has
        // already reported its own status, so only a failed read counts
        const int st0 = solver_collect(h, nullptr, nullptr);
        if (st0 == LQCD_ERR_CUDA) return st0;
    }
    LQ_CUDA(h, cudaGraphLaunch(h->md_exec, h->stream));
    h->launches += h->md_launches;
    h->solve_count += h->md_solves;
    *nforce += h->md_nforce;
    int64_t it = 0, sit = 0, osit = 0, ssit = 0, asit = 0;
    const int st = solver_collect(h, &it, &sit, &osit, &ssit, &asit);
    h->iter_count += it;
    h->site_iters += sit + ssit + asit;
    h->hop_sites += solver_hops_per_iter(SOLVER_BICGSTAB, 0) * sit + solver_hops_per_iter(SOLVER_SERIES, 0) * ssit +
                    (int64_t)solver_hops_per_iter(h->global_method, h->sap_terms) * asit;
    // kernel times of this replay (the stream is synchronised); the solver's
    // algorithmic bytes follow from the replay's iteration sums
    if (!h->prof.graph_recs.empty()) {
        for (const auto& r : h->prof.graph_recs) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, r.a, r.b);
            h->prof.launches[r.id] += 1;
            h->prof.ms[r.id] += ms;
            if (r.id != 1) h->prof.bytes[r.id] += r.bytes;
            if (h->prof.hist[r.id].size() < 65536) h->prof.hist[r.id].push_back(ms);
        }
        double bi, bo, bs;
        double ba;
        solver_site_bytes(p.precision, SOLVER_BICGSTAB, &bi, &bo);
        solver_site_bytes(p.precision, SOLVER_SERIES, &bs, &bo);
        solver_site_bytes(p.precision, h->global_method == SOLVER_SAPB ? SOLVER_SAPB : SOLVER_SAP, &ba, &bo,
                          h->sap_terms);
        h->prof.bytes[1] += (double)sit * bi + (double)ssit * bs + (double)asit * ba + (double)osit * bo;
    }
    return st;
}

// host Philox4x32-10 for the Metropolis uniform and the x0 shift
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t a = (uint64_t)0xD2511F53u * c[0], b = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c[1] ^ k0, n1 = (uint32_t)b;
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c[3] ^ k1, n3 = (uint32_t)a;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
}

// the (up to) eight energy terms: kinetic, gauge, W1, Schur, W2, Schur2, S2, S1
// -> red_out[base..base+7]
constexpr int NTERM = 8;

// the energies at the end of the molecular dynamics.  With chronological
// guesses every term's solve starts from the solution of its last force
// evaluation, which was on these same final links (every integrator level
// ends with a kick), so it needs no iteration.  The slots are only read:
// a replayed MD graph relies on the host-side slot state it was recorded
// with.
struct ChronoFreeze {
    lqcd_ctx* h;
    explicit ChronoFreeze(lqcd_ctx* c) : h(c) { h->chrono_frozen = true; }
    ~ChronoFreeze() { h->chrono_frozen = false; }
};

int energy(lqcd_ctx* h, const lqcd_hmc_params& p, const PfFields& pf, int base)
{
    const bool ch = p.chrono != 0;
    chrono_configure(h, p);
    ChronoFreeze freeze(h);
    double* e = h->red_out + base;
    LQ_TRY(kinetic_sum(h, h->P, e));
    if (p.level_gauge >= 0) LQ_TRY(plaquette_sum(h, e + 1));
    const SolveCfg cw1{p.precision, p.tol, p.max_iter, p.block_solver, ch ? SLOT_W1 : -1};
    const SolveCfg csch{p.precision, p.tol, p.max_iter, SOLVER_BICGSTAB, ch ? SLOT_SCHUR : -1};
    const SolveCfg cw2{p.precision, p.tol, p.max_iter, p.block_solver, ch ? SLOT_W2 : -1};
    const SolveCfg csch2{p.precision, p.tol, p.max_iter, SOLVER_BICGSTAB, ch ? SLOT_SCHUR2 : -1};
    const SolveCfg cs2{p.precision, p.tol, p.max_iter, p.eo_solver, ch ? SLOT_S2 : -1};
    const SolveCfg cs1{p.precision, p.tol, p.max_iter, p.eo_solver, ch ? SLOT_S1 : -1};
    if (p.level_w1 >= 0) LQ_TRY(pf_w1(h, nullptr, pf.phi1, p.kappa, 0.0, cw1, e + 2));
    if (p.level_schur >= 0) LQ_TRY(pf_schur(h, nullptr, pf.phi2, p.kappa, 0.0, csch, e + 3));
    if (p.level_w2 >= 0) LQ_TRY(pf_w2(h, nullptr, pf.phi3, p.kappa, 0.0, cw2, e + 4));
    if (p.level_schur2 >= 0) LQ_TRY(pf_schur2(h, nullptr, pf.phi4, p.kappa, 0.0, csch2, e + 5));
    if (p.level_s2 >= 0) LQ_TRY(pf_s2(h, nullptr, pf.phi5, p.kappa, p.rho, 0.0, cs2, e + 6));
    if (p.level_s1 >= 0) LQ_TRY(pf_s1(h, nullptr, pf.phi6, p.kappa, p.rho, 0.0, cs1, e + 7));
    return LQCD_OK;
}

double combine(const lqcd_hmc_params& p, const double* e)
{
    double H = 0.5 * e[0];
    if (p.level_gauge >= 0) H += -p.beta / 3.0 * e[1];
    if (p.level_w1 >= 0) H += e[2];
    if (p.level_schur >= 0) H += e[3];
    if (p.level_w2 >= 0) H += e[4];
    if (p.level_schur2 >= 0) H += e[5];
    if (p.level_s2 >= 0) H += e[6];
    if (p.level_s1 >= 0) H += e[7];
    return H;
}

}  // namespace

// small elementwise helper for boundary vectors: out = in - out
namespace {
__global__ void k_bnd_sub(double* out, const double* in, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = in[t] - out[t];
}
}  // namespace
int bnd_sub(lqcd_ctx* h, double* out, const double* in, int n)
{
    k_bnd_sub<<<(n + 255) / 256, 256, 0, h->stream>>>(out, in, n);
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->err = std::string("bnd_sub: ") + cudaGetErrorString(e);
        return LQCD_ERR_CUDA;
    }
    return LQCD_OK;
}

// ---------------------------------------------------------------------------
// views and profiling
// ---------------------------------------------------------------------------
GaugeF gauge_view(lqcd_ctx* h, int prec)
{
    GaugeF g;
    g.Vh = h->g.Vh;
    g.v = (prec == PREC64 || prec == PRECDF) ? (const void*)h->U64
          : prec == PREC32                     ? (const void*)h->U32
          : prec == PREC16                     ? (const void*)h->U16
                                               : (const void*)(h->U16 + (size_t)24 * h->g.Vh);
    return g;
}

void prof_begin(lqcd_ctx* h, int id, cudaEvent_t* a)
{
    *a = nullptr;
    if (!(h->prof.on & (1u << id))) return;
    if (h->prof.pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        h->prof.pool.push_back(e);
    }
    *a = h->prof.pool.back();
    h->prof.pool.pop_back();
    // while a graph is recorded, an external record makes the event a node
    // of the graph, updated by every replay
    if (h->capturing) cudaEventRecordWithFlags(*a, h->stream, cudaEventRecordExternal);
    else cudaEventRecord(*a, h->stream);
}

void prof_end(lqcd_ctx* h, int id, cudaEvent_t a, double bytes)
{
    if (!(h->prof.on & (1u << id)) || !a) return;
    cudaEvent_t b;
    if (h->prof.pool.empty()) {
        if (cudaEventCreate(&b) != cudaSuccess) return;
    } else {
        b = h->prof.pool.back();
        h->prof.pool.pop_back();
    }
    if (h->capturing) cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal);
    else cudaEventRecord(b, h->stream);
    // inside a graph recording the pair becomes two event-record nodes,
    // read after every replay
    if (h->capturing) h->prof.graph_recs.push_back({a, b, id, bytes});
    else h->prof.recs.push_back({a, b, id, bytes});
}

static void prof_flush(lqcd_ctx* h)
{
    if (h->prof.recs.empty()) return;
    cudaStreamSynchronize(h->stream);
    for (auto& r : h->prof.recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        h->prof.launches[r.id] += 1;
        h->prof.ms[r.id] += ms;
        h->prof.bytes[r.id] += r.bytes;
        if (h->prof.hist[r.id].size() < 65536) h->prof.hist[r.id].push_back(ms);
        h->prof.pool.push_back(r.a);
        h->prof.pool.push_back(r.b);
    }
    h->prof.recs.clear();
}

// ---------------------------------------------------------------------------
// extern "C" entry points
// ---------------------------------------------------------------------------
#define CHECK_H(h)                          \
    do {                                    \
        if (!(h)) return LQCD_ERR_ARG;      \
    } while (0)
#define NEED_GAUGE(h)                                         \
    do {                                                      \
        if (!(h)->have_gauge) {                               \
            (h)->err = "no gauge field set (lqcd_set_gauge)"; \
            return LQCD_ERR_STATE;                            \
        }                                                     \
    } while (0)
#define NEED(cond, msg)               \
    do {                              \
        if (!(cond)) {                \
            h->err = (msg);           \
            return LQCD_ERR_ARG;      \
        }                             \
    } while (0)

extern "C" {

int lqcd_create(lqcd_t* out, const int L[4], int l0, int bc_t, void* stream)
{
    if (!out || !L) return LQCD_ERR_ARG;
    *out = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        if (L[mu] < 2 || (L[mu] & 1)) return LQCD_ERR_GEOM;
    if (l0 < 1 || L[0] % (2 * l0)) return LQCD_ERR_GEOM;
    if (bc_t != 1 && bc_t != -1) return LQCD_ERR_ARG;
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    if (32 * V >= ((int64_t)1 << 31)) return LQCD_ERR_GEOM;
    lqcd_ctx* h = new lqcd_ctx();
    Geo& g = h->g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = L[mu];
    g.V = (int)V;
    g.Vh = g.V / 2;
    g.V3 = L[1] * L[2] * L[3];
    g.l0 = l0;
    g.nb = L[0] / l0;
    g.bc_t = bc_t;
    g.Sh = l0 * g.V3 / 2;
    g.l0s = 0;
    geo_finish(g);
    h->g1 = g;
    h->stream = (cudaStream_t)stream;
    *out = h;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        h->err = "no CUDA device";
        return LQCD_ERR_CUDA;
    }
    const size_t Vh = g.Vh;
    LQ_CUDA(h, cudaMalloc(&h->U64, sizeof(double2) * 72 * Vh));
    LQ_CUDA(h, cudaMalloc(&h->U64_save, sizeof(double2) * 72 * Vh));
    LQ_CUDA(h, cudaMalloc(&h->U32, sizeof(float4) * 24 * Vh));
    LQ_CUDA(h, cudaMalloc(&h->U16, sizeof(uint2) * 48 * Vh));  // fp16, then bf16
    h->f64.assign(NFIELD, nullptr);
    for (int k = 0; k < NFIELD; ++k) LQ_CUDA(h, cudaMalloc(&h->f64[k], sizeof(double2) * 24 * Vh));
    LQ_CUDA(h, cudaMalloc(&h->P, sizeof(double) * 32 * (size_t)g.V));
    LQ_CUDA(h, cudaMalloc(&h->F, sizeof(double) * 32 * (size_t)g.V));
    LQ_CUDA(h, cudaMalloc(&h->d_sscale, sizeof(double) * 2 * (size_t)g.L[0]));
    const size_t nb2 = 2 * (size_t)nbnd_of(g);
    for (int k = 0; k < 4; ++k) LQ_CUDA(h, cudaMalloc(&h->bnd[k], sizeof(double) * std::max<size_t>(nb2, 2)));
    h->red_blocks = reduction_blocks();
    LQ_CUDA(h, cudaMalloc(&h->red_part, sizeof(double) * h->red_blocks));
    LQ_CUDA(h, cudaMalloc(&h->red_out, sizeof(double) * 32));
    LQ_CUDA(h, cudaMallocHost(&h->red_host, sizeof(double) * 32));
    LQ_CUDA(h, cudaMemsetAsync(h->red_out, 0, sizeof(double) * 32, h->stream));
    return solver_init(h);
}

int lqcd_destroy(lqcd_t h)
{
    if (!h) return LQCD_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->md_exec) cudaGraphExecDestroy(h->md_exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    solver_free(h);
    cudaFree(h->U64);
    cudaFree(h->U64_save);
    for (double2* f : h->chrono_buf) cudaFree(f);
    chrono_mre_free(h);
    cudaFree(h->U32);
    cudaFree(h->U16);
    for (double2* f : h->f64) cudaFree(f);
    cudaFree(h->P);
    cudaFree(h->F);
    cudaFree(h->d_sscale);
    for (int k = 0; k < 4; ++k) cudaFree(h->bnd[k]);
    cudaFree(h->red_part);
    cudaFree(h->red_out);
    cudaFreeHost(h->red_host);
    for (auto& r : h->prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto& r : h->prof.graph_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    delete h;
    return LQCD_OK;
}

const char* lqcd_last_error(lqcd_t h) { return h ? h->err.c_str() : "null handle"; }

int lqcd_set_stream(lqcd_t h, void* stream)
{
    CHECK_H(h);
    h->stream = (cudaStream_t)stream;
    return LQCD_OK;
}

int lqcd_set_subslabs(lqcd_t h, int l0s)
{
    CHECK_H(h);
    if (l0s != 0 && (h->g1.l0 % 2 || l0s * 2 != h->g1.l0)) {
        h->err = "sub-slab thickness must be l0 / 2 (l0 even), or 0";
        return LQCD_ERR_GEOM;
    }
    h->g1.l0s = l0s;
    geo_finish(h->g1);
    h->g = h->g1;
    return LQCD_OK;
}

int lqcd_set_gauge(lqcd_t h, const double* U)
{
    CHECK_H(h);
    NEED(U, "null gauge pointer");
    LQ_TRY(pack_gauge(h, U));
    h->have_gauge = true;
    return LQCD_OK;
}

int lqcd_get_gauge(lqcd_t h, double* U)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(U, "null gauge pointer");
    return unpack_gauge(h, U);
}

int lqcd_index_maps(lqcd_t h, int32_t* maps)
{
    CHECK_H(h);
    NEED(maps, "null maps pointer");
    return index_maps(h, maps);
}

int lqcd_dslash_eo(lqcd_t h, double* out, const double* in, double kappa, int parity, int dagger, int op,
                   int precision)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(out && in, "null field pointer");
    NEED(parity == 0 || parity == 1, "parity must be 0 or 1");
    NEED(op == LQCD_OP_HOP || (op == LQCD_OP_MHAT && parity == 0), "op must be HOP, or MHAT with parity 0");
    NEED(prec_ok(precision), "bad precision");
    const int Vh = h->g.Vh;
    double2 *A = fld(h, F_A), *B = fld(h, F_B);
    const int pin = op == LQCD_OP_HOP ? 1 - parity : 0;
    LQ_TRY(pack_spinor(h, A, in, pin, 1));
    // low-precision work fields live in F_C / F_D (same byte size as double)
    SpinorF src = sp64(A, pin, Vh), res = sp64(B, parity, Vh);
    if (precision != LQCD_PREC_F64) {
        auto lowview = [&](double2* buf, int par) {
            SpinorF f;
            f.v = (char*)buf + (size_t)par * 12 * Vh * sizeof(double2);
            f.N = Vh;
            f.nrm = precision == PREC16 ? (float*)((uint4*)f.v + (size_t)3 * Vh) : nullptr;
            return f;
        };
        SpinorF ls = lowview(fld(h, F_C), pin), lr = lowview(fld(h, F_D), parity);
        LQ_TRY(convert_spinor(h, ls, precision, src, PREC64, Vh));
        if (op == LQCD_OP_HOP) {
            LQ_TRY(hop_sweep(h, precision, MODE_ALL, dagger, parity, -1, lr, ls, 0.0, none(), 1.0));
        } else {
            SpinorF lt = lowview(fld(h, F_E), 1);
            LQ_TRY(hop_sweep(h, precision, MODE_ALL, dagger, 1, -1, lt, ls, 0.0, none(), 1.0));
            LQ_TRY(hop_sweep(h, precision, MODE_ALL, dagger, 0, -1, lr, lt, 1.0, ls, -kappa * kappa));
        }
        LQ_TRY(convert_spinor(h, res, PREC64, lr, precision, Vh));
    } else if (op == LQCD_OP_HOP) {
        LQ_TRY(hop_sweep(h, PREC64, MODE_ALL, dagger, parity, -1, res, src, 0.0, none(), 1.0));
    } else {
        SpinorF tt = sp64(fld(h, F_C), 1, Vh);
        LQ_TRY(hop_sweep(h, PREC64, MODE_ALL, dagger, 1, -1, tt, src, 0.0, none(), 1.0));
        LQ_TRY(hop_sweep(h, PREC64, MODE_ALL, dagger, 0, -1, res, tt, 1.0, src, -kappa * kappa));
    }
    return unpack_spinor(h, out, B, parity, 1);
}

}  // extern "C"

// W1 (level-1 geometry) or W2 (inside a GeoScope on the sub-slab geometry)
static int block_dslash_impl(lqcd_t h, double* out, const double* in, double kappa, int colour, int dagger,
                             int precision)
{
    const int Vh = h->g.Vh;
    double2 *A = fld(h, F_A), *B = fld(h, F_B);
    LQ_TRY(pack_spinor(h, A, in, 0, 2));
    if (precision == LQCD_PREC_F64) {
        LQ_TRY(hop_full(h, MODE_INTRA, dagger, colour, B, A, 1.0, A, -kappa));
    } else {
        auto lowview = [&](double2* buf, int par) {
            SpinorF f;
            f.v = (char*)buf + (size_t)par * 12 * Vh * sizeof(double2);
            f.N = Vh;
            f.nrm = precision == PREC16 ? (float*)((uint4*)f.v + (size_t)3 * Vh) : nullptr;
            return f;
        };
        for (int p = 0; p < 2; ++p) LQ_TRY(convert_spinor(h, lowview(fld(h, F_C), p), precision, sp64(A, p, Vh), PREC64, Vh));
        for (int p = 0; p < 2; ++p)
            LQ_TRY(hop_sweep(h, precision, MODE_INTRA, dagger, p, colour, lowview(fld(h, F_D), p),
                             lowview(fld(h, F_C), 1 - p), 1.0, lowview(fld(h, F_C), p), -kappa));
        LQ_CUDA(h, cudaMemsetAsync(B, 0, sizeof(double2) * 24 * (size_t)Vh, h->stream));
        for (int p = 0; p < 2; ++p) LQ_TRY(convert_spinor(h, sp64(B, p, Vh), PREC64, lowview(fld(h, F_D), p), precision, Vh));
        if (colour >= 0) LQ_TRY(keep_colour(h, B, colour));
    }
    return unpack_spinor(h, out, B, 0, 2);
}

static int block_solve_impl(lqcd_t h, double* x, const double* b, double kappa, int colour, int dagger,
                            int precision, double tol, int max_iter, int* iters_out, double* resid_out)
{
    double2 *A = fld(h, F_A), *B = fld(h, F_B);
    LQ_TRY(pack_spinor(h, A, b, 0, 2));
    const int nsys = colour < 0 ? h->g.nb : h->g.nb / 2;
    std::vector<int> it(nsys, 0);
    std::vector<double> rs(nsys, 0.0);
    const int st = solve_full(h, MODE_INTRA, colour, dagger, precision, kappa, B, A, tol, max_iter, it.data(), rs.data());
    if (iters_out || resid_out)
        for (int k = 0; k < h->g.nb; ++k) {
            if (iters_out) iters_out[k] = 0;
            if (resid_out) resid_out[k] = 0.0;
        }
    for (int s = 0; s < nsys; ++s) {
        const int slab = colour < 0 ? s : colour + 2 * s;
        if (iters_out) iters_out[slab] = it[s];
        if (resid_out) resid_out[slab] = rs[s];
    }
    LQ_TRY(st);
    LQ_TRY(unpack_spinor(h, x, B, 0, 2));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

extern "C" {

int lqcd_block_dslash(lqcd_t h, double* out, const double* in, double kappa, int colour, int dagger, int precision)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(out && in, "null field pointer");
    NEED(colour >= -1 && colour <= 1, "colour must be -1, 0 or 1");
    NEED(prec_ok(precision), "bad precision");
    return block_dslash_impl(h, out, in, kappa, colour, dagger, precision);
}

int lqcd_subblock_dslash(lqcd_t h, double* out, const double* in, double kappa, int colour, int dagger,
                         int precision)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(out && in, "null field pointer");
    NEED(colour >= -1 && colour <= 1, "colour must be -1, 0 or 1");
    NEED(prec_ok(precision), "bad precision");
    if (!h->g1.l0s) {
        h->err = "no sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    GeoScope sc(h, sub_geo(h->g1));
    return block_dslash_impl(h, out, in, kappa, colour, dagger, precision);
}

int lqcd_block_solve_batched(lqcd_t h, double* x, const double* b, double kappa, int colour, int dagger,
                             int precision, double tol, int max_iter, int* iters_out, double* resid_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(x && b, "null field pointer");
    NEED(colour >= -1 && colour <= 1, "colour must be -1, 0 or 1");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    return block_solve_impl(h, x, b, kappa, colour, dagger, precision, tol, max_iter, iters_out, resid_out);
}

int lqcd_subblock_solve_batched(lqcd_t h, double* x, const double* b, double kappa, int colour, int dagger,
                                int precision, double tol, int max_iter, int* iters_out, double* resid_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(x && b, "null field pointer");
    NEED(colour >= -1 && colour <= 1, "colour must be -1, 0 or 1");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    if (!h->g1.l0s) {
        h->err = "no sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    GeoScope sc(h, sub_geo(h->g1));
    return block_solve_impl(h, x, b, kappa, colour, dagger, precision, tol, max_iter, iters_out, resid_out);
}

int lqcd_solve_wilson(lqcd_t h, double* x, const double* b, double kappa, int dagger, int precision, double tol,
                      int max_iter, int* iters_out, double* resid_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(x && b, "null field pointer");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    double2 *A = fld(h, F_A), *B = fld(h, F_B);
    LQ_TRY(pack_spinor(h, A, b, 0, 2));
    int it = 0;
    double rs = 0.0;
    LQ_TRY(solve_full(h, MODE_ALL, -1, dagger, precision, kappa, B, A, tol, max_iter, &it, &rs));
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = rs;
    LQ_TRY(unpack_spinor(h, x, B, 0, 2));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

int lqcd_schur_apply(lqcd_t h, double* out, const double* in, double kappa, int op, int precision, double tol,
                     int max_iter)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(out && in && out != in, "null or aliased boundary pointer");
    NEED(op >= LQCD_SCHUR_R && op <= LQCD_SCHUR2_RINVDAG, "bad Schur op");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    SolveCfg c{precision, tol, max_iter};
    if (op >= LQCD_SCHUR2_R) {
        if (!h->g1.l0s) {
            h->err = "no sub-slabs (lqcd_set_subslabs)";
            return LQCD_ERR_STATE;
        }
        LQ_TRY(schur2_op(h, out, in, kappa, op - LQCD_SCHUR2_R, c));
    } else {
        LQ_TRY(schur_op(h, out, in, kappa, op, c));
    }
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

int lqcd_pf_force(lqcd_t h, double* F, const double* phi, double kappa, int term, int precision, double tol,
                  int max_iter, double* S_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(phi, "null phi");
    NEED(term >= LQCD_TERM_W1 && term <= LQCD_TERM_SCHUR2, "bad term");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    if (term >= LQCD_TERM_W2 && !h->g1.l0s) {
        h->err = "no sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    SolveCfg c{precision, tol, max_iter};
    if (term == LQCD_TERM_W1) {
        LQ_TRY(pack_spinor(h, fld(h, F_PHI1), phi, 0, 2));
        LQ_TRY(pf_w1(h, F, fld(h, F_PHI1), kappa, 1.0, c, h->red_out));
    } else if (term == LQCD_TERM_SCHUR) {
        LQ_TRY(pf_schur(h, F, phi, kappa, 1.0, c, h->red_out));
    } else if (term == LQCD_TERM_W2) {
        LQ_TRY(pack_spinor(h, fld(h, F_PHI3), phi, 0, 2));
        LQ_TRY(pf_w2(h, F, fld(h, F_PHI3), kappa, 1.0, c, h->red_out));
    } else {
        LQ_TRY(pf_schur2(h, F, phi, kappa, 1.0, c, h->red_out));
    }
    double S;
    LQ_TRY(read_scalars(h, 1, &S));
    if (S_out) *S_out = S;
    return LQCD_OK;
}

int lqcd_gauge_force(lqcd_t h, double* F, double beta, double* S_out, double* plaq_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    if (F) LQ_TRY(gauge_force_kick(h, F, beta / 6.0, PREC64));
    LQ_TRY(plaquette_sum(h, h->red_out));
    double s;
    LQ_TRY(read_scalars(h, 1, &s));
    if (S_out) *S_out = -beta / 3.0 * s;
    if (plaq_out) *plaq_out = s / (18.0 * h->g.V);
    return LQCD_OK;
}

int lqcd_link_update(lqcd_t h, double* U, const double* P, double dt)
{
    CHECK_H(h);
    NEED(U && P, "null U / P");
    LQ_TRY(pack_gauge(h, U));
    h->have_gauge = true;
    LQ_TRY(update_links(h, P, dt));
    LQ_TRY(unpack_gauge(h, U));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

int lqcd_rng_normals(lqcd_t h, double* out, int64_t n, uint64_t seed, uint32_t stream, uint32_t traj)
{
    CHECK_H(h);
    NEED(out || n == 0, "null output");
    NEED(n >= 0, "negative n");
    return rng_normals(h, out, n, seed, stream, traj, 1.0);
}

int lqcd_md(lqcd_t h, double* U, double* P, const lqcd_pf_fields* f, const lqcd_hmc_params* prm)
{
    CHECK_H(h);
    NEED(U && P && f, "null U / P / fields");
    LQ_TRY(check_params(h, prm));
    LQ_TRY(chrono_alloc(h, prm));
    NEED(prm->level_w1 < 0 || f->w1, "the W1 field is needed");
    NEED(prm->level_schur < 0 || f->schur, "the boundary field is needed");
    NEED(prm->level_w2 < 0 || f->w2, "the W2 field is needed");
    NEED(prm->level_schur2 < 0 || f->schur2, "the second-level boundary field is needed");
    NEED(prm->level_s2 < 0 || f->s2, "the S2 field is needed");
    NEED(prm->level_s1 < 0 || f->s1, "the S1 field is needed");
    LQ_TRY(pack_gauge(h, U));
    h->have_gauge = true;
    if (prm->level_w1 >= 0) LQ_TRY(pack_spinor(h, fld(h, F_PHI1), f->w1, 0, 2));
    if (prm->level_schur >= 0)
        LQ_CUDA(h, cudaMemcpyAsync(h->bnd[0], f->schur, sizeof(double) * 2 * nbnd_of(h->g), cudaMemcpyDeviceToDevice,
                                   h->stream));
    if (prm->level_w2 >= 0) LQ_TRY(pack_spinor(h, fld(h, F_PHI3), f->w2, 0, 2));
    if (prm->level_schur2 >= 0)
        LQ_CUDA(h, cudaMemcpyAsync(h->bnd[3], f->schur2, sizeof(double) * 2 * nbnd2_of(h->g1),
                                   cudaMemcpyDeviceToDevice, h->stream));
    if (prm->level_s2 >= 0) LQ_TRY(pack_spinor(h, fld(h, F_PHI5), f->s2, 0, 1));
    if (prm->level_s1 >= 0) LQ_TRY(pack_spinor(h, fld(h, F_PHI6), f->s1, 0, 1));
    int nf = 0;
    const PfFields pf{fld(h, F_PHI1), h->bnd[0], fld(h, F_PHI3), h->bnd[3], fld(h, F_PHI5), fld(h, F_PHI6)};
    const double* ss = nullptr;
    LQ_TRY(md_scale_table(h, *prm, &ss));
    LQ_TRY(do_md(h, *prm, P, pf, &nf, ss));
    LQ_TRY(unpack_gauge(h, U));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

int lqcd_subblock_eo(lqcd_t h, double* out, const double* in, double kappa, double rho, int dagger, int op,
                     int precision, int method, double tol, int max_iter, int* iters_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(out && in, "null field pointer");
    NEED(op == LQCD_EO_APPLY || op == LQCD_EO_SOLVE, "bad op");
    NEED(prec_ok(precision) && (op == LQCD_EO_APPLY || (tol > 0 && max_iter > 0)), "bad precision / tol / max_iter");
    if (!h->g1.l0s) {
        h->err = "no sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    double2 *A = fld(h, F_D), *B = fld(h, F_E);
    LQ_TRY(pack_spinor(h, A, in, 0, 1));
    if (op == LQCD_EO_APPLY) {
        LQ_TRY(w3eo_apply(h, B, A, kappa, rho, dagger));
    } else {
        const int nbs = h->g1.L[0] / h->g1.l0s;
        std::vector<int> it(nbs, 0);
        NEED(method == LQCD_SOLVER_BICGSTAB || method == LQCD_SOLVER_SERIES, "bad method");
        SolveCfg c{precision, tol, max_iter, method};
        LQ_TRY(w3eo_solve(h, B, A, kappa, rho, dagger, c, it.data(), nullptr));
        if (iters_out)
            for (int k = 0; k < nbs; ++k) iters_out[k] = it[k];
    }
    LQ_TRY(unpack_spinor(h, out, B, 0, 1));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return LQCD_OK;
}

int lqcd_pf_force_eo(lqcd_t h, double* F, const double* phi, double kappa, double rho, int term, int precision,
                     double tol, int max_iter, double* S_out)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(phi, "null phi");
    NEED(term == LQCD_TERM_S2 || term == LQCD_TERM_S1, "bad term");
    NEED(prec_ok(precision) && tol > 0 && max_iter > 0, "bad precision / tol / max_iter");
    if (!h->g1.l0s) {
        h->err = "no sub-slabs (lqcd_set_subslabs)";
        return LQCD_ERR_STATE;
    }
    SolveCfg c{precision, tol, max_iter};
    double2* ph = fld(h, term == LQCD_TERM_S2 ? F_PHI5 : F_PHI6);
    LQ_TRY(pack_spinor(h, ph, phi, 0, 1));
    if (term == LQCD_TERM_S2) LQ_TRY(pf_s2(h, F, ph, kappa, rho, 1.0, c, h->red_out));
    else LQ_TRY(pf_s1(h, F, ph, kappa, rho, 1.0, c, h->red_out));
    double S;
    LQ_TRY(read_scalars(h, 1, &S));
    if (S_out) *S_out = S;
    return LQCD_OK;
}

int lqcd_hmc_trajectory(lqcd_t h, double* U, const lqcd_hmc_params* prm, uint64_t seed, uint32_t traj,
                        const double* P0, const double* eta1, const double* eta2, lqcd_hmc_result* res)
{
    CHECK_H(h);
    NEED(U && res, "null U / result");
    LQ_TRY(check_params(h, prm));
    LQ_TRY(chrono_alloc(h, prm));
    const lqcd_hmc_params& p = *prm;
    const Geo& g = h->g;
    const int nbd = 2 * nbnd_of(g);
    h->iter_count = 0;
    h->site_iters = 0;
    h->hop_sites = 0;
    h->solve_count = 0;
    LQ_TRY(pack_gauge(h, U));
    h->have_gauge = true;
    LQ_CUDA(h, cudaMemcpyAsync(h->U64_save, h->U64, sizeof(double2) * 72 * (size_t)g.Vh, cudaMemcpyDeviceToDevice,
                               h->stream));
    // heatbath: momenta N(0,1), pseudo-fermion noise exp(-|eta|^2)
    if (P0)
        LQ_CUDA(h, cudaMemcpyAsync(h->P, P0, sizeof(double) * 32 * (size_t)g.V, cudaMemcpyDeviceToDevice, h->stream));
    else
        LQ_TRY(rng_normals(h, h->P, (int64_t)32 * g.V, seed, 1, traj, 1.0));
    SolveCfg c{p.precision, p.tol, p.max_iter};
    double* e0 = h->red_out;  // [0..7] H0 terms, [8..15] H1 terms, [16] plaquette
    LQ_CUDA(h, cudaMemsetAsync(h->red_out, 0, sizeof(double) * 32, h->stream));
    LQ_TRY(kinetic_sum(h, h->P, e0));
    if (p.level_gauge >= 0) LQ_TRY(plaquette_sum(h, e0 + 1));
    if (p.level_w1 >= 0) {
        double2* et = fld(h, F_ETA1);
        if (eta1) LQ_TRY(pack_spinor(h, et, eta1, 0, 2));
        else LQ_TRY(rng_spinor(h, et, seed, 2, traj));
        if (p.pf_init == 0) {
            LQ_TRY(hop_full(h, MODE_INTRA, 0, -1, fld(h, F_PHI1), et, 1.0, et, -p.kappa));
            LQ_TRY(norm2_dev(h, (const double*)et, (int64_t)48 * g.Vh, e0 + 2));
        } else {
            LQ_CUDA(h, cudaMemcpyAsync(fld(h, F_PHI1), et, sizeof(double2) * 24 * (size_t)g.Vh,
                                       cudaMemcpyDeviceToDevice, h->stream));
            const SolveCfg cblk{p.precision, p.tol, p.max_iter, p.block_solver};
            LQ_TRY(pf_w1(h, nullptr, fld(h, F_PHI1), p.kappa, 0.0, cblk, e0 + 2));
        }
    }
    if (p.level_schur >= 0) {
        double* e2 = h->bnd[2];
        if (eta2) LQ_CUDA(h, cudaMemcpyAsync(e2, eta2, sizeof(double) * nbd, cudaMemcpyDeviceToDevice, h->stream));
        else LQ_TRY(rng_normals(h, e2, nbd, seed, 3, traj, sqrt(0.5)));
        if (p.pf_init == 0) {
            LQ_TRY(schur_op(h, h->bnd[0], e2, p.kappa, LQCD_SCHUR_R, c));
            LQ_TRY(norm2_dev(h, e2, nbd, e0 + 3));
        } else {
            LQ_CUDA(h, cudaMemcpyAsync(h->bnd[0], e2, sizeof(double) * nbd, cudaMemcpyDeviceToDevice, h->stream));
            LQ_TRY(pf_schur(h, nullptr, h->bnd[0], p.kappa, 0.0, c, e0 + 3));
        }
    }
    // second level (iterated decomposition): phi3 = W2 eta3, phi4 = R2 eta4
    // (Philox streams 5 and 6)
    if (p.level_w2 >= 0) {
        double2* et = fld(h, F_ETA1);
        LQ_TRY(rng_spinor(h, et, seed, 5, traj));
        LQ_TRY(sub_hop(h, 0, -1, fld(h, F_PHI3), et, 1.0, et, -p.kappa));
        LQ_TRY(norm2_dev(h, (const double*)et, (int64_t)48 * g.Vh, e0 + 4));
    }
    if (p.level_schur2 >= 0) {
        const int nbd2 = 2 * nbnd2_of(h->g1);
        double* e4 = h->bnd[2];
        LQ_TRY(rng_normals(h, e4, nbd2, seed, 6, traj, sqrt(0.5)));
        LQ_TRY(schur2_op(h, h->bnd[3], e4, p.kappa, LQCD_SCHUR_R, c));
        LQ_TRY(norm2_dev(h, e4, nbd2, e0 + 5));
    }
    // mass-preconditioned W2 (even sites): phi5 = W2,eo W3,eo^-1 eta5,
    // phi6 = W3,eo eta6 (Philox streams 7 and 8; the even half of a full draw)
    if (p.level_s2 >= 0) {
        double2* et = fld(h, F_ETA1);
        LQ_TRY(rng_spinor(h, et, seed, 7, traj));
        const SolveCfg ceo{p.precision, p.tol, p.max_iter, p.eo_solver};
        LQ_TRY(w3eo_solve(h, fld(h, F_G), et, p.kappa, p.rho, 0, ceo));
        LQ_TRY(w3eo_apply(h, fld(h, F_PHI5), fld(h, F_G), p.kappa, 0.0, 0));
        LQ_TRY(norm2_dev(h, (const double*)et, (int64_t)24 * g.Vh, e0 + 6));
    }
    if (p.level_s1 >= 0) {
        double2* et = fld(h, F_ETA1);
        LQ_TRY(rng_spinor(h, et, seed, 8, traj));
        LQ_TRY(w3eo_apply(h, fld(h, F_PHI6), et, p.kappa, p.rho, 0));
        LQ_TRY(norm2_dev(h, (const double*)et, (int64_t)24 * g.Vh, e0 + 7));
    }
    int nforce = 0;
    const PfFields pf{fld(h, F_PHI1), h->bnd[0], fld(h, F_PHI3), h->bnd[3], fld(h, F_PHI5), fld(h, F_PHI6)};
    const double* ss = nullptr;
    LQ_TRY(md_scale_table(h, p, &ss));
    if (p.use_graph) LQ_TRY(md_graph(h, p, pf, ss, &nforce));
    else LQ_TRY(do_md(h, p, h->P, pf, &nforce, ss));
    LQ_TRY(energy(h, p, pf, NTERM));
    double e[2 * NTERM];
    LQ_TRY(read_scalars(h, 2 * NTERM, e));
    const double H0 = combine(p, e), H1 = combine(p, e + NTERM);
    const double dH = H1 - H0;
    if (!isfinite(dH)) {
        h->err = "non-finite energy";
        return LQCD_ERR_NAN;
    }
    uint32_t w[4] = {0u, 0u, 4u, traj};
    philox_host(w, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6) + 0.5) / 9007199254740992.0;
    int shift = (int)(((uint64_t)w[2] * (uint64_t)g.L[0]) >> 32);
    int acc = 1;
    if (p.metropolis) acc = (dH <= 0.0) || (u < exp(-dH));
    if (!acc) {
        LQ_CUDA(h, cudaMemcpyAsync(h->U64, h->U64_save, sizeof(double2) * 72 * (size_t)g.Vh, cudaMemcpyDeviceToDevice,
                                   h->stream));
        LQ_TRY(refresh_low_precision(h));
    }
    if (!p.roll) shift = 0;
    if (shift) {
        LQ_CUDA(h, cudaMemcpyAsync(h->U64_save, h->U64, sizeof(double2) * 72 * (size_t)g.Vh, cudaMemcpyDeviceToDevice,
                                   h->stream));
        LQ_TRY(roll_links(h, shift));
    }
    LQ_TRY(plaquette_sum(h, h->red_out + 2 * NTERM));  // [16] of 32
    LQ_TRY(unpack_gauge(h, U));
    double pl;
    LQ_CUDA(h, cudaMemcpyAsync(h->red_host, h->red_out + 2 * NTERM, sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    pl = h->red_host[0];
    res->dH = dH;
    res->H0 = H0;
    res->H1 = H1;
    res->plaq = pl / (18.0 * g.V);
    res->u = u;
    res->accepted = acc;
    res->shift = shift;
    res->solver_iters = h->iter_count;
    res->site_iters = h->site_iters;
    res->hop_sites = h->hop_sites;
    res->n_solves = h->solve_count;
    res->n_force = nforce;
    return LQCD_OK;
}

int lqcd_autotune(lqcd_t h, int what, double kappa)
{
    CHECK_H(h);
    NEED_GAUGE(h);
    NEED(what >= 1 && what <= 3, "what: 1 hopping sweep, 2 solver, 3 both");
    const int Vh = h->g.Vh;
    double2 *A = fld(h, F_A), *B = fld(h, F_B);
    LQ_TRY(rng_spinor(h, A, 0x5eedULL, 9, 0));
    cudaEvent_t e0, e1;
    LQ_CUDA(h, cudaEventCreate(&e0));
    LQ_CUDA(h, cudaEventCreate(&e1));
    int st = LQCD_OK;
    if (what & 1) {
        // k_hop: threads per block, per storage precision, timed on this lattice
        const int cand[3] = {64, 128, 256};
        for (int prec = 0; prec < NPREC && st == LQCD_OK; ++prec) {
            SpinorF in = sp64(A, 1, Vh), out = sp64(B, 0, Vh);
            if (prec != PREC64) {
                auto lowview = [&](double2* buf, int par) {
                    SpinorF f;
                    f.v = (char*)buf + (size_t)par * 12 * Vh * sizeof(double2);
                    f.N = Vh;
                    f.nrm = prec == PREC16 ? (float*)((uint4*)f.v + (size_t)3 * Vh) : nullptr;
                    return f;
                };
                in = lowview(fld(h, F_C), 1);
                out = lowview(fld(h, F_D), 0);
                st = convert_spinor(h, in, prec, sp64(A, 1, Vh), PREC64, Vh);
            }
            // candidates interleaved over four rounds, the minimum per
            // candidate kept; the default stays unless another is 2 % faster
            const int def = h->tune.hop_bs[prec];
            float tmin[3] = {1e30f, 1e30f, 1e30f};
            for (int round = 0; round < 4 && st == LQCD_OK; ++round)
                for (int k = 0; k < 3 && st == LQCD_OK; ++k) {
                    h->tune.hop_bs[prec] = cand[k];
                    st = hop_sweep(h, prec, MODE_ALL, 0, 0, -1, out, in, 0.0, none(), 1.0);  // warm-up
                    cudaEventRecord(e0, h->stream);
                    for (int r = 0; r < 5 && st == LQCD_OK; ++r)
                        st = hop_sweep(h, prec, MODE_ALL, 0, 0, -1, out, in, 0.0, none(), 1.0);
                    cudaEventRecord(e1, h->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    tmin[k] = std::min(tmin[k], ms);
                }
            if (st != LQCD_OK) {
                h->tune.hop_bs[prec] = def;
                break;
            }
            int pick = def;
            float tdef = 1e30f;
            for (int k = 0; k < 3; ++k)
                if (cand[k] == def) tdef = tmin[k];
            float best = tdef;
            for (int k = 0; k < 3; ++k)
                if (tmin[k] < 0.98f * tdef && tmin[k] < best) {
                    best = tmin[k];
                    pick = cand[k];
                }
            h->tune.hop_bs[prec] = pick;
        }
    }
    if ((what & 2) && st == LQCD_OK) {
        // k_solve: sites per thread (CTAs per system; 0: every co-resident
        // CTA with an equal share of the sites), per precision, for the
        // batched slab solve and the global solve, timed on this lattice
        const int cand[3] = {1, 2, 0};
        for (int prec = 0; prec < NPREC && st == LQCD_OK; ++prec)
            for (int kind = 0; kind < 2 && st == LQCD_OK; ++kind) {
                // candidates interleaved over two rounds, the minimum per
                // candidate kept; the default stays unless another is 3 % faster
                const int def = h->tune.solve_spt[prec][kind];
                double tmin[3] = {1e30, 1e30, 1e30};
                for (int round = 0; round < 2 && st == LQCD_OK; ++round)
                    for (int k = 0; k < 3 && st == LQCD_OK; ++k) {
                        h->tune.solve_spt[prec][kind] = cand[k];
                        cudaEventRecord(e0, h->stream);
                        st = solve_full(h, kind == 0 ? MODE_INTRA : MODE_ALL, -1, 0, prec, kappa, B, A, 1e-10, 20000,
                                        nullptr, nullptr);
                        cudaEventRecord(e1, h->stream);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (st == LQCD_ERR_NOCONVERGE || st == LQCD_ERR_NAN) {
                            // this precision does not solve the test system at
                            // kappa: its schedule stays at the default
                            st = LQCD_OK;
                            tmin[k] = 2e30;
                        } else {
                            tmin[k] = std::min(tmin[k], (double)ms);
                        }
                    }
                if (st != LQCD_OK) {
                    h->tune.solve_spt[prec][kind] = def;
                    break;
                }
                int pick = def;
                double tdef = 1e30;
                for (int k = 0; k < 3; ++k)
                    if (cand[k] == def) tdef = tmin[k];
                double best = tdef;
                for (int k = 0; k < 3; ++k)
                    if (tmin[k] < 0.97 * tdef && tmin[k] < best) {
                        best = tmin[k];
                        pick = cand[k];
                    }
                h->tune.solve_spt[prec][kind] = pick;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

int lqcd_set_cluster_series(lqcd_t h, int enable)
{
    CHECK_H(h);
    h->tune.cluster_series = enable ? 1 : 0;
    return LQCD_OK;
}

int lqcd_set_solver_schedule(lqcd_t h, int spt)
{
    CHECK_H(h);
    if (spt < 0 || spt > 2) {
        h->err = "solver schedule: 0, 1 or 2 sites per thread";
        return LQCD_ERR_ARG;
    }
    for (int p = 0; p < NPREC; ++p) h->tune.solve_spt[p][0] = h->tune.solve_spt[p][1] = spt;
    return LQCD_OK;
}

int lqcd_tune_read(lqcd_t h, int* out)
{
    CHECK_H(h);
    NEED(out, "null output");
    for (int p = 0; p < NPREC; ++p) {
        out[p] = h->tune.hop_bs[p];
        out[NPREC + p] = h->tune.solve_spt[p][0];
        out[2 * NPREC + p] = h->tune.solve_spt[p][1];
    }
    return LQCD_OK;
}

int lqcd_profile_enable(lqcd_t h, int enable)
{
    CHECK_H(h);
    if (!enable) prof_flush(h);
    h->prof.on = enable == 1 ? 0x1fu : (unsigned)enable & 0x1fu;
    return LQCD_OK;
}

int lqcd_profile_reset(lqcd_t h)
{
    CHECK_H(h);
    prof_flush(h);
    for (int k = 0; k < 5; ++k) {
        h->prof.launches[k] = 0;
        h->prof.ms[k] = 0.0;
        h->prof.bytes[k] = 0.0;
        h->prof.hist[k].clear();
    }
    return LQCD_OK;
}

int lqcd_force_profile(lqcd_t h, const double* F, double* out)
{
    CHECK_H(h);
    NEED(F && out, "null force / output pointer");
    return force_profile(h, F, out);
}

int lqcd_set_global_solver(lqcd_t h, int method, int sap_terms)
{
    CHECK_H(h);
    if (method != LQCD_SOLVER_BICGSTAB && method != LQCD_SOLVER_SAP && method != LQCD_SOLVER_SAP_BLOCKS) {
        h->err = "global solver: LQCD_SOLVER_BICGSTAB, LQCD_SOLVER_SAP or LQCD_SOLVER_SAP_BLOCKS";
        return LQCD_ERR_ARG;
    }
    const bool sap = method == LQCD_SOLVER_SAP || method == LQCD_SOLVER_SAP_BLOCKS;
    if (sap && (sap_terms < 0 || sap_terms > 64)) {
        h->err = "global solver: 0 <= sap_terms <= 64";
        return LQCD_ERR_ARG;
    }
    if (sap) LQ_TRY(solver_sap_alloc(h));
    h->global_method = method == LQCD_SOLVER_SAP ? SOLVER_SAP : method == LQCD_SOLVER_SAP_BLOCKS ? SOLVER_SAPB
                                                                                                : SOLVER_BICGSTAB;
    if (sap) h->sap_terms = sap_terms;
    return LQCD_OK;
}

int lqcd_set_wait_limit(lqcd_t h, int64_t cycles)
{
    CHECK_H(h);
    h->wait_limit = cycles > 0 ? (long long)cycles : lqcd_ctx::WAIT_LIMIT_DEFAULT;
    return LQCD_OK;
}

int lqcd_launch_count(lqcd_t h, int64_t* count)
{
    CHECK_H(h);
    if (!count) return LQCD_ERR_ARG;
    *count = h->launches;
    return LQCD_OK;
}

int lqcd_profile_times(lqcd_t h, int id, float* ms_out, int64_t cap, int64_t* n_out)
{
    CHECK_H(h);
    if (id < 0 || id > 4 || !n_out || (cap > 0 && !ms_out)) return LQCD_ERR_ARG;
    prof_flush(h);
    const std::vector<float>& v = h->prof.hist[id];
    const int64_t n = std::min<int64_t>(cap, (int64_t)v.size());
    for (int64_t k = 0; k < n; ++k) ms_out[k] = v[k];
    *n_out = (int64_t)v.size();
    return LQCD_OK;
}

int lqcd_profile_read(lqcd_t h, int id, int64_t* launches, double* ms, double* bytes)
{
    CHECK_H(h);
    if (id < 0 || id > 4) return LQCD_ERR_ARG;
    prof_flush(h);
    if (launches) *launches = h->prof.launches[id];
    if (ms) *ms = h->prof.ms[id];
    if (bytes) *bytes = h->prof.bytes[id];
    return LQCD_OK;
}

}  // extern "C"
