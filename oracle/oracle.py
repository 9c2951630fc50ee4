"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Arrays are numpy complex128 / float64 in the documented layouts:
spinor ``(V, 4, 3)``, gauge ``(4, V, 3, 3)``, momenta/forces ``(4, V, 8)``,
boundary coordinates ``(nb/2, 2, V3, 2, 3)``, sites in checkerboard order.
Every function here forwards to ``lqcd_oracle.c``; the arithmetic lives
there (see its header comment for the paper passages each part follows).
"""
import ctypes as C
import numpy as np

from . import build as _build

HOP_ALL, HOP_INTRA, HOP_CROSS, HOP_INTRA2, HOP_CROSS2 = 0, 1, 2, 3, 4
R, RDAG, RINV, RINVDAG = 0, 1, 2, 3
LF, SW = 0, 1

_lib = None


class Geom(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("l0", C.c_int), ("bc_t", C.c_int), ("l0s", C.c_int)]


class HmcParams(C.Structure):
    _fields_ = [
        ("beta", C.c_double), ("kappa", C.c_double), ("tau", C.c_double), ("lam", C.c_double),
        ("nlevels", C.c_int), ("scheme", C.c_int * 5), ("nsteps", C.c_int * 5),
        ("level_gauge", C.c_int), ("level_w1", C.c_int), ("level_schur", C.c_int),
        ("pf_init", C.c_int), ("roll", C.c_int), ("schur_route", C.c_int),
        ("metropolis", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
        ("step_scale", C.c_void_p), ("level_w2", C.c_int), ("level_schur2", C.c_int),
        ("rho", C.c_double), ("level_s2", C.c_int), ("level_s1", C.c_int),
    ]


class PfFields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "schur", "w2", "schur2", "s2", "s1")]


class HmcResult(C.Structure):
    _fields_ = [
        ("dH", C.c_double), ("H0", C.c_double), ("H1", C.c_double), ("plaq", C.c_double),
        ("u", C.c_double), ("accepted", C.c_int), ("shift", C.c_int), ("status", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.lqo_gauge_action.restype = C.c_double
        _lib.lqo_plaquette.restype = C.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Lattice:
    """Geometry L = (L0, L1, L2, L3) with x0-slabs of thickness l0 and,
    for the iterated decomposition, sub-slabs of thickness l0s = l0/2."""

    def __init__(self, L, l0, bc_t=-1, l0s=0):
        self.L = tuple(int(v) for v in L)
        self.l0 = int(l0)
        self.bc_t = int(bc_t)
        self.l0s = int(l0s)
        self.g = Geom((C.c_int * 4)(*self.L), self.l0, self.bc_t, self.l0s)
        self.V3 = self.L[1] * self.L[2] * self.L[3]
        self.V = self.L[0] * self.V3
        self.Vh = self.V // 2
        self.nb = self.L[0] // self.l0
        self.nbnd = (self.nb // 2) * 2 * self.V3 * 6
        self.nbs = self.L[0] // self.l0s if self.l0s else 0
        self.nbnd2 = (self.nbs // 2) * self.V3 * 6
        st = lib().lqo_geom_check(C.byref(self.g))
        if st != 0:
            raise ValueError("invalid geometry L=%s l0=%d (status %d)" % (self.L, self.l0, st))

    # ---- shapes -------------------------------------------------------
    def spinor_shape(self):
        return (self.V, 4, 3)

    def half_shape(self):
        return (self.Vh, 4, 3)

    def bnd_shape(self):
        return (self.nb // 2, 2, self.V3, 2, 3)

    # ---- maps / algebra -------------------------------------------------
    def index_maps(self):
        m = np.zeros((14, self.V), dtype=np.int32)
        lib().lqo_index_maps(C.byref(self.g), _p(m))
        return m

    @staticmethod
    def gamma():
        g = np.zeros((5, 4, 4), dtype=np.complex128)
        lib().lqo_gamma(_p(g))
        return g

    # ---- operators --------------------------------------------------------
    def hop(self, U, x, mode=HOP_ALL, dagger=0):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_hop(C.byref(self.g), _p(U), _p(np.ascontiguousarray(x)), _p(out), mode, dagger)
        return out

    def M(self, U, kappa, x, dagger=0):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_apply_M(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(x)),
                          _p(out), dagger)
        return out

    def W1(self, U, kappa, x, dagger=0):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_apply_W1(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(x)),
                           _p(out), dagger)
        return out

    def dslash_eo(self, U, x_half, parity, dagger=0):
        out = np.zeros(self.half_shape(), np.complex128)
        lib().lqo_dslash_eo(C.byref(self.g), _p(U), _p(np.ascontiguousarray(x_half)), _p(out),
                            parity, dagger)
        return out

    def mhat(self, U, kappa, x_e, dagger=0):
        out = np.zeros(self.half_shape(), np.complex128)
        lib().lqo_mhat(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(x_e)),
                       _p(out), dagger)
        return out

    def block_dslash(self, U, kappa, x, colour=-1, dagger=0):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_block_dslash(C.byref(self.g), _p(U), C.c_double(kappa),
                               _p(np.ascontiguousarray(x)), _p(out), colour, dagger)
        return out

    def block_solve(self, U, kappa, b, colour=-1, dagger=0, tol=1e-13, maxit=20000):
        x = np.zeros(self.spinor_shape(), np.complex128)
        it = C.c_int(0)
        st = lib().lqo_block_solve(C.byref(self.g), _p(U), C.c_double(kappa), _p(x),
                                   _p(np.ascontiguousarray(b)), colour, dagger, C.c_double(tol),
                                   maxit, C.byref(it))
        if st:
            raise RuntimeError("oracle block solve did not converge")
        return x

    def solve_M(self, U, kappa, b, dagger=0, tol=1e-13, maxit=50000):
        x = np.zeros(self.spinor_shape(), np.complex128)
        it = C.c_int(0)
        st = lib().lqo_solve_M(C.byref(self.g), _p(U), C.c_double(kappa), _p(x),
                               _p(np.ascontiguousarray(b)), dagger, C.c_double(tol), maxit,
                               C.byref(it))
        if st:
            raise RuntimeError("oracle solve did not converge")
        return x

    def embed(self, c):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_embed_boundary(C.byref(self.g), _p(np.ascontiguousarray(c)), _p(out))
        return out

    def project(self, full):
        out = np.zeros(self.bnd_shape(), np.complex128)
        lib().lqo_project_boundary(C.byref(self.g), _p(np.ascontiguousarray(full)), _p(out))
        return out

    def schur(self, U, kappa, c, op=R, route=1, tol=1e-12, maxit=50000):
        out = np.zeros(self.bnd_shape(), np.complex128)
        st = lib().lqo_schur(C.byref(self.g), _p(U), C.c_double(kappa), _p(out),
                             _p(np.ascontiguousarray(c)), op, route, C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle Schur operator: a solve did not converge")
        return out

    # ---- forces ------------------------------------------------------------
    def bilinear(self, U, a, b, mask=HOP_ALL, coef=1.0):
        F = np.zeros((4, self.V, 8))
        lib().lqo_bilinear(C.byref(self.g), _p(U), _p(np.ascontiguousarray(a)),
                           _p(np.ascontiguousarray(b)), mask, C.c_double(coef), _p(F))
        return F

    def pf_w1(self, U, kappa, phi, force=True, tol=1e-13, maxit=20000):
        F = np.zeros((4, self.V, 8)) if force else None
        S = C.c_double(0)
        st = lib().lqo_pf_w1(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(phi)),
                             _p(F) if force else None, C.byref(S), C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle W1 force: a solve did not converge")
        return S.value, F

    def pf_schur(self, U, kappa, phi, force=True, route=1, tol=1e-12, maxit=50000):
        F = np.zeros((4, self.V, 8)) if force else None
        S = C.c_double(0)
        st = lib().lqo_pf_schur(C.byref(self.g), _p(U), C.c_double(kappa),
                                _p(np.ascontiguousarray(phi)), _p(F) if force else None,
                                C.byref(S), route, C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle Schur force: a solve did not converge")
        return S.value, F

    # ---- iterated decomposition (second level) -------------------------
    def bnd2_shape(self):
        return (self.nbs // 2, self.V3, 2, 3)

    def W2(self, U, kappa, x, dagger=0):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_apply_W2(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(x)),
                           _p(out), dagger)
        return out

    def block_solve2(self, U, kappa, b, colour=-1, dagger=0, tol=1e-13, maxit=20000):
        x = np.zeros(self.spinor_shape(), np.complex128)
        it = C.c_int(0)
        st = lib().lqo_block_solve2(C.byref(self.g), _p(U), C.c_double(kappa), _p(x),
                                    _p(np.ascontiguousarray(b)), colour, dagger, C.c_double(tol),
                                    maxit, C.byref(it))
        if st:
            raise RuntimeError("oracle sub-slab solve did not converge")
        return x

    def embed2(self, c):
        out = np.zeros(self.spinor_shape(), np.complex128)
        lib().lqo_embed_boundary2(C.byref(self.g), _p(np.ascontiguousarray(c)), _p(out))
        return out

    def project2(self, full):
        out = np.zeros(self.bnd2_shape(), np.complex128)
        lib().lqo_project_boundary2(C.byref(self.g), _p(np.ascontiguousarray(full)), _p(out))
        return out

    def schur2(self, U, kappa, c, op=R, route=1, tol=1e-12, maxit=50000):
        out = np.zeros(self.bnd2_shape(), np.complex128)
        st = lib().lqo_schur2(C.byref(self.g), _p(U), C.c_double(kappa), _p(out),
                              _p(np.ascontiguousarray(c)), op, route, C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle second-level Schur operator: a solve did not converge")
        return out

    def pf_w2(self, U, kappa, phi, force=True, tol=1e-13, maxit=20000):
        F = np.zeros((4, self.V, 8)) if force else None
        S = C.c_double(0)
        st = lib().lqo_pf_w2(C.byref(self.g), _p(U), C.c_double(kappa), _p(np.ascontiguousarray(phi)),
                             _p(F) if force else None, C.byref(S), C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle W2 force: a solve did not converge")
        return S.value, F

    def pf_schur2(self, U, kappa, phi, force=True, route=1, tol=1e-12, maxit=50000):
        F = np.zeros((4, self.V, 8)) if force else None
        S = C.c_double(0)
        st = lib().lqo_pf_schur2(C.byref(self.g), _p(U), C.c_double(kappa),
                                 _p(np.ascontiguousarray(phi)), _p(F) if force else None,
                                 C.byref(S), route, C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle second-level Schur force: a solve did not converge")
        return S.value, F

    # ---- even-odd + mass preconditioning of W2 (even-site fields) ---------
    def w3eo(self, U, kappa, rho, x_e, dagger=0):
        out = np.zeros(self.half_shape(), np.complex128)
        lib().lqo_apply_w3eo(C.byref(self.g), _p(U), C.c_double(kappa), C.c_double(rho),
                             _p(np.ascontiguousarray(x_e)), _p(out), dagger)
        return out

    def solve_w3eo(self, U, kappa, rho, b_e, dagger=0, tol=1e-13, maxit=20000):
        x = np.zeros(self.half_shape(), np.complex128)
        it = C.c_int(0)
        st = lib().lqo_solve_w3eo(C.byref(self.g), _p(U), C.c_double(kappa), C.c_double(rho), _p(x),
                                  _p(np.ascontiguousarray(b_e)), dagger, C.c_double(tol), maxit, C.byref(it))
        if st:
            raise RuntimeError("oracle W3,eo solve did not converge")
        return x

    def _pf_eo(self, fn, U, kappa, rho, phi, force, tol, maxit):
        F = np.zeros((4, self.V, 8)) if force else None
        S = C.c_double(0)
        st = fn(C.byref(self.g), _p(U), C.c_double(kappa), C.c_double(rho), _p(np.ascontiguousarray(phi)),
                _p(F) if force else None, C.byref(S), C.c_double(tol), maxit)
        if st:
            raise RuntimeError("oracle mass-preconditioned force: a solve did not converge")
        return S.value, F

    def pf_s1(self, U, kappa, rho, phi, force=True, tol=1e-13, maxit=20000):
        return self._pf_eo(lib().lqo_pf_s1, U, kappa, rho, phi, force, tol, maxit)

    def pf_s2(self, U, kappa, rho, phi, force=True, tol=1e-13, maxit=20000):
        return self._pf_eo(lib().lqo_pf_s2, U, kappa, rho, phi, force, tol, maxit)

    def force_profile(self, F):
        out = np.zeros((2, self.L[0]))
        lib().lqo_force_profile(C.byref(self.g), _p(np.ascontiguousarray(F)), _p(out))
        return out

    def gauge_action(self, U, beta):
        return lib().lqo_gauge_action(C.byref(self.g), _p(U), C.c_double(beta))

    def plaquette(self, U):
        return lib().lqo_plaquette(C.byref(self.g), _p(U))

    def gauge_force(self, U, beta):
        F = np.zeros((4, self.V, 8))
        lib().lqo_gauge_force(C.byref(self.g), _p(U), C.c_double(beta), _p(F))
        return F

    def update_U(self, U, P, dt):
        U2 = np.array(U, dtype=np.complex128, copy=True)
        lib().lqo_update_U(C.byref(self.g), _p(U2), _p(np.ascontiguousarray(P)), C.c_double(dt))
        return U2

    def roll_x0(self, U, shift):
        U2 = np.array(U, dtype=np.complex128, copy=True)
        lib().lqo_roll_x0(C.byref(self.g), _p(U2), int(shift))
        return U2

    def hmc_trajectory(self, U, prm, seed, traj, P0=None, eta1=None, eta2=None):
        U2 = np.array(U, dtype=np.complex128, copy=True)
        res = HmcResult()
        args = [np.ascontiguousarray(a) if a is not None else None for a in (P0, eta1, eta2)]
        st = lib().lqo_hmc_trajectory(C.byref(self.g), _p(U2), C.byref(prm), C.c_uint64(seed),
                                      C.c_uint32(traj), *[(_p(a) if a is not None else None)
                                                          for a in args], C.byref(res))
        return U2, res, st


def su3_expi(X):
    E = np.zeros((3, 3), np.complex128)
    lib().lqo_su3_expi(_p(np.ascontiguousarray(X, dtype=np.complex128)), _p(E))
    return E


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().lqo_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed, stream, traj, n):
    out = np.zeros(n)
    lib().lqo_normals(C.c_uint64(seed), C.c_uint32(stream), C.c_uint32(traj), C.c_int64(n), _p(out))
    return out


def metropolis_uniforms(seed, traj, L0):
    u = C.c_double(0)
    s = C.c_int(0)
    lib().lqo_uniforms_metropolis(C.c_uint64(seed), C.c_uint32(traj), int(L0), C.byref(u), C.byref(s))
    return u.value, s.value


def hmc_params(beta, kappa, tau, nlevels, scheme, nsteps, level_gauge=0, level_w1=0,
               level_schur=0, lam=1.0 / 6.0, pf_init=0, roll=0, schur_route=1, metropolis=1,
               tol=1e-12, maxit=50000, step_scale=None, level_w2=-1, level_schur2=-1, rho=0.0,
               level_s2=-1, level_s1=-1):
    """step_scale: None, or a float64 array (2, L0) of s(x0) for space-like /
    time-like links (see step_scheme)"""
    sc = list(scheme) + [0] * (5 - len(scheme))
    ns = list(nsteps) + [1] * (5 - len(nsteps))
    p = HmcParams(beta, kappa, tau, lam, nlevels, (C.c_int * 5)(*sc), (C.c_int * 5)(*ns),
                  level_gauge, level_w1, level_schur, pf_init, roll, schur_route, metropolis,
                  tol, maxit, None, level_w2, level_schur2, rho, level_s2, level_s1)
    if step_scale is not None:
        p._scale = np.ascontiguousarray(step_scale, dtype=np.float64)
        p.step_scale = p._scale.ctypes.data
    return p


def step_scheme(scheme, L0):
    """s(x0) tables of the step-size schemes A (1), B (2), C (3): (2, L0)"""
    out = np.zeros((2, L0))
    if lib().lqo_step_scheme(int(scheme), int(L0), _p(out)) != 0:
        raise ValueError("scheme %d does not tile L0 = %d" % (scheme, L0))
    return out


def md(lat, U, P, phi1, phi2, prm, phi3=None, phi4=None, phi_s2=None, phi_s1=None):
    """molecular dynamics only: integrates (U, P) for fixed pseudofermions
    (phi1 W1, phi2 R, phi3 W2, phi4 R2, phi_s2 / phi_s1 the even-site fields
    of the mass-preconditioned W2 terms)"""
    U2 = np.array(U, dtype=np.complex128, copy=True)
    P2 = np.array(P, dtype=np.float64, copy=True)
    keep = [np.ascontiguousarray(a) if a is not None else None
            for a in (phi1, phi2, phi3, phi4, phi_s2, phi_s1)]
    pf = PfFields(*[(a.ctypes.data if a is not None else None) for a in keep])
    st = lib().lqo_md(C.byref(lat.g), _p(U2), _p(P2), C.byref(pf), C.byref(prm))
    return U2, P2, st
