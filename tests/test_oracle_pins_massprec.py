"""Pins of the oracle's even-odd and mass preconditioning of W2 (Sec. 1:
W3,eo = W2,eo + rho) and of the four-part pseudo-fermion action
S4 + S3 + S2 + S1 (Sec. 1) on five integration levels (Sec. 2).

W2,eo is checked against the Schur complement of the odd-odd block of the
dense W2 (det W2 = det W2,eo), its adjoint against the conjugate transpose,
the S1 / S2 forces against finite differences, the heatbath identities,
and the molecular dynamics of the full action (reversibility, dt^2).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

from test_oracle_pins import dense, relerr, _fd_check

RHO = 0.2


def _lat(L, l0, bc=-1):
    return O.Lattice(L, l0, bc, l0s=l0 // 2)


@pytest.mark.parametrize("L,l0", [((4, 2, 2, 2), 2), ((8, 2, 2, 2), 4)])
def test_w2eo_is_the_schur_complement_of_w2(L, l0):
    lat = _lat(L, l0)
    kappa = 0.14
    U = syn.random_links(L, 0.4, 51)
    n, nh = lat.V * 12, lat.Vh * 12
    W2 = dense(lambda x: lat.W2(U, kappa, x), n, lat.spinor_shape())
    A, B, C, D = W2[:nh, :nh], W2[:nh, nh:], W2[nh:, :nh], W2[nh:, nh:]
    # odd-odd block of W2 is the identity (H only connects parities)
    assert np.array_equal(D, np.eye(n - nh))
    assert np.array_equal(A, np.eye(nh))
    W2eo = dense(lambda x: lat.w3eo(U, kappa, 0.0, x), nh, lat.half_shape())
    assert relerr(W2eo, A - B @ np.linalg.solve(D, C)) < 1e-13
    s2, l2 = np.linalg.slogdet(W2)
    se, le = np.linalg.slogdet(W2eo)
    assert abs(l2 - le) < 1e-10 * max(1, abs(l2)) and abs(s2 - se) < 1e-9
    # W3,eo = W2,eo + rho, its adjoint, and the solver
    W3 = dense(lambda x: lat.w3eo(U, kappa, RHO, x), nh, lat.half_shape())
    assert relerr(W3, W2eo + RHO * np.eye(nh)) < 1e-14
    W3d = dense(lambda x: lat.w3eo(U, kappa, RHO, x, 1), nh, lat.half_shape())
    assert relerr(W3d, W3.conj().T) < 1e-14
    b = syn.gaussian_spinor(lat.Vh, 52)
    for dag in (0, 1):
        x = lat.solve_w3eo(U, kappa, RHO, b, dag, tol=1e-14)
        ref = np.linalg.solve(W3.conj().T if dag else W3, b.ravel())
        assert relerr(x.ravel(), ref) < 1e-11


@pytest.mark.parametrize("term", ["s1", "s2"])
def test_force_massprec_fd(term):
    L = (4, 2, 2, 2)
    lat = _lat(L, 2)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 53)
    phi = syn.gaussian_spinor(lat.Vh, 54)
    fn = lat.pf_s1 if term == "s1" else lat.pf_s2
    S, F = fn(U, kappa, RHO, phi)
    rng = np.random.default_rng(3)
    links = [(mu, s) for mu in range(4) for s in range(lat.V)]
    pick = [links[i] for i in rng.choice(len(links), 12, replace=False)] + [(0, s) for s in range(0, lat.V, 4)]
    _fd_check(lambda W: fn(W, kappa, RHO, phi, force=False)[0], F, U, pick)
    # time-like links across a sub-slab face do not enter W2
    m = lat.index_maps()
    sub = (m[0] // lat.V3) // lat.l0s
    for s in range(lat.V):
        if sub[s] != sub[m[4, s]]:
            assert np.all(F[0, s] == 0)


def test_heatbath_actions_massprec():
    lat = _lat((8, 2, 2, 2), 4)
    U = syn.random_links(lat.L, 0.3, 55)
    kappa = 0.15
    e1 = syn.gaussian_spinor(lat.Vh, 56)
    e2 = syn.gaussian_spinor(lat.Vh, 57)
    S1 = lat.pf_s1(U, kappa, RHO, lat.w3eo(U, kappa, RHO, e1), force=False)[0]
    phi2 = lat.w3eo(U, kappa, 0.0, lat.solve_w3eo(U, kappa, RHO, e2, tol=1e-14))
    S2 = lat.pf_s2(U, kappa, RHO, phi2, force=False)[0]
    assert abs(S1 - np.vdot(e1, e1).real) < 1e-10 * S1
    assert abs(S2 - np.vdot(e2, e2).real) < 1e-10 * S2
    # rho = 0: S2 is |phi|^2 and carries no force
    S0, F0 = lat.pf_s2(U, kappa, 0.0, phi2)
    assert abs(S0 - np.vdot(phi2, phi2).real) < 1e-12 * S0
    assert np.all(F0 == 0)


def _prm5(ns, **kw):
    """the production layout: S_G on level 0, S1 on 1, S2 on 2, S3 (R2) on
    3, S4 (R) on 4; SW on levels 0, 1 and LF on 2, 3, 4 (Sec. 2)"""
    kw.setdefault("tol", 1e-14)
    return O.hmc_params(5.6, 0.15, kw.pop("tau", 0.3), 5, (O.SW, O.SW, O.LF, O.LF, O.LF), ns,
                        level_gauge=0, level_w1=-1, level_schur=4, level_w2=-1, level_schur2=3,
                        rho=RHO, level_s2=2, level_s1=1, **kw)


def _fields5(lat, seed):
    return dict(phi2=syn.gaussian_complex(lat.bnd_shape(), seed), phi4=syn.gaussian_complex(lat.bnd2_shape(), seed + 1),
                phi_s2=syn.gaussian_spinor(lat.Vh, seed + 2), phi_s1=syn.gaussian_spinor(lat.Vh, seed + 3))


def test_md5_reversibility():
    L = (4, 2, 2, 2)
    lat = _lat(L, 2)
    U = syn.random_links(L, 0.3, 65)
    P = syn.gaussian_momenta(lat.V, 66)
    f = _fields5(lat, 67)
    prm = _prm5([2, 2, 1, 1, 1])
    U1, P1, st = O.md(lat, U, P, None, f["phi2"], prm, None, f["phi4"], f["phi_s2"], f["phi_s1"])
    assert st == 0
    assert np.max(np.abs(U1 - U)) > 1e-3
    U2, P2, st = O.md(lat, U1, -P1, None, f["phi2"], prm, None, f["phi4"], f["phi_s2"], f["phi_s1"])
    assert np.max(np.abs(U2 - U)) < 1e-12
    assert np.max(np.abs(P2 + P)) < 1e-10


def test_md5_dH_scales_as_dt_squared():
    L = (4, 2, 2, 2)
    lat = _lat(L, 2)
    U = syn.random_links(L, 0.3, 75)
    P = syn.gaussian_momenta(lat.V, 76)
    f = _fields5(lat, 77)
    kappa, beta = 0.15, 5.6

    def H(Ux, Px):
        return (0.5 * np.sum(Px ** 2) + lat.gauge_action(Ux, beta)
                + lat.pf_schur(Ux, kappa, f["phi2"], force=False, tol=1e-14)[0]
                + lat.pf_schur2(Ux, kappa, f["phi4"], force=False, tol=1e-14)[0]
                + lat.pf_s2(Ux, kappa, RHO, f["phi_s2"], force=False, tol=1e-14)[0]
                + lat.pf_s1(Ux, kappa, RHO, f["phi_s1"], force=False, tol=1e-14)[0])

    H0 = H(U, P)
    dh = []
    # all five terms on one leap-frog level, refined
    ns = [3, 6, 12]
    for n in ns:
        prm = O.hmc_params(beta, kappa, 0.3, 1, (O.LF,), [n], level_gauge=0, level_w1=-1, level_schur=0,
                           level_schur2=0, rho=RHO, level_s2=0, level_s1=0, tol=1e-14)
        U1, P1, st = O.md(lat, U, P, None, f["phi2"], prm, None, f["phi4"], f["phi_s2"], f["phi_s1"])
        assert st == 0
        dh.append(abs(H(U1, P1) - H0))
    slope = np.polyfit(np.log(0.3 / np.array(ns)), np.log(dh), 1)[0]
    assert 1.8 < slope < 2.2, (slope, dh)


def test_trajectory_five_level_action():
    """the production integrator on a small lattice: dH = H1 - H0 and it
    decreases when every level is refined"""
    L = (4, 2, 2, 2)
    lat = _lat(L, 2)
    U = syn.random_links(L, 0.3, 95)
    dh = []
    for k in (1, 4):
        prm = _prm5([2, 2, 1, 1, 2 * k], metropolis=0, tol=1e-13)
        U1, res, st = lat.hmc_trajectory(U, prm, 13, 0)
        assert st == 0
        assert abs(res.dH - (res.H1 - res.H0)) < 1e-12 * abs(res.H0)
        dh.append(abs(res.dH))
    assert dh[1] < 0.25 * dh[0], dh
