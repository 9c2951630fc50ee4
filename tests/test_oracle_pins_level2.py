"""Pins of the oracle's iterated decomposition (Sec. 1: the slabs of the
first level split once more into sub-slabs of thickness l0/2).

With the sites of one slab ordered red|black by sub-slab colour, W1 is a
two-by-two block matrix whose diagonal blocks form W2; block LU then gives
det W1 = det W2 det R2 and, with the first level, det M = det R1 det R2 det W2.
The tests check these determinant identities with dense linear algebra,
the adjoint and inverse of R2 against the dense matrix, the subspace R2
acts on, the forces against finite differences of the actions, and the
molecular dynamics of the four-part action (reversibility, dt^2 scaling of
the energy violation, heatbath).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

from test_oracle_pins import dense, relerr, _fd_check


def _lat(L, l0, bc=-1):
    return O.Lattice(L, l0, bc, l0s=l0 // 2)


def _sub(lat):
    """sub-slab of every site, from the lexicographic index (map 0)"""
    x0 = lat.index_maps()[0] // lat.V3
    return x0 // lat.l0s


@pytest.mark.parametrize("L,l0,bc", [((4, 2, 2, 2), 2, -1), ((8, 2, 2, 2), 2, 1),
                                     ((8, 2, 2, 2), 4, -1)])
def test_det_iterated_factorisation_dense(L, l0, bc):
    lat = _lat(L, l0, bc)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 23)
    n = lat.V * 12
    sh = lat.spinor_shape()
    Md = dense(lambda x: lat.M(U, kappa, x), n, sh)
    W1 = dense(lambda x: lat.W1(U, kappa, x), n, sh)
    W2 = dense(lambda x: lat.W2(U, kappa, x), n, sh)
    R1 = dense(lambda c: lat.schur(U, kappa, c, O.R, tol=1e-10), lat.nbnd, lat.bnd_shape())
    R2 = dense(lambda c: lat.schur2(U, kappa, c, O.R, tol=1e-14), lat.nbnd2, lat.bnd2_shape())
    sM, lM = np.linalg.slogdet(Md)
    s1, l1 = np.linalg.slogdet(W1)
    s2, l2 = np.linalg.slogdet(W2)
    sr1, lr1 = np.linalg.slogdet(R1)
    sr2, lr2 = np.linalg.slogdet(R2)
    # det W1 = det W2 det R2
    assert abs(l1 - (l2 + lr2)) < 1e-10 * max(1, abs(l1))
    assert abs(s1 - s2 * sr2) < 1e-9
    # det M = det R1 det R2 det W2
    assert abs(lM - (lr1 + lr2 + l2)) < 1e-10 * max(1, abs(lM))
    assert abs(sM - sr1 * sr2 * s2) < 1e-9
    # det R2 is real (gamma5-hermiticity of W1 and W2)
    assert abs(sr2.imag) < 1e-9
    # W2 is block diagonal in the sub-slabs and agrees with W1 inside them
    sub = np.repeat(_sub(lat), 12)
    same = sub[:, None] == sub[None, :]
    assert np.all(W2[~same] == 0)
    assert np.array_equal(W2[same], W1[same])
    # R2^dag and both R2^-1 routes against dense linear algebra
    R2d = dense(lambda c: lat.schur2(U, kappa, c, O.RDAG, tol=1e-14), lat.nbnd2, lat.bnd2_shape())
    assert relerr(R2d, R2.conj().T) < 1e-10
    c = syn.gaussian_complex(lat.bnd2_shape(), 8)
    ref = np.linalg.solve(R2, c.ravel())
    refd = np.linalg.solve(R2.conj().T, c.ravel())
    for route in (0, 1):
        assert relerr(lat.schur2(U, kappa, c, O.RINV, route, tol=1e-13).ravel(), ref) < 1e-9
        assert relerr(lat.schur2(U, kappa, c, O.RINVDAG, route, tol=1e-13).ravel(), refd) < 1e-9
    # the sub-slab solve inverts W2
    b = syn.gaussian_spinor(lat.V, 9)
    for dag in (0, 1):
        x = lat.block_solve2(U, kappa, b, -1, dag, tol=1e-14)
        ref = np.linalg.solve(W2.conj().T if dag else W2, b.ravel())
        assert relerr(x.ravel(), ref) < 1e-11


def test_R2_from_dense_blocks():
    """R2 from the dense blocks of W1 (red|black by sub-slab colour) and the
    spin-projected first slices of the black sub-slabs"""
    L = (8, 2, 2, 2)
    lat = _lat(L, 4)
    kappa = 0.14
    U = syn.random_links(L, 0.4, 24)
    n = lat.V * 12
    W1 = dense(lambda x: lat.W1(U, kappa, x), n, lat.spinor_shape())
    col = np.repeat(_sub(lat) % 2, 12)
    r, b = col == 0, col == 1
    A, B, Cm, D = W1[np.ix_(r, r)], W1[np.ix_(r, b)], W1[np.ix_(b, r)], W1[np.ix_(b, b)]
    X = Cm @ np.linalg.solve(A, B) @ np.linalg.inv(D)
    E = dense(lambda c: lat.embed2(c), lat.nbnd2, lat.bnd2_shape())
    # the embedding is an isometry onto the black sub-slabs' first slices
    assert relerr(E.conj().T @ E, np.eye(lat.nbnd2)) < 1e-14
    assert np.all(E[r] == 0)
    Rd = np.eye(lat.nbnd2) - E[b].conj().T @ X @ E[b]
    for k in range(3):
        c = syn.gaussian_complex(lat.bnd2_shape(), 200 + k)
        assert relerr(lat.schur2(U, kappa, c, O.R, tol=1e-14).ravel(), Rd @ c.ravel()) < 1e-10
    # X vanishes outside the embedded subspace: the range of C2 is spanned by E
    Pb = E[b] @ E[b].conj().T
    assert relerr(Pb @ Cm, Cm) < 1e-13


def test_boundary2_subspace():
    L = (8, 2, 2, 4)
    lat = _lat(L, 4)
    U = syn.random_links(L, 0.3, 25)
    col = _sub(lat) % 2
    red = syn.gaussian_spinor(lat.V, 26)
    red[col == 1] = 0
    out = lat.hop(U, red, O.HOP_CROSS2)
    out[col == 0] = 0
    assert relerr(lat.embed2(lat.project2(out)), out) < 1e-13
    c = syn.gaussian_complex(lat.bnd2_shape(), 27)
    assert relerr(lat.project2(lat.embed2(c)), c) < 1e-14
    # CROSS2 hops stay inside a first-level slab: HOP_INTRA = INTRA2 + CROSS2
    x = syn.gaussian_spinor(lat.V, 28)
    assert relerr(lat.hop(U, x, O.HOP_INTRA2) + lat.hop(U, x, O.HOP_CROSS2),
                  lat.hop(U, x, O.HOP_INTRA)) < 1e-14


@pytest.mark.parametrize("L,l0", [((4, 2, 2, 2), 2), ((8, 2, 2, 2), 4)])
def test_force_w2_fd(L, l0):
    lat = _lat(L, l0)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 33)
    phi = syn.gaussian_spinor(lat.V, 34)
    S, F = lat.pf_w2(U, kappa, phi)
    rng = np.random.default_rng(2)
    links = [(mu, s) for mu in range(4) for s in range(lat.V)]
    links = [links[i] for i in rng.choice(len(links), 8, replace=False)] + [(0, 3), (0, 17)]
    _fd_check(lambda W: lat.pf_w2(W, kappa, phi, force=False)[0], F, U, links)
    # time-like links crossing a sub-slab face are frozen for this term
    m = lat.index_maps()
    sub = _sub(lat)
    for s in range(lat.V):
        if sub[s] != sub[m[4, s]]:
            assert np.all(F[0, s] == 0)


@pytest.mark.parametrize("L,l0,route,kappa", [((4, 2, 2, 2), 2, 1, 0.15), ((8, 2, 2, 2), 4, 1, 0.13),
                                              ((4, 2, 2, 2), 2, 0, 0.15)])
def test_force_schur2_fd(L, l0, route, kappa):
    lat = _lat(L, l0)
    U = syn.random_links(L, 0.3, 43)
    phi = syn.gaussian_complex(lat.bnd2_shape(), 44)
    S, F = lat.pf_schur2(U, kappa, phi, route=route, tol=1e-13)
    rng = np.random.default_rng(1)
    links = [(mu, s) for mu in range(4) for s in range(lat.V)]
    n = 10 if route == 1 else 2
    pick = [links[i] for i in rng.choice(len(links), n, replace=False)]
    pick += [(0, s) for s in range(0, lat.V, 5 if route == 1 else 32)]
    _fd_check(lambda W: lat.pf_schur2(W, kappa, phi, force=False, route=route, tol=1e-13)[0],
              F, U, pick)
    # S_R2 depends only on links inside the first-level slabs
    m = lat.index_maps()
    for s in range(lat.V):
        if m[2, s] != m[2, m[4, s]]:
            assert np.all(F[0, s] == 0)


def _setup4(L, l0, eps, seed):
    lat = _lat(L, l0)
    U = syn.random_links(L, eps, seed)
    P = syn.gaussian_momenta(lat.V, seed + 1)
    phi2 = syn.gaussian_complex(lat.bnd_shape(), seed + 3)
    phi3 = syn.gaussian_spinor(lat.V, seed + 4)
    phi4 = syn.gaussian_complex(lat.bnd2_shape(), seed + 5)
    return lat, U, P, phi2, phi3, phi4


def _prm4(n, scheme=O.LF, tau=0.3, nsteps=None, **kw):
    """S_G + S_R1 + S_R2 + S_W2 on two levels: gauge and W2 on the fine
    level 0, the two Schur terms on the coarse level 1"""
    kw.setdefault("tol", 1e-14)
    return O.hmc_params(5.6, 0.15, tau, 2, (scheme, scheme), nsteps or [n, 2], level_gauge=0,
                        level_w1=-1, level_schur=1, level_w2=0, level_schur2=1, **kw)


def test_md4_reversibility():
    lat, U, P, phi2, phi3, phi4 = _setup4((4, 2, 2, 2), 2, 0.3, 63)
    prm = _prm4(2)
    U1, P1, st = O.md(lat, U, P, None, phi2, prm, phi3, phi4)
    assert st == 0
    assert np.max(np.abs(U1 - U)) > 1e-3
    U2, P2, st = O.md(lat, U1, -P1, None, phi2, prm, phi3, phi4)
    assert np.max(np.abs(U2 - U)) < 1e-12
    assert np.max(np.abs(P2 + P)) < 1e-10


def test_md4_dH_scales_as_dt_squared():
    lat, U, P, phi2, phi3, phi4 = _setup4((4, 2, 2, 2), 2, 0.3, 73)
    kappa, beta = 0.15, 5.6

    def H(Ux, Px):
        return (0.5 * np.sum(Px ** 2) + lat.gauge_action(Ux, beta)
                + lat.pf_schur(Ux, kappa, phi2, force=False, tol=1e-14)[0]
                + lat.pf_w2(Ux, kappa, phi3, force=False, tol=1e-14)[0]
                + lat.pf_schur2(Ux, kappa, phi4, force=False, tol=1e-14)[0])

    H0 = H(U, P)
    ns = [3, 6, 12]
    dh = []
    for n in ns:
        prm = O.hmc_params(beta, kappa, 0.4, 1, (O.LF,), [n], level_gauge=0, level_w1=-1,
                           level_schur=0, level_w2=0, level_schur2=0, tol=1e-14)
        U1, P1, st = O.md(lat, U, P, None, phi2, prm, phi3, phi4)
        assert st == 0
        dh.append(abs(H(U1, P1) - H0))
    slope = np.polyfit(np.log(0.4 / np.array(ns)), np.log(dh), 1)[0]
    assert 1.8 < slope < 2.2, (slope, dh)


def test_heatbath_actions_level2():
    lat = _lat((8, 2, 2, 2), 4)
    U = syn.random_links(lat.L, 0.3, 83)
    kappa = 0.15
    eta3 = syn.gaussian_spinor(lat.V, 5)
    eta4 = syn.gaussian_complex(lat.bnd2_shape(), 6)
    S3 = lat.pf_w2(U, kappa, lat.W2(U, kappa, eta3), force=False)[0]
    S4 = lat.pf_schur2(U, kappa, lat.schur2(U, kappa, eta4, O.R, tol=1e-14), force=False)[0]
    assert abs(S3 - np.vdot(eta3, eta3).real) < 1e-10 * S3
    assert abs(S4 - np.vdot(eta4, eta4).real) < 1e-9 * S4


def test_trajectory_four_part_action_small_dH():
    """a full trajectory of the four-part action: its dH matches H1 - H0
    recomputed from the end configuration and is small at fine steps"""
    L = (4, 2, 2, 2)
    lat = _lat(L, 2)
    U = syn.random_links(L, 0.3, 93)
    dh = []
    for n in (4, 8):
        prm = _prm4(n, nsteps=[2 * n, n], metropolis=0, tol=1e-13)
        U1, res, st = lat.hmc_trajectory(U, prm, 11, 0)
        assert st == 0
        assert abs(res.dH - (res.H1 - res.H0)) < 1e-12 * abs(res.H0)
        assert res.accepted == 1
        assert np.max(np.abs(U1 - U)) > 1e-3
        dh.append(abs(res.dH))
    assert dh[1] < 0.01 and dh[0] > 3 * dh[1], dh
