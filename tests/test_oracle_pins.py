"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here calls the GPU library.  Each test checks the oracle against an
independent fact: a closed form (free-field momentum space), an algebraic
identity (Clifford algebra, gamma5-hermiticity, gauge covariance, block-LU
determinant factorisation det M = det W1 det R), a library routine (scipy's
expm, numpy's dense linear algebra) or finite differences of the actions.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

# ---------------------------------------------------------------------------
# test-side constructions (written independently of the oracle)
# ---------------------------------------------------------------------------
SX = np.array([[0, 1], [1, 0]], complex)
SY = np.array([[0, -1j], [1j, 0]], complex)
SZ = np.array([[1, 0], [0, -1]], complex)
I2 = np.eye(2)


def gammas():
    """chiral basis: gamma_0 = -sx (x) 1, gamma_k = sy (x) s_k"""
    return [-np.kron(SX, I2), np.kron(SY, SX), np.kron(SY, SY), np.kron(SY, SZ)]


def cb_coords(L):
    """checkerboard site order by brute force: coords[s] = (x0,x1,x2,x3)"""
    V = int(np.prod(L))
    out = np.zeros((V, 4), int)
    for x in itertools.product(*[range(n) for n in L]):
        lex = ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]
        p = sum(x) % 2
        out[p * (V // 2) + lex // 2] = x
    return out


def site_lookup(L):
    c = cb_coords(L)
    return {tuple(v): s for s, v in enumerate(c)}, c


def unit_links(V):
    U = np.zeros((4, V, 3, 3), complex)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def dense(apply, n_in, shape_in):
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, complex)
        e[k] = 1
        cols.append(apply(e.reshape(shape_in)).ravel())
    return np.array(cols).T


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------------------
# gamma matrices and index maps
# ---------------------------------------------------------------------------
def test_gamma_clifford_and_basis():
    g = O.Lattice.gamma()
    ref = gammas()
    for mu in range(4):
        assert np.allclose(g[mu], ref[mu])
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * (mu == nu) * np.eye(4))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3])


@pytest.mark.parametrize("L,l0", [((4, 2, 2, 2), 1), ((8, 4, 2, 6), 2), ((4, 4, 4, 4), 2)])
def test_index_maps_brute_force(L, l0):
    lat = O.Lattice(L, l0)
    m = lat.index_maps()
    look, c = site_lookup(L)
    V3 = L[1] * L[2] * L[3]
    for s in range(lat.V):
        x = c[s]
        assert m[0, s] == ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]
        assert m[1, s] == sum(x) % 2
        assert m[2, s] == x[0] // l0 and m[3, s] == (x[0] // l0) % 2
        for mu in range(4):
            y = list(x); y[mu] = (y[mu] + 1) % L[mu]
            z = list(x); z[mu] = (z[mu] - 1) % L[mu]
            assert m[4 + mu, s] == look[tuple(y)]
            assert m[8 + mu, s] == look[tuple(z)]
        first = x[0] % l0 == 0
        last = x[0] % l0 == l0 - 1
        assert m[12, s] == int(first) + 2 * int(last)
        k = x[0] // l0
        if k % 2 == 1 and (first or last):
            lex3 = (x[1] * L[2] + x[2]) * L[3] + x[3]
            assert m[13, s] == ((k // 2) * 2 + (0 if first else 1)) * V3 + lex3
        else:
            assert m[13, s] == -1


# ---------------------------------------------------------------------------
# eq. (2): free field against the momentum-space closed form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc_t", [1, -1])
def test_free_field_plane_waves(bc_t):
    L = (4, 4, 2, 6)
    lat = O.Lattice(L, 1, bc_t)
    kappa = 0.137
    U = unit_links(lat.V)
    c = cb_coords(L)
    g = gammas()
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = [rng.integers(0, L[mu]) for mu in range(4)]
        p = np.array([2 * math.pi * n[mu] / L[mu] for mu in range(4)])
        if bc_t == -1:
            p[0] += math.pi / L[0]
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = phase[:, None, None] * chi[None]
        Mp = np.eye(4, dtype=complex)
        for mu in range(4):
            Mp -= kappa * (2 * math.cos(p[mu]) * np.eye(4) - 2j * math.sin(p[mu]) * g[mu])
        expect = phase[:, None, None] * (Mp @ chi)[None]
        assert relerr(lat.M(U, kappa, psi), expect) < 1e-13


def test_free_w1_is_dirichlet_in_x0():
    """free W1 on one slab: spatial plane waves, Dirichlet (open) ends in x0"""
    L = (8, 2, 4, 2)
    l0 = 4
    lat = O.Lattice(L, l0, -1)
    kappa = 0.11
    U = unit_links(lat.V)
    c = cb_coords(L)
    g = gammas()
    rng = np.random.default_rng(9)
    q = np.array([0.0, 2 * math.pi / L[1], 2 * math.pi * 1 / L[2], math.pi])
    f = rng.standard_normal((L[0], 4, 3)) + 1j * rng.standard_normal((L[0], 4, 3))
    phase = np.exp(1j * (c[:, 1:] @ q[1:]))
    psi = phase[:, None, None] * f[c[:, 0]]
    # spatial part diagonal in q; x0 part: the l0 x l0 tridiagonal per slab
    Ks = np.eye(4, dtype=complex)
    for mu in (1, 2, 3):
        Ks -= kappa * (2 * math.cos(q[mu]) * np.eye(4) - 2j * math.sin(q[mu]) * g[mu])
    expect_t = np.zeros_like(f)
    for t in range(L[0]):
        expect_t[t] = Ks @ f[t]
        if (t + 1) % l0 != 0:
            expect_t[t] -= kappa * (np.eye(4) - g[0]) @ f[t + 1]
        if t % l0 != 0:
            expect_t[t] -= kappa * (np.eye(4) + g[0]) @ f[t - 1]
    expect = phase[:, None, None] * expect_t[c[:, 0]]
    assert relerr(lat.W1(U, kappa, psi), expect) < 1e-13


# ---------------------------------------------------------------------------
# gamma5-hermiticity and gauge covariance on random links
# ---------------------------------------------------------------------------
def _g5(x):
    y = x.copy()
    y[:, 2:, :] *= -1
    return y


@pytest.mark.parametrize("mode", [O.HOP_ALL, O.HOP_INTRA, O.HOP_CROSS])
def test_gamma5_hermiticity(mode):
    L = (8, 2, 4, 2)
    lat = O.Lattice(L, 2, -1)
    U = syn.random_links(L, 0.4, 11)
    chi = syn.gaussian_spinor(lat.V, 1)
    psi = syn.gaussian_spinor(lat.V, 2)
    H = lat.hop(U, psi, mode)
    Hd = lat.hop(U, chi, mode, dagger=1)
    # <chi, H psi> = <H^dag chi, psi>
    assert abs(np.vdot(chi, H) - np.vdot(Hd, psi)) < 1e-11 * np.linalg.norm(H) * np.linalg.norm(chi)
    # H^dag = gamma5 H gamma5
    assert relerr(Hd, _g5(lat.hop(U, _g5(chi), mode))) < 1e-13


def test_gauge_covariance():
    L = (4, 4, 2, 2)
    lat = O.Lattice(L, 1, -1)
    kappa = 0.15
    U = syn.random_links(L, 0.5, 3)
    gt = syn.random_gauge_transform(lat.V, 4)
    look, c = site_lookup(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        for s in range(lat.V):
            y = list(c[s]); y[mu] = (y[mu] + 1) % L[mu]
            Ug[mu, s] = gt[s] @ U[mu, s] @ gt[look[tuple(y)]].conj().T
    psi = syn.gaussian_spinor(lat.V, 5)
    gpsi = np.einsum("sij,saj->sai", gt, psi)
    for f in (lat.M, lat.W1):
        lhs = f(Ug, kappa, gpsi)
        rhs = np.einsum("sij,saj->sai", gt, f(U, kappa, psi))
        assert relerr(lhs, rhs) < 1e-12


# ---------------------------------------------------------------------------
# Schwarz factorisation det M = det W1 det R (block LU of eq. (2))
# ---------------------------------------------------------------------------
def _dense_ops(lat, U, kappa):
    n = lat.V * 12
    Md = dense(lambda x: lat.M(U, kappa, x), n, lat.spinor_shape())
    Wd = dense(lambda x: lat.W1(U, kappa, x), n, lat.spinor_shape())
    return Md, Wd


@pytest.mark.parametrize("L,l0,bc", [((2, 2, 2, 2), 1, -1), ((2, 2, 2, 2), 1, 1),
                                     ((4, 2, 2, 2), 1, -1), ((4, 2, 2, 2), 2, -1),
                                     ((8, 2, 2, 2), 2, 1)])
def test_det_factorisation_dense(L, l0, bc):
    lat = O.Lattice(L, l0, bc)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 21)
    Md, Wd = _dense_ops(lat, U, kappa)
    Rd = dense(lambda c: lat.schur(U, kappa, c, O.R, tol=1e-14), lat.nbnd, lat.bnd_shape())
    sM, lM = np.linalg.slogdet(Md)
    sW, lW = np.linalg.slogdet(Wd)
    sR, lR = np.linalg.slogdet(Rd)
    assert abs(lM - (lW + lR)) < 1e-10 * max(1, abs(lM))
    assert abs(sM - sW * sR) < 1e-9
    # det M, det W1 and det R are real (gamma5-hermiticity)
    assert abs(sM.imag) < 1e-9 and abs(sW.imag) < 1e-9 and abs(sR.imag) < 1e-9
    # W1 is block diagonal in the slabs
    slab = np.repeat(lat.index_maps()[2], 12)
    assert np.all(Wd[slab[:, None] != slab[None, :]] == 0)
    # R^dag and both R^-1 routes against dense linear algebra
    c = syn.gaussian_complex(lat.bnd_shape(), 7)
    Rdag = dense(lambda v: lat.schur(U, kappa, v, O.RDAG, tol=1e-14), lat.nbnd, lat.bnd_shape())
    assert relerr(Rdag, Rd.conj().T) < 1e-10
    ref = np.linalg.solve(Rd, c.ravel())
    refd = np.linalg.solve(Rd.conj().T, c.ravel())
    for route in ((0, 1) if lat.nbnd <= 96 else (1,)):
        assert relerr(lat.schur(U, kappa, c, O.RINV, route, tol=1e-13).ravel(), ref) < 1e-9
        assert relerr(lat.schur(U, kappa, c, O.RINVDAG, route, tol=1e-13).ravel(), refd) < 1e-9


def test_det_factorisation_4x4x4x4():
    """The small 4^4 workload geometry (l0=2): dense det M / det W1 against
    det R, with R assembled from dense blocks; the oracle's R matches it on
    random vectors"""
    L = (4, 4, 4, 4)
    lat = O.Lattice(L, 2, -1)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 2008)
    Md, Wd = _dense_ops(lat, U, kappa)
    col = np.repeat(lat.index_maps()[3], 12)
    r, b = col == 0, col == 1
    A, B, Cm, D = Md[np.ix_(r, r)], Md[np.ix_(r, b)], Md[np.ix_(b, r)], Md[np.ix_(b, b)]
    X = Cm @ np.linalg.solve(A, B) @ np.linalg.inv(D)
    E = dense(lambda c: lat.embed(c), lat.nbnd, lat.bnd_shape())[b]  # black rows
    Rd = np.eye(lat.nbnd) - E.conj().T @ X @ E
    sM, lM = np.linalg.slogdet(Md)
    sW, lW = np.linalg.slogdet(Wd)
    sR, lR = np.linalg.slogdet(Rd)
    assert abs(lM - (lW + lR)) < 1e-10 * abs(lM)
    assert abs(sM - sW * sR) < 1e-9
    for k in range(3):
        c = syn.gaussian_complex(lat.bnd_shape(), 100 + k)
        assert relerr(lat.schur(U, kappa, c, O.R, tol=1e-14).ravel(), Rd @ c.ravel()) < 1e-10


def test_boundary_subspace():
    """range of C (red -> black hops) lies in the spin-projected black faces,
    and the face basis is orthonormal"""
    L = (8, 2, 2, 4)
    lat = O.Lattice(L, 2, -1)
    U = syn.random_links(L, 0.3, 5)
    col = lat.index_maps()[3]
    red = syn.gaussian_spinor(lat.V, 8)
    red[col == 1] = 0
    out = lat.hop(U, red, O.HOP_CROSS)
    out[col == 0] = 0
    assert relerr(lat.embed(lat.project(out)), out) < 1e-13
    c = syn.gaussian_complex(lat.bnd_shape(), 9)
    assert relerr(lat.project(lat.embed(c)), c) < 1e-14
    assert abs(np.vdot(lat.embed(c), lat.embed(c)) - np.vdot(c, c)) < 1e-12 * np.vdot(c, c).real


def test_free_field_R_conserves_spatial_momentum():
    """U = 1: R commutes with spatial translations, so a boundary field that
    is a spatial plane wave exp(i p.x) stays one (with the same p), with a
    boundary-coordinate amplitude matrix that does not depend on x"""
    L = (8, 4, 2, 2)
    lat = O.Lattice(L, 2, -1)
    U = unit_links(lat.V)
    nj = lat.nb // 2
    x1, x2, x3 = np.meshgrid(np.arange(L[1]), np.arange(L[2]), np.arange(L[3]), indexing="ij")
    p = 2 * np.pi * np.array([1, 1, 0]) / np.array(L[1:])
    wave = np.exp(1j * (p[0] * x1 + p[1] * x2 + p[2] * x3)).reshape(-1)  # lexicographic (x1,x2,x3)
    rng = np.random.default_rng(4)
    amp = rng.standard_normal((nj, 2, 2, 3)) + 1j * rng.standard_normal((nj, 2, 2, 3))
    c = amp[:, :, None, :, :] * wave[None, None, :, None, None]
    out = lat.schur(U, 0.12, c, O.R, tol=1e-14)
    ratio = out / wave[None, None, :, None, None]
    assert np.max(np.abs(ratio - ratio[:, :, :1])) < 1e-12 * np.max(np.abs(ratio))
    assert np.max(np.abs(ratio)) > 1e-3  # and the result is not trivially zero


# ---------------------------------------------------------------------------
# forces against central finite differences of the actions
# ---------------------------------------------------------------------------
TA = syn._generators()


def _perturb(U, mu, s, a, h):
    V = U.copy()
    V[mu, s] = scipy.linalg.expm(1j * h * TA[a]) @ U[mu, s]
    return V


def _fd_check(action, force, U, links, h=1e-5, tol=1e-6):
    scale = np.max(np.abs(force))
    worst = 0.0
    for (mu, s) in links:
        for a in range(8):
            d = (action(_perturb(U, mu, s, a, h)) - action(_perturb(U, mu, s, a, -h))) / (2 * h)
            worst = max(worst, abs(d - force[mu, s, a]) / scale)
    assert worst < tol, worst


@pytest.mark.parametrize("L,l0", [((2, 2, 2, 2), 1), ((4, 2, 2, 2), 2)])
def test_force_w1_fd(L, l0):
    lat = O.Lattice(L, l0, -1)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 31)
    phi = syn.gaussian_spinor(lat.V, 32)
    S, F = lat.pf_w1(U, kappa, phi)
    links = [(mu, s) for mu in range(4) for s in range(lat.V)]
    if lat.V > 16:
        links = links[::5]
    _fd_check(lambda W: lat.pf_w1(W, kappa, phi, force=False)[0], F, U, links)
    # links that cross a slab face are frozen for this term (exactly zero)
    m = lat.index_maps()
    for s in range(lat.V):
        if m[2, s] != m[2, m[4, s]]:
            assert np.all(F[0, s] == 0)


@pytest.mark.parametrize("L,l0,route", [((2, 2, 2, 2), 1, 1), ((4, 2, 2, 2), 2, 1),
                                        ((4, 2, 2, 2), 1, 0)])
def test_force_schur_fd(L, l0, route):
    lat = O.Lattice(L, l0, -1)
    kappa = 0.15
    U = syn.random_links(L, 0.3, 41)
    phi = syn.gaussian_complex(lat.bnd_shape(), 42)
    S, F = lat.pf_schur(U, kappa, phi, route=route, tol=1e-13)
    rng = np.random.default_rng(0)
    links = [(mu, s) for mu in range(4) for s in range(lat.V)]
    if lat.V > 16:
        n = 12 if route == 1 else 3
        links = [links[i] for i in rng.choice(len(links), n, replace=False)]
        links += [(0, s) for s in range(lat.V)][:n // 2]
    _fd_check(lambda W: lat.pf_schur(W, kappa, phi, force=False, route=route, tol=1e-13)[0],
              F, U, links)


def test_force_gauge_fd():
    L = (4, 2, 4, 2)
    lat = O.Lattice(L, 1, -1)
    U = syn.random_links(L, 0.6, 51)
    beta = 5.6
    F = lat.gauge_force(U, beta)
    links = [(mu, s) for mu in range(4) for s in range(0, lat.V, 3)]
    _fd_check(lambda W: lat.gauge_action(W, beta), F, U, links)


def test_gauge_action_cold_and_plaquette():
    L = (4, 2, 2, 2)
    lat = O.Lattice(L, 1)
    U = unit_links(lat.V)
    # 6 plaquettes per site with Re tr = 3
    assert abs(lat.gauge_action(U, 5.6) - (-5.6 / 3 * 6 * lat.V * 3)) < 1e-9
    assert abs(lat.plaquette(U) - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# SU(3) exponential (T_U of eq. (3)) and link update
# ---------------------------------------------------------------------------
def test_su3_exp_against_scipy():
    rng = np.random.default_rng(3)
    for k in range(20):
        h = rng.standard_normal(8) * (0.05 + k * 0.3)
        X = np.einsum("a,aij->ij", h, TA)
        E = O.su3_expi(X)
        assert np.max(np.abs(E - scipy.linalg.expm(1j * X))) < 1e-13
        assert np.max(np.abs(E @ E.conj().T - np.eye(3))) < 1e-13
        assert abs(np.linalg.det(E) - 1) < 1e-12


def test_update_U_matches_expm():
    L = (2, 2, 2, 2)
    lat = O.Lattice(L, 1)
    U = syn.random_links(L, 0.5, 1)
    P = syn.gaussian_momenta(lat.V, 2)
    dt = 0.07
    U2 = lat.update_U(U, P, dt)
    for mu in range(4):
        for s in range(lat.V):
            X = np.einsum("a,aij->ij", P[mu, s] * dt, TA)
            assert np.max(np.abs(U2[mu, s] - scipy.linalg.expm(1j * X) @ U[mu, s])) < 1e-13


# ---------------------------------------------------------------------------
# random numbers: Philox4x32-10 known answers and Gaussian moments
# ---------------------------------------------------------------------------
def _read_kat():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, out in _read_kat():
        assert O.philox4x32_10(ctr, key) == out


def test_normals_moments():
    x = O.normals(2007, 1, 0, 200000)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1) < 0.01
    assert abs(np.mean(x ** 4) - 3) < 0.05
    u, s = O.metropolis_uniforms(2007, 3, 16)
    assert 0 < u < 1 and 0 <= s < 16


# ---------------------------------------------------------------------------
# HMC (Sec. 2): reversibility, dH scaling, <exp(-dH)> = 1, heatbath
# ---------------------------------------------------------------------------
def _setup(L, l0, eps, seed):
    lat = O.Lattice(L, l0, -1)
    U = syn.random_links(L, eps, seed)
    P = syn.gaussian_momenta(lat.V, seed + 1)
    phi1 = syn.gaussian_spinor(lat.V, seed + 2)
    phi2 = syn.gaussian_complex(lat.bnd_shape(), seed + 3)
    return lat, U, P, phi1, phi2


@pytest.mark.parametrize("scheme,levels", [((O.LF,), 1), ((O.SW, O.SW), 2)])
def test_md_reversibility(scheme, levels):
    lat, U, P, phi1, phi2 = _setup((2, 2, 2, 2), 1, 0.3, 61)
    if levels == 1:
        prm = O.hmc_params(5.6, 0.15, 0.3, 1, scheme, [3], 0, 0, 0, tol=1e-14)
    else:
        prm = O.hmc_params(5.6, 0.15, 0.3, 2, scheme, [2, 2], 0, 1, 1, tol=1e-14)
    U1, P1, st = O.md(lat, U, P, phi1, phi2, prm)
    assert st == 0
    U2, P2, st = O.md(lat, U1, -P1, phi1, phi2, prm)
    assert np.max(np.abs(U2 - U)) < 1e-12
    assert np.max(np.abs(P2 + P)) < 1e-10


def _dH(lat, U, P, phi1, phi2, prm, kappa, beta):
    def H(Ux, Px):
        return (0.5 * np.sum(Px ** 2) + lat.gauge_action(Ux, beta)
                + lat.pf_w1(Ux, kappa, phi1, force=False, tol=1e-14)[0]
                + lat.pf_schur(Ux, kappa, phi2, force=False, tol=1e-14)[0])
    U1, P1, st = O.md(lat, U, P, phi1, phi2, prm)
    return H(U1, P1) - H(U, P)


def test_dH_scales_as_dt_squared():
    lat, U, P, phi1, phi2 = _setup((2, 2, 2, 2), 1, 0.3, 71)
    kappa, beta = 0.15, 5.6
    ns = [4, 8, 16, 32]
    dh = [abs(_dH(lat, U, P, phi1, phi2,
                  O.hmc_params(beta, kappa, 0.5, 1, (O.LF,), [n], tol=1e-14), kappa, beta))
          for n in ns]
    slope = np.polyfit(np.log(0.5 / np.array(ns)), np.log(dh), 1)[0]
    assert 1.8 < slope < 2.2, (slope, dh)
    # the improved scheme (lambda = 1/6) is second order as well
    sw = [abs(_dH(lat, U, P, phi1, phi2,
                  O.hmc_params(beta, kappa, 0.5, 1, (O.SW,), [n], tol=1e-14), kappa, beta))
          for n in ns[1:]]
    slope = np.polyfit(np.log(0.5 / np.array(ns[1:])), np.log(sw), 1)[0]
    assert 1.8 < slope < 2.2, (slope, sw)


def test_heatbath_actions():
    lat, U, P, phi1, phi2 = _setup((4, 2, 2, 2), 1, 0.3, 81)
    kappa = 0.15
    eta1 = syn.gaussian_spinor(lat.V, 3)
    eta2 = syn.gaussian_complex(lat.bnd_shape(), 4)
    S1 = lat.pf_w1(U, kappa, lat.W1(U, kappa, eta1), force=False)[0]
    S2 = lat.pf_schur(U, kappa, lat.schur(U, kappa, eta2, O.R, tol=1e-14), force=False)[0]
    assert abs(S1 - np.vdot(eta1, eta1).real) < 1e-10 * S1
    assert abs(S2 - np.vdot(eta2, eta2).real) < 1e-9 * S2


def test_exp_minus_dH_average():
    """<exp(-dH)> = 1 (area preservation + reversibility), 2 sigma"""
    L = (2, 2, 2, 2)
    lat = O.Lattice(L, 1, -1)
    U = syn.random_links(L, 0.3, 91)
    prm = O.hmc_params(5.6, 0.15, 0.4, 2, (O.LF, O.LF), [2, 3], 0, 1, 1, metropolis=1,
                       roll=1, tol=1e-12)
    w = []
    for t in range(120):
        U, res, st = lat.hmc_trajectory(U, prm, 2007, t)
        assert st == 0
        w.append(math.exp(-res.dH))
    w = np.array(w)
    err = w.std(ddof=1) / math.sqrt(len(w))
    assert abs(w.mean() - 1) < 2.5 * err + 1e-3, (w.mean(), err)


# ---------------------------------------------------------------------------
# position-dependent step sizes (Sec. 2, schemes A, B, C)
# ---------------------------------------------------------------------------
def test_step_scheme_averages_match_the_paper():
    """the paper states the average of s over all links: 0.525 for scheme A
    (L0 = 24) and about 0.59 for B and C (L0 = 32)"""
    for scheme, L0, want, tol in [(1, 24, 0.525, 1e-12), (2, 32, 0.59, 0.01), (3, 32, 0.59, 0.015)]:
        s = O.step_scheme(scheme, L0)
        avg = (3 * s[0].mean() + s[1].mean()) / 4  # three space-like, one time-like link per site
        assert abs(avg - want) < tol, (scheme, avg)
    # the periods are 6, 8 and 16 time slices
    assert np.array_equal(O.step_scheme(1, 24)[:, :6], O.step_scheme(1, 24)[:, 6:12])
    with pytest.raises(ValueError):
        O.step_scheme(2, 12)


def test_step_scale_freezes_links_and_stays_reversible():
    L = (8, 2, 2, 2)
    lat, U, P, eta1, eta2 = _setup(L, 2, 0.3, 101)
    phi1 = lat.W1(U, 0.15, eta1)  # heatbath fields
    phi2 = lat.schur(U, 0.15, eta2, O.R, tol=1e-14)
    s = O.step_scheme(2, 8)
    prm = O.hmc_params(5.6, 0.15, 0.3, 2, (O.SW, O.LF), [2, 2], 0, 1, 1, tol=1e-13, step_scale=s)
    U1, P1, st = O.md(lat, U, P, phi1, phi2, prm)
    assert st == 0
    m = lat.index_maps()
    x0 = m[0] // (L[1] * L[2] * L[3])
    for mu in range(4):
        frozen = (s[1 if mu == 0 else 0][x0] == 0)
        assert np.array_equal(U1[mu, frozen], U[mu, frozen])
        assert np.array_equal(P1[mu, frozen], P[mu, frozen])
        assert np.max(np.abs(U1[mu, ~frozen] - U[mu, ~frozen])) > 1e-3
    U2, P2, st = O.md(lat, U1, -P1, phi1, phi2, prm)
    assert np.max(np.abs(U2 - U)) < 1e-11


def test_force_profile_closed_form():
    """Fig. 1 diagnostic: mean |F| per time slice; a force whose 8 coefficients
    equal c(mu, x0) on every link gives sqrt(8) c exactly"""
    L = (6, 2, 4, 2)
    lat = O.Lattice(L, 1, -1)
    m = lat.index_maps()
    x0 = m[0] // (L[1] * L[2] * L[3])
    F = np.zeros((4, lat.V, 8))
    for mu in range(4):
        F[mu] = (1.0 + 0.5 * mu + 0.25 * x0)[:, None]
    prof = lat.force_profile(F)
    t = np.arange(L[0])
    assert np.allclose(prof[0], np.sqrt(8) * (1.0 + 0.25 * t + 0.5 * 2), rtol=1e-14)  # mean of mu = 1, 2, 3
    assert np.allclose(prof[1], np.sqrt(8) * (1.0 + 0.25 * t), rtol=1e-14)
