"""Pins of the oracle's even-odd pieces and of its x0 shift.

* ``lqo_dslash_eo`` (Sec. 1 eq. (2), even-odd form): against a hopping term
  written out in this file from eq. (2) site by site (explicit gamma
  matrices, explicit neighbours, the fermion phase on the x0 wrap), for both
  parities and both daggers.  A field placed on the wrong parity block, a
  result read from the wrong block, a swapped projector or a missing wrap
  phase each fail it.
* ``lqo_mhat`` (Mhat = 1 - kappa^2 H_eo H_oe): the even-even Schur complement
  of the dense Wilson matrix (M_oo = 1), its adjoint, and det M = det Mhat.
  A wrong power or sign of kappa, or the two half sweeps taken in the wrong
  order, fail it.
* ``lqo_roll_x0`` (end of Sec. 2, the shift of the configuration along x0):
  a shift by L0 is the identity, shifts compose additively, a shift by one
  moves link (x0, x) to (x0 + 1, x) and by -1 back, the plaquette and the
  gauge action are invariant, and det M is invariant because the shifted
  Wilson matrix is the translated one up to sign flips of whole time slices
  (the antiperiodic phase moves with the configuration).
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

SX = np.array([[0, 1], [1, 0]], complex)
SY = np.array([[0, -1j], [1j, 0]], complex)
SZ = np.array([[1, 0], [0, -1]], complex)
I2 = np.eye(2)
GAM = [-np.kron(SX, I2), np.kron(SY, SX), np.kron(SY, SY), np.kron(SY, SZ)]  # chiral basis
ONE4 = np.eye(4)


def cb_coords(L):
    V = int(np.prod(L))
    out = np.zeros((V, 4), int)
    for x in itertools.product(*[range(n) for n in L]):
        lex = ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]
        out[(sum(x) % 2) * (V // 2) + lex // 2] = x
    return out


def brute_hop(L, bc_t, U, psi, dagger):
    """eq. (2)'s hopping term: (H psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x + mu)
    + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu); the adjoint swaps the two
    projectors.  Hops that wrap L0-1 <-> 0 carry bc_t."""
    c = cb_coords(L)
    look = {tuple(v): s for s, v in enumerate(c)}
    out = np.zeros_like(psi)
    sf = 1 if dagger else -1
    for s, x in enumerate(c):
        acc = np.zeros((4, 3), complex)
        for mu in range(4):
            y = list(x); y[mu] = (y[mu] + 1) % L[mu]
            z = list(x); z[mu] = (z[mu] - 1) % L[mu]
            fy, fz = look[tuple(y)], look[tuple(z)]
            ph_f = bc_t if (mu == 0 and x[0] == L[0] - 1) else 1
            ph_b = bc_t if (mu == 0 and x[0] == 0) else 1
            # spin matrix acts on the spin index, link on the colour index
            acc += ph_f * (ONE4 + sf * GAM[mu]) @ (psi[fy] @ U[mu, s].T)
            acc += ph_b * (ONE4 - sf * GAM[mu]) @ (psi[fz] @ U[mu, fz].conj())
        out[s] = acc
    return out


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
# lqo_dslash_eo
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,bc", [((2, 2, 2, 2), -1), ((4, 2, 2, 2), -1), ((4, 2, 2, 2), 1), ((2, 4, 2, 2), -1)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dslash_eo_against_brute_force(L, bc, dagger):
    lat = O.Lattice(L, 1, bc)
    U = syn.random_links(L, 0.6, 301)
    Vh = lat.Vh
    for parity in (0, 1):
        x_in = syn.gaussian_spinor(Vh, 302 + parity)
        full = np.zeros((lat.V, 4, 3), complex)
        full[(1 - parity) * Vh:(2 - parity) * Vh] = x_in
        ref = brute_hop(L, bc, U, full, dagger)
        # the input lives on parity 1-p only, so the hopping term is zero on it
        assert np.max(np.abs(ref[(1 - parity) * Vh:(2 - parity) * Vh])) == 0.0
        want = ref[parity * Vh:(parity + 1) * Vh]
        assert relerr(lat.dslash_eo(U, x_in, parity, dagger), want) < 1e-13
        # and the full-lattice oracle hopping term restricted the same way
        assert relerr(lat.hop(U, full, O.HOP_ALL, dagger)[parity * Vh:(parity + 1) * Vh], want) < 1e-13


def test_brute_hop_free_field_constant_mode():
    """the test-side hopping term itself: on U = 1 with periodic phases a
    constant spinor chi gives H chi = sum_mu 2 chi = 8 chi"""
    L = (2, 4, 2, 2)
    V = int(np.prod(L))
    U = np.zeros((4, V, 3, 3), complex)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    chi = syn.gaussian_complex((4, 3), 5)
    psi = np.broadcast_to(chi, (V, 4, 3)).copy()
    for dag in (0, 1):
        assert relerr(brute_hop(L, 1, U, psi, dag), 8 * psi) < 1e-14


# ---------------------------------------------------------------------------
# lqo_mhat: even-even Schur complement of M
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,bc", [((2, 2, 2, 2), -1), ((4, 2, 2, 2), -1), ((4, 2, 2, 2), 1)])
def test_mhat_is_even_schur_complement(L, bc):
    lat = O.Lattice(L, 1, bc)
    kappa = 0.14
    U = syn.random_links(L, 0.5, 311)
    n, nh = lat.V * 12, lat.Vh * 12
    Md = dense(lambda x: lat.M(U, kappa, x), n, lat.spinor_shape())
    Mee, Meo, Moe, Moo = Md[:nh, :nh], Md[:nh, nh:], Md[nh:, :nh], Md[nh:, nh:]
    # M has identity diagonal blocks (the hopping term only links parities)
    assert np.max(np.abs(Mee - np.eye(nh))) == 0.0 and np.max(np.abs(Moo - np.eye(nh))) == 0.0
    schur = Mee - Meo @ np.linalg.solve(Moo, Moe)
    Mh = dense(lambda x: lat.mhat(U, kappa, x), nh, lat.half_shape())
    assert relerr(Mh, schur) < 1e-13
    Mhd = dense(lambda x: lat.mhat(U, kappa, x, dagger=1), nh, lat.half_shape())
    assert relerr(Mhd, schur.conj().T) < 1e-13
    # det M = det Mhat (block LU with M_oo = 1)
    sM, lM = np.linalg.slogdet(Md)
    sH, lH = np.linalg.slogdet(Mh)
    assert abs(lM - lH) < 1e-11 * max(1.0, abs(lM))
    assert abs(sM - sH) < 1e-9
    # the power of kappa: Mhat(kappa) - 1 scales as kappa^2
    x = syn.gaussian_spinor(lat.Vh, 313)
    d1 = lat.mhat(U, kappa, x) - x
    d2 = lat.mhat(U, 2 * kappa, x) - x
    assert relerr(d2, 4 * d1) < 1e-13


# ---------------------------------------------------------------------------
# lqo_roll_x0
# ---------------------------------------------------------------------------
def test_roll_x0_moves_links_forward_by_brute_force():
    L = (6, 2, 4, 2)
    lat = O.Lattice(L, 1, -1)
    U = syn.random_links(L, 0.7, 321)
    c = cb_coords(L)
    look = {tuple(v): s for s, v in enumerate(c)}
    for shift in (1, 2, -1, 5):
        R = lat.roll_x0(U, shift)
        for s, x in enumerate(c):
            y = list(x); y[0] = (y[0] + shift) % L[0]
            for mu in range(4):
                assert np.array_equal(R[mu, look[tuple(y)]], U[mu, s])


def test_roll_x0_identity_and_composition():
    L = (8, 2, 2, 4)
    lat = O.Lattice(L, 2, -1)
    U = syn.random_links(L, 0.7, 331)
    assert np.array_equal(lat.roll_x0(U, L[0]), U)
    assert np.array_equal(lat.roll_x0(U, 0), U)
    assert np.array_equal(lat.roll_x0(lat.roll_x0(U, 3), 2), lat.roll_x0(U, 5))
    assert np.array_equal(lat.roll_x0(lat.roll_x0(U, 3), -3), U)
    assert np.array_equal(lat.roll_x0(U, 3 + L[0]), lat.roll_x0(U, 3))
    # a non-trivial shift changes the field
    assert not np.array_equal(lat.roll_x0(U, 1), U)


def test_roll_x0_keeps_plaquette_and_gauge_action():
    L = (8, 2, 4, 2)
    lat = O.Lattice(L, 2, -1)
    U = syn.random_links(L, 0.8, 341)
    S = lat.gauge_action(U, 5.6)
    for shift in (1, 3, 6):
        R = lat.roll_x0(U, shift)
        assert abs(lat.gauge_action(R, 5.6) - S) < 1e-11 * abs(S)
        assert abs(lat.plaquette(R) - lat.plaquette(U)) < 1e-14


@pytest.mark.parametrize("bc", [-1, 1])
def test_roll_x0_keeps_det_M(bc):
    """M[shifted U] = S T M[U] T^-1 S with T the translation and S a sign
    flip of whole time slices, so det M is unchanged; det W1 changes in
    general (the slabs stay where they are)"""
    L = (4, 2, 2, 2)
    lat = O.Lattice(L, 2, bc)
    kappa = 0.15
    U = syn.random_links(L, 0.5, 351)
    n = lat.V * 12
    s0, l0 = np.linalg.slogdet(dense(lambda x: lat.M(U, kappa, x), n, lat.spinor_shape()))
    for shift in (1, 2, 3):
        R = lat.roll_x0(U, shift)
        s1, l1 = np.linalg.slogdet(dense(lambda x: lat.M(R, kappa, x), n, lat.spinor_shape()))
        assert abs(l1 - l0) < 1e-11 * max(1.0, abs(l0))
        assert abs(s1 - s0) < 1e-9
    # W1 is not translation covariant by one slice: its determinant moves
    w0 = np.linalg.slogdet(dense(lambda x: lat.W1(U, kappa, x), n, lat.spinor_shape()))[1]
    w1 = np.linalg.slogdet(dense(lambda x: lat.W1(lat.roll_x0(U, 1), kappa, x), n, lat.spinor_shape()))[1]
    assert abs(w1 - w0) > 1e-6
