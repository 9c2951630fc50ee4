"""GPU path (through the C-ABI) against the FP64 oracle, element by element.

Tolerances (relative to the largest element of the reference):
  double kernels 1e-12; single-precision stencil 1e-6; half storage 5e-3
  and bfloat16 storage 2e-2 (ten unit roundoffs of the storage: 2^-11 for
  fp16, 2^-9 for bfloat16);
  solves: |b - W x| / |b| <= 1e-10 checked with the oracle's operator;
  forces 1e-5 (achieved ~1e-9 with double outer residuals); dH 1e-4.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402

# (L, l0, eps, kappa): the 4^4 and 16x8^3 rows are the small and the solver
# configurations (kappa = 0.15 and 0.156); eps = 0.6 at kappa = 0.156 keeps
# the synthetic field on the positive-mass side, like the paper's ensembles;
# 8x4^3 with l0 = 1 is the degenerate slab of one time slice (both faces of
# a black slab on the same slice, W1 without time-like hops)
GEOMS = [((4, 4, 4, 4), 2, 0.3, 0.15), ((8, 4, 2, 6), 2, 0.3, 0.14), ((16, 8, 8, 8), 4, 0.6, 0.156),
         ((8, 4, 4, 4), 1, 0.3, 0.14)]


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", params=GEOMS, ids=lambda p: "x".join(map(str, p[0])) + "_l0%d" % p[1])
def setup(request):
    L, l0, eps, kappa = request.param
    seed = 2007 + sum(L)
    U = syn.random_links(L, eps, seed)
    lat = lqcd.Lattice(L, l0, -1)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1)
    yield lat, olat, U, kappa, seed
    lat.close()


def test_index_maps_bit_exact(setup):
    lat, olat, U, kappa, seed = setup
    assert np.array_equal(lat.index_maps().cpu().numpy(), olat.index_maps())


def test_gauge_roundtrip(setup):
    lat, olat, U, kappa, seed = setup
    assert np.array_equal(lat.get_gauge().cpu().numpy(), U)


@pytest.mark.parametrize("prec,tol", [(lqcd.PREC_F64, 1e-13), (lqcd.PREC_F32, 1e-6), (lqcd.PREC_F16, 5e-3),
                                      (lqcd.PREC_BF16, 2e-2)])
def test_dslash_eo(setup, prec, tol):
    lat, olat, U, kappa, seed = setup
    for parity in (0, 1):
        for dagger in (0, 1):
            x = syn.gaussian_spinor(olat.Vh, seed + 10 * parity + dagger)
            ref = olat.dslash_eo(U, x, parity, dagger)
            out = lat.dslash_eo(cuda(x), parity, 0.0, dagger, lqcd.OP_HOP, prec)
            assert rel(out, ref) < tol, (parity, dagger, rel(out, ref))
    x = syn.gaussian_spinor(olat.Vh, seed + 7)
    for dagger in (0, 1):
        ref = olat.mhat(U, kappa, x, dagger)
        out = lat.dslash_eo(cuda(x), 0, kappa, dagger, lqcd.OP_MHAT, prec)
        assert rel(out, ref) < tol


@pytest.mark.parametrize("prec,tol", [(lqcd.PREC_F64, 1e-13), (lqcd.PREC_F32, 1e-6), (lqcd.PREC_F16, 5e-3),
                                      (lqcd.PREC_BF16, 2e-2)])
def test_block_dslash(setup, prec, tol):
    lat, olat, U, kappa, seed = setup
    x = syn.gaussian_spinor(olat.V, seed + 3)
    for colour in (-1, 0, 1):
        for dagger in (0, 1):
            ref = olat.block_dslash(U, kappa, x, colour, dagger)
            out = lat.block_dslash(cuda(x), kappa, colour, dagger, prec)
            assert rel(out, ref) < tol, (colour, dagger, rel(out, ref))


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16])
def test_block_solve_batched(setup, prec):
    lat, olat, U, kappa, seed = setup
    b = syn.gaussian_spinor(olat.V, seed + 4)
    m = olat.index_maps()
    for colour in (-1, 0, 1):
        for dagger in (0, 1):
            x, it, rs = lat.block_solve(cuda(b), kappa, colour, dagger, prec, tol=1e-10)
            x = x.cpu().numpy()
            bb = b.copy()
            if colour >= 0:
                bb[m[3] != colour] = 0
                assert np.all(x[m[3] != colour] == 0)
            r = bb - olat.W1(U, kappa, x, dagger)
            for k in range(olat.nb):
                if colour >= 0 and k % 2 != colour:
                    continue
                sel = m[2] == k
                assert np.linalg.norm(r[sel]) <= 1.5e-10 * np.linalg.norm(bb[sel]), (k, it, rs)
            ref = olat.block_solve(U, kappa, bb, colour, dagger, tol=1e-13)
            assert rel(x, ref) < 1e-8


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16])
def test_solve_wilson(setup, prec):
    lat, olat, U, kappa, seed = setup
    for k in range(3):
        b = syn.gaussian_spinor(olat.V, seed + 40 + k)
        for dagger in (0, 1):
            x, it, rs = lat.solve(cuda(b), kappa, dagger, prec, tol=1e-10)
            x = x.cpu().numpy()
            r = b - olat.M(U, kappa, x, dagger)
            assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b), (it, rs)


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16])
def test_zero_source_solves(setup, prec):
    """the degenerate system b = 0: every slab system and the global solve
    return x = 0 exactly, without an inner iteration"""
    lat, olat, U, kappa, seed = setup
    z = torch.zeros((olat.V, 4, 3), dtype=torch.complex128, device="cuda")
    x, it, rs = lat.block_solve(z, kappa, -1, 0, prec, tol=1e-10)
    assert x.abs().max().item() == 0.0 and max(it[:olat.nb]) == 0
    x, it, rs = lat.solve(z, kappa, 1, prec, tol=1e-10)
    assert x.abs().max().item() == 0.0 and it == 0


@pytest.mark.parametrize("op", [lqcd.SCHUR_R, lqcd.SCHUR_RDAG, lqcd.SCHUR_RINV, lqcd.SCHUR_RINVDAG])
def test_schur(setup, op):
    lat, olat, U, kappa, seed = setup
    c = syn.gaussian_complex(olat.bnd_shape(), seed + 5)
    ref = olat.schur(U, kappa, c, op, route=1, tol=1e-13)
    out = lat.schur(cuda(c), kappa, op, lqcd.PREC_F32, tol=1e-12)
    assert rel(out, ref) < 1e-9


def test_gauge_force_and_action(setup):
    lat, olat, U, kappa, seed = setup
    S, pl, F = lat.gauge_force(5.6)
    assert abs(S - olat.gauge_action(U, 5.6)) < 1e-10 * abs(S)
    assert abs(pl - olat.plaquette(U)) < 1e-13
    assert rel(F, olat.gauge_force(U, 5.6)) < 1e-12


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16])
def test_pf_force_w1(setup, prec):
    lat, olat, U, kappa, seed = setup
    phi = syn.gaussian_spinor(olat.V, seed + 6)
    S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_W1, prec, tol=1e-12)
    So, Fo = olat.pf_w1(U, kappa, phi, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    # double link arithmetic for the double form; the mixed forms evaluate the
    # force in single precision (unit roundoff 6e-8 over ~30-term sums),
    # within the 1e-5 force tolerance
    assert rel(F, Fo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-5)


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32])
def test_pf_force_schur(setup, prec):
    lat, olat, U, kappa, seed = setup
    phi = syn.gaussian_complex(olat.bnd_shape(), seed + 8)
    S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_SCHUR, prec, tol=1e-12)
    So, Fo = olat.pf_schur(U, kappa, phi, route=1, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    # double link arithmetic for the double form; the mixed forms evaluate the
    # force in single precision (unit roundoff 6e-8 over ~30-term sums),
    # within the 1e-5 force tolerance
    assert rel(F, Fo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-5)


def test_rng_normals_match_oracle(setup):
    lat, olat, U, kappa, seed = setup
    n = 10001
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    lqcd.lqcd_rng_normals(lat.h, out, 2007, 2, 5)
    ref = O.normals(2007, 2, 5, n)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-13


def test_md_matches_oracle():
    L, l0, kappa, beta = (4, 4, 4, 4), 2, 0.15, 5.6
    U = syn.random_links(L, 0.3, 11)
    olat = O.Lattice(L, l0, -1)
    P = syn.gaussian_momenta(olat.V, 12)
    phi1 = syn.gaussian_spinor(olat.V, 13)
    phi2 = syn.gaussian_complex(olat.bnd_shape(), 14)
    lat = lqcd.Lattice(L, l0, -1)
    for sch, nl, ns, lv in [((O.LF,), 1, [4], (0, 0, 0)), ((O.SW, O.SW, O.LF), 3, [2, 2, 2], (0, 1, 2))]:
        prm = lqcd.hmc_params(beta, kappa, 0.4, nl, sch, ns, *lv, tol=1e-12)
        oprm = O.hmc_params(beta, kappa, 0.4, nl, sch, ns, *lv, tol=1e-13)
        U1, P1 = lat.md(cuda(U), cuda(P), cuda(phi1), cuda(phi2), prm)
        Uo, Po, st = O.md(olat, U, P, phi1, phi2, oprm)
        assert st == 0
        assert rel(U1, Uo) < 1e-9
        assert rel(P1, Po) < 1e-8
    lat.close()


@pytest.mark.parametrize("pf_init", [0, 1])
def test_hmc_trajectory_matches_oracle(pf_init):
    """The small 4^4 workload: two slabs of thickness 2, kappa = 0.15,
    beta = 5.6, one leapfrog trajectory tau = 0.5 in 10 steps"""
    L, l0, kappa, beta = (4, 4, 4, 4), 2, 0.15, 5.6
    U = syn.random_links(L, 0.3, 2007)
    lat = lqcd.Lattice(L, l0, -1)
    olat = O.Lattice(L, l0, -1)
    prm = lqcd.hmc_params(beta, kappa, 0.5, 1, (lqcd.LF,), [10], 0, 0, 0, pf_init=pf_init, roll=1, tol=1e-12)
    oprm = O.hmc_params(beta, kappa, 0.5, 1, (O.LF,), [10], 0, 0, 0, pf_init=pf_init, roll=1, tol=1e-13)
    U1, res = lat.hmc_trajectory(cuda(U), prm, 2007, 3)
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2007, 3)
    assert st == 0
    assert abs(res.dH - ores.dH) < 1e-4
    assert abs(res.dH - ores.dH) < 1e-7
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < 1e-9
    lat.close()


def test_hmc_trajectory_block_series_matches_oracle():
    """the W1 solves by the geometric series (Sec. 3): kappa = 0.12 on a
    smooth field keeps the series convergent"""
    L, l0, kappa, beta = (8, 4, 4, 4), 2, 0.12, 5.6
    U = syn.random_links(L, 0.3, 2013)
    lat = lqcd.Lattice(L, l0, -1)
    olat = O.Lattice(L, l0, -1)
    prm = lqcd.hmc_params(beta, kappa, 0.5, 2, (lqcd.SW, lqcd.LF), [2, 4], 0, 0, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-11, block_solver=lqcd.SOLVER_SERIES)
    oprm = O.hmc_params(beta, kappa, 0.5, 2, (O.SW, O.LF), [2, 4], 0, 0, 1, roll=1, tol=1e-13)
    U1, res = lat.hmc_trajectory(cuda(U), prm, 2013, 1)
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2013, 1)
    assert st == 0
    assert abs(res.dH - ores.dH) < 1e-4
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < 1e-6
    lat.close()


@pytest.mark.parametrize("scheme,L,l0,kappa", [(2, (8, 4, 4, 4), 2, 0.15), (1, (12, 4, 4, 4), 2, 0.12)])
def test_md_step_scheme_matches_oracle(scheme, L, l0, kappa):
    """position-dependent step sizes (Sec. 2): per-link dt * s(x0); links
    with s = 0 stay frozen (kappa = 0.12 at 12x4^3: at 0.15 this random field
    makes M itself nearly singular)"""
    beta = 5.6
    U = syn.random_links(L, 0.3, 21)
    olat = O.Lattice(L, l0, -1)
    P = syn.gaussian_momenta(olat.V, 22)
    eta1 = syn.gaussian_spinor(olat.V, 23)
    eta2 = syn.gaussian_complex(olat.bnd_shape(), 24)
    phi1 = olat.W1(U, kappa, eta1)
    phi2 = olat.schur(U, kappa, eta2, O.R, tol=1e-14)
    s = O.step_scheme(scheme, L[0])
    lat = lqcd.Lattice(L, l0, -1)
    prm = lqcd.hmc_params(beta, kappa, 0.4, 2, (lqcd.SW, lqcd.LF), [2, 2], 0, 1, 1, tol=1e-12, step_scheme=scheme)
    oprm = O.hmc_params(beta, kappa, 0.4, 2, (O.SW, O.LF), [2, 2], 0, 1, 1, tol=1e-13, step_scale=s)
    U1, P1 = lat.md(cuda(U), cuda(P), cuda(phi1), cuda(phi2), prm)
    Uo, Po, st = O.md(olat, U, P, phi1, phi2, oprm)
    assert st == 0
    assert rel(U1, Uo) < 1e-9 and rel(P1, Po) < 1e-8
    # the same through an explicit table
    prm2 = lqcd.hmc_params(beta, kappa, 0.4, 2, (lqcd.SW, lqcd.LF), [2, 2], 0, 1, 1, tol=1e-12, step_scale=s)
    U2, P2 = lat.md(cuda(U), cuda(P), cuda(phi1), cuda(phi2), prm2)
    assert torch.equal(U1, U2) and torch.equal(P1, P2)
    m = olat.index_maps()
    x0 = m[0] // (L[1] * L[2] * L[3])
    U1n = U1.cpu().numpy()
    for mu in range(4):
        frozen = s[1 if mu == 0 else 0][x0] == 0
        assert np.array_equal(U1n[mu, frozen], U[mu, frozen])
    lat.close()


def test_force_profile_matches_oracle(setup):
    lat, olat, U, kappa, seed = setup
    phi = syn.gaussian_complex(olat.bnd_shape(), seed + 9)
    S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_SCHUR, lqcd.PREC_F64, tol=1e-12)
    prof = lat.force_profile(F).cpu().numpy()
    ref = olat.force_profile(F.cpu().numpy())
    assert rel(prof, ref) < 1e-13
