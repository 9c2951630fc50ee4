"""Even-odd + mass preconditioning of W2 (Sec. 1, W3,eo = W2,eo + rho) and
the paper's four-part action on five integration levels, on the GPU
through the C-ABI against the FP64 oracle.

Tolerances as for the other terms: double operators 1e-13, solves to
|b - W3,eo x| <= 1e-10 |b| checked with the oracle's operator, forces 1e-9
(double) / 1e-5 (mixed), trajectory dH 1e-4.
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

GEOMS = [((8, 4, 4, 4), 4, 0.3, 0.15), ((16, 8, 8, 8), 4, 0.6, 0.156), ((16, 4, 4, 6), 8, 0.3, 0.13)]
RHO = 0.2


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", params=GEOMS, ids=lambda p: "x".join(map(str, p[0])) + "_l0%d" % p[1])
def setup(request):
    L, l0, eps, kappa = request.param
    seed = 4001 + sum(L)
    U = syn.random_links(L, eps, seed)
    lat = lqcd.Lattice(L, l0, -1, l0s=l0 // 2)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1, l0s=l0 // 2)
    yield lat, olat, U, kappa, seed
    lat.close()


@pytest.mark.parametrize("rho", [0.0, RHO])
def test_w3eo_apply(setup, rho):
    lat, olat, U, kappa, seed = setup
    x = syn.gaussian_spinor(olat.Vh, seed + 1)
    for dagger in (0, 1):
        ref = olat.w3eo(U, kappa, rho, x, dagger)
        assert rel(lat.w3eo(cuda(x), kappa, rho, dagger), ref) < 1e-13


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16])
def test_w3eo_solve(setup, prec):
    lat, olat, U, kappa, seed = setup
    b = syn.gaussian_spinor(olat.Vh, seed + 2)
    sub = ((olat.index_maps()[0] // olat.V3) // olat.l0s)[:olat.Vh]
    for rho in (0.0, RHO):
        for dagger in (0, 1):
            x, it = lat.solve_w3eo(cuda(b), kappa, rho, dagger, prec, tol=1e-10)
            x = x.cpu().numpy()
            r = b - olat.w3eo(U, kappa, rho, x, dagger)
            for k in range(olat.nbs):
                sel = sub == k
                assert np.linalg.norm(r[sel]) <= 1.5e-10 * np.linalg.norm(b[sel]), (k, it[:olat.nbs])
                assert it[k] > 0
            ref = olat.solve_w3eo(U, kappa, rho, b, dagger, tol=1e-13)
            assert rel(x, ref) < 1e-8


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16])
def test_w3eo_geometric_series(setup, prec):
    """the geometric series (Sec. 3) at kappa = 0.1, where the spectral
    radius of kappa^2 H_eo H_oe / (1 + rho) is well below one"""
    lat, olat, U, kappa, seed = setup
    kappa = 0.1
    b = syn.gaussian_spinor(olat.Vh, seed + 12)
    for dagger in (0, 1):
        x, it = lat.solve_w3eo(cuda(b), kappa, RHO, dagger, prec, tol=1e-10, method=lqcd.SOLVER_SERIES)
        x = x.cpu().numpy()
        r = b - olat.w3eo(U, kappa, RHO, x, dagger)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b), it[:olat.nbs]
        xb, itb = lat.solve_w3eo(cuda(b), kappa, RHO, dagger, prec, tol=1e-10)
        assert rel(x, xb.cpu().numpy()) < 1e-8
        assert min(it[:olat.nbs]) > 0


def test_w3eo_geometric_series_diverges_cleanly():
    """kappa = 0.2 on a smooth field: the series grows, the solve returns
    LQCD_ERR_NOCONVERGE and the handle stays usable"""
    L = (8, 4, 4, 4)
    U = syn.random_links(L, 0.1, 7)
    lat = lqcd.Lattice(L, 4, -1, l0s=2)
    lat.set_gauge(cuda(U))
    b = cuda(syn.gaussian_spinor(lat.Vh, 8))
    with pytest.raises(lqcd.LqcdError) as e:
        lat.solve_w3eo(b, 0.2, 0.0, 0, lqcd.PREC_F32, tol=1e-10, method=lqcd.SOLVER_SERIES)
    assert e.value.status == lqcd.ERR_NOCONVERGE
    x, it = lat.solve_w3eo(b, 0.1, 0.0, 0, lqcd.PREC_F32, tol=1e-10)
    assert torch.isfinite(x).all()
    lat.close()


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32])
@pytest.mark.parametrize("term", ["s2", "s1"])
def test_pf_force_massprec(setup, prec, term):
    lat, olat, U, kappa, seed = setup
    phi = syn.gaussian_spinor(olat.Vh, seed + 3)
    t = lqcd.TERM_S2 if term == "s2" else lqcd.TERM_S1
    S, F = lat.pf_force_eo(cuda(phi), kappa, RHO, t, prec, tol=1e-12)
    So, Fo = (olat.pf_s2 if term == "s2" else olat.pf_s1)(U, kappa, RHO, phi, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    assert rel(F, Fo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-5)


def _levels5():
    """Sec. 2 layout: S_G level 0, S1 level 1, S2 level 2, S3 (R2) level 3,
    S4 (R) level 4"""
    return dict(level_gauge=0, level_w1=-1, level_schur=4, level_w2=-1, level_schur2=3, rho=RHO,
                level_s2=2, level_s1=1)


SCHEME5 = (lqcd.SW, lqcd.SW, lqcd.LF, lqcd.LF, lqcd.LF)


def test_md_five_levels_matches_oracle():
    L, l0, kappa, beta = (8, 4, 4, 4), 4, 0.15, 5.6
    U = syn.random_links(L, 0.3, 41)
    olat = O.Lattice(L, l0, -1, l0s=2)
    P = syn.gaussian_momenta(olat.V, 42)
    phi2 = syn.gaussian_complex(olat.bnd_shape(), 43)
    phi4 = syn.gaussian_complex(olat.bnd2_shape(), 44)
    ps2 = syn.gaussian_spinor(olat.Vh, 45)
    ps1 = syn.gaussian_spinor(olat.Vh, 46)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    prm = lqcd.hmc_params(beta, kappa, 0.2, 5, SCHEME5, [2, 2, 1, 1, 1], tol=1e-12, **_levels5())
    oprm = O.hmc_params(beta, kappa, 0.2, 5, SCHEME5, [2, 2, 1, 1, 1], tol=1e-13, **_levels5())
    U1, P1 = lat.md(cuda(U), cuda(P), None, cuda(phi2), prm, None, cuda(phi4), cuda(ps2), cuda(ps1))
    Uo, Po, st = O.md(olat, U, P, None, phi2, oprm, None, phi4, ps2, ps1)
    assert st == 0
    assert rel(U1, Uo) < 1e-9
    assert rel(P1, Po) < 1e-8
    lat.close()


@pytest.mark.parametrize("prec,method", [(lqcd.PREC_F64, lqcd.SOLVER_BICGSTAB), (lqcd.PREC_F32, lqcd.SOLVER_BICGSTAB),
                                         (lqcd.PREC_F32, lqcd.SOLVER_SERIES)])
def test_hmc_trajectory_five_levels_matches_oracle(prec, method):
    """kappa = 0.12 keeps the smooth field at positive quark mass (and the
    geometric series of W3,eo convergent)"""
    L, l0, kappa, beta = (8, 4, 4, 4), 4, 0.12, 5.6
    U = syn.random_links(L, 0.3, 51)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    olat = O.Lattice(L, l0, -1, l0s=2)
    ns = [2, 2, 1, 1, 3]
    prm = lqcd.hmc_params(beta, kappa, 0.4, 5, SCHEME5, ns, roll=1, precision=prec, tol=1e-11, eo_solver=method,
                          **_levels5())
    oprm = O.hmc_params(beta, kappa, 0.4, 5, SCHEME5, ns, roll=1, tol=1e-13, **_levels5())
    U1, res = lat.hmc_trajectory(cuda(U), prm, 2011, 6)
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2011, 6)
    assert st == 0
    assert abs(res.H0 - ores.H0) < 1e-9 * abs(ores.H0)
    assert abs(res.dH - ores.dH) < 1e-4
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-6)
    lat.close()
