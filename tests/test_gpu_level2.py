"""Iterated decomposition (Sec. 1, second level: sub-slabs of thickness
l0/2) on the GPU through the C-ABI against the FP64 oracle.

The same tolerances as the first level: double kernels 1e-12, single 1e-6,
half storage 5e-3; solves to |b - W2 x| <= 1e-10 |b| per sub-slab checked
with the oracle's W2; forces 1e-9 (double) / 1e-5 (mixed); dH 1e-4.
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

# (L, l0, eps, kappa): 8x4^3 with two slabs of four slices (four sub-slabs),
# 16x8^3 with four slabs of four (eight sub-slabs), 16x4x4x6 with l0 = 8
GEOMS = [((8, 4, 4, 4), 4, 0.3, 0.15), ((16, 8, 8, 8), 4, 0.6, 0.156), ((16, 4, 4, 6), 8, 0.3, 0.13)]


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", params=GEOMS, ids=lambda p: "x".join(map(str, p[0])) + "_l0%d" % p[1])
def setup(request):
    L, l0, eps, kappa = request.param
    seed = 3001 + sum(L)
    U = syn.random_links(L, eps, seed)
    lat = lqcd.Lattice(L, l0, -1, l0s=l0 // 2)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1, l0s=l0 // 2)
    sub = (olat.index_maps()[0] // olat.V3) // olat.l0s
    yield lat, olat, U, kappa, seed, sub
    lat.close()


@pytest.mark.parametrize("prec,tol", [(lqcd.PREC_F64, 1e-13), (lqcd.PREC_F32, 1e-6), (lqcd.PREC_F16, 5e-3)])
def test_subblock_dslash(setup, prec, tol):
    lat, olat, U, kappa, seed, sub = setup
    x = syn.gaussian_spinor(olat.V, seed + 3)
    for colour in (-1, 0, 1):
        for dagger in (0, 1):
            ref = olat.W2(U, kappa, x, dagger)
            if colour >= 0:
                ref[sub % 2 != colour] = 0
            out = lat.subblock_dslash(cuda(x), kappa, colour, dagger, prec)
            assert rel(out, ref) < tol, (colour, dagger, rel(out, ref))


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16])
def test_subblock_solve_batched(setup, prec):
    lat, olat, U, kappa, seed, sub = setup
    b = syn.gaussian_spinor(olat.V, seed + 4)
    for colour in (-1, 0, 1):
        for dagger in (0, 1):
            x, it, rs = lat.subblock_solve(cuda(b), kappa, colour, dagger, prec, tol=1e-10)
            x = x.cpu().numpy()
            bb = b.copy()
            if colour >= 0:
                bb[sub % 2 != colour] = 0
                assert np.all(x[sub % 2 != colour] == 0)
            r = bb - olat.W2(U, kappa, x, dagger)
            for k in range(olat.nbs):
                if colour >= 0 and k % 2 != colour:
                    assert it[k] == 0
                    continue
                sel = sub == k
                assert np.linalg.norm(r[sel]) <= 1.5e-10 * np.linalg.norm(bb[sel]), (k, it, rs)
                assert it[k] > 0
            ref = olat.block_solve2(U, kappa, bb, colour, dagger, tol=1e-13)
            assert rel(x, ref) < 1e-8


@pytest.mark.parametrize("op", [lqcd.SCHUR2_R, lqcd.SCHUR2_RDAG, lqcd.SCHUR2_RINV, lqcd.SCHUR2_RINVDAG])
def test_schur2(setup, op):
    lat, olat, U, kappa, seed, sub = setup
    c = syn.gaussian_complex(olat.bnd2_shape(), seed + 5)
    ref = olat.schur2(U, kappa, c, op - lqcd.SCHUR2_R, route=1, tol=1e-13)
    out = lat.schur(cuda(c), kappa, op, lqcd.PREC_F32, tol=1e-12)
    assert out.shape == ref.shape
    assert rel(out, ref) < 1e-9


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32])
def test_pf_force_w2(setup, prec):
    lat, olat, U, kappa, seed, sub = setup
    phi = syn.gaussian_spinor(olat.V, seed + 6)
    S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_W2, prec, tol=1e-12)
    So, Fo = olat.pf_w2(U, kappa, phi, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    assert rel(F, Fo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-5)


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32])
def test_pf_force_schur2(setup, prec):
    lat, olat, U, kappa, seed, sub = setup
    phi = syn.gaussian_complex(olat.bnd2_shape(), seed + 8)
    S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_SCHUR2, prec, tol=1e-12)
    So, Fo = olat.pf_schur2(U, kappa, phi, route=1, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    assert rel(F, Fo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-5)


def _levels4():
    """S_G and |W2^-1 phi3|^2 on the fine level 0, |R^-1 phi2|^2 and
    |R2^-1 phi4|^2 on level 1"""
    return dict(level_gauge=0, level_w1=-1, level_schur=1, level_w2=0, level_schur2=1)


def test_md_four_part_action_matches_oracle():
    L, l0, kappa, beta = (8, 4, 4, 4), 4, 0.15, 5.6
    U = syn.random_links(L, 0.3, 21)
    olat = O.Lattice(L, l0, -1, l0s=2)
    P = syn.gaussian_momenta(olat.V, 22)
    phi2 = syn.gaussian_complex(olat.bnd_shape(), 23)
    phi3 = syn.gaussian_spinor(olat.V, 24)
    phi4 = syn.gaussian_complex(olat.bnd2_shape(), 25)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    for sch in ((lqcd.SW, lqcd.SW),):
        prm = lqcd.hmc_params(beta, kappa, 0.3, 2, sch, [2, 2], tol=1e-12, **_levels4())
        oprm = O.hmc_params(beta, kappa, 0.3, 2, sch, [2, 2], tol=1e-13, **_levels4())
        U1, P1 = lat.md(cuda(U), cuda(P), None, cuda(phi2), prm, cuda(phi3), cuda(phi4))
        Uo, Po, st = O.md(olat, U, P, None, phi2, oprm, phi3, phi4)
        assert st == 0
        assert rel(U1, Uo) < 1e-9
        assert rel(P1, Po) < 1e-8
    lat.close()


@pytest.mark.parametrize("prec", [lqcd.PREC_F64, lqcd.PREC_F32])
def test_hmc_trajectory_four_part_action_matches_oracle(prec):
    """kappa = 0.12 keeps the smooth (eps = 0.3) field at positive quark mass;
    at 0.15 the thin sub-slabs carry near-zero surface modes of W2 and the
    trajectory runs away (both sides alike)"""
    L, l0, kappa, beta = (8, 4, 4, 4), 4, 0.12, 5.6
    U = syn.random_links(L, 0.3, 31)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    olat = O.Lattice(L, l0, -1, l0s=2)
    prm = lqcd.hmc_params(beta, kappa, 0.4, 2, (lqcd.LF, lqcd.LF), [4, 4], roll=1, precision=prec, tol=1e-11,
                          **_levels4())
    oprm = O.hmc_params(beta, kappa, 0.4, 2, (O.LF, O.LF), [4, 4], roll=1, tol=1e-13, **_levels4())
    U1, res = lat.hmc_trajectory(cuda(U), prm, 2009, 4)
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2009, 4)
    assert st == 0
    assert abs(res.H0 - ores.H0) < 1e-9 * abs(ores.H0)
    assert abs(res.dH - ores.dH) < 1e-4
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < (1e-9 if prec == lqcd.PREC_F64 else 1e-6)
    lat.close()


def test_subslab_errors():
    lat = lqcd.Lattice((8, 4, 4, 4), 4, -1)
    one = torch.zeros((4, lat.V, 3, 3), dtype=torch.complex128, device="cuda")
    one[..., 0, 0] = one[..., 1, 1] = one[..., 2, 2] = 1
    lat.set_gauge(one)
    x = lat.spinor()
    with pytest.raises(lqcd.LqcdError) as e:
        lat.subblock_dslash(x, 0.1)
    assert e.value.status == lqcd.ERR_STATE
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_set_subslabs(lat.h, 1)
    assert e.value.status == lqcd.ERR_GEOM
    lat.close()
    lat = lqcd.Lattice((8, 4, 4, 4), 2, -1)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.hmc_trajectory(torch.zeros((4, lat.V, 3, 3), dtype=torch.complex128, device="cuda"),
                           lqcd.hmc_params(5.6, 0.1, 1.0, 1, (lqcd.LF,), [1], level_w2=0), 1, 0)
    assert e.value.status == lqcd.ERR_STATE
    lat.close()
