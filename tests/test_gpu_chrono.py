"""Chronological initial guesses of the molecular-dynamics force solves
(lqcd_hmc_params.chrono): each solve starts from the linear (chrono = 1)
or quadratic (chrono = 2) extrapolation in MD time of its solutions at the
two or three previous force evaluations of its term, or (chrono = 3, the
whole-lattice solves of the boundary term) from the combination of its last
six solutions with the smallest residual (Brower et al.'s chronological
inverter).  The solves still run
to the requested residual, so trajectories agree with the FP64 oracle (which
always starts from zero) to the tolerances of the other trajectory tests;
a solve whose guess already meets the residual takes no iteration; the
CUDA graph replays the eager run bit for bit.
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

SW, LF = lqcd.SW, lqcd.LF
SCHEME5 = (SW, SW, LF, LF, LF)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _four_part():
    """Sec. 2 layout of the four-part action: S_G 0, S1 1, S2 2, R2 3, R 4"""
    return dict(level_gauge=0, level_w1=-1, level_schur=4, level_w2=-1, level_schur2=3, rho=0.2, level_s2=2,
                level_s1=1)


def _two_part():
    """Sec. 1 action: S_G 0, W1 1, R 2"""
    return dict(level_gauge=0, level_w1=1, level_schur=2)


CASES = {
    "two_part": (3, (SW, SW, LF), _two_part, [2, 2, 3]),
    "four_part": (5, SCHEME5, _four_part, [2, 2, 1, 1, 3]),
}


def _prm(case, tau, top, chrono, graph=0, prec=lqcd.PREC_F32, method=lqcd.SOLVER_BICGSTAB, mod=lqcd):
    nl, scheme, lv, ns = CASES[case]
    ns = list(ns)
    ns[-1] = top
    kw = dict(roll=1, tol=1e-11 if mod is lqcd else 1e-13, **lv())
    if mod is lqcd:
        kw.update(precision=prec, eo_solver=method, block_solver=method, chrono=chrono, use_graph=graph)
    return mod.hmc_params(5.6, 0.12, tau, nl, scheme, ns, **kw)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("order", [1, 3])
def test_repeated_solves_take_no_iterations(case, order):
    """tau = 1e-14: every force evaluation of a term solves the same systems
    up to 1e-14, so with chrono = 1 only the first evaluation of each term
    iterates and more integration steps cost (almost) no more iterations;
    without it every evaluation iterates"""
    L, l0 = (8, 4, 4, 4), 4
    U = cuda(syn.random_links(L, 0.3, 61))
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    it = {}
    for chrono in (0, order):
        for top in (1, 3):
            _, r = lat.hmc_trajectory(U, _prm(case, 1e-14, top, chrono), 7, 0)
            assert abs(r.dH) < 1e-8
            it[min(chrono, 1), top] = (r.solver_iters, r.n_force)
    assert it[0, 3][1] == it[1, 3][1] > it[0, 1][1] == it[1, 1][1]
    extra_plain = it[0, 3][0] - it[0, 1][0]
    extra_chrono = it[1, 3][0] - it[1, 1][0]
    assert extra_plain > 0
    # a guess whose residual sits just above the tolerance after the 1e-14
    # move still pays a short solve: allow a little
    assert extra_chrono <= 0.1 * extra_plain, (it, extra_chrono, extra_plain)
    assert it[1, 1][0] < it[0, 1][0]
    lat.close()


@pytest.mark.parametrize("case,method,chrono", [("two_part", lqcd.SOLVER_BICGSTAB, 1),
                                                ("four_part", lqcd.SOLVER_BICGSTAB, 1),
                                                ("four_part", lqcd.SOLVER_SERIES, 1),
                                                ("two_part", lqcd.SOLVER_BICGSTAB, 2),
                                                ("four_part", lqcd.SOLVER_SERIES, 2),
                                                ("two_part", lqcd.SOLVER_BICGSTAB, 3),
                                                ("four_part", lqcd.SOLVER_SERIES, 3)])
def test_chrono_trajectory_matches_oracle(case, method, chrono):
    """the mixed-precision trajectory with chronological guesses against
    the oracle's, which solves every system from zero"""
    L, l0 = (8, 4, 4, 4), 4
    Un = syn.random_links(L, 0.3, 51)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    olat = O.Lattice(L, l0, -1, l0s=2)
    U1, res = lat.hmc_trajectory(cuda(Un), _prm(case, 0.4, 3, chrono, method=method), 2011, 6)
    U0, res0 = lat.hmc_trajectory(cuda(Un), _prm(case, 0.4, 3, 0, method=method), 2011, 6)
    Uo, ores, st = olat.hmc_trajectory(Un, _prm(case, 0.4, 3, 0, mod=O), 2011, 6)
    assert st == 0
    assert abs(res.H0 - ores.H0) < 1e-9 * abs(ores.H0)
    assert abs(res.dH - ores.dH) < 1e-4
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < 1e-6
    assert res.n_force == res0.n_force and res.n_solves == res0.n_solves
    assert res.solver_iters < res0.solver_iters
    lat.close()


@pytest.mark.parametrize("chrono", [1, 2, 3])
def test_chrono_graph_equals_eager(chrono):
    L, l0 = (16, 8, 8, 8), 4
    U0 = cuda(syn.random_links(L, 0.6, 17))
    lat_e = lqcd.Lattice(L, l0, -1, l0s=2)
    lat_g = lqcd.Lattice(L, l0, -1, l0s=2)
    Ue, Ug = U0.clone(), U0.clone()
    for t in range(3):
        Ue, re = lat_e.hmc_trajectory(Ue, _prm("four_part", 0.5, 2, chrono, graph=0), 99, t)
        Ug, rg = lat_g.hmc_trajectory(Ug, _prm("four_part", 0.5, 2, chrono, graph=1), 99, t)
        assert torch.equal(Ue, Ug), t
        assert re.dH == rg.dH and re.accepted == rg.accepted
        assert re.solver_iters == rg.solver_iters
    lat_e.close()
    lat_g.close()


@pytest.mark.parametrize("chrono", [1, 2, 3])
def test_chrono_md_reversible(chrono):
    """forward then backward with the momenta negated returns to the start
    up to the solver tolerance (the guesses differ between the two legs)"""
    L, l0 = (8, 4, 4, 4), 4
    Un = syn.random_links(L, 0.3, 71)
    olat = O.Lattice(L, l0, -1, l0s=2)
    P = syn.gaussian_momenta(olat.V, 72)
    phi2 = syn.gaussian_complex(olat.bnd_shape(), 73)
    phi4 = syn.gaussian_complex(olat.bnd2_shape(), 74)
    ps2 = syn.gaussian_spinor(olat.Vh, 75)
    ps1 = syn.gaussian_spinor(olat.Vh, 76)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    prm = _prm("four_part", 0.3, 2, chrono)
    fields = (None, cuda(phi2), prm, None, cuda(phi4), cuda(ps2), cuda(ps1))
    U1, P1 = lat.md(cuda(Un), cuda(P), *fields)
    U2, P2 = lat.md(U1, -P1, *fields)
    assert rel(U2, Un) < 1e-8
    assert rel(-P2, P) < 1e-7
    lat.close()
