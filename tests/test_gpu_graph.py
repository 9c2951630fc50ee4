"""The molecular dynamics recorded as a CUDA graph and replayed
(lqcd_hmc_params.use_graph): the same kernels in the same order, so the
trajectories equal the eager ones bit for bit; a parameter change records
a new graph; a solve that fails inside the graph is reported after the
replay and leaves the handle usable.  kappa = 0.14 keeps the unthermalised
field (which the gauge force smooths) at positive quark mass."""
import numpy as np
import pytest

from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402

L, L0S = (16, 8, 8, 8), 4


def _prm(graph, **kw):
    kw.setdefault("nsteps", (2, 2, 3))
    ns = kw.pop("nsteps")
    return lqcd.hmc_params(5.6, 0.14, 0.5, 3, (lqcd.SW, lqcd.SW, lqcd.LF), ns, 0, 1, 2, roll=1,
                           precision=lqcd.PREC_F32, tol=1e-10, use_graph=graph, **kw)


def test_graph_trajectories_equal_eager():
    U0 = torch.from_numpy(syn.random_links(L, 0.6, 17)).cuda()
    lat_e = lqcd.Lattice(L, L0S, -1)
    lat_g = lqcd.Lattice(L, L0S, -1)
    Ue, Ug = U0.clone(), U0.clone()
    for t in range(3):
        Ue, re = lat_e.hmc_trajectory(Ue, _prm(0), 99, t)
        n0 = lqcd.lqcd_launch_count(lat_g.h)
        Ug, rg = lat_g.hmc_trajectory(Ug, _prm(1), 99, t)
        assert torch.equal(Ue, Ug), t
        assert re.dH == rg.dH and re.accepted == rg.accepted and re.shift == rg.shift
        assert re.n_force == rg.n_force and re.n_solves == rg.n_solves
        assert re.solver_iters == rg.solver_iters
        assert lqcd.lqcd_launch_count(lat_g.h) - n0 > 100
    # another schedule records another graph
    Ue, re = lat_e.hmc_trajectory(Ue, _prm(0, nsteps=(2, 2, 2)), 99, 7)
    Ug, rg = lat_g.hmc_trajectory(Ug, _prm(1, nsteps=(2, 2, 2)), 99, 7)
    assert torch.equal(Ue, Ug) and re.dH == rg.dH
    lat_e.close()
    lat_g.close()


def test_graph_kernel_times():
    """kernel timing inside the replayed graph: the same solver launches and
    algorithmic bytes as the eager trajectory, times of the same order"""
    U0 = torch.from_numpy(syn.random_links(L, 0.6, 19)).cuda()
    out = {}
    for graph in (0, 1):
        lat = lqcd.Lattice(L, L0S, -1)
        lqcd.lqcd_profile_enable(lat.h, 1 << lqcd.KERNEL_SOLVER)
        lat.hmc_trajectory(U0, _prm(graph), 3, 0)  # records the graph
        lqcd.lqcd_profile_reset(lat.h)
        lat.hmc_trajectory(U0, _prm(graph), 3, 0)
        out[graph] = lqcd.lqcd_profile_read(lat.h, lqcd.KERNEL_SOLVER)
        assert len(lqcd.lqcd_profile_times(lat.h, lqcd.KERNEL_SOLVER)) == out[graph][0]
        lat.close()
    (n0, ms0, b0), (n1, ms1, b1) = out[0], out[1]
    assert n0 == n1 > 10
    assert abs(b1 - b0) < 0.02 * b0
    assert 0.5 * ms0 < ms1 < 1.5 * ms0


def test_graph_reports_a_failed_solve():
    U0 = torch.from_numpy(syn.random_links(L, 0.6, 18)).cuda()
    lat = lqcd.Lattice(L, L0S, -1)
    # W1 term only: its heatbath needs no solve, so the first failing solve
    # is inside the recorded molecular dynamics
    bad = lqcd.hmc_params(5.6, 0.14, 0.5, 2, (lqcd.SW, lqcd.LF), (2, 2), 0, 1, -1, precision=lqcd.PREC_F32,
                          tol=1e-10, max_iter=3, use_graph=1)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.hmc_trajectory(U0, bad, 5, 0)
    assert e.value.status == lqcd.ERR_NOCONVERGE
    U1, res = lat.hmc_trajectory(U0, _prm(1), 5, 0)
    assert np.isfinite(res.dH)
    lat.close()
