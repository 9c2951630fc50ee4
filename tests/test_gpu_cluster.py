"""The single-precision geometric series of the slab systems on thread-block
clusters (opt-in, lqcd_set_cluster_series(h, 1): one 16-CTA cluster per
slab, the series' vectors in distributed shared memory, a bounded mbarrier
handshake between the CTAs of a slab) against the FP64 oracle and against
the grid-wide persistent solver (the default).

Checked: the W3,eo / W2,eo solves by the series (Sec. 3) on slab systems of
64 to 8192 sites (chunks of 4 to 512 sites per CTA, and a ragged chunk),
both daggers, to |b - W x| <= 1.5e-10 |b| under the oracle's operator and
to 1e-8 of the grid solver's solution; a trajectory with the W1 solves by
the series matching the oracle and the grid solver; the bounded handshake
giving up under a one-cycle wait limit with LQCD_ERR_TIMEOUT, after which
the handle solves normally.
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

RHO = 0.2


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# (L, l0 with sub-slabs l0 / 2, eps, kappa): sub-slab systems of 64 sites
# (8x4^3), 1024 (16x8^3, chunks of 64), 8192 (32x16^3 with l0 = 8: sub-slabs
# of 4 slices, the bench's slab size), and 12x6^3 with l0 = 6 (324 sites,
# chunks of 21 with a ragged last one)
GEOMS = [((8, 4, 4, 4), 4, 0.3, 0.1), ((16, 8, 8, 8), 4, 0.6, 0.1), ((32, 16, 16, 16), 8, 0.6, 0.1),
         ((12, 6, 6, 6), 6, 0.3, 0.1)]


@pytest.fixture(scope="module", params=GEOMS, ids=lambda p: "x".join(map(str, p[0])) + "_l0%d" % p[1])
def setup(request):
    L, l0, eps, kappa = request.param
    seed = 4501 + sum(L)
    U = syn.random_links(L, eps, seed)
    lat = lqcd.Lattice(L, l0, -1, l0s=l0 // 2)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1, l0s=l0 // 2)
    yield lat, olat, U, kappa, seed
    lat.close()


@pytest.mark.parametrize("rho", [0.0, RHO])
def test_cluster_series_solve(setup, rho):
    lat, olat, U, kappa, seed = setup
    b = syn.gaussian_spinor(olat.Vh, seed + 1)
    sub = ((olat.index_maps()[0] // olat.V3) // olat.l0s)[:olat.Vh]
    for dagger in (0, 1):
        lqcd.lqcd_set_cluster_series(lat.h, 1)
        x, it = lat.solve_w3eo(cuda(b), kappa, rho, dagger, lqcd.PREC_F32, tol=1e-10, method=lqcd.SOLVER_SERIES)
        x = x.cpu().numpy()
        r = b - olat.w3eo(U, kappa, rho, x, dagger)
        for k in range(olat.nbs):
            sel = sub == k
            assert np.linalg.norm(r[sel]) <= 1.5e-10 * np.linalg.norm(b[sel]), (k, it[:olat.nbs])
        assert min(it[:olat.nbs]) > 0
        lqcd.lqcd_set_cluster_series(lat.h, 0)
        xg, itg = lat.solve_w3eo(cuda(b), kappa, rho, dagger, lqcd.PREC_F32, tol=1e-10, method=lqcd.SOLVER_SERIES)
        lqcd.lqcd_set_cluster_series(lat.h, 1)
        assert rel(x, xg.cpu().numpy()) < 1e-8
        # the same iteration (series residual checked every second term)
        assert abs(int(max(it[:olat.nbs])) - int(max(itg[:olat.nbs]))) <= 2


def test_cluster_series_trajectory_matches_oracle_and_grid():
    L, l0, kappa, beta = (8, 4, 4, 4), 2, 0.12, 5.6
    U = syn.random_links(L, 0.3, 2013)
    olat = O.Lattice(L, l0, -1)
    prm = lqcd.hmc_params(beta, kappa, 0.5, 2, (lqcd.SW, lqcd.LF), [2, 4], 0, 0, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-11, block_solver=lqcd.SOLVER_SERIES, use_graph=1, chrono=2)
    oprm = O.hmc_params(beta, kappa, 0.5, 2, (O.SW, O.LF), [2, 4], 0, 0, 1, roll=1, tol=1e-13)
    out = []
    for on in (1, 0):
        lat = lqcd.Lattice(L, l0, -1)
        lqcd.lqcd_set_cluster_series(lat.h, on)
        out.append(lat.hmc_trajectory(cuda(U), prm, 2013, 1))
        lat.close()
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2013, 1)
    assert st == 0
    (U1, r1), (U2, r2) = out
    assert abs(r1.dH - ores.dH) < 1e-4
    assert r1.accepted == ores.accepted and r1.shift == ores.shift
    assert rel(U1, Uo) < 1e-6
    assert abs(r1.dH - r2.dH) < 1e-7
    assert rel(U1, U2.cpu().numpy()) < 1e-8


def test_cluster_wait_limit_times_out_then_handle_recovers():
    L, l0, kappa = (16, 8, 8, 8), 4, 0.1
    U = syn.random_links(L, 0.6, 4600)
    lat = lqcd.Lattice(L, l0, -1, l0s=l0 // 2)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1, l0s=l0 // 2)
    b = syn.gaussian_spinor(olat.Vh, 4601)
    lqcd.lqcd_set_cluster_series(lat.h, 1)
    lqcd.lqcd_set_wait_limit(lat.h, 1)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.solve_w3eo(cuda(b), kappa, 0.0, 0, lqcd.PREC_F32, tol=1e-10, method=lqcd.SOLVER_SERIES)
    assert e.value.status == lqcd.ERR_TIMEOUT
    lqcd.lqcd_set_wait_limit(lat.h, 0)
    x, it = lat.solve_w3eo(cuda(b), kappa, 0.0, 0, lqcd.PREC_F32, tol=1e-10, method=lqcd.SOLVER_SERIES)
    r = b - olat.w3eo(U, kappa, 0.0, x.cpu().numpy(), 0)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    lat.close()
