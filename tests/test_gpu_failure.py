"""Failure detection on the GPU without a GPU fault.

* Non-finite inputs injected on the host (a NaN in a source, in the links,
  in the momenta of a trajectory) end the call with LQCD_ERR_NAN, in the
  eager path and inside a replayed MD graph, and the same handle then gives
  the result a fresh handle gives.
* The persistent solver's barrier wait is bounded: with a wait limit of one
  clock cycle (lqcd_set_wait_limit) a solve whose system spans several CTAs
  must give up with LQCD_ERR_TIMEOUT, every CTA returns, and after the
  default limit is restored the same handle solves normally and its next
  graph trajectory is not failed by the earlier status.

Nothing here faults, traps or hangs the GPU: every wait is bounded and every
failure is a status the host reads.
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

L, L0_SLAB, EPS, KAPPA = (16, 8, 8, 8), 4, 0.6, 0.156


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def field():
    U = syn.random_links(L, EPS, 2101)
    return U, O.Lattice(L, L0_SLAB, -1)


def resid(olat, U, x, b, block):
    x = x.cpu().numpy()
    Wx = olat.W1(U, KAPPA, x) if block else olat.M(U, KAPPA, x)
    return np.linalg.norm(Wx - b) / np.linalg.norm(b)


@pytest.mark.parametrize("block", [True, False])
def test_nan_source_reported_then_handle_solves(field, block):
    U, olat = field
    lat = lqcd.Lattice(L, L0_SLAB, -1)
    lat.set_gauge(cuda(U))
    b = syn.gaussian_spinor(olat.V, 2102)
    bad = b.copy()
    bad[olat.Vh + 17, 2, 1] = np.nan  # an odd site: reaches the solve through the even-odd source
    solve = (lambda v: lat.block_solve(cuda(v), KAPPA, -1, 0, lqcd.PREC_F32)) if block else \
        (lambda v: lat.solve(cuda(v), KAPPA, 0, lqcd.PREC_F32))
    with pytest.raises(lqcd.LqcdError) as e:
        solve(bad)
    assert e.value.status == lqcd.ERR_NAN
    x = solve(b)[0]
    assert resid(olat, U, x, b, block) < 1e-10
    lat.close()


def test_nan_link_reported_then_handle_recovers(field):
    U, olat = field
    lat = lqcd.Lattice(L, L0_SLAB, -1)
    bad = U.copy()
    bad[0, 5, 1, 2] = np.nan
    lat.set_gauge(cuda(bad))
    phi = syn.gaussian_spinor(olat.V, 2103)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.pf_force(cuda(phi), KAPPA, lqcd.TERM_W1, lqcd.PREC_F32, tol=1e-10)
    assert e.value.status == lqcd.ERR_NAN
    lat.set_gauge(cuda(U))
    S, F = lat.pf_force(cuda(phi), KAPPA, lqcd.TERM_W1, lqcd.PREC_F32, tol=1e-10)
    So, Fo = olat.pf_w1(U, KAPPA, phi, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    assert np.max(np.abs(F.cpu().numpy() - Fo)) < 1e-5 * np.max(np.abs(Fo))
    lat.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_nan_momenta_in_trajectory_then_same_result_as_fresh_handle(use_graph):
    """a NaN momentum turns the links non-finite inside the molecular
    dynamics: with use_graph the failing solves run inside the replayed
    graph and report through the deferred status"""
    Ls, l0, kappa = (4, 4, 4, 4), 2, 0.15
    U = cuda(syn.random_links(Ls, 0.3, 2104))
    prm = lqcd.hmc_params(5.6, kappa, 0.5, 2, (lqcd.SW, lqcd.LF), (2, 3), 0, 1, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-10, use_graph=use_graph, chrono=1)
    P = cuda(syn.gaussian_momenta(256, 2105))
    P[1, 40, 3] = float("nan")
    lat = lqcd.Lattice(Ls, l0, -1)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.hmc_trajectory(U, prm, 2104, 0, P0=P)
    assert e.value.status == lqcd.ERR_NAN
    U1, r1 = lat.hmc_trajectory(U, prm, 2104, 1)
    fresh = lqcd.Lattice(Ls, l0, -1)
    U2, r2 = fresh.hmc_trajectory(U, prm, 2104, 1)
    assert abs(r1.dH - r2.dH) < 1e-10 and r1.accepted == r2.accepted and r1.shift == r2.shift
    assert float((U1 - U2).abs().max()) < 1e-12
    lat.close()
    fresh.close()


def test_barrier_wait_limit_times_out_then_handle_recovers(field):
    U, olat = field
    lat = lqcd.Lattice(L, L0_SLAB, -1)
    lat.set_gauge(cuda(U))
    b = syn.gaussian_spinor(olat.V, 2106)
    # the global solve spans several CTAs (V/2 = 4096 sites, 256 per CTA);
    # with a one-cycle limit the first CTA at a barrier gives up
    lqcd.lqcd_set_wait_limit(lat.h, 1)
    with pytest.raises(lqcd.LqcdError) as e:
        lat.solve(cuda(b), KAPPA, 0, lqcd.PREC_F32)
    assert e.value.status == lqcd.ERR_TIMEOUT
    lqcd.lqcd_set_wait_limit(lat.h, 0)
    x = lat.solve(cuda(b), KAPPA, 0, lqcd.PREC_F32)[0]
    assert resid(olat, U, x, b, False) < 1e-10
    # a graph trajectory on the same handle is not failed by the earlier status
    prm = lqcd.hmc_params(5.6, KAPPA, 0.2, 1, (lqcd.LF,), (2,), 0, 0, -1, roll=0, precision=lqcd.PREC_F32,
                          tol=1e-10, use_graph=1)
    U1, r1 = lat.hmc_trajectory(cuda(U), prm, 2106, 0)
    assert np.isfinite(r1.dH)
    fresh = lqcd.Lattice(L, L0_SLAB, -1)
    U2, r2 = fresh.hmc_trajectory(cuda(U), prm, 2106, 0)
    assert abs(r1.dH - r2.dH) < 1e-10
    lat.close()
    fresh.close()
