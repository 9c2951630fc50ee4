"""Parity at the full sizes and in the launch configurations bench.py times.

16^3 x 32 (the trajectory workload, l0 = 4) and 32^3 x 64 (the Dslash
bandwidth lattice and the iterated decomposition, l0 = 8, sub-slabs of 4):
the hopping sweep in all three storage precisions element by element
against the oracle, and the batched slab, sub-slab and global solves by
their residual under the oracle's own operator.  Tolerances as in
tests/test_gpu_parity.py.
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

TOL = {lqcd.PREC_F64: 1e-13, lqcd.PREC_F32: 1e-6, lqcd.PREC_F16: 5e-3, lqcd.PREC_BF16: 2e-2}


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _field(L, eps, seed):
    U = syn.random_links_torch(L, eps, seed, "cuda").contiguous()
    return U, U.cpu().numpy()


@pytest.mark.parametrize("L,l0", [((32, 16, 16, 16), 4), ((64, 32, 32, 32), 8)])
def test_dslash_full_size(L, l0):
    U, Un = _field(L, 0.6, 77)
    lat = lqcd.Lattice(L, l0, -1)
    lat.set_gauge(U)
    lqcd.lqcd_autotune(lat.h, 1, 0.0)  # the bench's schedule
    olat = O.Lattice(L, l0, -1)
    x = syn.gaussian_spinor(olat.Vh, 78)
    xd = torch.from_numpy(x).cuda()
    for parity in (0, 1):
        ref = olat.dslash_eo(Un, x, parity, 0)
        for p, tol in TOL.items():
            out = lat.dslash_eo(xd, parity, 0.0, 0, lqcd.OP_HOP, p).cpu().numpy()
            assert rel(out, ref) < tol, (parity, p, rel(out, ref))
    lat.close()


def test_solves_16x16x16x32():
    """the trajectory workload's solves: W1 slabs by BiCGstab and by the
    geometric series (through the sub-slab operator of an l0 = 8 handle,
    whose sub-slabs are the l0 = 4 slabs), and the global solve"""
    L, kappa = (32, 16, 16, 16), 0.1575
    U, Un = _field(L, 0.6, 79)
    lat = lqcd.Lattice(L, 4, -1)
    lat.set_gauge(U)
    olat = O.Lattice(L, 4, -1)
    b = syn.gaussian_spinor(olat.V, 80)
    bd = torch.from_numpy(b).cuda()
    for p in (lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16):
        x, it, rs = lat.block_solve(bd, kappa, -1, 0, p, tol=1e-10)
        r = b - olat.W1(Un, kappa, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
        x, it, rs = lat.solve(bd, kappa, 0, p, tol=1e-10)
        r = b - olat.M(Un, kappa, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    lat.close()
    # the series needs the spectral radius below one: on the bench's
    # thermalised field, not on the rough random start
    import bench

    lat8 = lqcd.Lattice(L, 8, -1, l0s=4)
    U, _ = bench.thermalise(lat8, U, 5.6, 20, 79)
    Un = U.cpu().numpy()
    lat8.set_gauge(U)
    olat8 = O.Lattice(L, 8, -1, l0s=4)
    be = b[:olat.Vh]
    for rho in (0.0, 0.2):
        x, it = lat8.solve_w3eo(torch.from_numpy(be).cuda(), kappa, rho, 0, lqcd.PREC_F32, tol=1e-10,
                                method=lqcd.SOLVER_SERIES)
        r = be - olat8.w3eo(Un, kappa, rho, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(be), it[:8]
    lat8.close()


def test_subslab_solve_32x32x32x64():
    """the iterated decomposition's W2 solve at 32^3 x 64 (l0 = 8, sub-slabs
    of 4, 16 systems in one launch)"""
    L, kappa = (64, 32, 32, 32), 0.158
    U, Un = _field(L, 0.6, 81)
    lat = lqcd.Lattice(L, 8, -1, l0s=4)
    lat.set_gauge(U)
    olat = O.Lattice(L, 8, -1, l0s=4)
    b = syn.gaussian_spinor(olat.V, 82)
    x, it, rs = lat.subblock_solve(torch.from_numpy(b).cuda(), kappa, -1, 0, lqcd.PREC_F32, tol=1e-10)
    r = b - olat.W2(Un, kappa, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    assert min(it[:16]) > 0
    lat.close()
