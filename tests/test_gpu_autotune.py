"""lqcd_autotune: the measured launch schedules are valid, and the hopping
sweep and the solvers give the same results under every schedule (up to
rounding, the solves to their tolerance)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402


def test_autotune_choices_and_results():
    L, l0, kappa = (16, 8, 8, 8), 4, 0.156
    U = syn.random_links(L, 0.6, 5)
    lat = lqcd.Lattice(L, l0, -1)
    lat.set_gauge(torch.from_numpy(U).cuda())
    olat = O.Lattice(L, l0, -1)
    x = syn.gaussian_spinor(olat.Vh, 6)
    b = syn.gaussian_spinor(olat.V, 7)
    before = {p: lat.dslash_eo(torch.from_numpy(x).cuda(), 0, 0.0, 0, lqcd.OP_HOP, p).cpu().numpy()
              for p in (lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16)}
    lqcd.lqcd_autotune(lat.h, 3, kappa)
    t = lqcd.lqcd_tune_read(lat.h)
    assert set(t["hop_block_size"].values()) <= {64, 128, 256}
    assert set(t["slab_solve_sites_per_thread"].values()) <= {0, 1, 2}  # 0: every resident CTA
    assert set(t["global_solve_sites_per_thread"].values()) <= {0, 1, 2}
    for p, ref in before.items():
        out = lat.dslash_eo(torch.from_numpy(x).cuda(), 0, 0.0, 0, lqcd.OP_HOP, p).cpu().numpy()
        assert np.array_equal(out, ref)  # one thread per site: the schedule changes nothing
    for p in (lqcd.PREC_F64, lqcd.PREC_F32, lqcd.PREC_F16, lqcd.PREC_BF16):
        xs, it, rs = lat.block_solve(torch.from_numpy(b).cuda(), kappa, -1, 0, p, tol=1e-10)
        r = b - olat.W1(U, kappa, xs.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
        xg, it, rs = lat.solve(torch.from_numpy(b).cuda(), kappa, 0, p, tol=1e-10)
        r = b - olat.M(U, kappa, xg.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    lat.close()


@pytest.mark.parametrize("spt", [0, 1, 2])
def test_solver_schedules_agree(spt):
    """every CTA count of the persistent solver (sites per thread 1 or 2, or
    0: all co-resident CTAs with an equal share of the sites, the last CTA's
    share ragged) solves the slab and global systems to the tolerance"""
    # 12 x 6^3 with slabs of 3: 324 sites per slab system and 1296 in the
    # global one, neither a multiple of the CTA share
    L, l0, kappa = (12, 6, 6, 6), 3, 0.156
    U = syn.random_links(L, 0.6, 8)
    lat = lqcd.Lattice(L, l0, -1)
    lat.set_gauge(torch.from_numpy(U).cuda())
    olat = O.Lattice(L, l0, -1)
    b = syn.gaussian_spinor(olat.V, 9)
    lqcd.lqcd_set_solver_schedule(lat.h, spt)
    for p in (lqcd.PREC_F64, lqcd.PREC_F32):
        xs, it, rs = lat.block_solve(torch.from_numpy(b).cuda(), kappa, -1, 0, p, tol=1e-10)
        r = b - olat.W1(U, kappa, xs.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
        xg, it, rs = lat.solve(torch.from_numpy(b).cuda(), kappa, 0, p, tol=1e-10)
        r = b - olat.M(U, kappa, xg.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    lat.close()
