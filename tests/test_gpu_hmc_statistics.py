"""Statistical and structural checks of the GPU HMC itself (Sec. 2):
reversibility of the double-precision molecular dynamics, and
<exp(-dH)> = 1 over an equilibrated chain of short trajectories on 4^4
(area preservation and reversibility together), run through the C-ABI."""
import math

import numpy as np
import pytest

from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402


def test_md_reversibility_double():
    L, l0, kappa = (8, 4, 4, 4), 2, 0.14
    lat = lqcd.Lattice(L, l0, -1)
    U = torch.from_numpy(syn.random_links(L, 0.3, 5)).cuda()
    P = torch.from_numpy(syn.gaussian_momenta(lat.V, 6)).cuda()
    phi1 = torch.from_numpy(syn.gaussian_spinor(lat.V, 7)).cuda()
    phi2 = torch.from_numpy(syn.gaussian_complex(lat.boundary().shape, 8)).cuda()
    prm = lqcd.hmc_params(5.6, kappa, 0.4, 3, (lqcd.SW, lqcd.SW, lqcd.LF), (2, 2, 2), 0, 1, 2,
                          lam=0.1931833275037836, tol=1e-13)
    U1, P1 = lat.md(U, P, phi1, phi2, prm)
    assert (U1 - U).abs().max().item() > 1e-3
    U2, P2 = lat.md(U1, -P1, phi1, phi2, prm)
    assert (U2 - U).abs().max().item() < 1e-11
    assert (P2 + P).abs().max().item() < 1e-9
    lat.close()


def test_exp_minus_dH_average_4x4x4x4():
    L, l0 = (4, 4, 4, 4), 2
    lat = lqcd.Lattice(L, l0, -1)
    U = torch.from_numpy(syn.random_links(L, 0.3, 2007)).cuda()
    prm = lqcd.hmc_params(5.6, 0.15, 0.4, 2, (lqcd.SW, lqcd.LF), (2, 3), 0, 0, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-12, use_graph=1)
    for t in range(50):  # equilibration at beta = 5.6 from the smooth start
        U, res = lat.hmc_trajectory(U, prm, 4242, t)
    w, acc = [], 0
    for t in range(50, 300):
        U, res = lat.hmc_trajectory(U, prm, 4242, t)
        w.append(math.exp(-res.dH))
        acc += res.accepted
    w = np.array(w)
    err = w.std(ddof=1) / math.sqrt(len(w))
    assert abs(w.mean() - 1.0) < 3.0 * err + 2e-3, (w.mean(), err)
    assert 0.3 < acc / len(w) <= 1.0
    lat.close()
