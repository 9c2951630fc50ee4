"""The allocation-free gauge-action entry point (lqcd_gauge_action_static).

It serves callers that cannot allocate device memory and therefore cannot
create a handle: its partial sums live in a fixed array inside the library.
Checked through the C-ABI against the handle-based lqcd_gauge_force on two
calls in a row (the second on a smaller lattice, so that partial sums left
over from the first call would show up if they were read).  Kept in a file
that runs last so that a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402


def test_static_gauge_action_matches_handle_path_twice():
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for k, (L, eps) in enumerate([((16, 8, 8, 8), 0.6), ((8, 4, 4, 4), 0.3)]):
        U = torch.from_numpy(syn.random_links(L, eps, 60 + k)).cuda()
        lat = lqcd.Lattice(L, 2, -1)
        lat.set_gauge(U)
        S, pl, _ = lat.gauge_force(5.6, force=False)
        lat.close()
        assert lqcd.lqcd_gauge_action_static(L, U, 5.6, out) == lqcd.OK
        torch.cuda.synchronize()
        S2, pl2 = out.tolist()
        assert abs(S2 - S) <= 1e-10 * abs(S), (k, S2, S)
        assert abs(pl2 - pl) <= 1e-13, (k, pl2, pl)


def test_static_gauge_action_rejects_oversized_lattice():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    U = torch.zeros(9, dtype=torch.complex128, device="cuda")  # never read
    assert lqcd.lqcd_gauge_action_static((128, 32, 32, 32), U, 5.6, out) == lqcd.ERR_GEOM
    assert lqcd.lqcd_gauge_action_static((4, 3, 4, 4), U, 5.6, out) == lqcd.ERR_GEOM
