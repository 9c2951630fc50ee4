"""The link update T_U of Sec. 2 eq. (4) on the GPU, U <- exp(i dt P) U,
against scipy's matrix exponential (Pade, an independent method) link by
link.  Small steps take the Cayley-Hamilton coefficients from their power
series, steps with tr (dt P)^2 / 2 > 1 from the closed trigonometric form;
both must agree with expm to double precision and leave the links unitary
with unit determinant.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402


def generators():
    t = np.zeros((8, 3, 3), np.complex128)
    t[0, 0, 1] = t[0, 1, 0] = 1
    t[1, 0, 1], t[1, 1, 0] = -1j, 1j
    t[2, 0, 0], t[2, 1, 1] = 1, -1
    t[3, 0, 2] = t[3, 2, 0] = 1
    t[4, 0, 2], t[4, 2, 0] = -1j, 1j
    t[5, 1, 2] = t[5, 2, 1] = 1
    t[6, 1, 2], t[6, 2, 1] = -1j, 1j
    t[7, 0, 0] = t[7, 1, 1] = 1 / np.sqrt(3)
    t[7, 2, 2] = -2 / np.sqrt(3)
    return 0.5 * t


@pytest.mark.parametrize("dt", [1e-7, 0.003, 0.05, 0.4, 1.5])
def test_link_update_matches_expm(dt):
    L = (4, 4, 2, 2)
    V = 64
    U = syn.random_links(L, 0.7, 401)
    P = syn.gaussian_momenta(V, 402)
    lat = lqcd.Lattice(L, 2, -1)
    U1 = lat.link_update(torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda(), dt).cpu().numpy()
    T = generators()
    err = 0.0
    nbig = 0
    for mu in range(4):
        for s in range(V):
            X = dt * np.einsum("a,aij->ij", P[mu, s], T)
            nbig += 0.5 * np.trace(X @ X).real > 1.0
            ref = scipy.linalg.expm(1j * X) @ U[mu, s]
            err = max(err, np.max(np.abs(U1[mu, s] - ref)))
            assert np.max(np.abs(U1[mu, s] @ U1[mu, s].conj().T - np.eye(3))) < 1e-14
            assert abs(np.linalg.det(U1[mu, s]) - 1) < 1e-13
    assert err < 2e-14, err
    if dt >= 1.5:
        assert nbig > 0  # the closed form was exercised
    lat.close()
