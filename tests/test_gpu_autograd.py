"""The autograd binding of the pseudo-fermion actions on the GPU: its
gradient equals the library force and the oracle force, and finite
differences of the action (through the library's own link update) agree
with it on 64 random links of the 16^3 x 32 lattice (Sec. 1 eq. (3),
Sec. 2 eq. (4)).

Finite differences: central, Richardson-extrapolated from h = 1e-2 and
2e-2 (error O(h^4)); the solves run to a relative residual of 1e-13 so that
solver noise in S stays below 1e-6 of the differences.  Tolerance 1e-5 of
the largest sampled force component.
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
from paper_0710_0066_gb300.autograd import pseudofermion_action  # noqa: E402


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _grad(lat, U, phi, kappa, term, rho=0.0, precision=lqcd.PREC_F32):
    omega = torch.zeros((4, lat.V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    S = pseudofermion_action(omega, lat, U, phi, kappa, term, precision, 1e-13, 40000, rho)
    S.backward()
    return S.item(), omega.grad


def _fd(lat, U, phi, kappa, term, links, rho=0.0, h=1e-2):
    def S_at(mu, s, a, eps):
        om = torch.zeros((4, lat.V, 8), dtype=torch.float64, device="cuda")
        om[mu, s, a] = eps
        with torch.no_grad():
            return pseudofermion_action(om, lat, U, phi, kappa, term, lqcd.PREC_F32, 1e-13, 40000, rho).item()

    out = []
    for (mu, s) in links:
        for a in range(8):
            d1 = (S_at(mu, s, a, h) - S_at(mu, s, a, -h)) / (2 * h)
            d2 = (S_at(mu, s, a, 2 * h) - S_at(mu, s, a, -2 * h)) / (4 * h)
            out.append(((mu, s, a), (4 * d1 - d2) / 3))
    return out


@pytest.fixture(scope="module")
def big():
    L, l0, kappa = (32, 16, 16, 16), 4, 0.1575
    U = cuda(syn.random_links(L, 0.6, 2009))
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    lat.set_gauge(U)
    yield lat, U, kappa
    lat.close()


@pytest.mark.parametrize("term,nlinks", [(lqcd.TERM_W1, 64), (lqcd.TERM_SCHUR, 16), (lqcd.TERM_S1, 16)])
def test_autograd_matches_finite_differences_16x16x16x32(big, term, nlinks):
    """phi lives on the sites of the sampled links (boundary sites for the
    Schur term, even sites for S1), so S stays O(10^2) and the
    differences resolve the force to ~1e-7"""
    lat, U, kappa = big
    rho = 0.2 if term == lqcd.TERM_S1 else 0.0
    rng = np.random.default_rng(term)
    maps = lat.index_maps().cpu().numpy()
    g = torch.Generator(device="cuda")
    g.manual_seed(77 + term)
    if term == lqcd.TERM_SCHUR:
        bsite = np.nonzero(maps[13] >= 0)[0]
        sites = rng.choice(bsite, nlinks, replace=False)
        phi = torch.zeros(lat.boundary().shape, dtype=torch.complex128, device="cuda")
        flat = phi.view(-1, 6)
        for st in sites:
            flat[int(maps[13, st])] = torch.randn(6, dtype=torch.complex128, device="cuda", generator=g)
    else:
        nsite = lat.Vh if term == lqcd.TERM_S1 else lat.V
        sites = rng.choice(nsite, nlinks, replace=False)
        phi = torch.zeros((nsite, 4, 3), dtype=torch.complex128, device="cuda")
        for st in sites:
            phi[int(st)] = torch.randn((4, 3), dtype=torch.complex128, device="cuda", generator=g)
    phi = phi.contiguous()
    links = [(int(rng.integers(4)), int(st)) for st in sites]
    S, grad = _grad(lat, U, phi, kappa, term, rho)
    # the gradient is the library force at omega = 0 (the rotation by
    # omega = 0 reunitarises the links, which can move their single-precision
    # copies by one rounding: the force, computed in single-precision link
    # arithmetic, agrees to that level)
    lat.set_gauge(U)
    if term == lqcd.TERM_S1:
        S2, F = lat.pf_force_eo(phi, kappa, rho, term, lqcd.PREC_F32, 1e-13, 40000)
    else:
        S2, F = lat.pf_force(phi, kappa, term, lqcd.PREC_F32, 1e-13, 40000)
    assert abs(S - S2) < 1e-10 * abs(S)
    assert torch.allclose(grad, F, rtol=0, atol=1e-6 * F.abs().max().item())
    fd = _fd(lat, U, phi, kappa, term, links, rho)
    G = grad.cpu().numpy()
    scale = max(abs(G[mu, s, a]) for (mu, s, a), _ in fd)
    worst = max(abs(G[mu, s, a] - d) for (mu, s, a), d in fd)
    assert scale > 1e-3
    assert worst < 1e-5 * scale, (worst, scale)


def test_autograd_matches_oracle_force():
    L, l0, kappa = (8, 4, 4, 4), 4, 0.15
    Un = syn.random_links(L, 0.3, 91)
    lat = lqcd.Lattice(L, l0, -1, l0s=2)
    olat = O.Lattice(L, l0, -1, l0s=2)
    phi = syn.gaussian_spinor(olat.V, 92)
    S, grad = _grad(lat, cuda(Un), cuda(phi), kappa, lqcd.TERM_W1, precision=lqcd.PREC_F64)
    So, Fo = olat.pf_w1(Un, kappa, phi, tol=1e-13)
    assert abs(S - So) < 1e-10 * So
    assert np.max(np.abs(grad.cpu().numpy() - Fo)) < 1e-9 * np.max(np.abs(Fo))
    # link update against the oracle's exponential
    P = syn.gaussian_momenta(olat.V, 93)
    U1 = lat.link_update(cuda(Un), cuda(P), 0.05)
    assert np.max(np.abs(U1.cpu().numpy() - olat.update_U(Un, P, 0.05))) < 1e-12
    lat.close()
