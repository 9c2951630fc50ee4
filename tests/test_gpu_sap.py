"""The Schwarz-preconditioned global solve (Sec. 3: the S4 solver, BiCGstab
with even-odd and Schwarz preconditioning) against the FP64 oracle.

The handle's global solver (lqcd_set_global_solver) is switched to
LQCD_SOLVER_SAP: BiCGstab on M with one multiplicative Schwarz cycle over
the red / black x0-slabs as right preconditioner, every slab solve a
truncated geometric series of its even-odd reduced operator; or to
LQCD_SOLVER_SAP_BLOCKS, the same cycle over red / black 4-D blocks of at
most 4^4 sites, each block solved by one CTA in shared memory.  Checked,
for both:
the solution of M x = b and of M^dag x = b by the oracle's residual
(<= 1e-10 relative) in all three inner precisions and for several series
lengths (0 terms: the first-order block inverse), R^-1 and R^-dag of the
boundary term against the oracle (1e-9), the boundary-term force (1e-5 in
the mixed form), and a trajectory against the oracle's (dH <= 1e-4).
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

# 16 x 8^3 with slabs of 4 (four slabs, two per colour) on the near-critical
# synthetic field of the solver tests; 8 x 4 x 2 x 6 with slabs of 2 (odd-
# sized slab faces, a ragged tail of the CTA loops)
GEOMS = [((16, 8, 8, 8), 4, 0.6, 0.156), ((8, 4, 2, 6), 2, 0.3, 0.14)]
# slab blocks, and 4-D blocks (4^4 on 16 x 8^3; 4 x 4 x 2 x 2 on 8 x 4 x 2 x 6,
# three blocks along x3: an odd block count, two same-colour neighbours)
METHODS = [lqcd.SOLVER_SAP, lqcd.SOLVER_SAP_BLOCKS]
MIDS = ["slabs", "blocks"]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", params=GEOMS, ids=lambda p: "x".join(map(str, p[0])) + "_l0%d" % p[1])
def setup(request):
    L, l0, eps, kappa = request.param
    U = syn.random_links(L, eps, 2200 + sum(L))
    lat = lqcd.Lattice(L, l0, -1)
    lat.set_gauge(cuda(U))
    olat = O.Lattice(L, l0, -1)
    yield lat, olat, U, kappa
    lat.close()


@pytest.mark.parametrize("method", METHODS, ids=MIDS)
@pytest.mark.parametrize("prec,nsap", [(lqcd.PREC_F64, 4), (lqcd.PREC_F32, 4), (lqcd.PREC_F16, 4),
                                       (lqcd.PREC_BF16, 4), (lqcd.PREC_F32, 0), (lqcd.PREC_F32, 1),
                                       (lqcd.PREC_F32, 8)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_sap_solve_residual(setup, method, prec, nsap, dagger):
    lat, olat, U, kappa = setup
    b = syn.gaussian_spinor(olat.V, 2201 + dagger)
    lqcd.lqcd_set_global_solver(lat.h, method, nsap)
    try:
        x, it, rs = lat.solve(cuda(b), kappa, dagger, prec, tol=1e-10)
    finally:
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_BICGSTAB, 0)
    xo = x.cpu().numpy()
    r = np.linalg.norm(olat.M(U, kappa, xo, dagger) - b) / np.linalg.norm(b)
    assert r < 1e-10, (r, it)
    assert rs <= 1e-10
    # the same solution as the plain even-odd BiCGstab (both to 1e-10)
    x2 = lat.solve(cuda(b), kappa, dagger, prec, tol=1e-10)[0]
    assert rel(x, x2.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("method", METHODS, ids=MIDS)
def test_sap_needs_fewer_iterations(setup, method):
    """the preconditioned operator is better conditioned: fewer (more
    expensive) iterations than the plain even-odd BiCGstab"""
    lat, olat, U, kappa = setup
    b = cuda(syn.gaussian_spinor(olat.V, 2203))
    it_plain = lat.solve(b, kappa, 0, lqcd.PREC_F64, tol=1e-10)[1]
    lqcd.lqcd_set_global_solver(lat.h, method, 4)
    try:
        it_sap = lat.solve(b, kappa, 0, lqcd.PREC_F64, tol=1e-10)[1]
    finally:
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_BICGSTAB, 0)
    assert it_sap < it_plain, (it_sap, it_plain)


@pytest.mark.parametrize("method", METHODS, ids=MIDS)
@pytest.mark.parametrize("op", [lqcd.SCHUR_RINV, lqcd.SCHUR_RINVDAG])
def test_sap_schur_inverse(setup, op, method):
    lat, olat, U, kappa = setup
    c = syn.gaussian_complex(olat.bnd_shape(), 2204 + op)
    ref = olat.schur(U, kappa, c, op, route=1, tol=1e-13)
    lqcd.lqcd_set_global_solver(lat.h, method, 4)
    try:
        out = lat.schur(cuda(c), kappa, op, lqcd.PREC_F32, tol=1e-12)
    finally:
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_BICGSTAB, 0)
    assert rel(out, ref) < 1e-9


@pytest.mark.parametrize("method", METHODS, ids=MIDS)
def test_sap_schur_force(setup, method):
    lat, olat, U, kappa = setup
    phi = syn.gaussian_complex(olat.bnd_shape(), 2206)
    lqcd.lqcd_set_global_solver(lat.h, method, 4)
    try:
        S, F = lat.pf_force(cuda(phi), kappa, lqcd.TERM_SCHUR, lqcd.PREC_F32, tol=1e-12)
    finally:
        lqcd.lqcd_set_global_solver(lat.h, lqcd.SOLVER_BICGSTAB, 0)
    So, Fo = olat.pf_schur(U, kappa, phi, route=1, tol=1e-13)
    assert abs(S - So) < 1e-9 * So
    assert rel(F, Fo) < 1e-5


@pytest.mark.parametrize("method", METHODS, ids=MIDS)
def test_sap_trajectory_matches_oracle(method):
    L, l0, kappa, beta = (4, 4, 4, 4), 2, 0.15, 5.6
    U = syn.random_links(L, 0.3, 2207)
    lat = lqcd.Lattice(L, l0, -1)
    lqcd.lqcd_set_global_solver(lat.h, method, 4)
    olat = O.Lattice(L, l0, -1)
    prm = lqcd.hmc_params(beta, kappa, 0.5, 2, (lqcd.SW, lqcd.LF), [2, 4], 0, 0, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-11, use_graph=1, chrono=1)
    oprm = O.hmc_params(beta, kappa, 0.5, 2, (O.SW, O.LF), [2, 4], 0, 0, 1, roll=1, tol=1e-13)
    U1, res = lat.hmc_trajectory(cuda(U), prm, 2207, 3)
    Uo, ores, st = olat.hmc_trajectory(U, oprm, 2207, 3)
    assert st == 0
    assert abs(res.dH - ores.dH) < 1e-4
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < 1e-7
    lat.close()


def test_set_global_solver_validates():
    lat = lqcd.Lattice((4, 4, 4, 4), 2, -1)
    for method, n in ((lqcd.SOLVER_SERIES, 4), (7, 4), (lqcd.SOLVER_SAP, -1), (lqcd.SOLVER_SAP, 65),
                      (lqcd.SOLVER_SAP_BLOCKS, -1), (lqcd.SOLVER_SAP_BLOCKS, 65)):
        with pytest.raises(lqcd.LqcdError) as e:
            lqcd.lqcd_set_global_solver(lat.h, method, n)
        assert e.value.status == lqcd.ERR_ARG
    lat.close()
