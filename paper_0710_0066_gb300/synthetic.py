"""Seeded synthetic inputs (gauge fields, spinor sources, momenta).

The paper's workloads are thermalised beta = 5.6 ensembles, which are not
available; these seeded fields stand in for them with the same shapes:

* links ``U = exp(i eps H)``, ``H`` traceless hermitian with independent
  N(0,1) coefficients on the eight generators lambda^a/2;
* spinors with complex Gaussian components of density ``exp(-|eta|^2)``
  (real and imaginary parts of variance 1/2);
* momenta with N(0,1) Lie-algebra coefficients.

Layouts follow the library: gauge ``(4, V, 3, 3)``, spinor ``(V, 4, 3)``,
momenta ``(4, V, 8)``, sites in checkerboard order.  The module only draws
random numbers (and exponentiates them with a library eigen-solver); it
holds none of the method's operators and is shared by the tests, by the
smoke check and by bench.py.
"""
import numpy as np

_SQ3 = 1.0 / np.sqrt(3.0)


def _generators():
    t = np.zeros((8, 3, 3), np.complex128)
    t[0, 0, 1] = t[0, 1, 0] = 1
    t[1, 0, 1], t[1, 1, 0] = -1j, 1j
    t[2, 0, 0], t[2, 1, 1] = 1, -1
    t[3, 0, 2] = t[3, 2, 0] = 1
    t[4, 0, 2], t[4, 2, 0] = -1j, 1j
    t[5, 1, 2] = t[5, 2, 1] = 1
    t[6, 1, 2], t[6, 2, 1] = -1j, 1j
    t[7, 0, 0] = t[7, 1, 1] = _SQ3
    t[7, 2, 2] = -2 * _SQ3
    return 0.5 * t


def volume(L):
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def random_links(L, eps, seed):
    """U = exp(i eps H) per link, numpy complex128 of shape (4, V, 3, 3)."""
    rng = np.random.default_rng(seed)
    V = volume(L)
    h = rng.standard_normal((4 * V, 8))
    H = np.einsum("na,aij->nij", h, _generators())
    w, vec = np.linalg.eigh(H)
    U = np.einsum("nij,nj,nkj->nik", vec, np.exp(1j * eps * w), vec.conj())
    return np.ascontiguousarray(U.reshape(4, V, 3, 3))


def random_links_torch(L, eps, seed, device):
    """Same distribution as random_links, drawn with torch on ``device``
    (for lattices too large to generate on the host quickly)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    V = volume(L)
    T = torch.as_tensor(_generators(), device=device)
    U = torch.empty((4 * V, 3, 3), dtype=torch.complex128, device=device)
    chunk = 1 << 20
    for a in range(0, 4 * V, chunk):
        b = min(4 * V, a + chunk)
        h = torch.randn((b - a, 8), generator=g, device=device, dtype=torch.float64)
        H = torch.einsum("na,aij->nij", h.to(torch.complex128), T)
        U[a:b] = torch.linalg.matrix_exp(1j * eps * H)
    return U.reshape(4, V, 3, 3)


def gaussian_spinor(n_sites, seed):
    """complex Gaussian spinor field of shape (n_sites, 4, 3)"""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n_sites, 4, 3, 2)) * np.sqrt(0.5)
    return np.ascontiguousarray(z[..., 0] + 1j * z[..., 1])


def gaussian_complex(shape, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(tuple(shape) + (2,)) * np.sqrt(0.5)
    return np.ascontiguousarray(z[..., 0] + 1j * z[..., 1])


def gaussian_momenta(V, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, V, 8))


def random_gauge_transform(V, seed):
    """random SU(3) matrices g(x), shape (V, 3, 3) (QR of complex Gaussians,
    phases fixed so that det g = 1)"""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((V, 3, 3)) + 1j * rng.standard_normal((V, 3, 3))
    q, r = np.linalg.qr(A)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q
