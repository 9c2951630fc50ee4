"""Thin Python binding of the C-ABI in include/lqcd.h.

Argument marshalling only: every function below forwards torch CUDA tensors
(their device pointers) to the same-named ``extern "C"`` entry point of
``liblqcd.so``; all arithmetic runs in the library's kernels.  There is no
fallback: if the library is missing or no GPU is present the calls raise.

Tensor layouts (complex128 unless noted, sites in checkerboard order):
spinor ``(V, 4, 3)``, one-parity spinor ``(V/2, 4, 3)``, gauge
``(4, V, 3, 3)``, momenta / forces float64 ``(4, V, 8)``, boundary field
``(L0/(2 l0), 2, V3, 2, 3)``, index maps int32 ``(14, V)``.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblqcd.so")

OK, ERR_ARG, ERR_GEOM, ERR_NOCONVERGE, ERR_CUDA, ERR_NAN, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7
PREC_F64, PREC_F32, PREC_F16, PREC_BF16 = 0, 1, 2, 3
OP_HOP, OP_MHAT = 0, 1
SCHUR_R, SCHUR_RDAG, SCHUR_RINV, SCHUR_RINVDAG = 0, 1, 2, 3
SCHUR2_R, SCHUR2_RDAG, SCHUR2_RINV, SCHUR2_RINVDAG = 4, 5, 6, 7
TERM_W1, TERM_SCHUR, TERM_W2, TERM_SCHUR2, TERM_S2, TERM_S1 = 0, 1, 2, 3, 4, 5
EO_APPLY, EO_SOLVE = 0, 1
SOLVER_BICGSTAB, SOLVER_SERIES, SOLVER_SAP, SOLVER_SAP_BLOCKS = 0, 1, 2, 3
MAX_LEVELS = 5
LF, SW = 0, 1
KERNEL_HOP, KERNEL_SOLVER, KERNEL_FORCE, KERNEL_GAUGE, KERNEL_BLAS = 0, 1, 2, 3, 4

EXPORTS = [
    "lqcd_create", "lqcd_destroy", "lqcd_last_error", "lqcd_set_stream", "lqcd_set_gauge",
    "lqcd_get_gauge", "lqcd_index_maps", "lqcd_dslash_eo", "lqcd_block_dslash",
    "lqcd_block_solve_batched", "lqcd_solve_wilson", "lqcd_schur_apply", "lqcd_pf_force",
    "lqcd_gauge_force", "lqcd_rng_normals", "lqcd_hmc_trajectory", "lqcd_md",
    "lqcd_profile_enable", "lqcd_profile_reset", "lqcd_profile_read", "lqcd_launch_count",
    "lqcd_gauge_action_static", "lqcd_force_profile", "lqcd_set_subslabs", "lqcd_subblock_dslash",
    "lqcd_subblock_solve_batched", "lqcd_subblock_eo", "lqcd_pf_force_eo", "lqcd_link_update",
    "lqcd_autotune", "lqcd_tune_read", "lqcd_profile_times", "lqcd_set_wait_limit",
    "lqcd_set_global_solver", "lqcd_set_solver_schedule", "lqcd_set_cluster_series",
]


class HmcParams(C.Structure):
    _fields_ = [
        ("beta", C.c_double), ("kappa", C.c_double), ("tau", C.c_double), ("lam", C.c_double),
        ("nlevels", C.c_int), ("scheme", C.c_int * MAX_LEVELS), ("nsteps", C.c_int * MAX_LEVELS),
        ("level_gauge", C.c_int), ("level_w1", C.c_int), ("level_schur", C.c_int),
        ("pf_init", C.c_int), ("roll", C.c_int), ("metropolis", C.c_int), ("precision", C.c_int),
        ("tol", C.c_double), ("max_iter", C.c_int), ("step_scheme", C.c_int), ("step_scale", C.c_void_p),
        ("level_w2", C.c_int), ("level_schur2", C.c_int),
        ("rho", C.c_double), ("level_s2", C.c_int), ("level_s1", C.c_int), ("eo_solver", C.c_int),
        ("block_solver", C.c_int), ("use_graph", C.c_int), ("chrono", C.c_int),
    ]


class PfFields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "schur", "w2", "schur2", "s2", "s1")]


class HmcResult(C.Structure):
    _fields_ = [
        ("dH", C.c_double), ("H0", C.c_double), ("H1", C.c_double), ("plaq", C.c_double),
        ("u", C.c_double), ("accepted", C.c_int), ("shift", C.c_int),
        ("solver_iters", C.c_int64), ("n_solves", C.c_int), ("n_force", C.c_int),
        ("site_iters", C.c_int64), ("hop_sites", C.c_int64),
    ]


def hmc_params(beta, kappa, tau, nlevels, scheme, nsteps, level_gauge=0, level_w1=0, level_schur=0,
               lam=1.0 / 6.0, pf_init=0, roll=0, metropolis=1, precision=PREC_F64, tol=1e-10,
               max_iter=20000, step_scheme=0, step_scale=None, level_w2=-1, level_schur2=-1, rho=0.0,
               level_s2=-1, level_s1=-1, eo_solver=SOLVER_BICGSTAB, block_solver=SOLVER_BICGSTAB, use_graph=0,
               chrono=0):
    """step_scale: None or a host float64 array (2, L0) of s(x0) (space-like,
    time-like rows); it is kept alive on the returned object"""
    sc = list(scheme) + [0] * (MAX_LEVELS - len(scheme))
    ns = list(nsteps) + [1] * (MAX_LEVELS - len(nsteps))
    p = HmcParams(beta, kappa, tau, lam, nlevels, (C.c_int * MAX_LEVELS)(*sc), (C.c_int * MAX_LEVELS)(*ns),
                  level_gauge, level_w1, level_schur, pf_init, roll, metropolis, precision, tol,
                  max_iter, step_scheme, None, level_w2, level_schur2, rho, level_s2, level_s1, eo_solver,
                  block_solver, use_graph, chrono)
    if step_scale is not None:
        import numpy as np

        p._scale = np.ascontiguousarray(step_scale, dtype=np.float64)
        p.step_scale = p._scale.ctypes.data
    return p


_lib = None


def load():
    """Load liblqcd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblqcd.so is missing: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, i64, u64, u32 = C.c_void_p, C.c_int, C.c_double, C.c_int64, C.c_uint64, C.c_uint32
    sig = {
        "lqcd_create": [C.POINTER(vp), C.POINTER(C.c_int * 4), i, i, vp],
        "lqcd_destroy": [vp],
        "lqcd_last_error": [vp],
        "lqcd_set_stream": [vp, vp],
        "lqcd_set_gauge": [vp, vp],
        "lqcd_get_gauge": [vp, vp],
        "lqcd_index_maps": [vp, vp],
        "lqcd_dslash_eo": [vp, vp, vp, d, i, i, i, i],
        "lqcd_block_dslash": [vp, vp, vp, d, i, i, i],
        "lqcd_block_solve_batched": [vp, vp, vp, d, i, i, i, d, i, vp, vp],
        "lqcd_solve_wilson": [vp, vp, vp, d, i, i, d, i, vp, vp],
        "lqcd_schur_apply": [vp, vp, vp, d, i, i, d, i],
        "lqcd_pf_force": [vp, vp, vp, d, i, i, d, i, vp],
        "lqcd_gauge_force": [vp, vp, d, vp, vp],
        "lqcd_rng_normals": [vp, vp, i64, u64, u32, u32],
        "lqcd_hmc_trajectory": [vp, vp, vp, u64, u32, vp, vp, vp, vp],
        "lqcd_md": [vp, vp, vp, vp, vp],
        "lqcd_subblock_eo": [vp, vp, vp, d, d, i, i, i, i, d, i, vp],
        "lqcd_pf_force_eo": [vp, vp, vp, d, d, i, i, d, i, vp],
        "lqcd_set_subslabs": [vp, i],
        "lqcd_link_update": [vp, vp, vp, d],
        "lqcd_autotune": [vp, i, d],
        "lqcd_tune_read": [vp, vp],
        "lqcd_profile_times": [vp, i, vp, i64, vp],
        "lqcd_subblock_dslash": [vp, vp, vp, d, i, i, i],
        "lqcd_subblock_solve_batched": [vp, vp, vp, d, i, i, i, d, i, vp, vp],
        "lqcd_profile_enable": [vp, i],
        "lqcd_profile_reset": [vp],
        "lqcd_profile_read": [vp, i, vp, vp, vp],
        "lqcd_launch_count": [vp, vp],
        "lqcd_gauge_action_static": [C.POINTER(C.c_int * 4), vp, d, vp, vp],
        "lqcd_force_profile": [vp, vp, vp],
        "lqcd_set_wait_limit": [vp, i64],
        "lqcd_set_solver_schedule": [vp, i],
        "lqcd_set_cluster_series": [vp, i],
        "lqcd_set_global_solver": [vp, i, i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_char_p if name == "lqcd_last_error" else C.c_int
    _lib = lib
    return lib


class LqcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lqcd status %d: %s" % (status, msg))
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


def _check(h, st):
    if st != OK:
        msg = load().lqcd_last_error(h)
        raise LqcdError(st, msg.decode() if msg else "")
    return st


# ---------------------------------------------------------------------------
# same-named entry points (handle first, tensors for device buffers)
# ---------------------------------------------------------------------------
def lqcd_create(L, l0, bc_t=-1, stream=None):
    h = C.c_void_p()
    s = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    st = load().lqcd_create(C.byref(h), C.byref((C.c_int * 4)(*L)), int(l0), int(bc_t), s)
    if st != OK:
        msg = load().lqcd_last_error(h) if h.value else b""
        if h.value:
            load().lqcd_destroy(h)
        raise LqcdError(st, (msg or b"lqcd_create failed").decode())
    return h


def lqcd_destroy(h):
    return load().lqcd_destroy(h)


def lqcd_last_error(h):
    msg = load().lqcd_last_error(h)
    return msg.decode() if msg else ""


def lqcd_set_stream(h, stream):
    return _check(h, load().lqcd_set_stream(h, C.c_void_p(stream.cuda_stream)))


def lqcd_set_gauge(h, U):
    return _check(h, load().lqcd_set_gauge(h, _ptr(U)))


def lqcd_get_gauge(h, U):
    return _check(h, load().lqcd_get_gauge(h, _ptr(U)))


def lqcd_index_maps(h, maps):
    return _check(h, load().lqcd_index_maps(h, _ptr(maps)))


def lqcd_dslash_eo(h, out, inp, kappa, parity, dagger=0, op=OP_HOP, precision=PREC_F64):
    return _check(h, load().lqcd_dslash_eo(h, _ptr(out), _ptr(inp), float(kappa), int(parity),
                                           int(dagger), int(op), int(precision)))


def lqcd_block_dslash(h, out, inp, kappa, colour=-1, dagger=0, precision=PREC_F64):
    return _check(h, load().lqcd_block_dslash(h, _ptr(out), _ptr(inp), float(kappa), int(colour),
                                              int(dagger), int(precision)))


def lqcd_block_solve_batched(h, x, b, kappa, colour=-1, dagger=0, precision=PREC_F64, tol=1e-10,
                             max_iter=10000, nb=None):
    n = nb or 64
    it = (C.c_int * n)()
    rs = (C.c_double * n)()
    _check(h, load().lqcd_block_solve_batched(h, _ptr(x), _ptr(b), float(kappa), int(colour),
                                              int(dagger), int(precision), float(tol), int(max_iter),
                                              it, rs))
    return list(it), list(rs)


def lqcd_autotune(h, what=3, kappa=0.15):
    return _check(h, load().lqcd_autotune(h, int(what), float(kappa)))


def lqcd_set_cluster_series(h, enable):
    return _check(h, load().lqcd_set_cluster_series(h, int(bool(enable))))


def lqcd_set_solver_schedule(h, spt):
    return _check(h, load().lqcd_set_solver_schedule(h, int(spt)))


def lqcd_tune_read(h):
    out = (C.c_int * 12)()
    _check(h, load().lqcd_tune_read(h, out))
    v = list(out)
    names = ("f64", "f32", "f16", "bf16")
    return {"hop_block_size": dict(zip(names, v[0:4])),
            "slab_solve_sites_per_thread": dict(zip(names, v[4:8])),
            "global_solve_sites_per_thread": dict(zip(names, v[8:12]))}


def lqcd_set_global_solver(h, method, sap_terms=4):
    return _check(h, load().lqcd_set_global_solver(h, int(method), int(sap_terms)))


def lqcd_set_wait_limit(h, cycles):
    return _check(h, load().lqcd_set_wait_limit(h, int(cycles)))


def lqcd_link_update(h, U, P, dt):
    return _check(h, load().lqcd_link_update(h, _ptr(U), _ptr(P), float(dt)))


def lqcd_set_subslabs(h, l0s):
    return _check(h, load().lqcd_set_subslabs(h, int(l0s)))


def lqcd_subblock_dslash(h, out, inp, kappa, colour=-1, dagger=0, precision=PREC_F64):
    return _check(h, load().lqcd_subblock_dslash(h, _ptr(out), _ptr(inp), float(kappa), int(colour),
                                                 int(dagger), int(precision)))


def lqcd_subblock_solve_batched(h, x, b, kappa, colour=-1, dagger=0, precision=PREC_F64, tol=1e-10,
                                max_iter=10000, nbs=None):
    n = nbs or 128
    it = (C.c_int * n)()
    rs = (C.c_double * n)()
    _check(h, load().lqcd_subblock_solve_batched(h, _ptr(x), _ptr(b), float(kappa), int(colour),
                                                 int(dagger), int(precision), float(tol), int(max_iter),
                                                 it, rs))
    return list(it), list(rs)


def lqcd_solve_wilson(h, x, b, kappa, dagger=0, precision=PREC_F64, tol=1e-10, max_iter=20000):
    it = C.c_int(0)
    rs = C.c_double(0)
    _check(h, load().lqcd_solve_wilson(h, _ptr(x), _ptr(b), float(kappa), int(dagger),
                                       int(precision), float(tol), int(max_iter), C.byref(it),
                                       C.byref(rs)))
    return it.value, rs.value


def lqcd_schur_apply(h, out, inp, kappa, op, precision=PREC_F64, tol=1e-10, max_iter=20000):
    return _check(h, load().lqcd_schur_apply(h, _ptr(out), _ptr(inp), float(kappa), int(op),
                                             int(precision), float(tol), int(max_iter)))


def lqcd_pf_force(h, F, phi, kappa, term, precision=PREC_F64, tol=1e-10, max_iter=20000):
    S = C.c_double(0)
    _check(h, load().lqcd_pf_force(h, _ptr(F), _ptr(phi), float(kappa), int(term), int(precision),
                                   float(tol), int(max_iter), C.byref(S)))
    return S.value


def lqcd_gauge_force(h, F, beta):
    S = C.c_double(0)
    pl = C.c_double(0)
    _check(h, load().lqcd_gauge_force(h, _ptr(F), float(beta), C.byref(S), C.byref(pl)))
    return S.value, pl.value


def lqcd_rng_normals(h, out, seed, stream, traj):
    return _check(h, load().lqcd_rng_normals(h, _ptr(out), out.numel(), int(seed), int(stream),
                                             int(traj)))


def lqcd_hmc_trajectory(h, U, prm, seed, traj, P0=None, eta1=None, eta2=None):
    res = HmcResult()
    _check(h, load().lqcd_hmc_trajectory(h, _ptr(U), C.byref(prm), int(seed), int(traj), _ptr(P0),
                                         _ptr(eta1), _ptr(eta2), C.byref(res)))
    return res


def lqcd_md(h, U, P, prm, w1=None, schur=None, w2=None, schur2=None, s2=None, s1=None):
    f = PfFields(*[_ptr(t) for t in (w1, schur, w2, schur2, s2, s1)])
    return _check(h, load().lqcd_md(h, _ptr(U), _ptr(P), C.byref(f), C.byref(prm)))


def lqcd_subblock_eo(h, out, inp, kappa, rho, dagger=0, op=EO_APPLY, precision=PREC_F64, tol=1e-10,
                     max_iter=10000, nbs=128, method=SOLVER_BICGSTAB):
    it = (C.c_int * nbs)()
    _check(h, load().lqcd_subblock_eo(h, _ptr(out), _ptr(inp), float(kappa), float(rho), int(dagger), int(op),
                                      int(precision), int(method), float(tol), int(max_iter), it))
    return list(it)


def lqcd_pf_force_eo(h, F, phi, kappa, rho, term, precision=PREC_F64, tol=1e-10, max_iter=20000):
    S = C.c_double(0)
    _check(h, load().lqcd_pf_force_eo(h, _ptr(F), _ptr(phi), float(kappa), float(rho), int(term), int(precision),
                                      float(tol), int(max_iter), C.byref(S)))
    return S.value


def lqcd_profile_enable(h, on):
    return _check(h, load().lqcd_profile_enable(h, int(bool(on))))


def lqcd_profile_reset(h):
    return _check(h, load().lqcd_profile_reset(h))


def lqcd_gauge_action_static(L, U, beta, out, stream=None):
    """Handle-free, allocation-free gauge action: out (device float64[2])
    receives S_G and the average plaquette.  For callers that cannot
    allocate device memory (see include/lqcd.h); returns the status code."""
    s = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    return load().lqcd_gauge_action_static(C.byref((C.c_int * 4)(*L)), _ptr(U), float(beta), _ptr(out), s)


def lqcd_force_profile(h, F, out):
    return _check(h, load().lqcd_force_profile(h, _ptr(F), _ptr(out)))


def lqcd_launch_count(h):
    n = C.c_int64(0)
    _check(h, load().lqcd_launch_count(h, C.byref(n)))
    return n.value


def lqcd_profile_times(h, kernel_id, cap=65536):
    """per-launch device times (ms) of kernel_id since the last reset"""
    n = C.c_int64(0)
    _check(h, load().lqcd_profile_times(h, int(kernel_id), None, 0, C.byref(n)))
    k = min(cap, n.value)
    buf = (C.c_float * max(k, 1))()
    _check(h, load().lqcd_profile_times(h, int(kernel_id), buf, k, C.byref(n)))
    return list(buf)[:k]


def lqcd_profile_read(h, kernel_id):
    n = C.c_int64(0)
    ms = C.c_double(0)
    by = C.c_double(0)
    _check(h, load().lqcd_profile_read(h, int(kernel_id), C.byref(n), C.byref(ms), C.byref(by)))
    return n.value, ms.value, by.value


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Lattice:
    """A handle on one lattice: L = (L0, L1, L2, L3), x0-slabs of thickness l0
    and, with l0s = l0/2, the sub-slabs of the iterated decomposition."""

    def __init__(self, L, l0, bc_t=-1, stream=None, l0s=0):
        self.L = tuple(int(v) for v in L)
        self.l0 = int(l0)
        self.l0s = int(l0s)
        self.V3 = self.L[1] * self.L[2] * self.L[3]
        self.V = self.L[0] * self.V3
        self.Vh = self.V // 2
        self.nb = self.L[0] // self.l0
        self.nbs = self.L[0] // self.l0s if self.l0s else 0
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.h = lqcd_create(self.L, self.l0, bc_t, stream)
        if self.l0s:
            lqcd_set_subslabs(self.h, self.l0s)

    def close(self):
        if self.h is not None:
            lqcd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spinor(self):
        return torch.zeros((self.V, 4, 3), dtype=torch.complex128, device=self.dev)

    def half(self):
        return torch.zeros((self.Vh, 4, 3), dtype=torch.complex128, device=self.dev)

    def boundary(self):
        return torch.zeros((self.nb // 2, 2, self.V3, 2, 3), dtype=torch.complex128, device=self.dev)

    def boundary2(self):
        return torch.zeros((self.nbs // 2, self.V3, 2, 3), dtype=torch.complex128, device=self.dev)

    def momenta(self):
        return torch.zeros((4, self.V, 8), dtype=torch.float64, device=self.dev)

    def set_gauge(self, U):
        lqcd_set_gauge(self.h, U.contiguous())

    def get_gauge(self):
        U = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=self.dev)
        lqcd_get_gauge(self.h, U)
        return U

    def index_maps(self):
        m = torch.empty((14, self.V), dtype=torch.int32, device=self.dev)
        lqcd_index_maps(self.h, m)
        return m

    def dslash_eo(self, x, parity, kappa=0.0, dagger=0, op=OP_HOP, precision=PREC_F64):
        out = self.half()
        lqcd_dslash_eo(self.h, out, x.contiguous(), kappa, parity, dagger, op, precision)
        return out

    def block_dslash(self, x, kappa, colour=-1, dagger=0, precision=PREC_F64):
        out = self.spinor()
        lqcd_block_dslash(self.h, out, x.contiguous(), kappa, colour, dagger, precision)
        return out

    def block_solve(self, b, kappa, colour=-1, dagger=0, precision=PREC_F64, tol=1e-10, max_iter=10000):
        x = self.spinor()
        it, rs = lqcd_block_solve_batched(self.h, x, b.contiguous(), kappa, colour, dagger, precision,
                                          tol, max_iter, nb=self.nb)
        return x, it, rs

    def subblock_dslash(self, x, kappa, colour=-1, dagger=0, precision=PREC_F64):
        out = self.spinor()
        lqcd_subblock_dslash(self.h, out, x.contiguous(), kappa, colour, dagger, precision)
        return out

    def subblock_solve(self, b, kappa, colour=-1, dagger=0, precision=PREC_F64, tol=1e-10, max_iter=10000):
        x = self.spinor()
        it, rs = lqcd_subblock_solve_batched(self.h, x, b.contiguous(), kappa, colour, dagger, precision,
                                             tol, max_iter, nbs=self.nbs)
        return x, it, rs

    def w3eo(self, x_e, kappa, rho, dagger=0):
        out = self.half()
        lqcd_subblock_eo(self.h, out, x_e.contiguous(), kappa, rho, dagger, EO_APPLY, nbs=self.nbs)
        return out

    def solve_w3eo(self, b_e, kappa, rho, dagger=0, precision=PREC_F64, tol=1e-10, max_iter=10000,
                   method=SOLVER_BICGSTAB):
        x = self.half()
        it = lqcd_subblock_eo(self.h, x, b_e.contiguous(), kappa, rho, dagger, EO_SOLVE, precision, tol, max_iter,
                              nbs=self.nbs, method=method)
        return x, it

    def pf_force_eo(self, phi_e, kappa, rho, term, precision=PREC_F64, tol=1e-10, max_iter=20000, force=True):
        F = self.momenta() if force else None
        S = lqcd_pf_force_eo(self.h, F, phi_e.contiguous(), kappa, rho, term, precision, tol, max_iter)
        return S, F

    def solve(self, b, kappa, dagger=0, precision=PREC_F64, tol=1e-10, max_iter=20000):
        x = self.spinor()
        it, rs = lqcd_solve_wilson(self.h, x, b.contiguous(), kappa, dagger, precision, tol, max_iter)
        return x, it, rs

    def schur(self, c, kappa, op=SCHUR_R, precision=PREC_F64, tol=1e-10, max_iter=20000):
        out = self.boundary2() if op >= SCHUR2_R else self.boundary()
        lqcd_schur_apply(self.h, out, c.contiguous(), kappa, op, precision, tol, max_iter)
        return out

    def pf_force(self, phi, kappa, term, precision=PREC_F64, tol=1e-10, max_iter=20000, force=True):
        F = self.momenta() if force else None
        S = lqcd_pf_force(self.h, F, phi.contiguous(), kappa, term, precision, tol, max_iter)
        return S, F

    def force_profile(self, F):
        """mean |F| per time slice: (2, L0) for space-like / time-like links"""
        out = torch.empty((2, self.L[0]), dtype=torch.float64, device=self.dev)
        lqcd_force_profile(self.h, F.contiguous(), out)
        return out

    def gauge_force(self, beta, force=True):
        F = self.momenta() if force else None
        S, pl = lqcd_gauge_force(self.h, F, beta)
        return S, pl, F

    def link_update(self, U, P, dt):
        """exp(i dt P) U (a new tensor); it also becomes the handle's field"""
        U2 = U.clone().contiguous()
        lqcd_link_update(self.h, U2, P.contiguous(), dt)
        return U2

    def hmc_trajectory(self, U, prm, seed, traj, P0=None, eta1=None, eta2=None):
        U2 = U.clone().contiguous()
        res = lqcd_hmc_trajectory(self.h, U2, prm, seed, traj, P0, eta1, eta2)
        return U2, res

    def md(self, U, P, phi1, phi2, prm, phi3=None, phi4=None, phi_s2=None, phi_s1=None):
        U2 = U.clone().contiguous()
        P2 = P.clone().contiguous()
        lqcd_md(self.h, U2, P2, prm, phi1, phi2, phi3, phi4, phi_s2, phi_s1)
        return U2, P2
