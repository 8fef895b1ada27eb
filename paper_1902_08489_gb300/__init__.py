"""Python binding of the tdmps CUDA library (GB300, sm_103a).

Thin ctypes marshalling around the C ABI declared in ``include/tdmps.h``:
every computation runs in the library's CUDA kernels.  PyTorch supplies the
CUDA stream (``torch.cuda.current_stream()``) and device selection.  If the
compiled library is missing, every entry point raises ``TdmpsError`` -- there
is no Python or CPU fallback.

Entry points keep the names of the C ABI without the ``tdmps_`` prefix
(``tdmps_sum`` is ``mps_sum`` here, to avoid shadowing the builtin).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtdmps.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "tdmps.h")

FP64, TF32, TF32X3, BF16 = 0, 1, 2, 3
PRECISION = {"fp64": FP64, "tf32": TF32, "tf32x3": TF32X3, "bf16": BF16}
KSTAT = {"gemm": 0, "wstage": 1, "qr": 2, "svd": 3, "other": 4, "gemm_fp64": 5,
         "host_plan": 6, "host_launch": 7, "host_sync": 8}
DEVICE_KSTAT = ("gemm", "wstage", "qr", "svd", "other", "gemm_fp64")
ERRORS = {-1: "INVALID_ARG", -2: "SECTOR", -3: "KRYLOV_SINGULAR", -4: "NONFINITE",
          -5: "CUDA", -6: "OOM", -7: "ZERO_STATE", -8: "NUMERIC"}


class TdmpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


class Complex(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class KStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None
P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
I64 = ctypes.c_int64
_SIGS = {
    "tdmps_create": (I, [ctypes.POINTER(P), P, I]),
    "tdmps_destroy": (I, [P]),
    "tdmps_last_error": (ctypes.c_char_p, [P]),
    "tdmps_create_error": (ctypes.c_char_p, []),
    "tdmps_set_precision": (I, [P, I]),
    "tdmps_set_schedule": (I, [P, I, I]),
    "tdmps_set_krylov_fp64": (I, [P, I]),
    "tdmps_set_concurrent_inner": (I, [P, I]),
    "tdmps_build_mpo": (I, [P, P, P, I, I, D, ctypes.POINTER(P)]),
    "tdmps_mpo_info": (I, [P, P, ctypes.POINTER(I64)]),
    "tdmps_mpo_elements": (I, [P, I, ctypes.POINTER(I64), P, P, P, P, P]),
    "tdmps_mpo_free": (I, [P]),
    "tdmps_mps_from_determinant": (I, [P, I, P, ctypes.POINTER(P)]),
    "tdmps_mps_import": (I, [P, I, P, P, P, ctypes.POINTER(P)]),
    "tdmps_mps_export": (I, [P, P, P, P, P]),
    "tdmps_mps_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                           ctypes.POINTER(I)]),
    "tdmps_mps_copy": (I, [P, P, ctypes.POINTER(P)]),
    "tdmps_mps_free": (I, [P]),
    "tdmps_apply_H": (I, [P, P, P, Complex, I, D, I, ctypes.POINTER(P)]),
    "tdmps_energy_gradient": (I, [P, P, P, I, ctypes.POINTER(D), ctypes.POINTER(P),
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "tdmps_heff_create": (I, [P, P, P, I, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)]),
    "tdmps_heff_apply": (I, [P, P, P, P]),
    "tdmps_heff_free": (I, [P]),
    "tdmps_energy": (I, [P, P, P, ctypes.POINTER(D)]),
    "tdmps_integral_gradient": (I, [P, P, P, P]),
    "tdmps_sum": (I, [P, I, P, P, I, D, ctypes.POINTER(P)]),
    "tdmps_overlap": (I, [P, P, P, ctypes.POINTER(Complex)]),
    "tdmps_overlap_noalloc": (I, [P, P, P, ctypes.POINTER(Complex)]),
    "tdmps_expectation": (I, [P, P, P, P, ctypes.POINTER(Complex)]),
    "tdmps_compress": (I, [P, P, I, D, ctypes.POINTER(D)]),
    "tdmps_rk4_step": (I, [P, P, P, D, I, D]),
    "tdmps_krylov_step": (I, [P, P, P, D, I, I, I, D]),
    "tdmps_one_rdm": (I, [P, P, P]),
    "tdmps_transition_rdm": (I, [P, P, P, P]),
    "tdmps_two_rdm": (I, [P, P, P]),
    "tdmps_apply_site_op": (I, [P, P, I, I, I, ctypes.POINTER(P)]),
    "tdmps_green_function": (I, [P, P, P, I, I, D, I, I, I, I, I, D, P]),
    "tdmps_evolve_batch": (I, [P, I, P, P, P, P, P, P, I, I, I, I, P]),
    "tdmps_fiedler_order": (I, [P, P, I, P]),
    "tdmps_stats_enable": (I, [P, I]),
    "tdmps_stats_reset": (I, [P]),
    "tdmps_stats_get": (I, [P, I, ctypes.POINTER(KStat)]),
}


def lib() -> ctypes.CDLL:
    """The loaded C library (raises TdmpsError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TdmpsError(-5, "CUDA library %s is not built; run "
                                 "paper_1902_08489_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Entry points declared in include/tdmps.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(tdmps_\w+)\(", txt, re.M)))


def _check(code, ctx=None):
    if code != 0:
        msg = lib().tdmps_last_error(ctx.h if ctx is not None else None)
        raise TdmpsError(code, (msg or b"").decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """Library context bound to a CUDA stream (default: torch's current)."""

    def __init__(self, precision="fp64", stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise TdmpsError(-5, "no CUDA device available")
        if device is not None:
            torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = getattr(stream, "cuda_stream", stream)
        h = ctypes.c_void_p()
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        code = lib().tdmps_create(ctypes.byref(h), ctypes.c_void_p(handle), prec)
        if code != 0:
            raise TdmpsError(code, lib().tdmps_create_error().decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().tdmps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision):
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(lib().tdmps_set_precision(self.h, prec), self)

    def set_schedule(self, n_two_site: int, n_one_site: int):
        _check(lib().tdmps_set_schedule(self.h, n_two_site, n_one_site), self)

    def set_krylov_fp64(self, on: bool = True):
        _check(lib().tdmps_set_krylov_fp64(self.h, 1 if on else 0), self)

    def set_concurrent_inner(self, on: bool = True):
        _check(lib().tdmps_set_concurrent_inner(self.h, 1 if on else 0), self)

    # statistics
    def stats_enable(self, on=True):
        _check(lib().tdmps_stats_enable(self.h, 1 if on else 0), self)

    def stats_reset(self):
        _check(lib().tdmps_stats_reset(self.h), self)

    def stats(self) -> dict:
        out = {}
        for name, k in KSTAT.items():
            s = KStat()
            _check(lib().tdmps_stats_get(self.h, k, ctypes.byref(s)), self)
            out[name] = dict(launches=s.launches, ms=s.ms, flops=s.flops, bytes=s.bytes)
        return out


class MPO:
    def __init__(self, handle, L):
        self.h = handle
        self.L = L

    def bond_dims(self):
        d = np.zeros(self.L + 1, dtype=np.int32)
        n = ctypes.c_int64()
        _check(lib().tdmps_mpo_info(self.h, _ptr(d), ctypes.byref(n)))
        return d, n.value

    def elements(self, site: int):
        n = ctypes.c_int64(0)
        _check(lib().tdmps_mpo_elements(self.h, site, ctypes.byref(n), None, None, None, None, None))
        a = [np.zeros(n.value, dtype=np.int32) for _ in range(4)]
        v = np.zeros(n.value)
        _check(lib().tdmps_mpo_elements(self.h, site, ctypes.byref(n), *[_ptr(x) for x in a], _ptr(v)))
        return (*a, v)

    def free(self):
        if self.h:
            lib().tdmps_mpo_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class MPS:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle

    def info(self):
        L, n, s, mb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().tdmps_mps_info(self.h, ctypes.byref(L), ctypes.byref(n), ctypes.byref(s),
                                    ctypes.byref(mb)))
        return dict(L=L.value, n_elec=n.value, two_sz=s.value, max_bond=mb.value)

    def export(self):
        """(tensors, labels) as dense complex arrays with bond labels."""
        L = self.info()["L"]
        dims = np.zeros(L + 1, dtype=np.int32)
        _check(lib().tdmps_mps_export(self.ctx.h, self.h, _ptr(dims), None, None), self.ctx)
        labels = np.zeros(2 * int(dims.sum()), dtype=np.int32)
        tens = [np.zeros((dims[i], 4, dims[i + 1]), dtype=np.complex128) for i in range(L)]
        arr = (ctypes.c_void_p * L)(*[t.ctypes.data for t in tens])
        _check(lib().tdmps_mps_export(self.ctx.h, self.h, _ptr(dims), _ptr(labels), arr), self.ctx)
        labs, off = [], 0
        for k in range(L + 1):
            labs.append(labels[2 * off:2 * (off + dims[k])].reshape(-1, 2).astype(np.int64))
            off += dims[k]
        return tens, labs

    def copy(self):
        h = ctypes.c_void_p()
        _check(lib().tdmps_mps_copy(self.ctx.h, self.h, ctypes.byref(h)), self.ctx)
        return MPS(self.ctx, h)

    def free(self):
        if self.h:
            lib().tdmps_mps_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points

def build_mpo(ctx, h, eri, L=None, n_elec=0, e0=0.0) -> MPO:
    """MPO of the Hamiltonian (h: L x L, eri: L^4 chemist order).  ctx may be
    None for a host-only MPO (inspection without a GPU)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    L = h.shape[0] if L is None else L
    out = ctypes.c_void_p()
    _check(lib().tdmps_build_mpo(ctx.h if ctx else None, _ptr(h), _ptr(eri), L, n_elec, e0,
                                 ctypes.byref(out)), ctx)
    return MPO(out, L)


def mps_from_determinant(ctx, occ) -> MPS:
    o = np.ascontiguousarray(occ, dtype=np.uint8)
    out = ctypes.c_void_p()
    _check(lib().tdmps_mps_from_determinant(ctx.h, len(o), _ptr(o), ctypes.byref(out)), ctx)
    return MPS(ctx, out)


def mps_import(ctx, tensors, labels) -> MPS:
    L = len(tensors)
    dims = np.array([len(q) for q in labels], dtype=np.int32)
    lab = np.ascontiguousarray(np.concatenate([np.asarray(q).reshape(-1, 2) for q in labels]),
                               dtype=np.int32)
    tens = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
    arr = (ctypes.c_void_p * L)(*[t.ctypes.data for t in tens])
    out = ctypes.c_void_p()
    _check(lib().tdmps_mps_import(ctx.h, L, _ptr(dims), _ptr(lab), arr, ctypes.byref(out)), ctx)
    return MPS(ctx, out)


def apply_H(ctx, mpo, mps, alpha=1.0, D=64, eps=0.0, n_sweeps=0) -> MPS:
    out = ctypes.c_void_p()
    a = complex(alpha)
    _check(lib().tdmps_apply_H(ctx.h, mpo.h, mps.h, Complex(a.real, a.imag), D, eps, n_sweeps,
                               ctypes.byref(out)), ctx)
    return MPS(ctx, out)


def energy_gradient(ctx, mpo, mps, stride=1):
    """(E, G, env_bytes_peak): E = <psi|H|psi>/<psi|psi> and G, an MPS-shaped
    handle whose site i is dE/dconj(A_i) (read it with G.export())."""
    out = ctypes.c_void_p()
    e = ctypes.c_double()
    peak = ctypes.c_size_t()
    _check(lib().tdmps_energy_gradient(ctx.h, mpo.h, mps.h, stride, ctypes.byref(e),
                                       ctypes.byref(out), ctypes.byref(peak)), ctx)
    return e.value, MPS(ctx, out), peak.value


class LocalHamiltonian:
    """The one-site effective Hamiltonian of a state at one site (environments
    held on the device); see local_hamiltonian."""

    def __init__(self, ctx, handle, site, env_bytes):
        self.ctx = ctx
        self.h = handle
        self.site = site
        self.env_bytes = env_bytes

    def apply(self, x, y):
        """Site `site` of y <- the operator applied to site `site` of x."""
        _check(lib().tdmps_heff_apply(self.ctx.h, self.h, x.h, y.h), self.ctx)

    def free(self):
        if self.h:
            lib().tdmps_heff_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def local_hamiltonian(ctx, mpo, mps, site) -> LocalHamiltonian:
    """H_site: x -> L W_site x R with the environments of <psi|H|psi> around
    `site` (the local problem of a one-site fit step)."""
    out = ctypes.c_void_p()
    nb = ctypes.c_size_t()
    _check(lib().tdmps_heff_create(ctx.h, mpo.h, mps.h, site, ctypes.byref(out),
                                   ctypes.byref(nb)), ctx)
    return LocalHamiltonian(ctx, out, site, nb.value)


def energy(ctx, mpo, mps) -> float:
    """<psi|H|psi> / <psi|psi>."""
    e = ctypes.c_double()
    _check(lib().tdmps_energy(ctx.h, mpo.h, mps.h, ctypes.byref(e)), ctx)
    return e.value


def integral_gradient(ctx, mps, two_body=True):
    """(dE/dh, dE/deri) of <psi|H|psi>/<psi|psi> (dE/deri None unless two_body)."""
    L = mps.info()["L"]
    dh = np.zeros((L, L))
    de = np.zeros((L, L, L, L)) if two_body else None
    _check(lib().tdmps_integral_gradient(ctx.h, mps.h, _ptr(dh),
                                         _ptr(de) if two_body else None), ctx)
    return dh, de


def mps_sum(ctx, coefs, terms, D=64, eps=0.0) -> MPS:
    n = len(terms)
    cs = (Complex * n)(*[Complex(complex(c).real, complex(c).imag) for c in coefs])
    ts = (ctypes.c_void_p * n)(*[t.h.value if isinstance(t.h, ctypes.c_void_p) else t.h for t in terms])
    out = ctypes.c_void_p()
    _check(lib().tdmps_sum(ctx.h, n, cs, ts, D, eps, ctypes.byref(out)), ctx)
    return MPS(ctx, out)


def overlap(ctx, bra, ket) -> complex:
    r = Complex()
    _check(lib().tdmps_overlap(ctx.h, bra.h, ket.h, ctypes.byref(r)), ctx)
    return complex(r.re, r.im)


def overlap_noalloc(ctx, bra, ket) -> complex:
    """<bra|ket> without any device allocation (fixed device scratch)."""
    r = Complex()
    _check(lib().tdmps_overlap_noalloc(ctx.h, bra.h, ket.h, ctypes.byref(r)), ctx)
    return complex(r.re, r.im)


def expectation(ctx, mpo, bra, ket) -> complex:
    r = Complex()
    _check(lib().tdmps_expectation(ctx.h, mpo.h, bra.h, ket.h, ctypes.byref(r)), ctx)
    return complex(r.re, r.im)


def compress(ctx, mps, D, eps=0.0) -> float:
    d = ctypes.c_double()
    _check(lib().tdmps_compress(ctx.h, mps.h, D, eps, ctypes.byref(d)), ctx)
    return d.value


def rk4_step(ctx, mpo, mps, dt, D, eps=0.0):
    _check(lib().tdmps_rk4_step(ctx.h, mpo.h, mps.h, dt, D, eps), ctx)


def krylov_step(ctx, mpo, mps, dt, m, orthogonal=True, D=64, eps=0.0):
    _check(lib().tdmps_krylov_step(ctx.h, mpo.h, mps.h, dt, m, 1 if orthogonal else 0, D, eps), ctx)


def one_rdm(ctx, mps) -> np.ndarray:
    L = mps.info()["L"]
    g = np.zeros((L, L), dtype=np.complex128)
    _check(lib().tdmps_one_rdm(ctx.h, mps.h, _ptr(g)), ctx)
    return g


def transition_rdm(ctx, bra, ket) -> np.ndarray:
    """T_ij = sum_s <bra| c+_is c_js |ket>."""
    L = bra.info()["L"]
    g = np.zeros((L, L), dtype=np.complex128)
    _check(lib().tdmps_transition_rdm(ctx.h, bra.h, ket.h, _ptr(g)), ctx)
    return g


def two_rdm(ctx, mps) -> np.ndarray:
    """Gamma_ijkl = sum_st <psi| c+_is c+_kt c_lt c_js |psi> (L^4)."""
    L = mps.info()["L"]
    g = np.zeros((L, L, L, L), dtype=np.complex128)
    _check(lib().tdmps_two_rdm(ctx.h, mps.h, _ptr(g)), ctx)
    return g


def apply_site_op(ctx, mps, site, spin, dagger=False) -> MPS:
    """c_(site, spin)|mps> or c+_(site, spin)|mps> exactly (spin 0 up, 1 down)."""
    out = ctypes.c_void_p()
    _check(lib().tdmps_apply_site_op(ctx.h, mps.h, site, spin, 1 if dagger else 0,
                                     ctypes.byref(out)), ctx)
    return MPS(ctx, out)


def green_function(ctx, mpo, psi0, i, j, dt, n_steps, method="krylov", m=10, orthogonal=True,
                   D=64, eps=0.0) -> np.ndarray:
    """G_ij(n dt), n = 0..n_steps, of Eq. (green_time) (backward propagation)."""
    g = np.zeros(n_steps + 1, dtype=np.complex128)
    meth = {"krylov": 0, "rk4": 1}[method]
    _check(lib().tdmps_green_function(ctx.h, mpo.h, psi0.h, i, j, dt, n_steps, meth, m,
                                      1 if orthogonal else 0, D, eps, _ptr(g)), ctx)
    return g


def evolve_batch(ctx, mpos, states, dt, n_steps, D, eps=0.0, method="rk4", m=10,
                 orthogonal=True, n_workers=0, raise_on_error=True) -> np.ndarray:
    """Advance many independent states in place (per-item dt, n_steps, D,
    eps may be scalars or sequences).  Returns the per-item status codes;
    with raise_on_error, raises TdmpsError for the first failed item after
    all items ran."""
    n = len(states)
    arr = lambda x, dt_: np.ascontiguousarray(np.broadcast_to(np.asarray(x), (n,)), dtype=dt_)
    dts, ns, Ds, es = arr(dt, np.float64), arr(n_steps, np.int32), arr(D, np.int32), arr(eps, np.float64)
    hm = (ctypes.c_void_p * n)(*[p.h.value if isinstance(p.h, ctypes.c_void_p) else p.h for p in mpos])
    hs = (ctypes.c_void_p * n)(*[p.h.value if isinstance(p.h, ctypes.c_void_p) else p.h for p in states])
    status = np.zeros(n, dtype=np.int32)
    meth = {"krylov": 0, "rk4": 1}[method]
    rc = lib().tdmps_evolve_batch(ctx.h, n, hm, hs, _ptr(dts), _ptr(ns), _ptr(Ds), _ptr(es), meth,
                                  m, 1 if orthogonal else 0, n_workers, _ptr(status))
    if raise_on_error:
        _check(rc, ctx)
    return status


def fiedler_order(h, eri) -> np.ndarray:
    """Fiedler ordering of the orbitals: perm[k] = orbital at position k."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    L = h.shape[0]
    perm = np.zeros(L, dtype=np.int32)
    rc = lib().tdmps_fiedler_order(_ptr(h), _ptr(eri), L, _ptr(perm))
    if rc != 0:
        raise TdmpsError(rc, (lib().tdmps_create_error() or b"").decode())
    return perm.astype(np.int64)


def permute_integrals(h, eri, perm):
    """Integrals in the orbital order perm (perm[k] = old orbital at k)."""
    p = np.asarray(perm)
    return np.asarray(h)[np.ix_(p, p)], np.asarray(eri)[np.ix_(p, p, p, p)]
