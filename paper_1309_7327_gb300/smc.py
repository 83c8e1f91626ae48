"""Python binding of the C ABI in include/smc.h (ctypes; marshalling only).

Every computation runs in ``libsmc.so``'s CUDA kernels.  There is no CPU
fallback: importing this module without the built library raises.

Functions with the C names (``smc_create``, ``smc_rhs``, ``smc_sdc_step``,
``smc_prim_to_cons``, ``smc_destroy`` ...) are exposed as-is; the ``Smc``
class wraps a handle and accepts PyTorch CUDA tensors (used in place, on the
handle's stream) or NumPy arrays (staged by the library through device
buffers).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmc.so")

SMC_OK, SMC_ERR_ARG, SMC_ERR_CUDA, SMC_ERR_OOM = 0, 1, 2, 3
SMC_ERR_NONCONVERGED, SMC_ERR_NONPHYSICAL, SMC_ERR_TIMEOUT, SMC_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "SMC_OK", 1: "SMC_ERR_ARG", 2: "SMC_ERR_CUDA", 3: "SMC_ERR_OOM",
                4: "SMC_ERR_NONCONVERGED", 5: "SMC_ERR_NONPHYSICAL", 6: "SMC_ERR_TIMEOUT",
                7: "SMC_ERR_STATE"}

OPT = dict(precision=0, m47=1, m48=2, diffusion_mode=3, ref_species=4, xi_ratio=5,
           newton_tol=6, newton_maxit=7, t_guess=8, reactions=9, segment=10, profile=11,
           use_graphs=12, x_layout=13, march=14, rates=15,
           fine_repeat=16, sdc_exit=17, chain_blocks=18, mr_mode=19, bdf_rtol=20, bdf_atol=21,
           persistent=22, alu=23)
KERNELS = ["prim", "grad", "march", "final", "update", "fine", "chem", "other", "bdf"]

EXPORTS = ["smc_create", "smc_destroy", "smc_rhs", "smc_sdc_step", "smc_prim_to_cons", "smc_autotune",
           "smc_set_stream", "smc_set_option", "smc_get_stats", "smc_synchronize",
           "smc_invalidate", "smc_collocation", "smc_multirate_collocation", "smc_rhs_noalloc",
           "smc_exp", "smc_dmul", "smc_heat2d", "smc_react_integrate", "smc_fma_throughput",
           "smc_last_error"]


class smc_grid(C.Structure):
    _fields_ = [("nboxes", C.c_int), ("lo", C.POINTER(C.c_int)), ("hi", C.POINTER(C.c_int)),
                ("domain", C.c_int * 3), ("dx", C.c_double * 3)]


class smc_mechanism(C.Structure):
    _fields_ = [("nspecies", C.c_int), ("nreactions", C.c_int),
                ("W", C.POINTER(C.c_double)), ("nasa7", C.POINTER(C.c_double)),
                ("nu_f", C.POINTER(C.c_int)), ("nu_r", C.POINTER(C.c_int)),
                ("A", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("Ea", C.POINTER(C.c_double)), ("Le", C.POINTER(C.c_double)),
                ("eta_ref", C.c_double), ("T_ref", C.c_double), ("eta_exp", C.c_double),
                ("Pr", C.c_double)]


SMC_BC_PERIODIC, SMC_BC_OUTFLOW = 0, 1


class smc_bc(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3)]


class smc_stats(C.Structure):
    _fields_ = [("n_rhs", C.c_longlong), ("n_react", C.c_longlong), ("n_steps", C.c_longlong),
                ("device_flags", C.c_uint), ("nvars", C.c_int), ("ncells", C.c_longlong),
                ("device_bytes", C.c_longlong), ("launches", C.c_longlong * 9),
                ("kernel_ms", C.c_double * 9), ("sweeps_done", C.c_int),
                ("residual", C.c_double * 64), ("bdf_steps", C.c_longlong),
                ("bdf_rejected", C.c_longlong), ("bdf_newton_failures", C.c_longlong),
                ("bdf_evals", C.c_longlong), ("bdf_max_steps", C.c_longlong),
                ("schedule", C.c_int * 4)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1309_7327_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, dp = C.c_void_p, C.c_double
    lib.smc_create.argtypes = [C.POINTER(smc_grid), C.POINTER(smc_mechanism), C.POINTER(smc_bc),
                               C.POINTER(vp)]
    lib.smc_destroy.argtypes = [vp]
    lib.smc_rhs.argtypes = [vp, vp, vp]
    lib.smc_sdc_step.argtypes = [vp, vp, dp, C.c_int, C.c_int, C.c_int]
    lib.smc_prim_to_cons.argtypes = [vp, vp, vp]
    lib.smc_set_stream.argtypes = [vp, vp]
    lib.smc_set_option.argtypes = [vp, C.c_int, dp]
    lib.smc_get_stats.argtypes = [vp, C.POINTER(smc_stats)]
    lib.smc_synchronize.argtypes = [vp]
    lib.smc_invalidate.argtypes = [vp]
    lib.smc_autotune.argtypes = [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.smc_collocation.argtypes = [C.c_int, vp, vp]
    lib.smc_multirate_collocation.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
    lib.smc_heat2d.argtypes = [C.c_int, dp, vp, vp, vp, dp, dp, dp, dp, C.c_int, C.c_int, C.c_int,
                               vp, C.POINTER(C.c_longlong), vp]
    lib.smc_exp.argtypes = [vp, vp, C.c_longlong, C.c_int]
    lib.smc_dmul.argtypes = [vp, vp, vp, C.c_longlong]
    lib.smc_dmul.restype = C.c_int
    lib.smc_react_integrate.argtypes = [vp, vp, vp, dp, vp]
    lib.smc_exp.restype = C.c_int
    lib.smc_rhs_noalloc.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(smc_mechanism), vp, vp, vp]
    lib.smc_fma_throughput.argtypes = [C.c_int, C.c_longlong, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.smc_last_error.argtypes = [vp]
    lib.smc_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name != "smc_last_error":
            getattr(lib, name).restype = C.c_int
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


# C-named entry points (thin pass-throughs)
def smc_create(grid, mech, bc, out):
    return lib().smc_create(grid, mech, bc, out)


def smc_destroy(h):
    return lib().smc_destroy(h)


def smc_rhs(h, U, dUdt):
    return lib().smc_rhs(h, U, dUdt)


def smc_sdc_step(h, U, dt, nodes, sweeps, reaction_substeps):
    return lib().smc_sdc_step(h, U, dt, nodes, sweeps, reaction_substeps)


def smc_prim_to_cons(h, prim, U):
    return lib().smc_prim_to_cons(h, prim, U)


def smc_collocation(nodes: int):
    """(tau, S) of smc_collocation as NumPy arrays."""
    tau = np.zeros(nodes)
    S = np.zeros((nodes - 1, nodes))
    st = lib().smc_collocation(nodes, C.c_void_p(tau.ctypes.data), C.c_void_p(S.ctypes.data))
    if st != SMC_OK:
        raise SmcError(st, "smc_collocation")
    return tau, S


def smc_multirate_collocation(coarse: int, fine: int, repeat: int = 1):
    """(t1, t2, S21, S22) of smc_multirate_collocation as NumPy arrays."""
    M2 = (coarse - 1) * (fine - 1) * max(repeat, 1)
    t1, t2 = np.zeros(coarse), np.zeros(M2 + 1)
    S21, S22 = np.zeros((M2, coarse)), np.zeros((M2, M2 + 1))
    st = lib().smc_multirate_collocation(coarse, fine, repeat,
                                         *(C.c_void_p(a.ctypes.data) for a in (t1, t2, S21, S22)))
    if st != SMC_OK:
        raise SmcError(st, "smc_multirate_collocation")
    return t1, t2, S21, S22


def smc_heat2d(N, h, a, b, G, u, t0, dt, nsteps, m47=3557.0 / 44100.0, m48=-2083.0 / 117600.0,
               nodes=3, sweeps=4, stream=None):
    """Advance the App. A heat problem in place (see smc.h); a, b, G (or
    None), u: CUDA float64 tensors of N*N elements.  Returns the number of
    operator evaluations."""
    for arr in (a, b, G, u):
        if arr is not None and arr.numel() != int(N) * int(N):
            raise ValueError(f"heat arrays need {int(N) * int(N)} values")
    ev = C.c_longlong(0)
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().smc_heat2d(int(N), float(h), _ptr(a), _ptr(b), _ptr(G) if G is not None else None,
                          float(m47), float(m48), float(t0), float(dt), int(nsteps), int(nodes),
                          int(sweeps), _ptr(u), C.byref(ev), C.c_void_p(raw))
    if st != SMC_OK:
        raise SmcError(st, "smc_heat2d")
    return ev.value


def smc_dmul(a, b, y):
    """y = a * b elementwise by the library's integer-pipe product (CUDA
    float64 tensors of equal size); synchronous."""
    if not (a.numel() == b.numel() <= y.numel()):
        raise ValueError("a, b and y must have the same size")
    st = lib().smc_dmul(_ptr(a), _ptr(b), _ptr(y), C.c_longlong(a.numel()))
    if st != SMC_OK:
        raise SmcError(st, "smc_dmul")
    return y


def smc_exp(x, y, variant=0):
    """y = exp(x) elementwise by one of the library's exponentials (CUDA
    float64 tensors of equal size): 0 the FP64 table method, 1 the integer /
    FP32 one; synchronous."""
    if y.numel() < x.numel():
        raise ValueError("y is smaller than x")
    st = lib().smc_exp(_ptr(x), _ptr(y), C.c_longlong(x.numel()), int(variant))
    if st != SMC_OK:
        raise SmcError(st, "smc_exp")
    return y


def smc_fma_throughput(kind: int, iters: int):
    """Measured FMA-pipe throughput of the current device (kind 0 FP64, 1 FP32,
    2 paired FP32): returns (flop/s, ms of the timed launch, SM count)."""
    fl, ms, sms = C.c_double(), C.c_double(), C.c_int()
    st = lib().smc_fma_throughput(int(kind), C.c_longlong(int(iters)), C.byref(fl), C.byref(ms),
                                  C.byref(sms))
    if st != SMC_OK:
        raise SmcError(st, "smc_fma_throughput")
    return fl.value, ms.value, sms.value


def mechanism_struct(mech):
    """(smc_mechanism, keep-alive list) for a synth.Mechanism-like object;
    the struct points into the arrays of the list."""
    keep = []

    def arr(a, t):
        a = np.ascontiguousarray(a, dtype=t)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int if t == np.int32 else C.c_double))
    m = smc_mechanism()
    m.nspecies, m.nreactions = mech.ns, mech.nr
    m.W, m.nasa7 = arr(mech.W, np.float64), arr(np.asarray(mech.nasa7).reshape(-1), np.float64)
    m.nu_f = arr(np.asarray(mech.nu_f).reshape(-1), np.int32)
    m.nu_r = arr(np.asarray(mech.nu_r).reshape(-1), np.int32)
    m.A, m.b, m.Ea, m.Le = (arr(mech.A, np.float64), arr(mech.b, np.float64),
                            arr(mech.Ea, np.float64), arr(mech.Le, np.float64))
    m.eta_ref, m.T_ref, m.eta_exp, m.Pr = mech.eta_ref, mech.T_ref, mech.eta_exp, mech.Pr
    return m, keep


def smc_rhs_noalloc(n, dx, mech, U, dUdt, stream=None):
    """The allocation-free right-hand side of one periodic box (see smc.h).
    n, dx: 3-sequences; mech: a synth.Mechanism-like object; U, dUdt: CUDA
    tensors in the box layout, on one device."""
    m, keep = mechanism_struct(mech)
    nn = (C.c_int * 3)(*[int(v) for v in n])
    dd = (C.c_double * 3)(*[float(v) for v in dx])
    raw = getattr(stream, "cuda_stream", stream)
    need = (5 + mech.ns) * int(n[0]) * int(n[1]) * int(n[2])
    for a in (U, dUdt):
        if not getattr(a, "is_cuda", False):
            raise ValueError("U and dUdt must be CUDA tensors (the call stages nothing)")
        if a.device != U.device:
            raise ValueError("U and dUdt must be on the same device")
        if a.numel() != need:
            raise ValueError(f"expected {need} values, got {a.numel()}")
    import torch
    with torch.cuda.device(U.device):
        st = lib().smc_rhs_noalloc(nn, dd, C.byref(m), _ptr(U), _ptr(dUdt), C.c_void_p(raw))
    if st != SMC_OK:
        raise SmcError(st, "smc_rhs_noalloc")
    return dUdt


class SmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _ptr(a):
    """Data pointer of a torch tensor or NumPy array (contiguous float64)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) != "torch.float64":
            raise ValueError("tensor must be float64")
        return C.c_void_p(a.data_ptr())
    if not (a.flags["C_CONTIGUOUS"] and a.dtype == np.float64):
        raise ValueError("array must be C-contiguous float64")
    return C.c_void_p(a.ctypes.data)


class Smc:
    """A library handle for one box layout and mechanism on the current GPU."""

    def __init__(self, grid, mech, options: dict | None = None, x_outflow: bool = False,
                 bc: tuple | None = None):
        """x_outflow: non-periodic x ends (boundary-lowered stencils).  bc:
        explicit (lo[3], hi[3]) boundary kinds (SMC_BC_*), overriding it."""
        L = lib()
        self._keep = []

        def arr(a, t):
            a = np.ascontiguousarray(a, dtype=t)
            self._keep.append(a)
            ct = C.c_int if t == np.int32 else C.c_double
            return a.ctypes.data_as(C.POINTER(ct))

        g = smc_grid()
        g.nboxes = grid.nboxes
        g.lo = arr(np.asarray(grid.lo).reshape(-1), np.int32)
        g.hi = arr(np.asarray(grid.hi).reshape(-1), np.int32)
        for d in range(3):
            g.domain[d] = int(grid.domain[d])
            g.dx[d] = float(grid.dx[d])
        m = smc_mechanism()
        m.nspecies = mech.ns
        m.nreactions = mech.nr
        m.W = arr(mech.W, np.float64)
        m.nasa7 = arr(np.asarray(mech.nasa7).reshape(-1), np.float64)
        m.nu_f = arr(np.asarray(mech.nu_f).reshape(-1), np.int32)
        m.nu_r = arr(np.asarray(mech.nu_r).reshape(-1), np.int32)
        m.A = arr(mech.A, np.float64)
        m.b = arr(mech.b, np.float64)
        m.Ea = arr(mech.Ea, np.float64)
        m.Le = arr(mech.Le, np.float64)
        m.eta_ref, m.T_ref, m.eta_exp, m.Pr = mech.eta_ref, mech.T_ref, mech.eta_exp, mech.Pr
        b = smc_bc()
        if bc is not None:
            for d in range(3):
                b.lo[d], b.hi[d] = int(bc[0][d]), int(bc[1][d])
        elif x_outflow:
            b.lo[0] = b.hi[0] = SMC_BC_OUTFLOW
        self.h = C.c_void_p()
        st = L.smc_create(C.byref(g), C.byref(m), C.byref(b), C.byref(self.h))
        self._keep = []
        if st != SMC_OK:
            msg = L.smc_last_error(self.h).decode() if self.h else ""
            if self.h:
                L.smc_destroy(self.h)
                self.h = C.c_void_p()
            raise SmcError(st, msg)
        self.ns = mech.ns
        self.nv = 5 + mech.ns
        self.ncells = grid.ncells
        # precision first: the per-precision options (x_layout, march) apply to it
        for k, v in sorted((options or {}).items(), key=lambda kv: kv[0] != "precision"):
            self.set_option(k, v)

    def _check(self, st):
        if st != SMC_OK:
            raise SmcError(st, lib().smc_last_error(self.h).decode())

    def set_option(self, key, value):
        self._check(lib().smc_set_option(self.h, OPT[key] if isinstance(key, str) else key,
                                         float(value)))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or raw cudaStream_t integer)."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(lib().smc_set_stream(self.h, C.c_void_p(raw)))

    def _state(self, a):
        """The pointer of a state-shaped array: NV x cells float64 (the C ABI
        takes raw pointers and cannot check sizes itself)."""
        n = a.numel() if hasattr(a, "numel") else a.size
        if n != self.nv * self.ncells:
            raise ValueError(f"expected {self.nv} x {self.ncells} values, got {n}")
        return _ptr(a)

    def rhs(self, U, out):
        self._check(lib().smc_rhs(self.h, self._state(U), self._state(out)))
        return out

    def sdc_step(self, U, dt, nodes=3, sweeps=4, reaction_substeps=0):
        self._check(lib().smc_sdc_step(self.h, self._state(U), float(dt), nodes, sweeps,
                                       reaction_substeps))
        return U

    def react_integrate(self, U, G, dt, out):
        """out = U(dt) of dU/dtau = R(U) + G per cell (implicit BDF; G may be
        None).  Device tensors of the state's shape; out may be U."""
        self._check(lib().smc_react_integrate(self.h, self._state(U),
                                              self._state(G) if G is not None else None,
                                              float(dt), self._state(out)))
        return out

    def prim_to_cons(self, prim, out):
        self._check(lib().smc_prim_to_cons(self.h, self._state(prim), self._state(out)))
        return out

    def autotune(self, U) -> dict:
        """Pick the fastest stencil segment length, x-line layout and line
        kernel at U."""
        seg, xl, mv = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().smc_autotune(self.h, self._state(U), C.byref(seg), C.byref(xl),
                                       C.byref(mv)))
        return {"segment": seg.value, "x_layout": xl.value, "march": mv.value,
                "persistent": self.stats()["schedule"][3]}

    def synchronize(self):
        self._check(lib().smc_synchronize(self.h))

    def invalidate(self):
        self._check(lib().smc_invalidate(self.h))

    def stats(self) -> dict:
        s = smc_stats()
        self._check(lib().smc_get_stats(self.h, C.byref(s)))
        out = {f: getattr(s, f) for f, _ in smc_stats._fields_}
        out["launches"] = dict(zip(KERNELS, list(s.launches)))
        out["kernel_ms"] = dict(zip(KERNELS, list(s.kernel_ms)))
        out["residual"] = list(s.residual)[:max(s.sweeps_done, 0)]
        out["schedule"] = list(s.schedule)
        return out

    def close(self):
        if self.h:
            lib().smc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
