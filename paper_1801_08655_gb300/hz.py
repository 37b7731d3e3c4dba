"""Thin Python binding of the C ABI in ``include/hz.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``_lib/libhz.so``; this module only
loads it, converts arguments and checks status codes.  There is no fallback: if the
library is missing, importing the binding raises.  PyTorch is used for device memory
and streams (complex128 tensors are passed by pointer; their interleaved (re, im)
layout is the ABI's complex layout).
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhz.so")

HZ_OK, HZ_ERR_ARG, HZ_ERR_OOM, HZ_ERR_ADMISSION, HZ_ERR_STATE, HZ_ERR_NONFINITE, HZ_ERR_PIVOT, \
    HZ_ERR_NO_CONVERGENCE, HZ_ERR_TIMEOUT, HZ_ERR_CUDA = range(10)
STATUS_NAMES = ["HZ_OK", "HZ_ERR_ARG", "HZ_ERR_OOM", "HZ_ERR_ADMISSION", "HZ_ERR_STATE", "HZ_ERR_NONFINITE",
                "HZ_ERR_PIVOT", "HZ_ERR_NO_CONVERGENCE", "HZ_ERR_TIMEOUT", "HZ_ERR_CUDA"]
PREC = {"fp64": 0, "mixed": 1, "mixed64": 2}

EXPORTED = [
    "hz_default_opts", "hz_create", "hz_create_ex", "hz_factor", "hz_solve", "hz_solve_host", "hz_destroy", "hz_last_error",
    "hz_layer_info", "hz_factor_stats", "hz_layer_solve_cost", "hz_layer_solve", "hz_polarized_rhs",
    "hz_apply_mpol", "hz_apply_precond", "hz_reconstruct", "hz_volume_residual",
    "hz_profile_begin", "hz_profile_begin_detail", "hz_profile_end", "hz_profile_kernel", "hz_profile_report", "hz_kernel_launches", "hz_volume_residual_noalloc",
    "hz_tuning_report", "hz_solve_group", "hz_create_shared", "hz_tensor_peak", "hz_factor_report",
    "hz_trace_blocks", "hz_symbolic_shape",
]


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("h", ct.c_double)]


class Pml(ct.Structure):
    _fields_ = [("npml", ct.c_int32), ("C", ct.c_double), ("npml_local", ct.c_int32)]


class SolveOpts(ct.Structure):
    _fields_ = [("gmres_tol", ct.c_double), ("restart", ct.c_int32), ("max_iter", ct.c_int32),
                ("refine_tol", ct.c_double), ("max_refine", ct.c_int32), ("krylov", ct.c_int32)]


class SolveInfo(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("refinements", ct.c_int32), ("trace_relres", ct.c_double),
                ("volume_relres", ct.c_double), ("ms_total", ct.c_float), ("iters_total", ct.c_int32)]


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Load libhz.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_1801_08655_gb300.build.build()")
    lib = ct.CDLL(path)
    P, I32, D, VP = ct.POINTER, ct.c_int32, ct.c_double, ct.c_void_p
    lib.hz_default_opts.argtypes = [ct.c_int, P(SolveOpts)]
    lib.hz_default_opts.restype = None
    lib.hz_create.argtypes = [P(Grid), VP, D, P(Pml), I32, ct.c_int, VP, P(VP)]
    lib.hz_create_ex.argtypes = [P(Grid), VP, VP, D, P(Pml), I32, ct.c_int, VP, P(VP)]
    lib.hz_factor.argtypes = [VP]
    lib.hz_solve.argtypes = [VP, VP, I32, VP, P(SolveOpts), P(SolveInfo)]
    lib.hz_solve_host.argtypes = [VP, VP, I32, VP, P(SolveOpts), P(SolveInfo)]
    lib.hz_destroy.argtypes = [VP]
    lib.hz_last_error.argtypes = [VP]
    lib.hz_last_error.restype = ct.c_char_p
    lib.hz_layer_info.argtypes = [VP, I32, P(I32), P(I32), P(I32), P(I32)]
    lib.hz_factor_stats.argtypes = [VP, P(ct.c_int64), P(ct.c_int64), P(D), P(ct.c_int64), P(ct.c_float)]
    lib.hz_layer_solve_cost.argtypes = [VP, I32, P(D), P(D)]
    lib.hz_layer_solve.argtypes = [VP, I32, VP, I32, VP]
    lib.hz_polarized_rhs.argtypes = [VP, VP, I32, VP]
    lib.hz_apply_mpol.argtypes = [VP, VP, I32, VP]
    lib.hz_apply_precond.argtypes = [VP, VP, I32, VP]
    lib.hz_reconstruct.argtypes = [VP, VP, VP, I32, VP]
    lib.hz_volume_residual.argtypes = [VP, VP, VP, I32, VP, P(D)]
    lib.hz_volume_residual_noalloc.argtypes = [VP, VP, VP, I32, VP, P(D)]
    lib.hz_profile_begin.argtypes = [VP]
    lib.hz_profile_begin_detail.argtypes = [VP]
    lib.hz_profile_end.argtypes = [VP, P(ct.c_int64), P(D), P(D), P(D)]
    lib.hz_profile_kernel.argtypes = [VP, I32, P(ct.c_int64), P(D), P(D), P(D)]
    lib.hz_kernel_launches.argtypes = []
    lib.hz_tuning_report.argtypes = [VP]
    lib.hz_profile_report.argtypes = [VP]
    lib.hz_create_shared.argtypes = [VP, VP, P(VP)]
    lib.hz_solve_group.argtypes = [P(VP), I32, P(VP), P(I32), P(VP), P(SolveOpts), P(VP), P(ct.c_int)]
    lib.hz_tensor_peak.argtypes = [I32, I32, D, P(D), P(D)]
    lib.hz_trace_blocks.argtypes = [VP, I32, P(ct.c_int64)]
    lib.hz_symbolic_shape.argtypes = [I32, I32, I32, I32, P(ct.c_int64), P(ct.c_int64), VP, VP, VP, VP, VP, VP]
    lib.hz_factor_report.argtypes = [VP]
    lib.hz_factor_report.restype = ct.c_char_p
    for name in EXPORTED:
        if name not in ("hz_default_opts", "hz_last_error", "hz_kernel_launches", "hz_tuning_report",
                        "hz_profile_report", "hz_factor_report"):
            getattr(lib, name).restype = ct.c_int
    lib.hz_kernel_launches.restype = ct.c_int64
    lib.hz_tuning_report.restype = ct.c_char_p
    lib.hz_profile_report.restype = ct.c_char_p
    _lib = lib
    return lib


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None else 0


def default_opts(precision: str = "mixed") -> SolveOpts:
    o = SolveOpts()
    load().hz_default_opts(PREC[precision], ct.byref(o))
    return o


class Solver:
    """One (grid, m, omega, PML, layers, precision) problem with resident factors."""

    def __init__(self, m: np.ndarray, omega: float, npml: int, C: float, n_layers: int,
                 precision: str = "mixed", npml_local: int = -1, h: float = 1.0, stream=None,
                 b: Optional[np.ndarray] = None):
        """b: optional 1/rho on the grid (variable density, hz_create_ex); None for constant density."""
        import torch
        self.lib = load()
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64))
        if b is not None:
            b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
            assert b.shape == m.shape
        nz, ny, nx = m.shape
        self.shape = (nz, ny, nx)
        self.precision = precision
        self.n_layers = n_layers
        self.K = n_layers - 1
        self.P = nx * ny
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = Grid(nx, ny, nz, h)
        p = Pml(npml, C, npml_local)
        hnd = ct.c_void_p()
        st = self.lib.hz_create_ex(ct.byref(g), m.ctypes.data, b.ctypes.data if b is not None else None, omega,
                                   ct.byref(p), n_layers, PREC[precision], ct.c_void_p(self.stream.cuda_stream),
                                   ct.byref(hnd))
        if st != HZ_OK:
            raise HzError(st, self.lib.hz_last_error(None).decode())
        self.h = hnd

    @classmethod
    def shared(cls, src: "Solver", stream=None) -> "Solver":
        """A second handle on src's resident factors with its own workspaces and stream."""
        import torch
        obj = cls.__new__(cls)
        obj.lib = src.lib
        obj.shape, obj.precision, obj.n_layers, obj.K, obj.P = src.shape, src.precision, src.n_layers, src.K, src.P
        obj.stream = stream if stream is not None else torch.cuda.Stream()
        hnd = ct.c_void_p()
        st = obj.lib.hz_create_shared(src.h, ct.c_void_p(obj.stream.cuda_stream), ct.byref(hnd))
        if st != HZ_OK:
            raise HzError(st, obj.lib.hz_last_error(src.h).decode())
        obj.h = hnd
        obj._src = src  # keep the factor owner alive
        return obj

    # -------------------------------------------------------------------- plumbing
    def _check(self, st: int, allow=(HZ_OK,)):
        if st not in allow:
            raise HzError(st, self.lib.hz_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.hz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------------- main path
    def factor(self):
        self._check(self.lib.hz_factor(self.h))

    def solve(self, rhs, opts: Optional[SolveOpts] = None, u=None, allow_noconv: bool = False):
        """rhs: complex128 CUDA tensor (R, nz, ny, nx).  Returns (u, [SolveInfo]*R, status)."""
        import torch
        self._check_volume(rhs)
        R = rhs.shape[0]
        if u is None:
            u = torch.empty_like(rhs)
        self._check_volume(rhs, u)
        info = (SolveInfo * R)()
        st = self.lib.hz_solve(self.h, _ptr(rhs), R, _ptr(u), ct.byref(opts) if opts else None, info)
        self._check(st, (HZ_OK, HZ_ERR_NO_CONVERGENCE) if allow_noconv else (HZ_OK,))
        return u, list(info), st

    def solve_host(self, rhs: np.ndarray, opts: Optional[SolveOpts] = None, u: Optional[np.ndarray] = None,
                   allow_noconv: bool = False):
        """Host (numpy complex128) rhs and u: the end-to-end entry point."""
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        if rhs.ndim != 4 or tuple(rhs.shape[1:]) != self.shape:
            raise ValueError(f"expected rhs of shape (R,) + {self.shape}, got {rhs.shape}")
        R = rhs.shape[0]
        if u is None:
            u = np.empty_like(rhs)
        if not (isinstance(u, np.ndarray) and u.dtype == np.complex128 and u.flags.c_contiguous
                and u.shape == rhs.shape):
            raise ValueError(f"u must be a C-contiguous complex128 array of shape {rhs.shape}")
        info = (SolveInfo * R)()
        st = self.lib.hz_solve_host(self.h, rhs.ctypes.data, R, u.ctypes.data,
                                    ct.byref(opts) if opts else None, info)
        self._check(st, (HZ_OK, HZ_ERR_NO_CONVERGENCE) if allow_noconv else (HZ_OK,))
        return u, list(info), st

    def trace_blocks(self, max_cols: int = 32) -> int:
        """Explicit trace-to-trace Green's blocks (hz_trace_blocks): M_pol and the preconditioner
        use dense block products for solves of at most max_cols right-hand sides; 0 releases the
        blocks.  Returns the device bytes they hold."""
        nb = ct.c_int64()
        self._check(self.lib.hz_trace_blocks(self.h, int(max_cols), ct.byref(nb)))
        return nb.value

    # -------------------------------------------------------------------- introspection
    def layer_info(self, ell: int):
        v = [ct.c_int32() for _ in range(4)]
        self._check(self.lib.hz_layer_info(self.h, ell, *[ct.byref(x) for x in v]))
        return tuple(x.value for x in v)  # lo, hi, zlo, zhi

    def factor_stats(self):
        a, b, d = ct.c_int64(), ct.c_int64(), ct.c_int64()
        f, ms = ct.c_double(), ct.c_float()
        self._check(self.lib.hz_factor_stats(self.h, ct.byref(a), ct.byref(b), ct.byref(f), ct.byref(d),
                                             ct.byref(ms)))
        return dict(nodes=a.value, factor_entries=b.value, factor_flops=f.value, workspace_bytes=d.value,
                    factor_ms=ms.value)

    def layer_solve_cost(self, ell: int):
        b, f = ct.c_double(), ct.c_double()
        self._check(self.lib.hz_layer_solve_cost(self.h, ell, ct.byref(b), ct.byref(f)))
        return b.value, f.value

    # -------------------------------------------------------------------- stages
    def layer_solve(self, ell: int, g):
        """g: complex128 CUDA tensor (ncols, nzl, ny, nx) on layer ell's local grid."""
        import torch
        lo, hi, zlo, zhi = self.layer_info(ell)
        nz, ny, nx = self.shape
        if not (g.is_cuda and g.dtype == torch.complex128 and g.is_contiguous() and g.dim() == 4
                and tuple(g.shape[1:]) == (zhi - zlo + 1, ny, nx)):
            raise ValueError(f"expected a contiguous complex128 CUDA tensor of shape (ncols, {zhi - zlo + 1}, {ny}, {nx})")
        w = torch.empty_like(g)
        self._check(self.lib.hz_layer_solve(self.h, ell, _ptr(g), g.shape[0], _ptr(w)))
        return w

    def trace_shape(self, R: int):
        nz, ny, nx = self.shape
        return (R, 2, self.K, 2, ny, nx)

    def _check_traces(self, x, shape):
        import torch
        if not (x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous() and tuple(x.shape) == tuple(shape)):
            raise ValueError(f"expected a contiguous complex128 CUDA tensor of shape {tuple(shape)}, "
                             f"got {tuple(x.shape)} {x.dtype} on {x.device}")

    def polarized_rhs(self, rhs):
        import torch
        self._check_volume(rhs)
        R = rhs.shape[0]
        out = torch.empty(self.trace_shape(R), dtype=torch.complex128, device=rhs.device)
        self._check(self.lib.hz_polarized_rhs(self.h, _ptr(rhs), R, _ptr(out)))
        return out

    def apply_mpol(self, x):
        import torch
        self._check_traces(x, self.trace_shape(x.shape[0]))
        y = torch.empty_like(x)
        self._check(self.lib.hz_apply_mpol(self.h, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def apply_precond(self, x):
        import torch
        self._check_traces(x, self.trace_shape(x.shape[0]))
        y = torch.empty_like(x)
        self._check(self.lib.hz_apply_precond(self.h, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def reconstruct(self, rhs, t):
        import torch
        self._check_volume(rhs)
        nz, ny, nx = self.shape
        if t is not None or self.K > 0:      # one layer has no traces: t may be None
            self._check_traces(t, (rhs.shape[0], self.K, 2, ny, nx))
        u = torch.empty_like(rhs)
        self._check(self.lib.hz_reconstruct(self.h, _ptr(rhs), _ptr(t), rhs.shape[0], _ptr(u)))
        return u

    def _check_volume(self, *ts):
        """Every tensor must be a contiguous complex128 CUDA tensor of shape (R, nz, ny, nx) with
        the same R (the kernels read R * nz * ny * nx elements of each)."""
        import torch
        R = ts[0].shape[0] if ts[0].dim() == 4 else -1
        for t in ts:
            if t is None:
                continue
            if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
                    and tuple(t.shape) == (R,) + self.shape):
                raise ValueError(f"expected a contiguous complex128 CUDA tensor of shape {(R,) + self.shape}, "
                                 f"got {tuple(t.shape)} {t.dtype} on {t.device}")

    def volume_residual_noalloc(self, rhs, u, r=None):
        """As volume_residual, through the entry point that allocates nothing; r (if given)
        must be a preallocated complex128 CUDA tensor shaped like rhs."""
        self._check_volume(rhs, u, r)
        R = rhs.shape[0]
        rel = (ct.c_double * R)()
        self._check(self.lib.hz_volume_residual_noalloc(self.h, _ptr(rhs), _ptr(u), R, _ptr(r), rel))
        return list(rel)

    def factor_report(self) -> str:
        """Per-kernel-kind device time of the last factorization (HZ_FACTOR_PROFILE=1 at creation)."""
        return self.lib.hz_factor_report(self.h).decode()

    def tuning_report(self) -> str:
        return self.lib.hz_tuning_report(self.h).decode()

    def profile_report(self) -> str:
        """Per kernel kind, phase and tree level table of the last detail-profiled interval."""
        return self.lib.hz_profile_report(self.h).decode()

    def profile_begin(self, detail: bool = False):
        fn = self.lib.hz_profile_begin_detail if detail else self.lib.hz_profile_begin
        self._check(fn(self.h))

    def profile_kernel(self, kind: int):
        """Per-kernel-kind totals of the last detail-profiled interval: 0 CUDA-core, 1 tensor-core
        substitution, 2 explicit trace-block products."""
        n, ms, by, fl = ct.c_int64(), ct.c_double(), ct.c_double(), ct.c_double()
        self._check(self.lib.hz_profile_kernel(self.h, kind, ct.byref(n), ct.byref(ms), ct.byref(by), ct.byref(fl)))
        return dict(launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)

    def profile_end(self):
        n, ms, by, fl = ct.c_int64(), ct.c_double(), ct.c_double(), ct.c_double()
        self._check(self.lib.hz_profile_end(self.h, ct.byref(n), ct.byref(ms), ct.byref(by), ct.byref(fl)))
        return dict(calls=n.value, ms=ms.value, bytes=by.value, flops=fl.value)

    def volume_residual(self, rhs, u, want_r: bool = False):
        import torch
        self._check_volume(rhs, u)
        R = rhs.shape[0]
        r = torch.empty_like(rhs) if want_r else None
        rel = (ct.c_double * R)()
        self._check(self.lib.hz_volume_residual(self.h, _ptr(rhs), _ptr(u), R, _ptr(r), rel))
        return list(rel), r


def solve_group(solvers, rhs_list, opts: Optional[SolveOpts] = None, allow_noconv: bool = False):
    """Solve several factored problems at once (hz_solve_group): rhs_list[i] is a complex128
    CUDA tensor (R_i, nz_i, ny_i, nx_i) for solvers[i].  Returns ([u_i], [[SolveInfo]_i], [status_i])."""
    import torch
    lib = load()
    n = len(solvers)
    us = [torch.empty_like(r) for r in rhs_list]
    infos = [(SolveInfo * r.shape[0])() for r in rhs_list]
    hs = (ct.c_void_p * n)(*[s.h.value for s in solvers])
    rp = (ct.c_void_p * n)(*[_ptr(r) for r in rhs_list])
    up = (ct.c_void_p * n)(*[_ptr(u) for u in us])
    Rs = (ct.c_int32 * n)(*[r.shape[0] for r in rhs_list])
    ip = (ct.c_void_p * n)(*[ct.addressof(i) for i in infos])
    sts = (ct.c_int * n)()
    for sv, r in zip(solvers, rhs_list):
        sv._check_volume(r)
    st = lib.hz_solve_group(hs, n, rp, Rs, up, ct.byref(opts) if opts else None, ip, sts)
    ok = (HZ_OK, HZ_ERR_NO_CONVERGENCE) if allow_noconv else (HZ_OK,)
    if st not in ok:
        bad = [i for i in range(n) if sts[i] not in ok]
        raise HzError(st, f"member {bad[0]}: " + lib.hz_last_error(solvers[bad[0]].h).decode())
    return us, [list(i) for i in infos], list(sts)


def tensor_peak(kind: str = "tf32", n: int = 128, seconds: float = 1.0):
    """Measured dense tcgen05 MMA rate of the current device (hz_tensor_peak): (TFLOP/s, ms)."""
    tf, ms = ct.c_double(), ct.c_double()
    st = load().hz_tensor_peak({"tf32": 0, "bf16": 1, "tf32_tmem_a": 2}[kind], n, seconds, ct.byref(tf), ct.byref(ms))
    if st != HZ_OK:
        raise HzError(st, f"hz_tensor_peak({kind}, {n}) failed")
    return tf.value, ms.value


def symbolic_shape(nx: int, ny: int, nz: int, leaf: int = 256):
    """The library's nested-dissection symbolic phase of one box shape (hz_symbolic_shape, host
    only): dict of perm, own0, nown, parent, upd_off and upd_idx as numpy arrays."""
    lib = load()
    nn, nu = ct.c_int64(), ct.c_int64()
    st = lib.hz_symbolic_shape(nx, ny, nz, leaf, ct.byref(nn), ct.byref(nu), None, None, None, None, None, None)
    if st != HZ_OK:
        raise HzError(st, lib.hz_last_error(None).decode())
    out = dict(perm=np.empty(nx * ny * nz, np.int32), own0=np.empty(nn.value, np.int32),
               nown=np.empty(nn.value, np.int32), parent=np.empty(nn.value, np.int32),
               upd_off=np.empty(nn.value, np.int64), upd_idx=np.empty(nu.value, np.int32))
    st = lib.hz_symbolic_shape(nx, ny, nz, leaf, ct.byref(nn), ct.byref(nu),
                               *[out[k].ctypes.data for k in ("perm", "own0", "nown", "parent", "upd_off", "upd_idx")])
    if st != HZ_OK:
        raise HzError(st, lib.hz_last_error(None).decode())
    return out


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load().hz_kernel_launches())


def exported_symbols(path: str = LIB_PATH) -> Sequence[str]:
    """Names of the declared entry points present in the library (no GPU needed)."""
    lib = ct.CDLL(path)
    return [n for n in EXPORTED if hasattr(lib, n)]
