"""Thin Python binding of libndmg (include/ndmg.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module checks tensor
dtypes, devices and contiguity, passes raw device pointers through ctypes and
turns status codes into exceptions.  Importing it loads ``libndmg.so`` and
raises if the library has not been built (``python -m
paper_2205_05840_gb300.build``); there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libndmg.so")
HEADER = os.path.join(_HERE, "..", "include", "ndmg.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libndmg.so is not built ({LIB_PATH}); run python -m paper_2205_05840_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

OK, INVALID_ARG, CUDA_ERROR, OUT_OF_MEMORY, NOT_CONVERGED, BREAKDOWN, DEVICE_TIMEOUT = range(7)
F64, F32 = 0, 1
SMOOTHER_VERTEX, SMOOTHER_EDGE = 0, 1
PREC_FP64, PREC_MIXED_BF16, PREC_MIXED_FP16, PREC_FP32 = 0, 1, 2, 3
K_STENCIL, K_RESTRICT, K_PROLONG, K_BUBBLE, K_PATCH, K_COARSE, K_BLAS = range(7)
KERNEL_CLASSES = {"stencil": K_STENCIL, "restrict": K_RESTRICT, "prolong": K_PROLONG, "bubble": K_BUBBLE,
                  "patch": K_PATCH, "coarse": K_COARSE, "blas": K_BLAS}
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA_ERROR", 3: "OUT_OF_MEMORY", 4: "NOT_CONVERGED",
                5: "BREAKDOWN", 6: "DEVICE_TIMEOUT"}


class Opts(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_coarsest", ctypes.c_int32), ("L", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("smoother", ctypes.c_int32),
                ("eta", ctypes.c_double), ("m", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nrhs", ctypes.c_int32), ("stream", ctypes.c_void_p), ("subdomain", ctypes.c_int32)]


_vp, _i32, _i64, _d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER
_SIGS = {
    "ndmg_opts_default": [_P(Opts)],
    "ndmg_create": [_P(Opts), _P(_vp)],
    "ndmg_destroy": [_vp],
    "ndmg_set_alpha": [_vp, _d],
    "ndmg_num_levels": [_vp, _P(_i32)],
    "ndmg_num_dofs": [_vp, _i32, _P(_i64)],
    "ndmg_apply": [_vp, _i32, _i32, _vp, _vp],
    "ndmg_residual": [_vp, _i32, _i32, _vp, _vp, _vp],
    "ndmg_pencil": [_vp, _i32, _i32, _d, _d, _vp, _vp, _vp],
    "ndmg_axpby": [_vp, _i32, _i32, _d, _vp, _d, _vp],
    "ndmg_smooth": [_vp, _i32, _i32, _vp, _vp, _i32],
    "ndmg_restrict": [_vp, _i32, _i32, _vp, _vp],
    "ndmg_prolong_add": [_vp, _i32, _i32, _vp, _vp],
    "ndmg_coarse_solve": [_vp, _i32, _vp, _vp],
    "ndmg_vcycle": [_vp, _i32, _vp, _vp],
    "ndmg_solve": [_vp, _vp, _vp, _d, _i32, _P(_i32), _P(_d)],
    "ndmg_solve_host": [_vp, _vp, _vp, _d, _i32, _P(_i32), _P(_d)],
    "ndmg_solve_ir": [_vp, _vp, _vp, _d, _d, _i32, _P(_i32), _P(_d)],
    "ndmg_vcycle_iterate": [_vp, _vp, _vp, _d, _i32, _P(_i32), _P(_d)],
    "ndmg_grad_alpha": [_vp, _vp, _vp, _P(_d)],
    "ndmg_dot": [_vp, _i32, _i32, _vp, _vp, _P(_d)],
    "ndmg_trace_enable": [_vp, _i32, _i32],
    "ndmg_trace_read": [_vp, _i32, _P(_i64), _P(_d), _P(_d)],
    "ndmg_counters": [_vp, _P(_i64), _P(_i64)],
    "ndmg_use_graphs": [_vp, _i32],
    "ndmg_dot_noalloc": [_i32, _vp, _vp, _i64, _P(_d), _vp],
    "ndmg_set_alpha_field": [_vp, _vp],
    "ndmg_autotune": [_vp, _P(_i32)],
    "ndmg_set_launch_shapes": [_vp, _P(_i32)],
    "ndmg_grad_alpha_field": [_vp, _vp, _vp, _vp],
    "ndmg_inject_status": [_vp, _i32],
    "ndmg_select_smoother": [_vp, _i32, _i32],
    "ndmg_probe_fma_rate": [_i32, _P(_d)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.ndmg_last_error.argtypes = [_vp]
_lib.ndmg_last_error.restype = ctypes.c_char_p


def fma_rate_tflops(dtype: int) -> float:
    """Measured CUDA-core FMA rate of the current device in TFLOP/s
    (ndmg_probe_fma_rate; dtype F64 or F32)."""
    out = _d()
    st = _lib.ndmg_probe_fma_rate(int(dtype), ctypes.byref(out))
    if st != OK:
        raise NdmgError(st, "ndmg_probe_fma_rate failed")
    return out.value


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the entry points the C header declares."""
    with open(path) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(ndmg_\w+)\s*\(", txt, flags=re.M)))


class NdmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


class Solver:
    """One multigrid hierarchy on the current CUDA device (see ndmg_create)."""

    def __init__(self, n: int, n_coarsest: int = 2, L: float = 1.0, alpha: float = 1.0, beta: float = 1.0,
                 smoother: int = SMOOTHER_VERTEX, eta: float = 0.0, m: int = 2, precision: int = PREC_FP64,
                 nrhs: int = 1, stream: torch.cuda.Stream | None = None, subdomain: int = 2):
        o = Opts()
        _lib.ndmg_opts_default(ctypes.byref(o))
        o.n, o.n_coarsest, o.L, o.alpha, o.beta = n, n_coarsest, L, alpha, beta
        o.smoother, o.eta, o.m, o.precision, o.nrhs = smoother, eta, m, precision, nrhs
        o.subdomain = subdomain
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o.stream = self.stream.cuda_stream
        self._h = _vp()
        st = _lib.ndmg_create(ctypes.byref(o), ctypes.byref(self._h))
        if st != OK:
            raise NdmgError(st, "ndmg_create failed")
        self.n, self.precision, self.nrhs, self.alpha = n, precision, nrhs, alpha
        self.field = None                   # coefficient per hexahedron last set (CPU float64), if any
        lv = _i32()
        _lib.ndmg_num_levels(self._h, ctypes.byref(lv))
        self.num_levels = lv.value

    # -- helpers ----------------------------------------------------------
    def _check(self, st: int, what: str, ok=(OK,)):
        if st not in ok:
            raise NdmgError(st, f"{what}: {_lib.ndmg_last_error(self._h).decode()}")
        return st

    def _vec(self, t: torch.Tensor, level: int, dtype=None) -> int:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise TypeError("expected a contiguous CUDA tensor")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        if t.numel() != self.num_dofs(level) * self.nrhs:
            raise ValueError(f"expected {self.num_dofs(level) * self.nrhs} entries, got {t.numel()}")
        return t.data_ptr()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.ndmg_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries ----------------------------------------------------------
    def num_dofs(self, level: int = -1) -> int:
        out = _i64()
        self._check(_lib.ndmg_num_dofs(self._h, level, ctypes.byref(out)), "num_dofs")
        return out.value

    def set_alpha(self, alpha: float):
        self._check(_lib.ndmg_set_alpha(self._h, alpha), "set_alpha")
        self.alpha = alpha
        self.field = None

    def set_alpha_field(self, alpha_cells):
        """Curl-curl coefficient per finest-level hexahedron (ndmg_set_alpha_field):
        n^3 values, cell (i, j, k) at (k n + j) n + i (numpy array or CPU tensor)."""
        a = torch.as_tensor(alpha_cells, dtype=torch.float64).detach().cpu().contiguous().reshape(-1)
        if a.numel() != self.n ** 3:
            raise ValueError(f"expected {self.n ** 3} cell coefficients, got {a.numel()}")
        if self.field is not None and torch.equal(self.field, a):
            return                          # the handle holds this field already
        self._check(_lib.ndmg_set_alpha_field(self._h, a.data_ptr()), "set_alpha_field")
        self.alpha = None
        self.field = a.clone()

    def grad_alpha_field(self, lam, u, out=None):
        """-lambda_r^T K_T u_r for every finest-level cell T (ndmg_grad_alpha_field):
        a float64 CUDA tensor of n^3 x nrhs values, queued on the handle's stream."""
        if out is None:
            out = torch.empty(self.n ** 3 * self.nrhs, dtype=torch.float64, device=lam.device)
        if not out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous() or \
                out.numel() != self.n ** 3 * self.nrhs:
            raise TypeError("expected a contiguous float64 CUDA tensor of n^3 x nrhs entries")
        self._check(_lib.ndmg_grad_alpha_field(self._h, self._vec(lam, -1, torch.float64),
                                               self._vec(u, -1, torch.float64), out.data_ptr()), "grad_alpha_field")
        return out

    # -- level operations ---------------------------------------------------
    def apply(self, x, y, level: int = -1):
        self._check(_lib.ndmg_apply(self._h, level, _dtype_code(x), self._vec(x, level), self._vec(y, level, x.dtype)),
                    "apply")

    def residual(self, g, z, r, level: int = -1):
        d = _dtype_code(g)
        self._check(_lib.ndmg_residual(self._h, level, d, self._vec(g, level), self._vec(z, level, g.dtype),
                                       self._vec(r, level, g.dtype)), "residual")

    def pencil(self, a: float, b: float, x, y, g=None, level: int = -1):
        """y = g + (a K + b M) x (ndmg_pencil); g=None gives y = (a K + b M) x."""
        d = _dtype_code(x)
        gp = None if g is None else self._vec(g, level, x.dtype)
        self._check(_lib.ndmg_pencil(self._h, level, d, a, b, gp, self._vec(x, level), self._vec(y, level, x.dtype)),
                    "pencil")

    def axpby(self, a: float, x, b: float, y, level: int = -1):
        """y = a x + b y (ndmg_axpby)."""
        self._check(_lib.ndmg_axpby(self._h, level, _dtype_code(x), a, self._vec(x, level), b,
                                    self._vec(y, level, x.dtype)), "axpby")

    def smooth(self, g, z, steps: int = 1, level: int = -1):
        self._check(_lib.ndmg_smooth(self._h, level, _dtype_code(g), self._vec(g, level), self._vec(z, level, g.dtype),
                                     steps), "smooth")

    def restrict(self, r_fine, g_coarse, level: int = -1):
        lv = self.num_levels - 1 if level == -1 else level
        self._check(_lib.ndmg_restrict(self._h, lv, _dtype_code(r_fine), self._vec(r_fine, lv),
                                       self._vec(g_coarse, lv - 1, r_fine.dtype)), "restrict")

    def prolong_add(self, z_coarse, z_fine, level: int = -1):
        lv = self.num_levels - 1 if level == -1 else level
        self._check(_lib.ndmg_prolong_add(self._h, lv, _dtype_code(z_fine), self._vec(z_coarse, lv - 1, z_fine.dtype),
                                          self._vec(z_fine, lv)), "prolong_add")

    def coarse_solve(self, g, z):
        self._check(_lib.ndmg_coarse_solve(self._h, _dtype_code(g), self._vec(g, 0), self._vec(z, 0, g.dtype)),
                    "coarse_solve")

    def vcycle(self, g, z):
        self._check(_lib.ndmg_vcycle(self._h, _dtype_code(g), self._vec(g, -1), self._vec(z, -1, g.dtype)), "vcycle")

    def dot(self, x, y, level: int = -1):
        """x_r . y_r in FP64 (a float, or a list of nrhs floats for batches)."""
        out = (_d * self.nrhs)()
        self._check(_lib.ndmg_dot(self._h, level, _dtype_code(x), self._vec(x, level), self._vec(y, level, x.dtype),
                                  out), "dot")
        return out[0] if self.nrhs == 1 else list(out)

    # -- solvers ------------------------------------------------------------
    def solve(self, f, u, tol: float = 1e-8, maxit: int = 200, raise_on_fail: bool = True):
        """PCG (FP64 handles) or FP64 iterative refinement (mixed handles).
        Returns (status, iterations, relative residual)."""
        it, rr = _i32(), _d()
        st = _lib.ndmg_solve(self._h, self._vec(f, -1, torch.float64), self._vec(u, -1, torch.float64), tol, maxit,
                             ctypes.byref(it), ctypes.byref(rr))
        if raise_on_fail:
            self._check(st, "solve")
        return st, it.value, rr.value

    def solve_ir(self, f, u, tol: float = 1e-8, inner_tol: float = 1e-4, maxit: int = 400):
        """FP64 iterative refinement around the float PCG (mixed / FP32 handles)."""
        it, rr = _i32(), _d()
        st = _lib.ndmg_solve_ir(self._h, self._vec(f, -1, torch.float64), self._vec(u, -1, torch.float64), tol,
                                inner_tol, maxit, ctypes.byref(it), ctypes.byref(rr))
        self._check(st, "solve_ir")
        return st, it.value, rr.value

    def solve_host(self, f_host, u_host, tol: float = 1e-8, maxit: int = 200):
        """Same as solve with host (CPU, preferably pinned) float64 tensors."""
        for t in (f_host, u_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != self.num_dofs() * self.nrhs:
                raise TypeError("expected contiguous host float64 tensors of the finest level")
        it, rr = _i32(), _d()
        st = _lib.ndmg_solve_host(self._h, f_host.data_ptr(), u_host.data_ptr(), tol, maxit, ctypes.byref(it),
                                  ctypes.byref(rr))
        self._check(st, "solve_host")
        return st, it.value, rr.value

    def vcycle_iterate(self, f, u, tol: float = 1e-8, maxit: int = 500):
        c, rr = _i32(), _d()
        st = _lib.ndmg_vcycle_iterate(self._h, self._vec(f, -1, torch.float64), self._vec(u, -1, torch.float64), tol,
                                      maxit, ctypes.byref(c), ctypes.byref(rr))
        self._check(st, "vcycle_iterate")
        return st, c.value, rr.value

    def grad_alpha(self, lam, u):
        """-lambda_r^T K u_r (a float, or a list of nrhs floats for batches)."""
        out = (_d * self.nrhs)()
        self._check(_lib.ndmg_grad_alpha(self._h, self._vec(lam, -1, torch.float64), self._vec(u, -1, torch.float64),
                                         out), "grad_alpha")
        return out[0] if self.nrhs == 1 else list(out)

    # -- tracing ------------------------------------------------------------
    def trace(self, kernel_class: int, on: bool = True):
        self._check(_lib.ndmg_trace_enable(self._h, kernel_class, int(on)), "trace_enable")

    def trace_read(self, kernel_class: int):
        """(launches, total ms, work units) of a traced kernel class since the
        last read; synchronises the handle's stream."""
        n, ms, u = _i64(), _d(), _d()
        self._check(_lib.ndmg_trace_read(self._h, kernel_class, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(u)),
                    "trace_read")
        return n.value, ms.value, u.value

    def autotune(self):
        """Pick launch shapes by timing (ndmg_autotune); returns {level:
        (stencil planes per CTA for float, for double, smoother: 0 CUDA cores,
        1 tensor cores per brick, 2 tensor cores on cell-owned rows)}; level
        0's smoother entry is 1 when the levels n <= 16 run in one cluster
        launch."""
        out = (_i32 * (3 * self.num_levels))()
        self._check(_lib.ndmg_autotune(self._h, out), "autotune")
        return {k: (out[3 * k], out[3 * k + 1], out[3 * k + 2]) for k in range(self.num_levels)}

    def set_launch_shapes(self, tuned):
        """Apply launch shapes in autotune()'s format without timing
        (ndmg_set_launch_shapes); tuned: {level: (planes f32, planes f64,
        smoother)}; level 0's smoother entry is the small-level cluster switch."""
        arr = (_i32 * (3 * self.num_levels))()
        for k in range(self.num_levels):
            a, b, c = tuned[k]
            arr[3 * k], arr[3 * k + 1], arr[3 * k + 2] = int(a), int(b), int(c)
        self._check(_lib.ndmg_set_launch_shapes(self._h, arr), "set_launch_shapes")

    def use_graphs(self, on: bool = True):
        """Replay the mixed-precision V-cycle as a CUDA graph (ndmg_use_graphs)."""
        self._check(_lib.ndmg_use_graphs(self._h, 1 if on else 0), "use_graphs")

    def counters(self):
        """(kernels launched, finest-level V-cycles) since creation."""
        a, b = _i64(), _i64()
        self._check(_lib.ndmg_counters(self._h, ctypes.byref(a), ctypes.byref(b)), "counters")
        return a.value, b.value

    def inject_status(self, code: int):
        """Test hook: set the handle's device status word (ndmg_inject_status),
        as a tensor-core kernel whose bounded wait gave up would."""
        self._check(_lib.ndmg_inject_status(self._h, int(code)), "inject_status")

    def select_smoother(self, kind: int, level: int = -1):
        """Smoother kernel of a level (ndmg_select_smoother): 0 CUDA cores,
        1 tensor cores per brick, 2 tensor cores on cell-owned rows; level 0:
        the levels n <= 16 in one cluster launch (1) or separate ones (0)."""
        self._check(_lib.ndmg_select_smoother(self._h, int(level), int(kind)), "select_smoother")
