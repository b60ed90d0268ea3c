"""Python binding of libcmg (include/cmg.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of libcmg.so.  Tensors are
PyTorch CUDA tensors (device memory and streams only); this module checks
their dtype, shape, device and contiguity and passes raw pointers through
the C ABI.  There is no CPU fallback: if the library is missing or no GPU
is present, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmg.so")

CMG_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "NONFINITE",
          6: "TIMEOUT", 7: "UNSUPPORTED"}
SMOOTH_RBGS, SMOOTH_JACOBI = 0, 1
FP64, FP32 = 0, 1
BATCH_AUTO, BATCH_PERSISTENT, BATCH_BRANCHES = 0, 1, 2
BATCH_LEGS_BY_WORK, BATCH_LEGS_PERSISTENT, BATCH_LEGS_PHASES = -1, 0, 1
METHOD_CYCLE, METHOD_FGMRES = 0, 1
COARSE = {"averaged": 0, "nodal": 1, "galerkin": 2}


class CMGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cmg {STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int), ("nu", ctypes.c_double),
                ("amp", ctypes.c_double), ("coarsest_n", ctypes.c_int), ("coarse_coeff", ctypes.c_int),
                ("ctl_box", ctypes.c_double * 4)]


def _box(control_box):
    """cmg_problem.ctl_box from (x0, x1, y0, y1), or all zero (control everywhere)."""
    b = (0.0, 0.0, 0.0, 0.0) if control_box is None else tuple(float(v) for v in control_box)
    if len(b) != 4:
        raise ValueError("control_box must be (x0, x1, y0, y1)")
    return (ctypes.c_double * 4)(*b)


class Cycle(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("theta", ctypes.c_double), ("n1", ctypes.c_int),
                ("n2", ctypes.c_int), ("gamma", ctypes.c_int), ("precision", ctypes.c_int),
                ("tail_n", ctypes.c_int), ("freeze_u", ctypes.c_int), ("ctl32", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("relres0", ctypes.c_double),
                ("relres", ctypes.c_double)]


class SSNStats(ctypes.Structure):
    _fields_ = [("newton", ctypes.c_int), ("inner_total", ctypes.c_int), ("merit0", ctypes.c_double),
                ("merit", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libcmg.so (built by paper_2302_13680_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcmg.so not found at {path}: run paper_2302_13680_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    sig = {
        "cmg_create": (_I, [ctypes.POINTER(Problem), _P, _P, ctypes.POINTER(H)]),
        "cmg_set_samples": (_I, [H, _P]),
        "cmg_destroy": (None, [H]),
        "cmg_last_error": (ctypes.c_char_p, [H]),
        "cmg_num_levels": (_I, [H]),
        "cmg_level_n": (_I, [H, _I]),
        "cmg_rhs": (_I, [H, _P, _P, _P, _P, _P]),
        "cmg_norm": (_I, [H, _I, _P, _P, _P, ctypes.POINTER(_D)]),
        "cmg_sync": (_I, [H]),
        "cmg_mean_log_kappa": (_I, [H, _P]),
        "cmg_profile_begin": (_I, [H, _I, _I]),
        "cmg_profile_end": (_I, [H, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
        "cmg_kernel_launches": (ctypes.c_longlong, []),
        "cmg_autotune": (_I, [H, _I, ctypes.POINTER(ctypes.c_int)]),
        "cmg_set_tuning": (_I, [H, _I, ctypes.POINTER(ctypes.c_int)]),
        "cmg_sweep_wait_timeouts": (_I, [ctypes.POINTER(ctypes.c_uint)]),
        "cmg_batch_autotune": (_I, [_P, _I]),
        "cmg_batch_create": (_I, [ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_void_p), _I, _P,
                                  ctypes.POINTER(ctypes.c_void_p)]),
        "cmg_batch_destroy": (None, [_P]),
        "cmg_batch_last_error": (ctypes.c_char_p, [_P]),
        "cmg_batch_instance": (_P, [_P, _I]),
        "cmg_batch_solve": (_I, [_P, ctypes.POINTER(Cycle), _D, _I] + [ctypes.POINTER(ctypes.c_void_p)] * 6
                            + [ctypes.POINTER(Stats)]),
        "cmg_solve": (_I, [H, ctypes.POINTER(Cycle), _I, _D, _I, _I, _P, _P, _P, _P, _P, _P,
                           ctypes.POINTER(Stats)]),
        "cmg_ssn_solve": (_I, [H, ctypes.POINTER(Cycle), _I, _D, _D, _D, _D, _D, _I, _P, _P, _P, _P,
                               ctypes.POINTER(SSNStats)]),
    }
    for suf in ("", "_f32"):
        sig["cmg_residual" + suf] = (_I, [H, _I] + [_P] * 9)
        sig["cmg_smooth" + suf] = (_I, [H, _I, ctypes.POINTER(Cycle), _I] + [_P] * 6)
        sig["cmg_restrict" + suf] = (_I, [H, _I] + [_P] * 6)
        sig["cmg_prolong_add" + suf] = (_I, [H, _I] + [_P] * 6)
        sig["cmg_coarse_solve" + suf] = (_I, [H] + [_P] * 6)
        sig["cmg_cycle_apply" + suf] = (_I, [H, ctypes.POINTER(Cycle)] + [_P] * 6)
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


@dataclass
class CycleOptions:
    smoother: int = SMOOTH_RBGS
    theta: float = 0.5
    n1: int = 2
    n2: int = 2
    gamma: int = 1
    precision: int = FP64
    tail_n: int = 0           # grids with n <= tail_n run as one cluster launch; 0 = one launch per step
                              # (the faster choice inside the refinement graph on GB300)
    freeze_u: int = 0         # 1: keep u fixed, solve the state and adjoint rows only
    ctl32: int = 0            # FP32 cycles: 1 = Eq. (13)'s per-node Schur scalar in FP32 too (all-FP32 option)

    def c(self) -> Cycle:
        return Cycle(self.smoother, self.theta, self.n1, self.n2, self.gamma, self.precision, self.tail_n,
                     self.freeze_u, self.ctl32)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Hierarchy:
    """One problem instance: grid hierarchy and coefficients on the GPU.

    Vectors are triples (y, u, p) of CUDA tensors with y, p of shape
    [n_l*n_l, N] and u of shape [n_l*n_l] on grid l, contiguous, dtype
    float64 (or float32 for the *_f32 calls).
    """

    def __init__(self, n: int, N: int, xi, nu: float, amp: float, coarsest_n: int = 3, stream=None,
                 coarse: str = "averaged", control_box=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libcmg needs a CUDA GPU; none is available")
        self._lib = load_library()
        xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
        if xi.ndim != 2 or xi.shape[0] != N:
            raise ValueError("xi must have shape [N, K]")
        self.n, self.N, self.K = int(n), int(N), int(xi.shape[1])
        self.nu, self.amp = float(nu), float(amp)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if coarse not in COARSE:
            raise ValueError(f"coarse must be one of {sorted(COARSE)}")
        prob = Problem(self.n, self.N, self.K, self.nu, self.amp, coarsest_n, COARSE[coarse], _box(control_box))
        self.control_box = control_box
        h = ctypes.c_void_p()
        st = self._lib.cmg_create(ctypes.byref(prob), xi.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != CMG_OK:
            raise CMGError(st, "cmg_create failed")
        self._h = h
        self.levels = self._lib.cmg_num_levels(h)
        self.level_n = [self._lib.cmg_level_n(h, l) for l in range(self.levels)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers ----
    def _check(self, st: int):
        if st != CMG_OK:
            msg = self._lib.cmg_last_error(self._h)
            raise CMGError(st, msg.decode() if msg else "")

    def _vec(self, v, level: int, dtype, name: str):
        import torch

        if v is None:
            return [None, None, None]
        y, u, p = v
        if not 0 <= level < self.levels:
            # out-of-range level: let the C ABI reject the call
            return [_ptr(y), _ptr(u), _ptr(p)]
        m = self.level_n[level] ** 2
        for t, shape in ((y, (m, self.N)), (u, (m,)), (p, (m, self.N))):
            if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype:
                raise TypeError(f"{name}: expected CUDA {dtype} tensors")
            if tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{name}: expected contiguous shape {shape}, got {tuple(t.shape)}")
        return [_ptr(y), _ptr(u), _ptr(p)]

    def zeros(self, level: int = 0, dtype=None):
        import torch

        dtype = dtype or torch.float64
        m = self.level_n[level] ** 2
        return (torch.zeros(m, self.N, dtype=dtype, device=self.device),
                torch.zeros(m, dtype=dtype, device=self.device),
                torch.zeros(m, self.N, dtype=dtype, device=self.device))

    @staticmethod
    def _suffix(dtype):
        import torch

        return "_f32" if dtype == torch.float32 else ""

    # ---- C ABI calls ----
    def set_samples(self, xi_dev):
        self._check(self._lib.cmg_set_samples(self._h, _ptr(xi_dev)))

    def rhs(self, yd, fsrc=None):
        import torch

        f = self.zeros(0)
        self._check(self._lib.cmg_rhs(self._h, _ptr(yd), _ptr(fsrc), *[_ptr(t) for t in f]))
        return f

    def residual(self, level, x, f, r):
        dt = x[0].dtype
        fn = getattr(self._lib, "cmg_residual" + self._suffix(dt))
        self._check(fn(self._h, level, *self._vec(x, level, dt, "x"), *self._vec(f, level, dt, "f"),
                       *self._vec(r, level, dt, "r")))

    def smooth(self, level, opts: CycleOptions, sweeps, x, f):
        dt = x[0].dtype
        fn = getattr(self._lib, "cmg_smooth" + self._suffix(dt))
        c = opts.c()
        self._check(fn(self._h, level, ctypes.byref(c), sweeps, *self._vec(x, level, dt, "x"),
                       *self._vec(f, level, dt, "f")))

    def restrict(self, level, r, c):
        if not 0 <= level < self.levels - 1:
            raise CMGError(1, "level out of range")
        dt = r[0].dtype
        fn = getattr(self._lib, "cmg_restrict" + self._suffix(dt))
        self._check(fn(self._h, level, *self._vec(r, level, dt, "r"), *self._vec(c, level + 1, dt, "c")))

    def prolong_add(self, level, e, x):
        if not 0 <= level < self.levels - 1:
            raise CMGError(1, "level out of range")
        dt = e[0].dtype
        fn = getattr(self._lib, "cmg_prolong_add" + self._suffix(dt))
        self._check(fn(self._h, level, *self._vec(e, level + 1, dt, "e"), *self._vec(x, level, dt, "x")))

    def coarse_solve(self, f, x):
        dt = f[0].dtype
        L = self.levels - 1
        fn = getattr(self._lib, "cmg_coarse_solve" + self._suffix(dt))
        self._check(fn(self._h, *self._vec(f, L, dt, "f"), *self._vec(x, L, dt, "x")))

    def cycle(self, opts: CycleOptions, x, f):
        dt = x[0].dtype
        fn = getattr(self._lib, "cmg_cycle_apply" + self._suffix(dt))
        c = opts.c()
        self._check(fn(self._h, ctypes.byref(c), *self._vec(x, 0, dt, "x"), *self._vec(f, 0, dt, "f")))

    def solve(self, opts: CycleOptions, f, x, method=METHOD_CYCLE, tol=1e-10, maxit=100, restart=30,
              raise_on_fail=True):
        import torch

        c = opts.c()
        st = Stats()
        status = self._lib.cmg_solve(self._h, ctypes.byref(c), method, tol, maxit, restart,
                                     *self._vec(f, 0, torch.float64, "f"), *self._vec(x, 0, torch.float64, "x"),
                                     ctypes.byref(st))
        if raise_on_fail:
            self._check(status)
        return st, status

    def ssn_solve(self, opts: CycleOptions, yd, u, beta: float, a: float, b: float, method=METHOD_CYCLE,
                  tol=1e-9, inner_tol=1e-10, maxit=50, raise_on_fail=True):
        """L1 + box problem by semismooth Newton (cmg_ssn_solve).  yd [n*n],
        u [n*n] (u0 in, control out) CUDA float64; returns (stats, status, y, p)."""
        import torch

        m = self.n * self.n
        for t, name in ((yd, "yd"), (u, "u")):
            if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64 \
                    or tuple(t.shape) != (m,) or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous CUDA float64 tensor of shape ({m},)")
        y = torch.empty(m, self.N, dtype=torch.float64, device=self.device)
        p = torch.empty(m, self.N, dtype=torch.float64, device=self.device)
        c = opts.c()
        st = SSNStats()
        status = self._lib.cmg_ssn_solve(self._h, ctypes.byref(c), method, beta, a, b, tol, inner_tol, maxit,
                                         _ptr(yd), _ptr(y), _ptr(u), _ptr(p), ctypes.byref(st))
        if raise_on_fail:
            self._check(status)
        return st, status, y, p

    def norm(self, level, v):
        import torch

        out = ctypes.c_double()
        self._check(self._lib.cmg_norm(self._h, level, *self._vec(v, level, torch.float64, "v"),
                                       ctypes.byref(out)))
        return out.value

    def sync(self):
        self._check(self._lib.cmg_sync(self._h))

    def mean_log_kappa(self, out=None):
        import torch

        out = torch.empty(self.n * self.n, dtype=torch.float64, device=self.device) if out is None else out
        self._check(self._lib.cmg_mean_log_kappa(self._h, _ptr(out)))
        return out

    def autotune(self, precision: int = FP32):
        """Time 1, 2 and 4 sample chunks per lane on every grid; keep the fastest."""
        out = (ctypes.c_int * self.levels)()
        self._check(self._lib.cmg_autotune(self._h, precision, out))
        return list(out)

    def set_tuning(self, precision: int, targets):
        arr = None if targets is None else (ctypes.c_int * self.levels)(*targets)
        self._check(self._lib.cmg_set_tuning(self._h, precision, arr))

    def profile_begin(self, kinds: int, level: int = 0):
        self._check(self._lib.cmg_profile_begin(self._h, kinds, level))

    def profile_end(self):
        ms, cnt = ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.cmg_profile_end(self._h, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value


KERNEL_SMOOTH, KERNEL_RESIDUAL, KERNEL_RESTRICT, KERNEL_PROLONG, KERNEL_COARSE, KERNEL_TAIL = 1, 2, 4, 8, 16, 32


def sample_map(N: int, elem_bytes: int, items: int = 0, target: int = 0):
    """(lanes per node, vector width, chunks per lane) of the node kernels
    (cmg_sample_map; host arithmetic, no GPU needed)."""
    lib = load_library()
    fn = lib.cmg_sample_map
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    out = [ctypes.c_int() for _ in range(3)]
    st = fn(N, elem_bytes, items, target, *[ctypes.byref(o) for o in out])
    if st not in (CMG_OK, 7):
        raise CMGError(st, "bad sample-map arguments")
    return tuple(o.value for o in out)


class BoundaryHierarchy:
    """Neumann boundary control on (0,1) x {0} (cmg_bnd_*): grid l has
    level_n[l] interior columns and level_n[l] + 1 rows (row 0 on Gamma).
    Vectors are triples (y, u, p) of CUDA float64 tensors, y and p of shape
    [(n_l+1) n_l, N], u of shape [n_l]."""

    def __init__(self, n: int, N: int, xi, nu: float, amp: float, coarsest_n: int = 3, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libcmg needs a CUDA GPU; none is available")
        self._lib = load_library()
        xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
        if xi.ndim != 2 or xi.shape[0] != N:
            raise ValueError("xi must have shape [N, K]")
        self.n, self.N = int(n), int(N)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        L = self._lib
        L.cmg_bnd_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        L.cmg_bnd_last_error.restype = ctypes.c_char_p
        L.cmg_bnd_last_error.argtypes = [ctypes.c_void_p]
        st = L.cmg_bnd_create(self.n, self.N, xi.shape[1], float(nu), float(amp), int(coarsest_n),
                              xi.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(self.stream.cuda_stream),
                              ctypes.byref(h))
        if st != CMG_OK:
            raise CMGError(st, "cmg_bnd_create failed")
        self._h = h
        self.levels = L.cmg_bnd_num_levels(h)
        self.level_n = [L.cmg_bnd_level_n(h, l) for l in range(self.levels)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cmg_bnd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != CMG_OK:
            msg = self._lib.cmg_bnd_last_error(self._h)
            raise CMGError(st, msg.decode() if msg else "")

    def zeros(self, level: int = 0):
        import torch

        n = self.level_n[level]
        m = (n + 1) * n
        return (torch.zeros(m, self.N, dtype=torch.float64, device="cuda"),
                torch.zeros(n, dtype=torch.float64, device="cuda"),
                torch.zeros(m, self.N, dtype=torch.float64, device="cuda"))

    def _vec(self, v, level):
        import torch

        if v is None:
            return [None, None, None]
        n = self.level_n[level]
        m = (n + 1) * n
        for t, shape in zip(v, ((m, self.N), (n,), (m, self.N))):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.device.type != "cuda" \
                    or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"expected contiguous CUDA float64 tensors of shapes {(m, self.N)}, {(n,)}")
        return [_ptr(t) for t in v]

    def rhs(self, yd, fsrc=None):
        f = self.zeros(0)
        self._check(self._lib.cmg_bnd_rhs(self._h, _ptr(yd), _ptr(fsrc), *[_ptr(t) for t in f]))
        return f

    def residual(self, level, x, f, r):
        self._check(self._lib.cmg_bnd_residual(self._h, level, *self._vec(x, level), *self._vec(f, level),
                                               *self._vec(r, level)))

    def smooth(self, level, theta, sweeps, x, f):
        self._check(self._lib.cmg_bnd_smooth(self._h, level, ctypes.c_double(theta), sweeps, *self._vec(x, level),
                                             *self._vec(f, level)))

    def restrict(self, level, r, c):
        self._check(self._lib.cmg_bnd_restrict(self._h, level, *self._vec(r, level), *self._vec(c, level + 1)))

    def prolong_add(self, level, e, x):
        self._check(self._lib.cmg_bnd_prolong_add(self._h, level, *self._vec(e, level + 1), *self._vec(x, level)))

    def coarse_solve(self, f, x):
        L = self.levels - 1
        self._check(self._lib.cmg_bnd_coarse_solve(self._h, *self._vec(f, L), *self._vec(x, L)))

    def cycle(self, x, f, theta=0.5, n1=2, n2=2, gamma=1):
        self._check(self._lib.cmg_bnd_cycle(self._h, ctypes.c_double(theta), n1, n2, gamma, *self._vec(x, 0),
                                            *self._vec(f, 0)))

    def solve(self, f, x, theta=0.5, n1=2, n2=2, gamma=1, tol=1e-10, maxit=100, raise_on_fail=True):
        st = Stats()
        status = self._lib.cmg_bnd_solve(self._h, ctypes.c_double(theta), n1, n2, gamma, ctypes.c_double(tol),
                                         maxit, *self._vec(f, 0), *self._vec(x, 0), ctypes.byref(st))
        if raise_on_fail:
            self._check(status)
        return st, status


def kernel_launches() -> int:
    """Kernels launched by libcmg in this process so far."""
    return int(load_library().cmg_kernel_launches())


class Batch:
    """Independent instances solved together (cmg_batch_*).

    problems: sequence of objects with n, N, xi, nu, amp (e.g.
    inputs.ProblemSpec).  Vectors are lists of (y, u, p) CUDA float64
    tensors, one triple per instance, shaped by that instance's n and N.
    """

    def __init__(self, problems, coarsest_n: int = 3, coarse: str = "averaged", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libcmg needs a CUDA GPU; none is available")
        self._lib = load_library()
        self.count = len(problems)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        probs = (Problem * self.count)()
        self._xi = []
        for i, pr in enumerate(problems):
            xi = np.ascontiguousarray(np.asarray(pr.xi, dtype=np.float64))
            self._xi.append(xi)
            probs[i] = Problem(pr.n, pr.N, xi.shape[1], pr.nu, pr.amp, coarsest_n, COARSE[coarse],
                               _box(getattr(pr, "control_box", None)))
        ptrs = (ctypes.c_void_p * self.count)(*[x.ctypes.data for x in self._xi])
        b = ctypes.c_void_p()
        st = self._lib.cmg_batch_create(probs, ptrs, self.count, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(b))
        if st != CMG_OK:
            raise CMGError(st, "cmg_batch_create failed")
        self._b = b
        self.shapes = [(pr.n, pr.N) for pr in problems]

    def close(self):
        if getattr(self, "_b", None):
            self._lib.cmg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_form(self, form: int):
        """BATCH_AUTO, BATCH_PERSISTENT or BATCH_BRANCHES (cmg_batch_set_form)."""
        self._bcheck(self._lib.cmg_batch_set_form(self._b, int(form)))

    def form(self) -> int:
        """The form the last FP32 solve used (cmg_batch_form)."""
        return int(self._lib.cmg_batch_form(self._b))

    def set_legs(self, legs: int):
        """Persistent form, per grid depth: BATCH_LEGS_BY_WORK (default),
        BATCH_LEGS_PERSISTENT (the persistent kernel everywhere) or
        BATCH_LEGS_PHASES (one launch per phase everywhere)."""
        self._bcheck(self._lib.cmg_batch_set_legs(self._b, int(legs)))

    def set_wait_limit(self, polls: int):
        """Polls per grid-wide barrier wait (0 = default) (cmg_batch_set_wait_limit)."""
        self._bcheck(self._lib.cmg_batch_set_wait_limit(self._b, ctypes.c_longlong(int(polls))))

    def _bcheck(self, st):
        if st != CMG_OK:
            msg = self._lib.cmg_batch_last_error(self._b)
            raise CMGError(st, msg.decode() if msg else "")

    def autotune(self, precision: int = FP32):
        st = self._lib.cmg_batch_autotune(self._b, precision)
        if st != CMG_OK:
            msg = self._lib.cmg_batch_last_error(self._b)
            raise CMGError(st, msg.decode() if msg else "")

    def zeros(self):
        import torch

        return [(torch.zeros(n * n, N, dtype=torch.float64, device="cuda"),
                 torch.zeros(n * n, dtype=torch.float64, device="cuda"),
                 torch.zeros(n * n, N, dtype=torch.float64, device="cuda")) for n, N in self.shapes]

    def solve(self, opts: CycleOptions, fs, xs, tol=1e-10, maxit=100, raise_on_fail=True):
        import torch

        for (n, N), f, x in zip(self.shapes, fs, xs):
            for v in (f, x):
                for t, shape in zip(v, ((n * n, N), (n * n,), (n * n, N))):
                    if t.dtype != torch.float64 or t.device.type != "cuda" or tuple(t.shape) != shape \
                            or not t.is_contiguous():
                        raise ValueError("batch vectors must be contiguous CUDA float64 of the instance's shape")
        arr = lambda k, vs: (ctypes.c_void_p * self.count)(*[v[k].data_ptr() for v in vs])
        stats = (Stats * self.count)()
        c = opts.c()
        status = self._lib.cmg_batch_solve(self._b, ctypes.byref(c), tol, maxit, arr(0, fs), arr(1, fs),
                                           arr(2, fs), arr(0, xs), arr(1, xs), arr(2, xs), stats)
        if raise_on_fail and status != CMG_OK:
            msg = self._lib.cmg_batch_last_error(self._b)
            raise CMGError(status, msg.decode() if msg else "")
        return list(stats), status
