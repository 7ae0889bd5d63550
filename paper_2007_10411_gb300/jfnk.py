"""Thin ctypes binding of libjfnk (the C ABI declared in include/jfnk.h).

Only argument marshalling lives here: every numerical step runs in the CUDA
kernels of ``libjfnk.so``.  PyTorch supplies device memory and streams.  The
binding refuses to run without the compiled library (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjfnk.so")

JFNK_OK = 0
JFNK_ERR_INVALID_ARG = 1
JFNK_ERR_CUDA = 2
JFNK_ERR_OOM = 3
JFNK_ERR_NOT_CONVERGED = 4
JFNK_ERR_BREAKDOWN = 5
JFNK_ERR_NAN = 6
JFNK_ERR_TIMEOUT = 7
JFNK_ERR_UNSUPPORTED = 8
MAX_KRYLOV = 32
MAX_NEWTON = 32
BUDGETS_STATIC_MAX_POINTS = 8388608   # JFNK_BUDGETS_STATIC_MAX_POINTS

EXPORTS = (
    "jfnk_create", "jfnk_destroy", "jfnk_set_surface_flux", "jfnk_rhs", "jfnk_residual",
    "jfnk_jv", "jfnk_precond_apply", "jfnk_step", "jfnk_step_host", "jfnk_budgets",
    "jfnk_get_launch_count", "jfnk_status_str", "jfnk_kernel_timing", "jfnk_kernel_timing_read",
    "jfnk_kernel_timing_sampled",
    "jfnk_budgets_static", "jfnk_autotune", "jfnk_set_tiles", "jfnk_set_cycle_graph",
    "jfnk_create_batch", "jfnk_destroy_batch", "jfnk_batch_handle", "jfnk_step_batch",
    "jfnk_unet_init", "jfnk_unet_num_weights", "jfnk_unet_get_weights", "jfnk_unet_set_weights",
    "jfnk_unet_capture", "jfnk_unet_pair_count", "jfnk_unet_get_pair", "jfnk_unet_train",
    "jfnk_unet_forward", "jfnk_unet_loss_grad", "jfnk_set_precond", "jfnk_unet_set_engine",
    "jfnk_unet_status",
)
UNET_TCGEN05, UNET_MMA_SYNC = 0, 1

PC_NONE, PC_BLOCK, PC_UNET, PC_SCHUR, PC_NONLINEAR = 0, 1, 2, 3, 4
PAIRS_NEWTON, PAIRS_ARNOLDI = 1, 2

KERNEL_FAMILIES = ("arnoldi_a", "arnoldi_b", "arnoldi_c", "jv", "precond", "residual", "unet")


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc_bottom", ctypes.c_int), ("bc_top", ctypes.c_int)]


class Strat(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("theta0", "beta", "pbar", "g", "gamma_p", "rho0", "cp")]


class Sgs(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int)] + [(k, ctypes.c_double) for k in ("K_M", "K_H", "Cs", "Pr")]


class Opts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("precision", "wavelet_p", "krylov_m", "flexible",
                                           "precond", "pc_sweeps")] + \
               [(k, ctypes.c_double) for k in ("newton_rtol", "newton_atol_factor", "eta")] + \
               [("max_newton", ctypes.c_int), ("max_restarts", ctypes.c_int)] + \
               [(k, ctypes.c_double) for k in ("dt", "scale_u", "scale_theta", "scale_p")]


class Stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int),
                ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("res0", ctypes.c_double), ("res_final", ctypes.c_double), ("tol", ctypes.c_double),
                ("res_hist", ctypes.c_double * (MAX_NEWTON + 1)),
                ("gmres_per_newton", ctypes.c_int * MAX_NEWTON),
                ("pc_fallback", ctypes.c_int), ("pc_switches", ctypes.c_int)]

    def as_dict(self) -> dict:
        k = self.newton_iters
        return {"newton_iters": k, "gmres_iters": self.gmres_iters, "restarts": self.restarts,
                "converged": bool(self.converged), "res0": self.res0, "res_final": self.res_final,
                "tol": self.tol, "residual_history": list(self.res_hist[: k + 1]),
                "gmres_per_newton": list(self.gmres_per_newton[:k]), "pc_fallback": bool(self.pc_fallback),
                "pc_switches": self.pc_switches}


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Budget(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("E_k", "E_p", "sum_theta", "sum_div")] + \
               [("max", ctypes.c_double * 5), ("min", ctypes.c_double * 5)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libjfnk.so (built by ``paper_2007_10411_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libjfnk.so is not built (%s); run paper_2007_10411_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    lib.jfnk_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Strat), ctypes.POINTER(Sgs),
                                ctypes.POINTER(Opts), P, ctypes.POINTER(P)]
    lib.jfnk_destroy.argtypes = [P]
    lib.jfnk_set_surface_flux.argtypes = [P, P]
    lib.jfnk_rhs.argtypes = [P, P, P]
    lib.jfnk_residual.argtypes = [P, P, P, P]
    lib.jfnk_jv.argtypes = [P, P, P, P, D, P, ctypes.POINTER(D)]
    lib.jfnk_precond_apply.argtypes = [P, P, P, P]
    lib.jfnk_step.argtypes = [P, P, ctypes.POINTER(Stats)]
    lib.jfnk_step_host.argtypes = [P, P, ctypes.POINTER(Stats)]
    lib.jfnk_budgets.argtypes = [P, P, ctypes.POINTER(Budget)]
    lib.jfnk_get_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.jfnk_kernel_timing.argtypes = [P, ctypes.c_uint]
    lib.jfnk_kernel_timing_read.argtypes = [P, ctypes.POINTER(KernelTime)]
    lib.jfnk_kernel_timing_sampled.argtypes = [P, ctypes.c_uint, I]
    lib.jfnk_budgets_static.argtypes = [ctypes.POINTER(Grid), P, P, P]
    lib.jfnk_autotune.argtypes = [P, P, ctypes.POINTER(ctypes.c_int)]
    lib.jfnk_set_tiles.argtypes = [P, I, I]
    lib.jfnk_set_cycle_graph.argtypes = [P, I]
    lib.jfnk_create_batch.argtypes = [I, ctypes.POINTER(Grid), ctypes.POINTER(Strat), ctypes.POINTER(Sgs),
                                      ctypes.POINTER(Opts), P, ctypes.POINTER(P)]
    lib.jfnk_destroy_batch.argtypes = [P]
    lib.jfnk_batch_handle.argtypes = [P, I, ctypes.POINTER(P)]
    lib.jfnk_step_batch.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(Stats), ctypes.POINTER(I)]
    lib.jfnk_unet_init.argtypes = [P, ctypes.c_ulonglong]
    lib.jfnk_unet_num_weights.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.jfnk_unet_get_weights.argtypes = [P, P, ctypes.c_size_t]
    lib.jfnk_unet_set_weights.argtypes = [P, P, ctypes.c_size_t]
    lib.jfnk_unet_capture.argtypes = [P, I, I]
    lib.jfnk_unet_pair_count.argtypes = [P, ctypes.POINTER(I)]
    lib.jfnk_unet_get_pair.argtypes = [P, I, P, P]
    lib.jfnk_unet_train.argtypes = [P, I, ctypes.c_float, P]
    lib.jfnk_unet_forward.argtypes = [P, P, P]
    lib.jfnk_unet_loss_grad.argtypes = [P, P, P, ctypes.POINTER(D), P]
    lib.jfnk_set_precond.argtypes = [P, I]
    lib.jfnk_unet_set_engine.argtypes = [P, I]
    lib.jfnk_unet_status.argtypes = [P]
    lib.jfnk_status_str.argtypes = [I]
    lib.jfnk_status_str.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "jfnk_status_str":
            getattr(lib, name).restype = I
    _lib = lib
    return lib


class JfnkError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load_library().jfnk_status_str(code).decode()
        super().__init__("%s: %s (status %d)" % (what, msg, code))


def _check(code: int, what: str, allow=(JFNK_OK,)):
    if code not in allow:
        raise JfnkError(code, what)
    return code


def structs_from_case(c: dict):
    """C structs from a parameter dict with sections grid/strat/sgs/opts."""
    g, s, q, o = c["grid"], c["strat"], c["sgs"], c["opts"]
    grid = Grid(g["dim"], g["nx"], g.get("ny", 1), g["nz"], g["lx"], g.get("ly", 1.0), g["lz"],
                g["bc_bottom"], g["bc_top"])
    strat = Strat(s["theta0"], s["beta"], s["pbar"], s["g"], s["gamma_p"], s["rho0"], s["cp"])
    sgs = Sgs(q["mode"], q["K_M"], q["K_H"], q["Cs"], q["Pr"])
    opts = Opts(o["precision"], o["wavelet_p"], o["krylov_m"], o["flexible"], o["precond"],
                o["pc_sweeps"], o["newton_rtol"], o["newton_atol_factor"], o["eta"],
                o["max_newton"], o["max_restarts"], o["dt"], o["scale_u"], o["scale_theta"],
                o["scale_p"])
    return grid, strat, sgs, opts


def _ptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor (validated)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _fptr(t) -> int:
    """Device pointer of a contiguous float32 CUDA tensor (validated)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


class Solver:
    """One grid's JFNK solver bound to a CUDA stream (defaults to torch's current stream)."""

    def __init__(self, case: dict, stream=None):
        import torch
        self.lib = load_library()
        self.case = case
        self.structs = structs_from_case(case)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ctypes.c_void_p()
        g, s, q, o = self.structs
        _check(self.lib.jfnk_create(ctypes.byref(g), ctypes.byref(s), ctypes.byref(q), ctypes.byref(o),
                                    sp, ctypes.byref(h)), "jfnk_create")
        self.h = h
        gr = case["grid"]
        nf = 4 if gr["dim"] == 2 else 5
        self.shape = (nf, gr["nz"], gr["nx"]) if gr["dim"] == 2 else (nf, gr["nz"], gr["ny"], gr["nx"])

    def close(self):
        if getattr(self, "h", None):
            self.lib.jfnk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_surface_flux(self, H):
        _check(self.lib.jfnk_set_surface_flux(self.h, None if H is None else _ptr(H)), "jfnk_set_surface_flux")

    def rhs(self, u, F):
        _check(self.lib.jfnk_rhs(self.h, _ptr(u), _ptr(F)), "jfnk_rhs")

    def residual(self, u_n, u, R):
        _check(self.lib.jfnk_residual(self.h, _ptr(u_n), _ptr(u), _ptr(R)), "jfnk_residual")

    def jv(self, u, v, Jv, eps: float = 0.0, F_u=None) -> float:
        e = ctypes.c_double(0.0)
        _check(self.lib.jfnk_jv(self.h, _ptr(u), None if F_u is None else _ptr(F_u), _ptr(v),
                                float(eps), _ptr(Jv), ctypes.byref(e)), "jfnk_jv")
        return e.value

    def precond_apply(self, u, r, z):
        _check(self.lib.jfnk_precond_apply(self.h, _ptr(u), _ptr(r), _ptr(z)), "jfnk_precond_apply")

    def step(self, u) -> dict:
        st = Stats()
        _check(self.lib.jfnk_step(self.h, _ptr(u), ctypes.byref(st)), "jfnk_step",
               allow=(JFNK_OK, JFNK_ERR_NOT_CONVERGED))
        return st.as_dict()

    def step_host(self, u_host) -> dict:
        """Step a pinned (or pageable) float64 CPU tensor in place through jfnk_step_host."""
        import torch
        if u_host.is_cuda or u_host.dtype != torch.float64 or not u_host.is_contiguous():
            raise ValueError("expected a contiguous float64 CPU tensor")
        st = Stats()
        _check(self.lib.jfnk_step_host(self.h, ctypes.c_void_p(u_host.data_ptr()), ctypes.byref(st)),
               "jfnk_step_host", allow=(JFNK_OK, JFNK_ERR_NOT_CONVERGED))
        return st.as_dict()

    def budgets(self, u) -> dict:
        b = Budget()
        _check(self.lib.jfnk_budgets(self.h, _ptr(u), ctypes.byref(b)), "jfnk_budgets")
        nf = self.shape[0]
        return {"E_k": b.E_k, "E_p": b.E_p, "sum_theta": b.sum_theta, "sum_div": b.sum_div,
                "max": list(b.max[:nf]), "min": list(b.min[:nf])}

    def kernel_timing(self, families=KERNEL_FAMILIES, every: int = 1):
        """Start CUDA-event timing of the named kernel families (resets the accumulators);
        launches inside GMRES cycles are timed at Krylov steps j = 0 mod `every`."""
        mask = 0
        for f in families:
            mask |= 1 << KERNEL_FAMILIES.index(f)
        _check(self.lib.jfnk_kernel_timing_sampled(self.h, mask, int(every)), "jfnk_kernel_timing_sampled")

    def kernel_timing_read(self) -> dict:
        arr = (KernelTime * len(KERNEL_FAMILIES))()
        _check(self.lib.jfnk_kernel_timing_read(self.h, arr), "jfnk_kernel_timing_read")
        return {name: {"launches": a.launches, "ms": a.ms, "bytes": a.bytes}
                for name, a in zip(KERNEL_FAMILIES, arr)}

    def autotune(self, u) -> tuple:
        """Pick the fastest stencil tile shapes for this grid (times every candidate)."""
        t = (ctypes.c_int * 2)()
        _check(self.lib.jfnk_autotune(self.h, _ptr(u), t), "jfnk_autotune")
        return (t[0], t[1])

    def set_tiles(self, tile_jv: int, tile_pc: int):
        _check(self.lib.jfnk_set_tiles(self.h, int(tile_jv), int(tile_pc)), "jfnk_set_tiles")

    def set_cycle_graph(self, steps: int):
        """Krylov steps per captured graph segment of a GMRES cycle (0: stream launches;
        -1: the library's default for the cycle's kind)."""
        _check(self.lib.jfnk_set_cycle_graph(self.h, int(steps)), "jfnk_set_cycle_graph")

    def launch_count(self) -> int:
        c = ctypes.c_longlong(0)
        _check(self.lib.jfnk_get_launch_count(self.h, ctypes.byref(c)), "jfnk_get_launch_count")
        return c.value

    # ------------------------------------------------ learned preconditioner
    def set_precond(self, mode: int):
        _check(self.lib.jfnk_set_precond(self.h, int(mode)), "jfnk_set_precond")

    def unet_init(self, seed: int = 0):
        _check(self.lib.jfnk_unet_init(self.h, int(seed)), "jfnk_unet_init")

    def unet_num_weights(self) -> int:
        c = ctypes.c_size_t(0)
        _check(self.lib.jfnk_unet_num_weights(self.h, ctypes.byref(c)), "jfnk_unet_num_weights")
        return c.value

    def unet_get_weights(self):
        """Float32 master weights as a numpy array (flat order of include/jfnk.h)."""
        import numpy as np
        w = np.zeros(self.unet_num_weights(), dtype=np.float32)
        _check(self.lib.jfnk_unet_get_weights(self.h, w.ctypes.data, w.size), "jfnk_unet_get_weights")
        return w

    def unet_set_weights(self, w):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(self.lib.jfnk_unet_set_weights(self.h, w.ctypes.data, w.size), "jfnk_unet_set_weights")

    def unet_capture(self, capacity: int, kinds: int = PAIRS_NEWTON | PAIRS_ARNOLDI):
        _check(self.lib.jfnk_unet_capture(self.h, int(capacity), int(kinds)), "jfnk_unet_capture")

    def unet_pair_count(self) -> int:
        c = ctypes.c_int(0)
        _check(self.lib.jfnk_unet_pair_count(self.h, ctypes.byref(c)), "jfnk_unet_pair_count")
        return c.value

    def unet_get_pair(self, i: int, X, T):
        _check(self.lib.jfnk_unet_get_pair(self.h, int(i), _fptr(X), _fptr(T)), "jfnk_unet_get_pair")

    def unet_train(self, epochs: int, lr: float) -> list:
        hist = (ctypes.c_double * max(1, int(epochs)))()
        _check(self.lib.jfnk_unet_train(self.h, int(epochs), float(lr), hist), "jfnk_unet_train")
        return list(hist[:epochs])

    def unet_forward(self, x, y):
        _check(self.lib.jfnk_unet_forward(self.h, _fptr(x), _fptr(y)), "jfnk_unet_forward")

    def unet_set_engine(self, engine: int):
        """Convolution engine of the network: UNET_TCGEN05 (default) or UNET_MMA_SYNC."""
        _check(self.lib.jfnk_unet_set_engine(self.h, int(engine)), "jfnk_unet_set_engine")

    def unet_status(self):
        """Raises JfnkError (JFNK_ERR_TIMEOUT) if a tensor-core wait of a convolution timed out."""
        _check(self.lib.jfnk_unet_status(self.h), "jfnk_unet_status")

    def unet_loss_grad(self, x, t, grads: bool = True):
        import numpy as np
        loss = ctypes.c_double(0.0)
        g = np.zeros(self.unet_num_weights(), dtype=np.float32) if grads else None
        _check(self.lib.jfnk_unet_loss_grad(self.h, _fptr(x), _fptr(t), ctypes.byref(loss),
                                            None if g is None else g.ctypes.data), "jfnk_unet_loss_grad")
        return loss.value, g


class Batch:
    """Independent grids stepped together (one handle and stream per instance)."""

    def __init__(self, cases, stream=None):
        import torch
        self.lib = load_library()
        self.cases = list(cases)
        n = len(self.cases)
        structs = [structs_from_case(c) for c in self.cases]
        arrs = [(t * n)(*[s[k] for s in structs]) for k, t in enumerate((Grid, Strat, Sgs, Opts))]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        b = ctypes.c_void_p()
        _check(self.lib.jfnk_create_batch(n, arrs[0], arrs[1], arrs[2], arrs[3], sp, ctypes.byref(b)),
               "jfnk_create_batch")
        self.b = b
        self.n = n

    def close(self):
        if getattr(self, "b", None):
            self.lib.jfnk_destroy_batch(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_surface_flux(self, i: int, H):
        h = ctypes.c_void_p()
        _check(self.lib.jfnk_batch_handle(self.b, i, ctypes.byref(h)), "jfnk_batch_handle")
        _check(self.lib.jfnk_set_surface_flux(h, None if H is None else _ptr(H)), "jfnk_set_surface_flux")

    def set_cycle_graph(self, steps: int):
        """jfnk_set_cycle_graph on every instance's handle."""
        for i in range(self.n):
            _check(self.lib.jfnk_set_cycle_graph(self.handle(i), int(steps)), "jfnk_set_cycle_graph")

    def handle(self, i: int):
        h = ctypes.c_void_p()
        _check(self.lib.jfnk_batch_handle(self.b, i, ctypes.byref(h)), "jfnk_batch_handle")
        return h

    def kernel_timing(self, families=KERNEL_FAMILIES):
        """CUDA-event timing of the named kernel families on every instance's handle."""
        mask = 0
        for f in families:
            mask |= 1 << KERNEL_FAMILIES.index(f)
        for i in range(self.n):
            _check(self.lib.jfnk_kernel_timing(self.handle(i), mask), "jfnk_kernel_timing")

    def kernel_timing_read(self) -> dict:
        """Per-family launches, summed launch time and algorithmic bytes over all instances."""
        out = {name: {"launches": 0, "ms": 0.0, "bytes": 0.0} for name in KERNEL_FAMILIES}
        for i in range(self.n):
            arr = (KernelTime * len(KERNEL_FAMILIES))()
            _check(self.lib.jfnk_kernel_timing_read(self.handle(i), arr), "jfnk_kernel_timing_read")
            for name, a in zip(KERNEL_FAMILIES, arr):
                out[name]["launches"] += a.launches
                out[name]["ms"] += a.ms
                out[name]["bytes"] += a.bytes
        return out

    def budgets(self, i: int, u) -> dict:
        """jfnk_budgets on instance i's handle (its stream is synchronised)."""
        b = Budget()
        _check(self.lib.jfnk_budgets(self.handle(i), _ptr(u), ctypes.byref(b)), "jfnk_budgets")
        nf = 4 if self.cases[i]["grid"]["dim"] == 2 else 5
        return {"E_k": b.E_k, "E_p": b.E_p, "sum_theta": b.sum_theta, "sum_div": b.sum_div,
                "max": list(b.max[:nf]), "min": list(b.min[:nf])}

    def step(self, states) -> list:
        ptrs = (ctypes.c_void_p * self.n)(*[_ptr(u) for u in states])
        stats = (Stats * self.n)()
        status = (ctypes.c_int * self.n)()
        _check(self.lib.jfnk_step_batch(self.b, ptrs, stats, status), "jfnk_step_batch",
               allow=(JFNK_OK, JFNK_ERR_NOT_CONVERGED))
        return [s.as_dict() for s in stats]
