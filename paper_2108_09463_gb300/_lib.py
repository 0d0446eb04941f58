"""ctypes binding of the C ABI in include/hmm.h (argument marshalling only).

Every step of the HMM path runs in the library's CUDA kernels; this module
only converts Python/torch arguments into the C structs and pointers. There is
no fallback: if libhmm_gb300.so is missing or fails to load, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmm_gb300.so")

HMM_OK = 0
STATUS_NAMES = {0: "HMM_OK", 1: "HMM_ERR_INVALID_ARG", 2: "HMM_ERR_UNSTABLE_DT",
                3: "HMM_ERR_OUT_OF_MEMORY", 4: "HMM_ERR_CUDA", 5: "HMM_ERR_TIMEOUT",
                6: "HMM_ERR_NONFINITE", 7: "HMM_ERR_NOT_INITIALISED"}
HMM_FP64_PLAIN, HMM_FP32_BATCHED = 0, 1

# The symbols include/hmm.h declares (checked by the CPU test suite).
EXPORTED = ("hmm_init", "hmm_micro_batch", "hmm_micro_batch_host", "hmm_macro_step",
            "hmm_macro_step_host", "hmm_macro_step_wave", "hmm_get_state", "hmm_set_state", "hmm_stats",
            "hmm_box_info", "hmm_set_face_table", "hmm_macro_dt", "hmm_micro_batch_noalloc",
            "hmm_flux_batch", "hmm_micro_batch_points", "hmm_plan_report", "hmm_fp32_fma_rate", "hmm_last_error",
            "hmm_destroy")
# The symbols include/hmm_dns.h declares.
EXPORTED_DNS = ("hmm_dns_init", "hmm_dns_set_face_table", "hmm_dns_step", "hmm_dns_step_host",
                "hmm_dns_reset", "hmm_dns_info", "hmm_dns_plan", "hmm_dns_last_error", "hmm_dns_destroy")


class HmmCoefTerm(ctypes.Structure):
    _fields_ = [("amp", c_double), ("kind", c_int * 3), ("scale", c_int * 3),
                ("omega", c_double * 3), ("phase", c_double * 3)]


class HmmParams(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n_macro", c_int * 3), ("L", c_double), ("alpha", c_double),
                ("alpha_micro", c_double), ("dt_macro", c_double), ("c0", c_double),
                ("n_terms", c_int), ("terms", POINTER(HmmCoefTerm)), ("eps", c_double),
                ("eps_field", POINTER(c_double)), ("box_n", c_int), ("box_n_field", POINTER(c_int)),
                ("pts_per_eps", c_double), ("mu_over_eps", c_double), ("micro_steps", c_int),
                ("dt_safety", c_double), ("px", c_int), ("qx", c_int), ("pt", c_int), ("qt", c_int),
                ("interp_order", c_int), ("stencil_order", c_int), ("precision", c_int),
                ("kernel_variant", c_int), ("micro_stepper", c_int), ("model", c_int), ("macro_stepper", c_int), ("tile_rows", c_int)]


class HmmDnsParams(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("L", c_double), ("alpha", c_double),
                ("dt", c_double), ("dt_safety", c_double), ("c0", c_double), ("n_terms", c_int),
                ("terms", POINTER(HmmCoefTerm)), ("eps", c_double), ("stencil_order", c_int),
                ("precision", c_int), ("reserved", c_int * 4)]


class HmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhmm_gb300.so and declare the signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_2108_09463_gb300.build.build() "
                          "(the HMM path has no CPU fallback)")
    lib = ctypes.CDLL(path)
    lib.hmm_init.argtypes = [POINTER(HmmParams), c_void_p, POINTER(c_void_p)]
    lib.hmm_micro_batch.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.hmm_micro_batch_host.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.hmm_flux_batch.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.hmm_micro_batch_points.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int]
    lib.hmm_macro_step.argtypes = [c_void_p, c_void_p, c_int]
    lib.hmm_macro_step_host.argtypes = [c_void_p, c_void_p, c_int]
    lib.hmm_macro_step_wave.argtypes = [c_void_p, c_void_p, c_int, c_int]
    lib.hmm_fp32_fma_rate.argtypes = [c_int, ctypes.POINTER(c_double)]
    lib.hmm_get_state.argtypes = [c_void_p, c_void_p, POINTER(c_longlong)]
    lib.hmm_set_state.argtypes = [c_void_p, c_void_p, c_longlong]
    lib.hmm_stats.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double)]
    lib.hmm_box_info.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hmm_macro_dt.argtypes = [c_void_p, POINTER(c_double)]
    lib.hmm_set_face_table.argtypes = [c_void_p, c_void_p, ctypes.c_longlong]
    lib.hmm_micro_batch_noalloc.argtypes = [POINTER(HmmParams), c_void_p, c_void_p, c_void_p]
    lib.hmm_last_error.argtypes = [c_void_p]
    lib.hmm_last_error.restype = c_char_p
    lib.hmm_plan_report.argtypes = [c_void_p]
    lib.hmm_plan_report.restype = c_char_p
    lib.hmm_destroy.argtypes = [c_void_p]
    lib.hmm_destroy.restype = None
    lib.hmm_dns_init.argtypes = [POINTER(HmmDnsParams), c_void_p, POINTER(c_void_p)]
    lib.hmm_dns_set_face_table.argtypes = [c_void_p, c_void_p, c_longlong]
    lib.hmm_dns_step.argtypes = [c_void_p, c_void_p, c_int]
    lib.hmm_dns_step_host.argtypes = [c_void_p, c_void_p, c_int]
    lib.hmm_dns_reset.argtypes = [c_void_p]
    lib.hmm_dns_info.argtypes = [c_void_p, POINTER(c_double), POINTER(c_longlong), POINTER(c_double)]
    lib.hmm_dns_plan.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]
    lib.hmm_dns_last_error.argtypes = [c_void_p]
    lib.hmm_dns_last_error.restype = c_char_p
    lib.hmm_dns_destroy.argtypes = [c_void_p]
    lib.hmm_dns_destroy.restype = None
    for name in EXPORTED + EXPORTED_DNS:
        if name not in ("hmm_last_error", "hmm_plan_report", "hmm_destroy", "hmm_dns_last_error",
                        "hmm_dns_destroy"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def make_params(cfg, precision=None, kernel_variant=0):
    """Fill HmmParams from a problem description (an object with HMMConfig's fields).

    Returns (params, keepalive): keepalive holds the arrays params points to.
    """
    import numpy as np
    terms = (HmmCoefTerm * max(1, len(cfg.terms)))()
    for i, t in enumerate(cfg.terms):
        terms[i].amp = float(t.amp)
        for k in range(3):
            terms[i].kind[k] = int(t.kind[k]) if k < cfg.dim else 0
            terms[i].scale[k] = int(t.scale[k])
            terms[i].omega[k] = float(t.omega[k])
            terms[i].phase[k] = float(t.phase[k])
    p = HmmParams()
    p.dim = int(cfg.dim)
    for k in range(3):
        p.n_macro[k] = int(list(cfg.n_macro)[k]) if k < len(cfg.n_macro) else 1
    p.L = float(cfg.L)
    p.alpha = float(cfg.alpha)
    p.alpha_micro = float(cfg.alpha_micro)
    p.dt_macro = float(cfg.dt_macro)
    p.c0 = float(cfg.c0)
    p.n_terms = len(cfg.terms)
    p.terms = ctypes.cast(terms, POINTER(HmmCoefTerm))
    p.eps = float(cfg.eps)
    keep = [terms]
    if cfg.eps_field is not None:
        ef = np.ascontiguousarray(cfg.eps_field, dtype=np.float64)
        keep.append(ef)
        p.eps_field = ef.ctypes.data_as(POINTER(c_double))
    p.box_n = int(cfg.box_n)
    if cfg.box_n_field is not None:
        nf = np.ascontiguousarray(cfg.box_n_field, dtype=np.int32)
        keep.append(nf)
        p.box_n_field = nf.ctypes.data_as(POINTER(c_int))
    p.pts_per_eps = float(cfg.pts_per_eps)
    p.mu_over_eps = float(cfg.mu_over_eps)
    p.micro_steps = int(cfg.micro_steps)
    p.dt_safety = float(cfg.dt_safety)
    p.px, p.qx, p.pt, p.qt = int(cfg.px), int(cfg.qx), int(cfg.pt), int(cfg.qt)
    p.interp_order = int(cfg.interp_order)
    p.stencil_order = int(cfg.stencil_order)
    p.precision = int(cfg.precision if precision is None else precision)
    p.kernel_variant = int(kernel_variant)
    p.micro_stepper = int(getattr(cfg, "micro_stepper", 0))
    p.model = int(getattr(cfg, "model", 0))
    p.macro_stepper = int(getattr(cfg, "macro_stepper", 0))
    p.tile_rows = int(getattr(cfg, "tile_rows", 0))
    return p, keep


def _fill_terms(cfg):
    terms = (HmmCoefTerm * max(1, len(cfg.terms)))()
    for i, t in enumerate(cfg.terms):
        terms[i].amp = float(t.amp)
        for k in range(3):
            terms[i].kind[k] = int(t.kind[k]) if k < cfg.dim else 0
            terms[i].scale[k] = int(t.scale[k])
            terms[i].omega[k] = float(t.omega[k])
            terms[i].phase[k] = float(t.phase[k])
    return terms


def make_dns_params(cfg, precision=None):
    """Fill HmmDnsParams from a problem description (an object with DNSConfig's
    fields). Returns (params, keepalive)."""
    terms = _fill_terms(cfg)
    p = HmmDnsParams()
    p.dim = int(cfg.dim)
    for k in range(3):
        p.n[k] = int(list(cfg.n)[k]) if k < len(cfg.n) else 1
    p.L = float(cfg.L)
    p.alpha = float(cfg.alpha)
    p.dt = float(cfg.dt)
    p.dt_safety = float(cfg.dt_safety)
    p.c0 = float(cfg.c0)
    p.n_terms = len(cfg.terms)
    p.terms = ctypes.cast(terms, POINTER(HmmCoefTerm))
    p.eps = float(cfg.eps)
    p.stencil_order = int(cfg.stencil_order)
    p.precision = int(cfg.precision if precision is None else precision)
    return p, [terms]


def _ptr(t) -> int:
    return t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data


class HMM:
    """One HMM problem on the current CUDA device (a handle of the C ABI)."""

    def __init__(self, cfg, precision=None, stream=None, kernel_variant=0, face_table=None):
        import torch
        self.lib = load_library()
        self.cfg = cfg
        self.P = int(cfg.n_points)
        params, keep = make_params(cfg, precision, kernel_variant)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = c_void_p()
        st = self.lib.hmm_init(ctypes.byref(params), c_void_p(stream.cuda_stream), ctypes.byref(h))
        del keep
        if st != HMM_OK:
            raise HmmError(st, self.lib.hmm_last_error(None).decode())
        self.h = h
        if face_table is not None:
            self.set_face_table(face_table)

    def set_face_table(self, table):
        """Tabulated a^eps at every face of every box (see hmm_set_face_table)."""
        import numpy as np
        t = np.ascontiguousarray(table, dtype=np.float64)
        self._check(self.lib.hmm_set_face_table(self.h, t.ctypes.data, int(t.size)))

    def _check(self, st):
        if st != HMM_OK:
            raise HmmError(st, self.lib.hmm_last_error(self.h).decode())

    def _field(self, M):
        import torch
        if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float64
                and M.is_contiguous() and tuple(M.shape) == (3, self.P)):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape (3, {self.P})")
        return M

    def micro_batch(self, M, out=None):
        import torch
        M = self._field(M)
        if out is None:
            out = torch.empty_like(M)
        self._check(self.lib.hmm_micro_batch(self.h, c_void_p(M.data_ptr()), c_void_p(self._field(out).data_ptr())))
        return out

    def micro_batch_points(self, M, points, out=None):
        """H_avg at the listed macro points only (hmm_micro_batch_points); ``out``
        (3, P) keeps its other entries. Returns out."""
        import numpy as np
        import torch
        M = self._field(M)
        if out is None:
            out = torch.zeros_like(M)
        pts = np.ascontiguousarray(points, dtype=np.int32)
        self._check(self.lib.hmm_micro_batch_points(self.h, c_void_p(M.data_ptr()), c_void_p(self._field(out).data_ptr()),
                                                    c_void_p(pts.ctypes.data), int(pts.size)))
        return out

    def flux_batch(self, M, out=None):
        """Flux model: the averaged flux columns F_avg, (d, 3, P) (see hmm_flux_batch)."""
        import torch
        M = self._field(M)
        d = int(self.cfg.dim)
        if out is None:
            out = torch.empty((d, 3, self.P), dtype=torch.float64, device=M.device)
        if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and tuple(out.shape) == (d, 3, self.P)):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape ({d}, 3, {self.P})")
        self._check(self.lib.hmm_flux_batch(self.h, c_void_p(M.data_ptr()), c_void_p(out.data_ptr())))
        return out

    def micro_batch_host(self, M, out):
        """M, out: contiguous float64 host arrays/tensors of shape (3, P)."""
        self._check(self.lib.hmm_micro_batch_host(self.h, c_void_p(_ptr(M)), c_void_p(_ptr(out))))
        return out

    def macro_step(self, M, n_steps=1):
        M = self._field(M)
        self._check(self.lib.hmm_macro_step(self.h, c_void_p(M.data_ptr()), int(n_steps)))
        return M

    def macro_step_host(self, M, n_steps=1):
        self._check(self.lib.hmm_macro_step_host(self.h, c_void_p(_ptr(M)), int(n_steps)))
        return M

    def macro_step_wave(self, M, wave, n_waves):
        """Wave `wave` of n_waves of one macro step (hmm_macro_step_wave); the last
        wave updates M in place."""
        M = self._field(M)
        self._check(self.lib.hmm_macro_step_wave(self.h, c_void_p(M.data_ptr()), int(wave), int(n_waves)))
        return M

    def get_state(self):
        import torch
        hist = torch.empty((2, 3, self.P), dtype=torch.float64, device="cuda")
        j = c_longlong()
        self._check(self.lib.hmm_get_state(self.h, c_void_p(hist.data_ptr()), ctypes.byref(j)))
        return hist, int(j.value)

    def set_state(self, hist, j):
        ptr = c_void_p(hist.data_ptr()) if hist is not None else c_void_p()
        self._check(self.lib.hmm_set_state(self.h, ptr, int(j)))

    def stats(self):
        lu, ms = c_double(), c_double()
        self._check(self.lib.hmm_stats(self.h, ctypes.byref(lu), ctypes.byref(ms)))
        return lu.value, ms.value

    def box_info(self):
        import numpy as np
        dt, mu, dx = (np.empty(self.P) for _ in range(3))
        n = np.empty(self.P, dtype=np.int32)
        self._check(self.lib.hmm_box_info(self.h, c_void_p(dt.ctypes.data), c_void_p(mu.ctypes.data),
                                          c_void_p(dx.ctypes.data), c_void_p(n.ctypes.data)))
        return dict(dt=dt, mu=mu, dx=dx, N=n)

    def plan_report(self):
        """The resident-plan autotuner's timings (hmm_plan_report), one line per box size."""
        return self.lib.hmm_plan_report(self.h).decode()

    def macro_dt(self):
        v = c_double()
        self._check(self.lib.hmm_macro_dt(self.h, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_fma_rate(packed=True):
    """The current device's FP32 FMA rate in flop/s (hmm_fp32_fma_rate): paired
    FP32x2 FMAs (packed) or scalar FMAs."""
    lib = load_library()
    r = c_double()
    st = lib.hmm_fp32_fma_rate(1 if packed else 0, ctypes.byref(r))
    if st != HMM_OK:
        raise HmmError(st, lib.hmm_last_error(None).decode())
    return r.value


def micro_batch_noalloc(cfg, M, out, stream=None):
    """hmm_micro_batch_noalloc: the FP32 micro batch without any device allocation.

    For callers that cannot allocate device memory (see include/hmm.h): all
    working memory comes from a fixed 32 MiB array inside the library. M and
    out are contiguous float64 CUDA tensors of shape (3, P); ``cfg`` describes a
    batch of uniform boxes. Raises HmmError on failure.
    """
    import torch
    lib = load_library()
    params, keep = make_params(cfg, precision=HMM_FP32_BATCHED)
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib.hmm_micro_batch_noalloc(ctypes.byref(params), c_void_p(M.data_ptr()),
                                     c_void_p(out.data_ptr()), c_void_p(stream.cuda_stream))
    del keep
    if st != HMM_OK:
        raise HmmError(st, lib.hmm_last_error(None).decode())
    return out


class DNS:
    """One direct simulation resolving eps on the current CUDA device (a handle
    of include/hmm_dns.h). ``face_table``: d blocks of G positive face values
    for coefficients that are not separable sums (see hmm_dns_set_face_table)."""

    def __init__(self, cfg, precision=None, stream=None, face_table=None):
        import torch
        self.lib = load_library()
        self.cfg = cfg
        self.G = int(cfg.n_points)
        params, keep = make_dns_params(cfg, precision)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = c_void_p()
        st = self.lib.hmm_dns_init(ctypes.byref(params), c_void_p(stream.cuda_stream), ctypes.byref(h))
        del keep
        if st != HMM_OK:
            raise HmmError(st, self.lib.hmm_dns_last_error(None).decode())
        self.h = h
        if face_table is not None:
            self.set_face_table(face_table)

    def _check(self, st):
        if st != HMM_OK:
            raise HmmError(st, self.lib.hmm_dns_last_error(self.h).decode())

    def set_face_table(self, table):
        import numpy as np
        t = np.ascontiguousarray(table, dtype=np.float64)
        self._check(self.lib.hmm_dns_set_face_table(self.h, t.ctypes.data, int(t.size)))

    def step(self, M, n_steps=1):
        """n_steps steps in place on M, a contiguous float64 CUDA tensor (3, G)."""
        import torch
        if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float64
                and M.is_contiguous() and tuple(M.shape) == (3, self.G)):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape (3, {self.G})")
        self._check(self.lib.hmm_dns_step(self.h, c_void_p(M.data_ptr()), int(n_steps)))
        return M

    def step_host(self, M, n_steps=1):
        """As step with M a contiguous float64 host array/tensor (3, G)."""
        self._check(self.lib.hmm_dns_step_host(self.h, c_void_p(_ptr(M)), int(n_steps)))
        return M

    def reset(self):
        self._check(self.lib.hmm_dns_reset(self.h))

    def info(self):
        dt, j, ms = c_double(), c_longlong(), c_double()
        self._check(self.lib.hmm_dns_info(self.h, ctypes.byref(dt), ctypes.byref(j), ctypes.byref(ms)))
        return dict(dt=dt.value, j=int(j.value), last_ms=ms.value)

    def plan(self):
        """The time-stepping kernel's work plan (see hmm_dns_plan)."""
        st, ch, it = c_int(), c_int(), c_int()
        self._check(self.lib.hmm_dns_plan(self.h, ctypes.byref(st), ctypes.byref(ch), ctypes.byref(it)))
        return dict(strips=st.value, chunk=ch.value, items=it.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_dns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
