"""Python binding of libhelm (include/helm.h): argument marshalling only.

Every function below has the name of the C entry point it forwards to and
takes raw device pointers (ints) plus sizes, exactly like the C ABI.  The
``Solver`` class is a convenience wrapper that passes torch tensors'
pointers and the current CUDA stream; all arithmetic happens in the CUDA
kernels of libhelm.  There is no CPU fallback: if the library is missing
the import of this module succeeds but every call raises.
"""
from __future__ import annotations

import ctypes
import os

HELM_OK = 0
HELM_ENOCONV = 1
HELM_EINVAL = -1
HELM_ENOMEM = -2
HELM_ECUDA = -3
HELM_ETIMEOUT = -4
HELM_ENOTSUP = -5
HELM_FP32 = 0           # stored factor formats (opts.precision)
HELM_FP16 = 1
HELM_SPLIT_FP16 = 2
PRECISIONS = {"fp32": HELM_FP32, "fp16": HELM_FP16, "split_fp16": HELM_SPLIT_FP16}
HELM_ONE_FRONT = 0      # opts.schedule
HELM_TWO_FRONT = 1
SCHEDULES = {"one_front": HELM_ONE_FRONT, "two_front": HELM_TWO_FRONT}
HELM_CHAIN = 0          # opts.apply_form
HELM_DENSE = 1
APPLY_FORMS = {"chain": HELM_CHAIN, "dense": HELM_DENSE}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libhelm.so")
_lib = None


class helm_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("b_aux", ctypes.c_int), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("pml_C", ctypes.c_double), ("rhs_per_cta", ctypes.c_int),
                ("schedule", ctypes.c_int), ("apply_form", ctypes.c_int), ("debug_unmet_wait", ctypes.c_int),
                ("wait_cycles", ctypes.c_longlong), ("dense_clusters", ctypes.c_int), ("reserved_", ctypes.c_int)]


class helm_problem(ctypes.Structure):
    _fields_ = [("c", ctypes.c_void_p), ("omega", ctypes.c_double), ("n", ctypes.c_int), ("b", ctypes.c_int),
                ("d", ctypes.c_int), ("nrhs", ctypes.c_int)]


class helm_stats(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_longlong), ("sweep_ms", ctypes.c_double),
                ("stencil_launches", ctypes.c_longlong), ("stencil_ms", ctypes.c_double),
                ("rhs_applied", ctypes.c_longlong)]


class helm_candidate(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("apply_form", ctypes.c_int), ("precision", ctypes.c_int),
                ("schedule", ctypes.c_int), ("b_aux", ctypes.c_int)]


class helm_tune_result(ctypes.Structure):
    _fields_ = [("cand", helm_candidate), ("status", ctypes.c_int), ("iters_max", ctypes.c_int),
                ("relres_max", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("score", ctypes.c_double), ("stored_bytes", ctypes.c_size_t)]


class HelmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {helm_strerror(code)} (code {code})")
        self.code = code


_VP = ctypes.c_void_p
_SIGS = {
    "helm_default_opts": (None, [ctypes.POINTER(helm_opts)]),
    "helm_setup": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(helm_opts), _VP, ctypes.POINTER(_VP)]),
    "helm_setup_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(helm_problem), ctypes.POINTER(helm_opts),
                                        _VP, ctypes.POINTER(_VP)]),
    "helm_apply_precond": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "helm_apply_slab": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP]),
    "helm_apply_precond_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "helm_matvec": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    "helm_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _VP]),
    "helm_status": (ctypes.c_int, [_VP, _VP]),
    "helm_apply_batch": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
    "helm_solve_batch": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _VP]),
    "helm_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP]),
    "helm_tune": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(helm_opts),
                                 ctypes.POINTER(helm_candidate), ctypes.c_int, _VP, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.POINTER(helm_tune_result), ctypes.POINTER(ctypes.c_int),
                                 _VP]),
    "helm_solve_adjoint": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _VP]),
    "helm_velocity_gradient": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "helm_update_velocity": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _VP]),
    "helm_affected_problems": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "helm_enable_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "helm_get_stats": (ctypes.c_int, [_VP, ctypes.c_void_p]),
    "helm_reset_stats": (None, [_VP]),
    "helm_grid_size": (ctypes.c_int, [_VP]),
    "helm_num_blocks": (ctypes.c_int, [_VP]),
    "helm_slab_layers": (ctypes.c_int, [_VP, ctypes.c_int]),
    "helm_factor_bytes": (ctypes.c_size_t, [_VP]),
    "helm_dense_operator": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _VP, _VP]),
    "helm_launch_count": (ctypes.c_longlong, [_VP]),
    "helm_destroy": (None, [_VP]),
    "helm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """Load libhelm.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libhelm.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str, allow=(HELM_OK,)):
    if code not in allow:
        raise HelmError(code, what)
    return code


def helm_strerror(code: int) -> str:
    return lib().helm_strerror(code).decode()


def helm_default_opts() -> helm_opts:
    o = helm_opts()
    lib().helm_default_opts(ctypes.byref(o))
    return o


def helm_setup(c_ptr: int, omega: float, n: int, b: int, d: int, opts: helm_opts | None = None,
               stream: int = 0) -> int:
    h = _VP()
    code = lib().helm_setup(_VP(c_ptr), omega, n, b, d,
                            ctypes.byref(opts) if opts is not None else None, _VP(stream),
                            ctypes.byref(h))
    _check(code, "helm_setup")
    return h.value


def helm_setup_batch(problems, opts: helm_opts | None = None, stream: int = 0) -> int:
    """One handle over several problems: problems is a list of
    (c_ptr, omega, n, b, d, nrhs); vectors for the handle are the problems'
    vectors back to back."""
    arr = (helm_problem * len(problems))(*[helm_problem(_VP(c), om, n, b, d, r)
                                           for c, om, n, b, d, r in problems])
    h = _VP()
    code = lib().helm_setup_batch(len(problems), arr, ctypes.byref(opts) if opts is not None else None,
                                  _VP(stream), ctypes.byref(h))
    _check(code, "helm_setup_batch")
    return h.value


def pad_velocity(c_phys, b: int):
    """Extend a physical velocity (n x n x n, indexed [z, y, x]) by b layers on
    every face with the nearest physical value, the padded-grid convention the
    library expects.  Accepts a numpy array or a torch tensor (same type out)."""
    try:
        import torch
        if isinstance(c_phys, torch.Tensor):
            return torch.nn.functional.pad(c_phys[None, None], (b,) * 6, mode="replicate")[0, 0].contiguous()
    except ImportError:
        pass
    import numpy as np
    return np.pad(np.asarray(c_phys), b, mode="edge")


def helm_apply_precond(h: int, r_ptr: int, z_ptr: int, nrhs: int, stream: int = 0) -> int:
    return _check(lib().helm_apply_precond(_VP(h), _VP(r_ptr), _VP(z_ptr), nrhs, _VP(stream)),
                  "helm_apply_precond")


HELM_NOALLOC_SCRATCH_BYTES = 16 << 20


def helm_apply_precond_noalloc(h: int, r_ptr: int, z_ptr: int, nrhs: int, stream: int = 0) -> int:
    """helm_apply_precond without any device allocation (fixed library scratch)."""
    return _check(lib().helm_apply_precond_noalloc(_VP(h), _VP(r_ptr), _VP(z_ptr), nrhs, _VP(stream)),
                  "helm_apply_precond_noalloc")


def helm_apply_slab(h: int, M: int, g_ptr: int, v_ptr: int, nrhs: int, stream: int = 0) -> int:
    return _check(lib().helm_apply_slab(_VP(h), M, _VP(g_ptr), _VP(v_ptr), nrhs, _VP(stream)),
                  "helm_apply_slab")


def helm_matvec(h: int, x_ptr: int, y_ptr: int, nrhs: int, fp64: int = 0, stream: int = 0) -> int:
    return _check(lib().helm_matvec(_VP(h), _VP(x_ptr), _VP(y_ptr), nrhs, fp64, _VP(stream)),
                  "helm_matvec")


def helm_solve(h: int, f_ptr: int, u_ptr: int, nrhs: int, tol: float, stream: int = 0):
    """Returns (code, iters list, relres list); code is HELM_OK or HELM_ENOCONV."""
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    code = lib().helm_solve(_VP(h), _VP(f_ptr), _VP(u_ptr), nrhs, tol, its, rel, _VP(stream))
    _check(code, "helm_solve", allow=(HELM_OK, HELM_ENOCONV))
    return code, list(its), list(rel)


def helm_solve_adjoint(h: int, g_ptr: int, lam_ptr: int, nrhs: int, tol: float, stream: int = 0):
    """A^T lambda = g; returns (code, iters, relres) like helm_solve."""
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    code = lib().helm_solve_adjoint(_VP(h), _VP(g_ptr), _VP(lam_ptr), nrhs, tol, its, rel, _VP(stream))
    _check(code, "helm_solve_adjoint", allow=(HELM_OK, HELM_ENOCONV))
    return code, list(its), list(rel)


def helm_velocity_gradient(h: int, lam_ptr: int, u_ptr: int, nrhs: int, grad_ptr: int, stream: int = 0) -> int:
    return _check(lib().helm_velocity_gradient(_VP(h), _VP(lam_ptr), _VP(u_ptr), nrhs, _VP(grad_ptr),
                                               _VP(stream)), "helm_velocity_gradient")


def helm_tune(c_ptr: int, omega: float, n: int, b: int, f_ptr: int, nrhs: int, candidates, tol: float = 1e-6,
              setup_weight: float = 0.0, base=None, stream: int = 0):
    """The setup-level autotuner (see helm_tune in helm.h).  candidates: a
    sequence of (d, apply_form, precision) or (d, apply_form, precision,
    schedule, b_aux) with forms / precisions / schedules given as names
    ("chain", "dense"; "fp32", "fp16", "split_fp16"; "one_front", "two_front")
    or codes (schedule one front and b_aux = b when omitted).  Returns (index of
    the fastest passing candidate or -1, list of result dicts)."""
    def code(v, table):
        return table[v] if isinstance(v, str) else int(v)

    def cand(t):
        d, fm, pr = t[:3]
        sc, ba = (t[3], t[4]) if len(t) > 3 else ("one_front", 0)
        return helm_candidate(int(d), code(fm, APPLY_FORMS), code(pr, PRECISIONS), code(sc, SCHEDULES), int(ba))
    nc = len(candidates)
    cs = (helm_candidate * nc)(*[cand(t) for t in candidates])
    res = (helm_tune_result * nc)()
    best = ctypes.c_int(-1)
    rc = lib().helm_tune(_VP(c_ptr), omega, n, b, ctypes.byref(base) if base is not None else None, cs, nc,
                         _VP(f_ptr), nrhs, tol, setup_weight, res, ctypes.byref(best), _VP(stream))
    _check(rc, "helm_tune", allow=(HELM_OK, HELM_ENOCONV, HELM_ENOTSUP, HELM_ENOMEM))
    out = [{"d": r.cand.d, "apply_form": r.cand.apply_form, "precision": r.cand.precision,
            "schedule": r.cand.schedule, "b_aux": r.cand.b_aux, "status": r.status,
            "iters_max": r.iters_max, "relres_max": r.relres_max, "setup_ms": r.setup_ms,
            "solve_ms": r.solve_ms, "score": r.score, "stored_bytes": r.stored_bytes} for r in res]
    return best.value, out


def helm_update_velocity(h: int, c_ptr: int, box, stream: int = 0) -> int:
    """Local factor update; box = (x0, x1, y0, y1, z0, z1) node ranges of the
    padded grid (half-open).  Returns the number of quasi-1D problems rebuilt."""
    bx = (ctypes.c_int * 6)(*[int(v) for v in box])
    n = ctypes.c_int(0)
    _check(lib().helm_update_velocity(_VP(h), _VP(c_ptr), bx, ctypes.byref(n), _VP(stream)), "helm_update_velocity")
    return n.value


def helm_affected_problems(n: int, b: int, d: int, box, b_aux: int = 0, schedule: int = 0):
    """(first slab, last slab, first line block, last line block) touched by a
    velocity change in box (host only; -1 entries when none)."""
    bx = (ctypes.c_int * 6)(*[int(v) for v in box])
    out = (ctypes.c_int * 4)()
    _check(lib().helm_affected_problems(n, b, d, b_aux, int(schedule), bx, out), "helm_affected_problems")
    return tuple(out)


HELM_MAX_BATCH = 8


def _ptrs(xs):
    return (_VP * len(xs))(*[_VP(x) for x in xs])


def helm_apply_batch(hs, r_ptrs, z_ptrs, nrhs, stream: int = 0) -> int:
    n = len(hs)
    return _check(lib().helm_apply_batch(_ptrs(hs), _ptrs(r_ptrs), _ptrs(z_ptrs), (ctypes.c_int * n)(*nrhs),
                                         n, _VP(stream)), "helm_apply_batch")


def helm_solve_batch(hs, f_ptrs, u_ptrs, nrhs, tol: float, stream: int = 0):
    n = len(hs)
    tot = sum(nrhs)
    its = (ctypes.c_int * tot)()
    rel = (ctypes.c_double * tot)()
    code = lib().helm_solve_batch(_ptrs(hs), _ptrs(f_ptrs), _ptrs(u_ptrs), (ctypes.c_int * n)(*nrhs), n, tol,
                                  its, rel, _VP(stream))
    _check(code, "helm_solve_batch", allow=(HELM_OK, HELM_ENOCONV))
    return code, list(its), list(rel)


def helm_autotune(h: int, nrhs: int, stream: int = 0) -> int:
    out = ctypes.c_int()
    _check(lib().helm_autotune(_VP(h), nrhs, ctypes.byref(out), _VP(stream)), "helm_autotune")
    return out.value


def helm_status(h: int, stream: int = 0) -> int:
    return _check(lib().helm_status(_VP(h), _VP(stream)), "helm_status")


def helm_enable_timing(h: int, on: bool) -> int:
    return _check(lib().helm_enable_timing(_VP(h), 1 if on else 0), "helm_enable_timing")


def helm_get_stats(h: int) -> helm_stats:
    st = helm_stats()
    _check(lib().helm_get_stats(_VP(h), ctypes.addressof(st)), "helm_get_stats")
    return st


def helm_reset_stats(h: int) -> None:
    lib().helm_reset_stats(_VP(h))


def helm_grid_size(h: int) -> int:
    return lib().helm_grid_size(_VP(h))


def helm_num_blocks(h: int) -> int:
    return lib().helm_num_blocks(_VP(h))


def helm_slab_layers(h: int, M: int) -> int:
    return lib().helm_slab_layers(_VP(h), M)


def helm_factor_bytes(h: int) -> int:
    return lib().helm_factor_bytes(_VP(h))


def helm_dense_operator(h: int, M: int, Mp: int, dir: int = 0, g_ptr: int = 0, stream: int = 0):
    """Size and index sets of one stored restricted operator of a dense handle,
    and (if g_ptr) its values decoded into the device buffer g_ptr
    (complex64 [n_out][n_in]).  Returns (n_out, n_in, in_rect, out_rects) with
    rects as (first line, lines, first window z row, z rows)."""
    no, ni = ctypes.c_int(), ctypes.c_int()
    rects = (ctypes.c_int * 13)()
    _check(lib().helm_dense_operator(_VP(h), M, Mp, dir, ctypes.byref(no), ctypes.byref(ni), rects,
                                     _VP(g_ptr) if g_ptr else None, _VP(stream)), "helm_dense_operator")
    r = list(rects)
    nrect = r[0]
    return no.value, ni.value, tuple(r[1:5]), [tuple(r[5:9]), tuple(r[9:13])][:nrect]


def helm_launch_count(h: int) -> int:
    return lib().helm_launch_count(_VP(h))


def helm_destroy(h: int) -> None:
    lib().helm_destroy(_VP(h))


class Solver:
    """Owns one helm handle; methods take torch CUDA tensors.

    c: float32 (N, N, N) on the padded grid; vectors: complex64 (R, N, N, N).
    """

    def __init__(self, c, omega: float, n: int, b: int, d: int = 1, b_aux: int = 0,
                 restart: int = 30, maxit: int = 300, pml_C: float = 10.0, rhs_per_cta: int = 0,
                 precision: str = "fp32", apply_form: str = "chain", wait_cycles: int = 0,
                 debug_unmet_wait: bool = False, dense_clusters: int = 0, schedule: str = "one_front"):
        import torch
        if not c.is_cuda or c.dtype != torch.float32 or not c.is_contiguous():
            raise ValueError("c must be a contiguous float32 CUDA tensor")
        self.n, self.b, self.d, self.omega = n, b, d, omega
        self.N = n + 2 * b
        o = helm_default_opts()
        o.b_aux, o.restart, o.maxit, o.pml_C, o.rhs_per_cta = b_aux, restart, maxit, pml_C, rhs_per_cta
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        o.precision = PRECISIONS[precision]
        if apply_form not in APPLY_FORMS:
            raise ValueError(f"apply_form must be one of {sorted(APPLY_FORMS)}")
        o.apply_form = APPLY_FORMS[apply_form]
        o.wait_cycles = int(wait_cycles)
        o.debug_unmet_wait = 1 if debug_unmet_wait else 0
        o.dense_clusters = int(dense_clusters)
        if schedule not in SCHEDULES:
            raise ValueError(f"schedule must be one of {sorted(SCHEDULES)}")
        o.schedule = SCHEDULES[schedule]
        self.schedule = schedule
        self.precision = precision
        self.apply_form = apply_form
        self.opts = o
        self.handle = helm_setup(c.data_ptr(), omega, n, b, d, o, self._stream())

    @staticmethod
    def _stream() -> int:
        import torch
        return torch.cuda.current_stream().cuda_stream

    def _vec(self, x, dtype_name="complex64"):
        import torch
        dt = getattr(torch, dtype_name)
        if not x.is_cuda or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {dtype_name} CUDA tensor")
        if x.is_complex() and x.is_conj():
            raise ValueError("tensor has a pending conjugation; call resolve_conj() first")
        if x.numel() % (self.N ** 3):
            raise ValueError("vector size is not a multiple of N^3")
        return x.numel() // (self.N ** 3)

    def apply(self, r, z=None):
        import torch
        R = self._vec(r)
        z = torch.empty_like(r) if z is None else z
        helm_apply_precond(self.handle, r.data_ptr(), z.data_ptr(), R, self._stream())
        return z

    def apply_slab(self, M: int, g, v=None):
        import torch
        if not g.is_cuda or g.dtype != torch.complex64 or not g.is_contiguous():
            raise ValueError("g must be a contiguous complex64 CUDA tensor")
        Lz = helm_slab_layers(self.handle, M)
        R = g.numel() // (Lz * self.N * self.N)
        v = torch.empty_like(g) if v is None else v
        helm_apply_slab(self.handle, M, g.data_ptr(), v.data_ptr(), R, self._stream())
        return v

    def matvec(self, x, y=None):
        import torch
        fp64 = 1 if x.dtype == torch.complex128 else 0
        R = self._vec(x, "complex128" if fp64 else "complex64")
        y = torch.empty_like(x) if y is None else y
        helm_matvec(self.handle, x.data_ptr(), y.data_ptr(), R, fp64, self._stream())
        return y

    def solve(self, f, tol: float = 1e-6, u=None):
        import torch
        R = self._vec(f)
        u = torch.empty_like(f) if u is None else u
        code, its, rel = helm_solve(self.handle, f.data_ptr(), u.data_ptr(), R, tol, self._stream())
        return u, its, rel, code

    def status(self):
        return helm_status(self.handle, self._stream())

    def update_velocity(self, c_new, box) -> int:
        """Local factor update after the velocity changed inside box (see
        helm_update_velocity); c_new is the whole padded-grid velocity."""
        import torch
        if not c_new.is_cuda or c_new.dtype != torch.float32 or not c_new.is_contiguous():
            raise ValueError("c_new must be a contiguous float32 CUDA tensor")
        if c_new.numel() != self.N ** 3:
            raise ValueError("c_new must hold N^3 values")
        return helm_update_velocity(self.handle, c_new.data_ptr(), box, self._stream())

    def dense_operator(self, M: int, Mp: int, dir: int = 0):
        """(G as a complex64 CUDA tensor [n_out][n_in], in_rect, out_rects) of a dense handle."""
        import torch
        no, ni, rin, rout = helm_dense_operator(self.handle, M, Mp, dir)
        G = torch.empty((no, ni), dtype=torch.complex64, device="cuda")
        helm_dense_operator(self.handle, M, Mp, dir, G.data_ptr(), self._stream())
        return G, rin, rout

    @property
    def launches(self) -> int:
        return helm_launch_count(self.handle)

    @property
    def factor_bytes(self) -> int:
        return helm_factor_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            helm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
