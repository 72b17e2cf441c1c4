"""ctypes binding of libpdhcg.so with the C ABI's names (include/pdhcg.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Pointers may be host or device addresses (the library detects which).
Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdhcg.so")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

PDHCG_OK, PDHCG_ERR_INVALID, PDHCG_ERR_CUDA, PDHCG_ERR_OOM = 0, 1, 2, 3
PDHCG_ERR_NOT_CONVERGED, PDHCG_ERR_NUMERIC, PDHCG_ERR_TIMEOUT, PDHCG_ERR_NO_STATE = 4, 5, 6, 7
PDHCG_FP64, PDHCG_MIXED = 0, 1
PDHCG_VAL_F64, PDHCG_VAL_F32 = 0, 1


class pdhcg_market(ctypes.Structure):
    _fields_ = [("n", c_int32), ("m", c_int32), ("nnz", c_int64), ("row_ptr", c_void_p), ("col", c_void_p),
                ("val", c_void_p), ("val_type", ctypes.c_int), ("w", c_void_p)]


class pdhcg_params(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int64), ("time_limit_s", c_double), ("prec", ctypes.c_int),
                ("kkt_check_every", c_int32), ("beta_suff", c_double), ("beta_nec", c_double),
                ("beta_art", c_double), ("theta", c_double), ("eta_lo", c_double), ("eta_hi", c_double),
                ("eta0_scale", c_double), ("omega_reset_every", c_int32), ("omega_range", c_double),
                ("row_solve_max_iter", c_int32), ("tight_kappa", c_double), ("verbose", c_int32),
                ("timing", c_int32), ("batch_lanes", c_int32),
                ("section_count", c_int32), ("section_tol", c_double)]


class pdhcg_info(ctypes.Structure):
    _fields_ = [("iters", c_int64), ("passes", c_int64), ("restarts", c_int32), ("kkt", c_double),
                ("r_primal", c_double), ("r_dual", c_double), ("r_gap", c_double), ("solve_ms", c_double),
                ("setup_ms", c_double), ("bytes_moved", c_double), ("row_solve_capped", c_int32),
                ("status", ctypes.c_int), ("prox_ms", c_double), ("prox_launches", c_int64), ("kkt_ms", c_double),
                ("kernel_launches", c_int64), ("row_solve_evals", c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.POINTER
_SIGS = {
    "pdhcg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pdhcg_version": (c_int32, []),
    "pdhcg_last_error": (ctypes.c_char_p, []),
    "pdhcg_default_params": (None, [_P(pdhcg_params)]),
    "pdhcg_create": (ctypes.c_int, [_P(c_void_p), c_void_p]),
    "pdhcg_destroy": (ctypes.c_int, [c_void_p]),
    "pdhcg_fisher_solve": (ctypes.c_int, [c_void_p, _P(pdhcg_market), _P(pdhcg_params), c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, _P(pdhcg_info)]),
    "pdhcg_fisher_solve_pdhg": (ctypes.c_int, [c_void_p, _P(pdhcg_market), _P(pdhcg_params), c_int32, c_void_p,
                                               c_void_p, c_void_p, _P(pdhcg_info)]),
    "pdhcg_fisher_begin": (ctypes.c_int, [c_void_p, _P(pdhcg_market), _P(pdhcg_params), c_void_p, c_void_p]),
    "pdhcg_fisher_step": (ctypes.c_int, [c_void_p, c_int32, _P(pdhcg_info)]),
    "pdhcg_fisher_end": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, _P(pdhcg_info)]),
    "pdhcg_ad_solve": (ctypes.c_int, [c_void_p, _P(pdhcg_market), c_void_p, c_void_p, c_void_p, c_double, c_int32,
                                      _P(pdhcg_params), c_void_p, c_void_p, _P(c_int32), _P(pdhcg_info)]),
    "pdhcg_fisher_solve_batched": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                                  c_void_p, c_void_p, ctypes.c_int, c_void_p, _P(pdhcg_params),
                                                  c_void_p, c_void_p, c_void_p]),
    "pdhcg_fisher_backward": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pdhcg_row_prox": (ctypes.c_int, [c_void_p, _P(pdhcg_market), ctypes.c_int, c_void_p, c_void_p, c_double,
                                      c_void_p, c_void_p, c_void_p]),
    "pdhcg_kkt": (ctypes.c_int, [c_void_p, _P(pdhcg_market), ctypes.c_int, c_void_p, c_void_p, c_void_p]),
    "pdhcg_kkt_noalloc": (ctypes.c_int, [_P(pdhcg_market), c_void_p, c_void_p, c_void_p, c_void_p]),
}

_lib = None


def declared_symbols():
    """Every function name declared in include/pdhcg.h."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "pdhcg.h")).read()
    return sorted(set(re.findall(r"\b(pdhcg_[a-z_0-9]+)\s*\(", hdr)) - {"pdhcg_status", "pdhcg_handle"})


def load(path: str = LIB_PATH):
    """Load the library (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpdhcg.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _fn(name):
    return getattr(load(), name)


def status_string(st: int) -> str:
    return _fn("pdhcg_status_string")(st).decode()


def last_error() -> str:
    return _fn("pdhcg_last_error")().decode()


class PdhcgError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        extra = f"; CUDA: {last_error()}" if status == PDHCG_ERR_CUDA else ""
        super().__init__(f"{where}: status {status} ({status_string(status)}){extra}")


def default_params(**overrides) -> pdhcg_params:
    p = pdhcg_params()
    _fn("pdhcg_default_params")(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# thin same-name wrappers (raw pointers as ints)
def pdhcg_create(stream: int = 0) -> int:
    h = c_void_p()
    st = _fn("pdhcg_create")(ctypes.byref(h), c_void_p(stream))
    if st:
        raise PdhcgError(st, "pdhcg_create")
    return h.value


def pdhcg_destroy(h: int) -> int:
    return _fn("pdhcg_destroy")(c_void_p(h))


def pdhcg_fisher_solve(h, mk, prm, p0, x0, p_out, util_out, x_out, info) -> int:
    return _fn("pdhcg_fisher_solve")(c_void_p(h), ctypes.byref(mk), ctypes.byref(prm), c_void_p(p0), c_void_p(x0),
                                     c_void_p(p_out), c_void_p(util_out), c_void_p(x_out),
                                     ctypes.byref(info) if info is not None else None)


def pdhcg_fisher_solve_pdhg(h, mk, prm, restart_every, p_out, util_out, x_out, info) -> int:
    return _fn("pdhcg_fisher_solve_pdhg")(c_void_p(h), ctypes.byref(mk), ctypes.byref(prm), c_int32(restart_every),
                                          c_void_p(p_out), c_void_p(util_out), c_void_p(x_out),
                                          ctypes.byref(info) if info is not None else None)


def pdhcg_fisher_begin(h, mk, prm, p0, x0) -> int:
    return _fn("pdhcg_fisher_begin")(c_void_p(h), ctypes.byref(mk), ctypes.byref(prm), c_void_p(p0), c_void_p(x0))


def pdhcg_fisher_step(h, chunks, info) -> int:
    return _fn("pdhcg_fisher_step")(c_void_p(h), c_int32(chunks), ctypes.byref(info) if info is not None else None)


def pdhcg_fisher_end(h, p_out, util_out, x_out, info) -> int:
    return _fn("pdhcg_fisher_end")(c_void_p(h), c_void_p(p_out), c_void_p(util_out), c_void_p(x_out),
                                   ctypes.byref(info) if info is not None else None)


def pdhcg_ad_solve(h, mk, e_rp, e_col, e_val, outer_tol, max_outer, prm, p_out, w_out, outer, info) -> int:
    return _fn("pdhcg_ad_solve")(c_void_p(h), ctypes.byref(mk), c_void_p(e_rp), c_void_p(e_col), c_void_p(e_val),
                                 c_double(outer_tol), c_int32(max_outer), ctypes.byref(prm), c_void_p(p_out),
                                 c_void_p(w_out), ctypes.byref(outer) if outer is not None else None,
                                 ctypes.byref(info) if info is not None else None)


def pdhcg_fisher_solve_batched(h, B, row_off, good_off, nnz_off, row_ptr, col, val, val_type, w, prm, p_out,
                               util_out, info_out) -> int:
    return _fn("pdhcg_fisher_solve_batched")(c_void_p(h), c_int32(B), c_void_p(row_off), c_void_p(good_off),
                                             c_void_p(nnz_off), c_void_p(row_ptr), c_void_p(col), c_void_p(val),
                                             val_type, c_void_p(w), ctypes.byref(prm), c_void_p(p_out),
                                             c_void_p(util_out), c_void_p(info_out))


def pdhcg_fisher_backward(h, grad_p, grad_util, grad_u, grad_w) -> int:
    return _fn("pdhcg_fisher_backward")(c_void_p(h), c_void_p(grad_p), c_void_p(grad_util), c_void_p(grad_u),
                                        c_void_p(grad_w))


def pdhcg_row_prox(h, mk, prec, x_in, p, tau, x_new, s_out, c_out) -> int:
    return _fn("pdhcg_row_prox")(c_void_p(h), ctypes.byref(mk), prec, c_void_p(x_in), c_void_p(p), c_double(tau),
                                 c_void_p(x_new), c_void_p(s_out), c_void_p(c_out))


def pdhcg_kkt(h, mk, prec, x, p, out) -> int:
    return _fn("pdhcg_kkt")(c_void_p(h), ctypes.byref(mk), prec, c_void_p(x), c_void_p(p), c_void_p(out))


def pdhcg_kkt_noalloc(mk, x, p, out, stream=0) -> int:
    """KKT residuals without any allocation (device inputs only); see pdhcg.h."""
    return _fn("pdhcg_kkt_noalloc")(ctypes.byref(mk), c_void_p(x), c_void_p(p), c_void_p(out), c_void_p(stream))
