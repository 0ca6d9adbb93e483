"""Python binding of liblgk.so (ctypes).  Argument marshalling only: every
step of the planning path runs in the library's CUDA kernels.

The names mirror the C ABI of include/lgk.h without the `lgk_` prefix:
create_case, solve_weightings, fetch_times, fetch_doses, fetch_stats,
fetch_state.  The library must have been built (paper_2509_08602_b300.build);
importing this module without it raises ImportError rather than falling back
to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblgk.so")

PREC_FP32 = 0
PREC_BF16 = 1
PREC_BF16X3 = 2
LGK_NOALLOC_MAX_TIMES = 1 << 22     # doubles of static scratch for lgk_fetch_doses_device
STATUS = {0: "LGK_OK", 1: "LGK_EINVAL", 2: "LGK_ENOMEM", 3: "LGK_EBUDGET", 4: "LGK_ENOTPD",
          5: "LGK_ECUDA", 6: "LGK_ETIMEOUT"}


class LgkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class CaseDesc(C.Structure):
    _fields_ = [("n_iso", C.c_int), ("n_pts", C.c_int), ("n_targets", C.c_int), ("n_oars", C.c_int),
                ("phi", C.POINTER(C.c_double)), ("kind", C.POINTER(C.c_uint8)),
                ("struct_id", C.POINTER(C.c_uint16)), ("d_presc", C.POINTER(C.c_double)),
                ("q_area", C.POINTER(C.c_double)), ("q_vol", C.POINTER(C.c_double)),
                ("d_oar", C.POINTER(C.c_double)), ("d_ld1", C.c_double), ("d_ld2", C.c_double),
                ("phi_cal", C.c_double)]


class Params(C.Structure):
    _fields_ = [("precision", C.c_int), ("normalize_rows", C.c_int), ("scale_bot", C.c_int),
                ("check_every", C.c_int), ("eps_abs", C.c_double), ("device", C.c_int),
                ("stream", C.c_void_p), ("hbm_budget", C.c_size_t), ("timeout_ms", C.c_int),
                ("profile", C.c_int), ("lo_refresh", C.c_int), ("lo_refresh_iters", C.c_int),
                ("rho_adapt", C.c_int), ("solve_refine", C.c_int), ("setup_fp64", C.c_int),
                ("check_fp64", C.c_int), ("autotune", C.c_int), ("refine_after", C.c_int),
                ("l2_keep_inverse", C.c_int), ("gemm2_tile_rows", C.c_int),
                ("accum_kblocks", C.c_int)]


class ServerParams(C.Structure):
    _fields_ = [("case_params", Params), ("hbm_budget", C.c_size_t), ("workers", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("w0_bot", C.c_double),
                ("rho0_per_beta", C.c_double), ("stream_width", C.c_int)]


class Pass2Params(C.Structure):
    _fields_ = [("phi_cand", C.POINTER(C.c_double)), ("n_cand", C.c_int), ("delta_ld1", C.c_double),
                ("delta_ld2", C.c_double), ("n_ld1", C.c_int), ("n_ld2", C.c_int),
                ("seed", C.c_uint64)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("K", C.c_int), ("n_iso", C.c_int), ("queue_ms", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("total_ms", C.c_double),
                ("max_iters", C.c_int), ("converged", C.c_int), ("footprint", C.c_size_t)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built; run `python -m paper_2509_08602_b300.build`")
    lib = C.CDLL(_LIB_PATH)
    P = C.POINTER
    lib.lgk_default_params.argtypes = [P(Params)]
    lib.lgk_create_case.argtypes = [P(CaseDesc), P(Params), P(C.c_void_p)]
    lib.lgk_case_info.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_double), P(C.c_size_t)]
    lib.lgk_solve_weightings.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double),
                                         C.c_double, C.c_double, C.c_double, C.c_int, P(C.c_void_p)]
    lib.lgk_fetch_times.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
    lib.lgk_fetch_doses.argtypes = [C.c_void_p, P(C.c_double), C.c_int, P(C.c_double)]
    lib.lgk_fetch_stats.argtypes = [C.c_void_p, P(C.c_int), P(C.c_double), P(C.c_double),
                                    P(C.c_double), P(C.c_uint8)]
    lib.lgk_fetch_state.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
    lib.lgk_solve_weightings_warm.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double),
                                              C.c_double, C.c_double, C.c_double, C.c_int,
                                              P(C.c_double), P(C.c_double), P(C.c_void_p)]
    lib.lgk_solve_weightings_masked.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double),
                                                C.c_double, C.c_double, C.c_double, C.c_int,
                                                P(C.c_uint32), P(C.c_double), P(C.c_double),
                                                P(C.c_void_p)]
    lib.lgk_solve_stream.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double), C.c_double,
                                     C.c_double, C.c_double, C.c_int, C.c_int, P(C.c_double),
                                     P(C.c_double), P(C.c_int), P(C.c_double), P(C.c_double),
                                     P(C.c_double), P(C.c_uint8), P(C.c_double), P(C.c_longlong),
                                     P(C.c_double)]
    lib.lgk_solve_stream.restype = C.c_int
    lib.lgk_fetch_check.argtypes = [C.c_void_p, P(C.c_double)]
    lib.lgk_fetch_check.restype = C.c_int
    lib.lgk_solve_weightings_async.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double),
                                               C.c_double, C.c_double, C.c_double, C.c_int,
                                               P(C.c_void_p)]
    lib.lgk_solve_weightings_async.restype = C.c_int
    lib.lgk_solve_group.argtypes = [C.c_int, P(C.c_void_p), P(C.c_int), P(P(C.c_double)), P(P(C.c_double)),
                                    C.c_double, P(C.c_double), C.c_double, C.c_int, P(C.c_void_p)]
    lib.lgk_solve_group.restype = C.c_int
    lib.lgk_wait.argtypes = [C.c_void_p, C.c_int]
    lib.lgk_wait.restype = C.c_int
    lib.lgk_low_dose_volumes.argtypes = [C.c_void_p, P(C.c_double), C.c_int, C.c_int, P(C.c_double),
                                         P(C.c_double), P(C.c_uint32), P(C.c_int)]
    lib.lgk_sample_low_dose.argtypes = [C.c_int, C.c_int, P(C.c_uint32), P(C.c_int), C.c_uint64,
                                        C.c_int, P(C.c_int), P(C.c_int), P(C.c_uint32)]
    lib.lgk_two_pass.argtypes = [P(CaseDesc), P(Params), C.c_int, P(C.c_double), C.c_double,
                                 C.c_double, C.c_double, C.c_int, P(Pass2Params), P(C.c_void_p),
                                 P(C.c_void_p), P(C.c_void_p), P(C.c_int), P(C.c_int)]
    lib.lgk_fetch_profile.argtypes = [C.c_void_p, P(C.c_double), P(C.c_longlong)]
    lib.lgk_fetch_metrics.argtypes = [C.c_void_p, P(C.c_double), C.c_int, P(C.c_int), P(C.c_double),
                                       P(C.c_double), P(C.c_double), P(C.c_double)]
    lib.lgk_fetch_metrics.restype = C.c_int
    lib.lgk_fetch_doses_device.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    lib.lgk_fetch_doses_device.restype = C.c_int
    lib.lgk_server_create.argtypes = [P(ServerParams), P(C.c_void_p)]
    lib.lgk_server_submit.argtypes = [C.c_void_p, P(CaseDesc), C.c_int, P(C.c_double),
                                      P(C.c_longlong)]
    lib.lgk_server_wait.argtypes = [C.c_void_p, C.c_longlong, C.c_int, P(RequestInfo),
                                    P(C.c_double), P(C.c_double)]
    lib.lgk_server_destroy.argtypes = [C.c_void_p]
    lib.lgk_server_open.argtypes = [C.c_void_p, P(CaseDesc), P(C.c_longlong)]
    lib.lgk_server_submit_to.argtypes = [C.c_void_p, C.c_longlong, C.c_int, P(C.c_double),
                                         P(C.c_longlong)]
    lib.lgk_server_close.argtypes = [C.c_void_p, C.c_longlong]
    for f in ("lgk_server_open", "lgk_server_submit_to", "lgk_server_close"):
        getattr(lib, f).restype = C.c_int
    for f in ("lgk_server_create", "lgk_server_submit", "lgk_server_wait"):
        getattr(lib, f).restype = C.c_int
    lib.lgk_free_result.argtypes = [C.c_void_p]
    lib.lgk_destroy_case.argtypes = [C.c_void_p]
    lib.lgk_last_error.restype = C.c_char_p
    lib.lgk_launch_count.restype = C.c_longlong
    for f in ("lgk_default_params", "lgk_create_case", "lgk_case_info", "lgk_solve_weightings",
              "lgk_fetch_times", "lgk_fetch_doses", "lgk_fetch_stats", "lgk_fetch_state",
              "lgk_solve_weightings_warm", "lgk_fetch_profile"):
        getattr(lib, f).restype = C.c_int
    return lib


_lib = _load()


def _check(rc: int):
    if rc != 0:
        raise LgkError(rc, _lib.lgk_last_error().decode(errors="replace"))


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def default_params(**kw) -> Params:
    p = Params()
    _check(_lib.lgk_default_params(C.byref(p)))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Case:
    """Device-resident planning case (lgk_case)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep
        m, n, beta, nbytes = C.c_int(), C.c_int(), C.c_double(), C.c_size_t()
        _check(_lib.lgk_case_info(handle, C.byref(m), C.byref(n), C.byref(beta), C.byref(nbytes)))
        self.m, self.n, self.beta, self.device_bytes = m.value, n.value, beta.value, nbytes.value

    def close(self):
        if self._h:
            _lib.lgk_destroy_case(self._h)
            self._h = None

    def __del__(self):
        self.close()


class _Dims:
    """Sizes of a case held only by its results."""

    def __init__(self, m: int, n: int):
        self.m, self.n = m, n


class Result:
    """Solved batch of weightings (lgk_result)."""

    def __init__(self, handle, K, case):
        self._h = handle
        self.K = K
        self.case = case

    def close(self):
        if self._h:
            _lib.lgk_free_result(self._h)
            self._h = None

    def __del__(self):
        self.close()


def _desc(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal, d_oar):
    """CaseDesc over contiguous copies; returns (desc, arrays to keep alive)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    struct_id = np.ascontiguousarray(struct_id, dtype=np.uint16)
    d_presc = np.ascontiguousarray(np.atleast_1d(d_presc), dtype=np.float64)
    q_area = np.ascontiguousarray(np.atleast_1d(q_area), dtype=np.float64)
    q_vol = np.ascontiguousarray(np.atleast_1d(q_vol), dtype=np.float64)
    d_oar = None if d_oar is None or len(d_oar) == 0 else np.ascontiguousarray(d_oar, dtype=np.float64)
    if phi.shape[1] != 24 * int(n_iso) or kind.shape[0] != phi.shape[0] or struct_id.shape[0] != phi.shape[0]:
        raise LgkError(1, "phi must be n_pts x 24 n_iso; kind and struct_id of length n_pts")
    d = CaseDesc(n_iso=int(n_iso), n_pts=int(phi.shape[0]), n_targets=int(d_presc.shape[0]),
                 n_oars=0 if d_oar is None else int(d_oar.shape[0]),
                 phi=_ptr(phi, C.c_double), kind=_ptr(kind, C.c_uint8),
                 struct_id=_ptr(struct_id, C.c_uint16), d_presc=_ptr(d_presc, C.c_double),
                 q_area=_ptr(q_area, C.c_double), q_vol=_ptr(q_vol, C.c_double),
                 d_oar=_ptr(d_oar, C.c_double), d_ld1=float(d_ld1), d_ld2=float(d_ld2),
                 phi_cal=float(phi_cal))
    return d, (phi, kind, struct_id, d_presc, q_area, q_vol, d_oar)


def create_case(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal,
                d_oar=None, params: Params | None = None) -> Case:
    d, _keep = _desc(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal, d_oar)
    h = C.c_void_p()
    _check(_lib.lgk_create_case(C.byref(d), C.byref(params) if params is not None else None,
                                C.byref(h)))
    return Case(h, None)


def solve_weightings(case: Case, W, rho=None, *, w0_bot: float = 0.0, rho0: float = 0.0,
                     tol: float = 1e-4, max_iter: int = 10000) -> Result:
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    if W.shape[1] != 4:
        raise LgkError(1, "W must be K x 4")
    K = W.shape[0]
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (K,)), dtype=np.float64)
    h = C.c_void_p()
    _check(_lib.lgk_solve_weightings(case._h, K, _ptr(W, C.c_double), _ptr(r, C.c_double),
                                     float(w0_bot), float(rho0), float(tol), int(max_iter),
                                     C.byref(h)))
    return Result(h, K, case)


def solve_group(cases, Ws, rhos=None, *, w0_bot: float = 0.0, rho0=None, tol: float = 1e-4,
                max_iter: int = 10000) -> list:
    """lgk_solve_group: up to 4 cases, each with its own weightings (Ws[g],
    K_g x 4), solved together (one launch per product over all of them).
    rhos: None or per case None / K_g penalties; rho0: per case (Eq. rho_rule).
    Returns one Result per case."""
    G = len(cases)
    Ws = [np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64) for W in Ws]
    if len(Ws) != G or any(W.shape[1] != 4 for W in Ws):
        raise LgkError(1, "one K x 4 weight matrix per case")
    Ks = (C.c_int * G)(*[W.shape[0] for W in Ws])
    rr = [None] * G if rhos is None else [
        None if r is None else np.ascontiguousarray(np.broadcast_to(r, (W.shape[0],)), dtype=np.float64)
        for r, W in zip(rhos, Ws)]
    hs = (C.c_void_p * G)(*[c._h for c in cases])
    wp = (C.POINTER(C.c_double) * G)(*[_ptr(W, C.c_double) for W in Ws])
    rp = (C.POINTER(C.c_double) * G)(*[_ptr(r, C.c_double) for r in rr])
    r0 = None if rho0 is None else np.ascontiguousarray(np.broadcast_to(rho0, (G,)), dtype=np.float64)
    out = (C.c_void_p * G)()
    _check(_lib.lgk_solve_group(G, hs, Ks, wp, rp, float(w0_bot), _ptr(r0, C.c_double), float(tol),
                                int(max_iter), out))
    return [Result(C.c_void_p(out[g]), Ws[g].shape[0], cases[g]) for g in range(G)]


def solve_weightings_async(case: Case, W, rho=None, *, w0_bot: float = 0.0, rho0: float = 0.0,
                           tol: float = 1e-4, max_iter: int = 10000) -> Result:
    """lgk_solve_weightings_async: starts the solve and returns its Result at
    once; call wait(res, timeout_ms) before fetching from it."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (K,)), dtype=np.float64)
    h = C.c_void_p()
    _check(_lib.lgk_solve_weightings_async(case._h, K, _ptr(W, C.c_double), _ptr(r, C.c_double),
                                           float(w0_bot), float(rho0), float(tol), int(max_iter),
                                           C.byref(h)))
    return Result(h, K, case)


def wait(res: Result, timeout_ms: int) -> bool:
    """lgk_wait: True once the solve finished (raises LgkError if it failed),
    False if it is still running after timeout_ms."""
    rc = _lib.lgk_wait(res._h, int(timeout_ms))
    if rc == 6:
        return False
    _check(rc)
    return True


def solve_stream(case: Case, W, rho=None, *, w0_bot: float = 0.0, rho0: float = 0.0,
                 tol: float = 1e-4, max_iter: int = 10000, width: int = 32,
                 profile: bool = False, check: bool = False) -> dict:
    """lgk_solve_stream: the K_total weightings of W run through `width`
    columns, each freed column taking the next weighting.  Returns, per
    weighting in W's order, t (K_total x 24N), tau (K_total x N), iters, obj,
    rel_pri, rel_dual, converged; with profile=True (the case created with
    profile=1) also {kernel: (ms, launches)} under "profile"; with check=True
    the FP64 check of each weighting (as fetch_check) under "check"."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    if W.shape[1] != 4:
        raise LgkError(1, "W must be K x 4")
    K = W.shape[0]
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (K,)), dtype=np.float64)
    n_iso = case.m // 25
    t = np.empty((K, 24 * n_iso))
    tau = np.empty((K, n_iso))
    it = np.empty(K, np.int32)
    obj, rp, rd = np.empty(K), np.empty(K), np.empty(K)
    conv = np.empty(K, np.uint8)
    ms = np.zeros(len(KERNELS)) if profile else None
    nl = np.zeros(len(KERNELS), np.int64) if profile else None
    ck = np.full((K, len(CHECK_FIELDS)), np.nan) if check else None
    _check(_lib.lgk_solve_stream(case._h, K, _ptr(W, C.c_double), _ptr(r, C.c_double), float(w0_bot),
                                 float(rho0), float(tol), int(max_iter), int(width), _ptr(t, C.c_double),
                                 _ptr(tau, C.c_double), _ptr(it, C.c_int), _ptr(obj, C.c_double),
                                 _ptr(rp, C.c_double), _ptr(rd, C.c_double), _ptr(conv, C.c_uint8),
                                 _ptr(ms, C.c_double), _ptr(nl, C.c_longlong), _ptr(ck, C.c_double)))
    out = dict(t=t, tau=tau, iters=it, obj=obj, rel_pri=rp, rel_dual=rd, converged=conv.astype(bool))
    if check:
        out["check"] = {k: ck[:, i].copy() for i, k in enumerate(CHECK_FIELDS)}
    if profile:
        out["profile"] = {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(KERNELS)}
    return out


def solve_weightings_warm(case: Case, W, rho=None, *, q1_init=None, q2_init=None,
                          w0_bot: float = 0.0, rho0: float = 0.0, tol: float = 1e-4,
                          max_iter: int = 10000) -> Result:
    """Resume from a q-form state (K x n, K x m) such as fetch_state returns."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (K,)), dtype=np.float64)
    q1 = None if q1_init is None else np.ascontiguousarray(q1_init, dtype=np.float64)
    q2 = None if q2_init is None else np.ascontiguousarray(q2_init, dtype=np.float64)
    if q1 is not None and q1.shape != (K, case.n) or q2 is not None and q2.shape != (K, case.m):
        raise LgkError(1, "q1_init must be K x n and q2_init K x m")
    h = C.c_void_p()
    _check(_lib.lgk_solve_weightings_warm(case._h, K, _ptr(W, C.c_double), _ptr(r, C.c_double),
                                          float(w0_bot), float(rho0), float(tol), int(max_iter),
                                          _ptr(q1, C.c_double), _ptr(q2, C.c_double), C.byref(h)))
    return Result(h, K, case)


def pack_bits(sel) -> np.ndarray:
    """(rows, K) bool -> (rows, ceil(K/32)) uint32, bit j % 32 of word j / 32."""
    sel = np.asarray(sel, dtype=bool)
    rows, K = sel.shape
    kw = (K + 31) // 32
    pad = np.zeros((rows, kw * 32), dtype=bool)
    pad[:, :K] = sel
    return np.ascontiguousarray(np.packbits(pad, axis=1, bitorder="little").view("<u4"))


def unpack_bits(words, K: int) -> np.ndarray:
    """Inverse of pack_bits: (rows, ceil(K/32)) uint32 -> (rows, K) bool."""
    w = np.ascontiguousarray(words, dtype="<u4")
    return np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")[..., :K].astype(bool)


def solve_weightings_masked(case: Case, W, rho=None, *, select=None, q1_init=None, q2_init=None,
                            w0_bot: float = 0.0, rho0: float = 0.0, tol: float = 1e-4,
                            max_iter: int = 10000) -> Result:
    """Batched solve with a point selection per weighting: select is
    (n_pts, K) bool (None: every point), packed for lgk_solve_weightings_masked."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (K,)), dtype=np.float64)
    mask = None if select is None else pack_bits(select)
    q1 = None if q1_init is None else np.ascontiguousarray(q1_init, dtype=np.float64)
    q2 = None if q2_init is None else np.ascontiguousarray(q2_init, dtype=np.float64)
    h = C.c_void_p()
    _check(_lib.lgk_solve_weightings_masked(case._h, K, _ptr(W, C.c_double), _ptr(r, C.c_double),
                                            float(w0_bot), float(rho0), float(tol), int(max_iter),
                                            _ptr(mask, C.c_uint32), _ptr(q1, C.c_double),
                                            _ptr(q2, C.c_double), C.byref(h)))
    return Result(h, K, case)


def low_dose_volumes(res: Result, phi_cand, d_lo, delta):
    """Membership (levels, K, n_cand) bool and sizes (levels, K) of the
    low-dose volumes [d_lo, d_lo + delta) of every plan (Sec. 2.C)."""
    phi_cand = np.ascontiguousarray(phi_cand, dtype=np.float64)
    d_lo = np.ascontiguousarray(np.atleast_1d(d_lo), dtype=np.float64)
    delta = np.ascontiguousarray(np.atleast_1d(delta), dtype=np.float64)
    L, nc = d_lo.shape[0], phi_cand.shape[0]
    words = (nc + 31) // 32
    member = np.zeros((L, res.K, words), dtype=np.uint32)
    count = np.zeros((L, res.K), dtype=np.int32)
    _check(_lib.lgk_low_dose_volumes(res._h, _ptr(phi_cand, C.c_double), nc, L, _ptr(d_lo, C.c_double),
                                     _ptr(delta, C.c_double), _ptr(member, C.c_uint32),
                                     _ptr(count, C.c_int)))
    return unpack_bits(member, nc), count


def sample_low_dose(member, n_desired, seed: int, level: int = 0):
    """Algorithm 1 (Sec. 2.C) on volumes member (K, n_cand) bool.  Returns
    (union candidate indices ascending, sel (n_union, K) bool)."""
    member = np.asarray(member, dtype=bool)
    K, nc = member.shape
    words = pack_bits(member)
    nd = np.ascontiguousarray(np.broadcast_to(n_desired, (K,)), dtype=np.int32)
    kw = (K + 31) // 32
    n_union = C.c_int()
    idx = np.zeros(nc, dtype=np.int32)
    sel = np.zeros((nc, kw), dtype=np.uint32)
    _check(_lib.lgk_sample_low_dose(K, nc, _ptr(words, C.c_uint32), _ptr(nd, C.c_int),
                                    C.c_uint64(int(seed) & (2 ** 64 - 1)), int(level), C.byref(n_union),
                                    _ptr(idx, C.c_int), _ptr(sel, C.c_uint32)))
    nu = n_union.value
    return idx[:nu].copy(), unpack_bits(sel[:nu], K)


def two_pass(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal, W, *,
             phi_cand, delta_ld1, delta_ld2, w0_bot, rho0_per_beta, n_ld1=0, n_ld2=0, seed=0,
             d_oar=None, tol=1e-4, max_iter=10000, params: Params | None = None):
    """Both passes of Sec. 2.C (lgk_two_pass).  Returns (res1, case2, res2,
    (ld1 union candidate indices, ld2 union candidate indices))."""
    d, _keep = _desc(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal, d_oar)
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    pc = np.ascontiguousarray(phi_cand, dtype=np.float64)
    nc = pc.shape[0]
    p2 = Pass2Params(phi_cand=_ptr(pc, C.c_double), n_cand=nc, delta_ld1=float(delta_ld1),
                     delta_ld2=float(delta_ld2), n_ld1=int(n_ld1), n_ld2=int(n_ld2),
                     seed=int(seed) & (2 ** 64 - 1))
    r1, c2, r2 = C.c_void_p(), C.c_void_p(), C.c_void_p()
    nu = np.zeros(2, dtype=np.int32)
    idx = np.zeros((2, nc), dtype=np.int32)
    _check(_lib.lgk_two_pass(C.byref(d), C.byref(params) if params is not None else None, K,
                             _ptr(W, C.c_double), float(w0_bot), float(rho0_per_beta), float(tol),
                             int(max_iter), C.byref(p2), C.byref(r1), C.byref(c2), C.byref(r2),
                             _ptr(nu, C.c_int), _ptr(idx, C.c_int)))
    # the first case lives on inside res1 (the library keeps it alive)
    case1 = _Dims(m=25 * int(n_iso), n=int(np.asarray(phi).shape[0]) + 8 * int(n_iso))
    res1 = Result(r1, K, case1)
    case2 = Case(c2, None)
    return res1, case2, Result(r2, K, case2), (idx[0, :nu[0]].copy(), idx[1, :nu[1]].copy())


def fetch_times(res: Result):
    """(t (K x 24N), tau (K x N)) as FP64."""
    n_iso = (res.case.m) // 25
    t = np.empty((res.K, 24 * n_iso))
    tau = np.empty((res.K, n_iso))
    _check(_lib.lgk_fetch_times(res._h, _ptr(t, C.c_double), _ptr(tau, C.c_double)))
    return t, tau


def fetch_doses(res: Result, phi_eval) -> np.ndarray:
    phi_eval = np.ascontiguousarray(phi_eval, dtype=np.float64)
    dose = np.empty((res.K, phi_eval.shape[0]))
    _check(_lib.lgk_fetch_doses(res._h, _ptr(phi_eval, C.c_double), int(phi_eval.shape[0]),
                                _ptr(dose, C.c_double)))
    return dose


def fetch_doses_device(res: Result, phi_eval_ptr: int, n_eval: int, dose_ptr: int) -> None:
    """Allocation-free dose evaluation on caller device buffers (integer device
    addresses, e.g. torch's data_ptr()): phi_eval n_eval x 24N FP64 in,
    dose K x n_eval FP64 out.  See lgk_fetch_doses_device in include/lgk.h."""
    _check(_lib.lgk_fetch_doses_device(res._h, C.c_void_p(phi_eval_ptr), int(n_eval),
                                       C.c_void_p(dose_ptr)))


def fetch_metrics(res: Result, phi_eval, label) -> dict:
    """Coverage, selectivity, gradient index and beam-on time of every plan,
    computed on the device (Sec. 2.A, Sec. 3.B)."""
    phi_eval = np.ascontiguousarray(phi_eval, dtype=np.float64)
    label = np.ascontiguousarray(label, dtype=np.int32)
    out = {k: np.empty(res.K) for k in ("coverage", "selectivity", "gi", "bot")}
    _check(_lib.lgk_fetch_metrics(res._h, _ptr(phi_eval, C.c_double), int(phi_eval.shape[0]),
                                  _ptr(label, C.c_int), _ptr(out["coverage"], C.c_double),
                                  _ptr(out["selectivity"], C.c_double), _ptr(out["gi"], C.c_double),
                                  _ptr(out["bot"], C.c_double)))
    return out


def fetch_stats(res: Result) -> dict:
    K = res.K
    it = np.empty(K, np.int32)
    obj, rp, rd = np.empty(K), np.empty(K), np.empty(K)
    conv = np.empty(K, np.uint8)
    _check(_lib.lgk_fetch_stats(res._h, _ptr(it, C.c_int), _ptr(obj, C.c_double), _ptr(rp, C.c_double),
                                _ptr(rd, C.c_double), _ptr(conv, C.c_uint8)))
    return dict(iters=it, obj=obj, rel_pri=rp, rel_dual=rd, converged=conv.astype(bool))


CHECK_FIELDS = ("obj", "plan", "gap", "infeas", "infeas_abs", "hard", "bound", "primal")   # LGK_CHECK_*


def fetch_check(res: Result) -> dict:
    """lgk_fetch_check: the FP64 check of every plan, {field: (K,) array}
    with the fields of CHECK_FIELDS (LGK_CHECK_* in include/lgk.h)."""
    out = np.empty((res.K, len(CHECK_FIELDS)))
    _check(_lib.lgk_fetch_check(res._h, _ptr(out, C.c_double)))
    return {k: out[:, i].copy() for i, k in enumerate(CHECK_FIELDS)}


def fetch_state(res: Result):
    """(q1 (K x n), q2 (K x m)): the q-form ADMM state of the scaled problem,
    q = z + y, FP64."""
    q1 = np.empty((res.K, res.case.n))
    q2 = np.empty((res.K, res.case.m))
    _check(_lib.lgk_fetch_state(res._h, _ptr(q1, C.c_double), _ptr(q2, C.c_double)))
    return q1, q2


KERNELS = ("gemm1", "reduce_rhs", "solve", "reduce_solve", "gemm2", "q1_update", "finalize",
           "gemm1_lo", "gemm2_lo", "sv", "reduce_err")


def fetch_profile(res: Result) -> dict:
    """{kernel: (total ms, timed launches)} of a solve made with profile=1."""
    ms = np.zeros(len(KERNELS))
    n = np.zeros(len(KERNELS), np.int64)
    _check(_lib.lgk_fetch_profile(res._h, _ptr(ms, C.c_double), _ptr(n, C.c_longlong)))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}


class Server:
    """Serving loop with continuous batching (lgk_server): resident cases
    admitted first come, first served under a device-memory budget, each a
    streaming solve on a worker thread with its own stream; every request for
    a resident case joins its running stream."""

    def __init__(self, *, workers=2, hbm_budget=0, tol=1e-4, max_iter=20000, w0_bot=1e-4,
                 rho0_per_beta=1.1e3, stream_width=32, params: Params | None = None):
        sp = ServerParams(case_params=params if params is not None else default_params(),
                          hbm_budget=int(hbm_budget), workers=int(workers), tol=float(tol),
                          max_iter=int(max_iter), w0_bot=float(w0_bot),
                          rho0_per_beta=float(rho0_per_beta), stream_width=int(stream_width))
        self._h = C.c_void_p()
        _check(_lib.lgk_server_create(C.byref(sp), C.byref(self._h)))

    def submit(self, phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal,
               W, d_oar=None) -> int:
        d, keep = _desc(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2,
                        phi_cal, d_oar)
        W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
        rid = C.c_longlong()
        _check(_lib.lgk_server_submit(self._h, C.byref(d), int(W.shape[0]), _ptr(W, C.c_double),
                                      C.byref(rid)))
        del keep                     # the library copied everything
        return rid.value

    def open(self, phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2, phi_cal,
             d_oar=None) -> int:
        """lgk_server_open: a resident case; returns its case id."""
        d, keep = _desc(phi, kind, struct_id, n_iso, d_presc, q_area, q_vol, d_ld1, d_ld2,
                        phi_cal, d_oar)
        cid = C.c_longlong()
        _check(_lib.lgk_server_open(self._h, C.byref(d), C.byref(cid)))
        del keep
        return cid.value

    def submit_to(self, case_id: int, W) -> int:
        """lgk_server_submit_to: K weightings for a resident case; returns the request id."""
        W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
        rid = C.c_longlong()
        _check(_lib.lgk_server_submit_to(self._h, int(case_id), int(W.shape[0]), _ptr(W, C.c_double),
                                         C.byref(rid)))
        return rid.value

    def close_case(self, case_id: int) -> None:
        """lgk_server_close: the case leaves once its queued weightings are done."""
        _check(_lib.lgk_server_close(self._h, int(case_id)))

    def wait(self, rid: int, n_iso: int, K: int, timeout_ms: int = 600000):
        """(info dict, t (K x 24N), tau (K x N)) of request rid."""
        info = RequestInfo()
        t = np.zeros((K, 24 * n_iso))
        tau = np.zeros((K, n_iso))
        rc = _lib.lgk_server_wait(self._h, int(rid), int(timeout_ms), C.byref(info),
                                  _ptr(t, C.c_double), _ptr(tau, C.c_double))
        out = {f: getattr(info, f) for f, _ in RequestInfo._fields_}
        if rc != 0:
            raise LgkError(rc, _lib.lgk_last_error().decode(errors="replace"))
        return out, t, tau

    def close(self):
        if self._h:
            _lib.lgk_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def launch_count() -> int:
    """Kernel launches issued by the library on this thread since the last call."""
    return int(_lib.lgk_launch_count())
