"""Thin ctypes binding of the C ABI in include/lsr.h (argument marshalling only).

Every step of the registration runs in the CUDA library ``_lib/liblsr.so``;
nothing here computes. Inputs may be torch tensors (CUDA or CPU) or numpy
arrays; they are passed to the library as raw pointers. Loading fails loudly if
the library has not been built (``paper_1801_01572_gb300._build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, field

import numpy as np

# LSR_CHECKED=1 in the environment loads the checked build (device bounds
# checks that report instead of trapping), built by _build.build(checked=True).
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                         "liblsr_checked.so" if os.environ.get("LSR_CHECKED") == "1" else "liblsr.so")
_lib = None
_lock = threading.Lock()

LSR_OK, LSR_E_ARG, LSR_E_CUDA, LSR_E_OOM, LSR_E_TIMEOUT, LSR_E_STATE, LSR_E_TOO_LARGE = 0, -1, -2, -3, -4, -5, -6
STATUS_ALIGNED, STATUS_NO_ALIGNMENT = 0, 1
MATCH_FP32, MATCH_BF16, MATCH_BF16_PLAIN = 0, 1, 2
NN_EXACT, NN_SINGLE_CELL = 0, 1
NORMALS_SAMPLES, NORMALS_INLIERS = 0, 1
DESC_DIM = 33

# Names of every entry point declared in include/lsr.h (checked by the tests).
ABI_FUNCTIONS = (
    "lsr_default_params", "lsr_create", "lsr_destroy", "lsr_set_params", "lsr_get_params", "lsr_set_profiling",
    "lsr_error_string", "lsr_last_error", "lsr_workspace_bytes", "lsr_launch_count", "lsr_transfer_bytes",
    "lsr_register_pair", "lsr_register_batch",
    "lsr_stage_normals", "lsr_stage_spfh", "lsr_stage_fpfh", "lsr_stage_match", "lsr_stage_hypotheses",
    "lsr_stage_rigid4", "lsr_stage_consensus", "lsr_stage_refine", "lsr_objective_fwd", "lsr_objective_bwd",
    "lsr_consensus_static", "lsr_match_scores_bf16", "lsr_information_matrix", "lsr_surfel_correct",
    "lsr_voxel_downsample", "lsr_debug_inject", "lsr_set_kernel_timing", "lsr_kernel_timing_count",
    "lsr_kernel_timing_entry", "lsr_checked_build", "lsr_pose_implicit_grad", "lsr_stage_nn",
    "lsr_stage_consensus_modes",
)
INJECT_NONE, INJECT_ALLOC, INJECT_MATCH_STALL, INJECT_CHECK = 0, 1, 2, 3
LSR_E_CHECK = -7


class LsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lsr error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("r_normal", C.c_float), ("r_feature", C.c_float), ("eps_inlier", C.c_float), ("tau", C.c_float),
                ("cos_normal", C.c_float), ("min_inlier_ratio", C.c_float), ("mu_scale", C.c_float),
                ("refine_iters", C.c_int32), ("n_hypotheses", C.c_int64), ("seed", C.c_uint64),
                ("pair_id", C.c_uint64), ("match_precision", C.c_int32), ("refine_levels", C.c_int32),
                ("batch_streams", C.c_int32), ("batch_graph", C.c_int32), ("match_tile", C.c_int32),
                ("nn_mode", C.c_int32), ("normal_mode", C.c_int32), ("reserved_", C.c_int32 * 2)]


class Result(C.Structure):
    _fields_ = [("T", C.c_double * 16), ("T_hyp", C.c_double * 16), ("inliers", C.c_int64),
                ("hyp_inliers", C.c_int64), ("survivors", C.c_int64), ("n_normal_ok", C.c_int64),
                ("best_h", C.c_int64), ("match_fallbacks", C.c_int64),
                ("match_terms", C.c_int64), ("fitness", C.c_float),
                ("hyp_fitness", C.c_float), ("status", C.c_int32), ("refine_iters_done", C.c_int32),
                ("stage_ms", C.c_float * 8)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {_LIB_PATH} is missing; run "
                               "paper_1801_01572_gb300._build.build() (needs nvcc) first")
        L = C.CDLL(_LIB_PATH)
        vp, i64, i32, u64, f32, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_float, C.c_double
        pp = C.POINTER(C.c_void_p)
        sig = {
            "lsr_default_params": (None, [C.POINTER(Params)]),
            "lsr_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Params), C.c_int, vp]),
            "lsr_destroy": (C.c_int, [vp]),
            "lsr_set_params": (C.c_int, [vp, C.POINTER(Params)]),
            "lsr_get_params": (C.c_int, [vp, C.POINTER(Params)]),
            "lsr_set_profiling": (C.c_int, [vp, C.c_int]),
            "lsr_error_string": (C.c_char_p, [C.c_int]),
            "lsr_last_error": (C.c_char_p, [vp]),
            "lsr_workspace_bytes": (i64, [vp]),
            "lsr_launch_count": (C.c_uint64, []),
            "lsr_transfer_bytes": (C.c_int, [i64, i64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
            "lsr_register_pair": (C.c_int, [vp, vp, i64, vp, i64, vp, vp, C.POINTER(Result)]),
            "lsr_register_batch": (C.c_int, [vp, i32, pp, vp, pp, vp, vp, C.POINTER(Result)]),
            "lsr_stage_normals": (C.c_int, [vp, vp, i64, vp, f32, vp, vp, vp]),
            "lsr_stage_spfh": (C.c_int, [vp, vp, vp, i64, f32, vp, vp]),
            "lsr_stage_fpfh": (C.c_int, [vp, vp, vp, vp, i64, f32, vp]),
            "lsr_stage_match": (C.c_int, [vp, vp, i64, vp, i64, i32, vp, vp, vp]),
            "lsr_match_scores_bf16": (C.c_int, [vp, vp, i64, vp, i64, i32, vp]),
            "lsr_stage_hypotheses": (C.c_int, [vp, vp, i64, vp, i64, vp, vp, vp, i64, u64, u64, f32, vp, i64, vp]),
            "lsr_stage_rigid4": (C.c_int, [vp, vp, vp, i64, vp]),
            "lsr_stage_consensus": (C.c_int, [vp, vp, i64, vp, i64, vp, i64, f32, vp, vp]),
            "lsr_stage_refine": (C.c_int, [vp, vp, i64, vp, i64, vp, f32, f32, i32, i32, vp, vp]),
            "lsr_objective_fwd": (C.c_int, [vp, i32, pp, vp, pp, vp, vp, vp, f32, f32, vp]),
            "lsr_objective_bwd": (C.c_int, [vp, i32, pp, vp, pp, vp, vp, vp, f32, f32, vp, pp, pp, vp]),
            "lsr_consensus_static": (C.c_int, [vp, i64, vp, i64, vp, i64, f32, vp, vp, vp]),
            "lsr_information_matrix": (C.c_int, [vp, vp, i64, vp, i64, vp, f32, vp, vp]),
            "lsr_surfel_correct": (C.c_int, [vp, i64, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
            "lsr_voxel_downsample": (C.c_int, [vp, vp, i64, f32, vp, i64, vp]),
            "lsr_debug_inject": (C.c_int, [vp, i32, i32]),
            "lsr_set_kernel_timing": (C.c_int, [vp, C.c_char_p]),
            "lsr_checked_build": (C.c_int, []),
            "lsr_stage_nn": (C.c_int, [vp, vp, i64, vp, i64, f32, i32, vp, vp]),
            "lsr_stage_consensus_modes": (C.c_int, [vp, vp, vp, i64, vp, vp, i64, vp, i64, f32, i32, i32, f32, vp,
                                                    vp]),
            "lsr_pose_implicit_grad": (C.c_int, [vp, vp, i64, vp, i64, vp, f32, f32, vp, vp, vp, vp, vp, vp,
                                                 C.POINTER(C.c_int64)]),
            "lsr_kernel_timing_count": (i32, [vp]),
            "lsr_kernel_timing_entry": (C.c_int, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                                                  C.POINTER(C.c_double)]),
        }
        for name in ABI_FUNCTIONS:
            res, args = sig[name]
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


# ------------------------------------------------------------------ marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _prep(x, dtype, cols=None):
    """(pointer, keep-alive object, n_rows) of a contiguous array of `dtype`."""
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
               np.uint8: torch.uint8, np.int64: torch.int64}[dtype]
        t = x.detach()
        if t.dtype != tdt:
            t = t.to(tdt)
        t = t.contiguous()
        if cols is not None:
            t = t.reshape(-1, cols)
        return C.c_void_p(t.data_ptr()), t, (t.shape[0] if t.dim() else 1)
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    if cols is not None:
        a = a.reshape(-1, cols)
    return C.c_void_p(a.ctypes.data), a, (a.shape[0] if a.ndim else 1)


def _vec3(v):
    if v is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(v, np.float32).reshape(3))
    return C.c_void_p(a.ctypes.data), a


def launch_count() -> int:
    """Kernels launched by the CUDA library in this process so far."""
    return int(lib().lsr_launch_count())


def transfer_bytes(nP: int, nQ: int) -> tuple[int, int]:
    """(host-to-device, device-to-host) bytes of one registration of host clouds."""
    a, b = C.c_int64(0), C.c_int64(0)
    rc = lib().lsr_transfer_bytes(int(nP), int(nQ), C.byref(a), C.byref(b))
    if rc != LSR_OK:
        raise LsrError(rc, "transfer_bytes")
    return int(a.value), int(b.value)


def default_params(**overrides) -> Params:
    p = Params()
    lib().lsr_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


@dataclass
class Registration:
    T: np.ndarray
    T_hyp: np.ndarray
    inliers: int
    hyp_inliers: int
    survivors: int
    n_normal_ok: int
    best_h: int
    match_fallbacks: int
    match_terms: int
    fitness: float
    hyp_fitness: float
    status: int
    refine_iters: int
    stage_ms: list = field(default_factory=list)

    @property
    def aligned(self) -> bool:
        return self.status == STATUS_ALIGNED

    @staticmethod
    def from_c(r: Result) -> "Registration":
        return Registration(T=np.array(r.T, np.float64).reshape(4, 4), T_hyp=np.array(r.T_hyp, np.float64).reshape(4, 4),
                            inliers=int(r.inliers), hyp_inliers=int(r.hyp_inliers), survivors=int(r.survivors),
                            n_normal_ok=int(r.n_normal_ok), best_h=int(r.best_h),
                            match_fallbacks=int(r.match_fallbacks), match_terms=int(r.match_terms), fitness=float(r.fitness),
                            hyp_fitness=float(r.hyp_fitness), status=int(r.status),
                            refine_iters=int(r.refine_iters_done), stage_ms=list(r.stage_ms))


class Context:
    """An lsr_ctx: device workspace, stream and parameters (one per thread)."""

    def __init__(self, device: int = 0, params: Params | None = None, stream: int | None = None, **overrides):
        self._L = lib()
        p = params if params is not None else default_params()
        for k, v in overrides.items():
            setattr(p, k, v)
        h = C.c_void_p()
        rc = self._L.lsr_create(C.byref(h), C.byref(p), int(device), C.c_void_p(stream) if stream else None)
        if rc != LSR_OK:
            raise LsrError(rc, self._L.lsr_error_string(rc).decode())
        self._h = h
        self.device = device

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._L.lsr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != LSR_OK:
            raise LsrError(rc, self._L.lsr_last_error(self._h).decode())

    # -- parameters
    @property
    def params(self) -> Params:
        p = Params()
        self._check(self._L.lsr_get_params(self._h, C.byref(p)))
        return p

    def set_params(self, params: Params | None = None, **overrides):
        p = params if params is not None else self.params
        for k, v in overrides.items():
            setattr(p, k, v)
        self._check(self._L.lsr_set_params(self._h, C.byref(p)))

    def set_profiling(self, on: bool = True):
        self._check(self._L.lsr_set_profiling(self._h, 1 if on else 0))

    def debug_inject(self, kind: int, count: int = 1):
        """Test hook (lsr_debug_inject): make the next `count` workspace
        allocations fail (INJECT_ALLOC) or tensor-core matcher launches stall
        into their bounded wait (INJECT_MATCH_STALL); INJECT_NONE clears."""
        self._check(self._L.lsr_debug_inject(self._h, int(kind), int(count)))

    def set_kernel_timing(self, prefix: str | None = ""):
        """Time every launch whose kernel name starts with `prefix` ("" = all,
        None = off) with CUDA events in later registrations; clears the table."""
        self._check(self._L.lsr_set_kernel_timing(self._h, None if prefix is None else prefix.encode()))

    def kernel_times(self) -> dict:
        """{kernel name: (timed launches, total ms)} since set_kernel_timing."""
        out = {}
        for i in range(int(self._L.lsr_kernel_timing_count(self._h))):
            nm, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
            self._check(self._L.lsr_kernel_timing_entry(self._h, i, C.byref(nm), C.byref(n), C.byref(ms)))
            out[nm.value.decode()] = (int(n.value), float(ms.value))
        return out

    def workspace_bytes(self) -> int:
        return int(self._L.lsr_workspace_bytes(self._h))

    # -- registration
    def register_pair(self, P, Q, vpP=None, vpQ=None) -> Registration:
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        a, ka = _vec3(vpP)
        b, kb = _vec3(vpQ)
        r = Result()
        self._check(self._L.lsr_register_pair(self._h, pP, nP, pQ, nQ, a, b, C.byref(r)))
        return Registration.from_c(r)

    def register_batch(self, Ps, Qs, vps=None) -> list[Registration]:
        n = len(Ps)
        prepP = [_prep(x, np.float32, 3) for x in Ps]
        prepQ = [_prep(x, np.float32, 3) for x in Qs]
        arrP = (C.c_void_p * n)(*[p[0].value for p in prepP])
        arrQ = (C.c_void_p * n)(*[p[0].value for p in prepQ])
        nP = np.array([p[2] for p in prepP], np.int64)
        nQ = np.array([p[2] for p in prepQ], np.int64)
        vp = None
        if vps is not None:
            vp = np.ascontiguousarray(np.asarray(vps, np.float32).reshape(n, 6))
        res = (Result * n)()
        self._check(self._L.lsr_register_batch(self._h, n, C.cast(arrP, C.POINTER(C.c_void_p)),
                                               C.c_void_p(nP.ctypes.data), C.cast(arrQ, C.POINTER(C.c_void_p)),
                                               C.c_void_p(nQ.ctypes.data),
                                               C.c_void_p(vp.ctypes.data) if vp is not None else None, res))
        return [Registration.from_c(r) for r in res]

    # -- stages (outputs are numpy arrays in caller order)
    def stage_normals(self, P, vp=None, r=0.05):
        pP, kP, n = _prep(P, np.float32, 3)
        a, ka = _vec3(vp)
        N = np.zeros((n, 3), np.float32)
        cnt = np.zeros(n, np.int32)
        curv = np.zeros(n, np.float32)
        self._check(self._L.lsr_stage_normals(self._h, pP, n, a, C.c_float(r), C.c_void_p(N.ctypes.data),
                                              C.c_void_p(cnt.ctypes.data), C.c_void_p(curv.ctypes.data)))
        return N, cnt, curv

    def stage_spfh(self, P, N, r=0.125):
        pP, kP, n = _prep(P, np.float32, 3)
        pN, kN, _ = _prep(N, np.float32, 3)
        S = np.zeros((n, DESC_DIM), np.float32)
        k = np.zeros(n, np.int32)
        self._check(self._L.lsr_stage_spfh(self._h, pP, pN, n, C.c_float(r), C.c_void_p(S.ctypes.data),
                                           C.c_void_p(k.ctypes.data)))
        return S, k

    def stage_fpfh(self, P, N, S, r=0.125):
        pP, kP, n = _prep(P, np.float32, 3)
        pN, kN, _ = _prep(N, np.float32, 3)
        pS, kS, _ = _prep(S, np.float32, DESC_DIM)
        F = np.zeros((n, DESC_DIM), np.float32)
        self._check(self._L.lsr_stage_fpfh(self._h, pP, pN, pS, n, C.c_float(r), C.c_void_p(F.ctypes.data)))
        return F

    def stage_match(self, FP, FQ, precision=MATCH_FP32):
        pA, kA, nA = _prep(FP, np.float32, DESC_DIM)
        pB, kB, nB = _prep(FQ, np.float32, DESC_DIM)
        nn = np.zeros(nA, np.int32)
        d1 = np.zeros(nA, np.float32)
        fb = C.c_int64(0)
        self._check(self._L.lsr_stage_match(self._h, pA, nA, pB, nB, int(precision), C.c_void_p(nn.ctypes.data),
                                            C.c_void_p(d1.ctypes.data), C.byref(fb)))
        return nn, d1, int(fb.value)

    def match_scores_bf16(self, FP, FQ, precision=None):
        """Tensor-core approximations of |FP_i - FQ_j|^2 (nP x nQ float32)."""
        precision = MATCH_BF16 if precision is None else precision
        pA, kA, nA = _prep(FP, np.float32, DESC_DIM)
        pB, kB, nB = _prep(FQ, np.float32, DESC_DIM)
        out = np.zeros((nA, nB), np.float32)
        self._check(self._L.lsr_match_scores_bf16(self._h, pA, nA, pB, nB, int(precision),
                                                  C.c_void_p(out.ctypes.data)))
        return out

    def stage_hypotheses(self, P, Q, nn, validP, validQ, H, seed, pair_id=0, tau=0.9, cap=None):
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        pn, kn, _ = _prep(nn, np.int32)
        pa, ka, _ = _prep(validP, np.uint8)
        pb, kb, _ = _prep(validQ, np.uint8)
        cap = int(H if cap is None else cap)
        surv = np.zeros(max(cap, 1), np.int32)
        ns = C.c_int64(0)
        self._check(self._L.lsr_stage_hypotheses(self._h, pP, nP, pQ, nQ, pn, pa, pb, int(H), C.c_uint64(seed),
                                                 C.c_uint64(pair_id), C.c_float(tau), C.c_void_p(surv.ctypes.data),
                                                 cap, C.byref(ns)))
        return surv[:min(cap, ns.value)], int(ns.value)

    def stage_rigid4(self, ps, qs):
        pa, ka, nh = _prep(ps, np.float32, 12)
        pb, kb, _ = _prep(qs, np.float32, 12)
        Rt = np.zeros((nh, 12), np.float32)
        self._check(self._L.lsr_stage_rigid4(self._h, pa, pb, nh, C.c_void_p(Rt.ctypes.data)))
        return Rt

    def stage_consensus(self, P, Q, Rt, eps=0.0375):
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        pR, kR, nh = _prep(Rt, np.float32, 12)
        cnt = np.zeros(nh, np.int32)
        sd = np.zeros(nh, np.float64)
        self._check(self._L.lsr_stage_consensus(self._h, pP, nP, pQ, nQ, pR, nh, C.c_float(eps),
                                                C.c_void_p(cnt.ctypes.data), C.c_void_p(sd.ctypes.data)))
        return cnt, sd

    def stage_refine(self, P, Q, T, eps=0.0375, mu_scale=1.0, levels=4, iters=50):
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        Tin = np.ascontiguousarray(np.asarray(T, np.float64).reshape(16))
        Tout = np.zeros(16, np.float64)
        it = C.c_int32(0)
        self._check(self._L.lsr_stage_refine(self._h, pP, nP, pQ, nQ, C.c_void_p(Tin.ctypes.data), C.c_float(eps),
                                             C.c_float(mu_scale), int(levels), int(iters),
                                             C.c_void_p(Tout.ctypes.data), C.byref(it)))
        return Tout.reshape(4, 4), int(it.value)

    def stage_consensus_modes(self, P, Q, Rt, eps=0.0375, nn_mode=NN_EXACT, normal_mode=NORMALS_SAMPLES,
                              NP=None, NQ=None, cos_normal=0.8660254037844387):
        """Consensus counts and squared-distance sums per pose with the variant
        modes (lsr_stage_consensus_modes)."""
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        pR, kR, nh = _prep(Rt, np.float32, 12)
        pNP = pNQ = None
        if NP is not None:
            pNP, kNP, _ = _prep(NP, np.float32, 3)
            pNQ, kNQ, _ = _prep(NQ, np.float32, 3)
        cnt = np.zeros(nh, np.int32)
        sd = np.zeros(nh, np.float64)
        self._check(self._L.lsr_stage_consensus_modes(self._h, pP, pNP, nP, pQ, pNQ, nQ, pR, nh, C.c_float(eps),
                                                      int(nn_mode), int(normal_mode), C.c_float(cos_normal),
                                                      C.c_void_p(cnt.ctypes.data), C.c_void_p(sd.ctypes.data)))
        return cnt, sd

    def stage_nn(self, Q, X, r, mode=NN_EXACT):
        """Nearest Q point of every query (lsr_stage_nn): (nn int32, d2 float32)."""
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        pX, kX, nX = _prep(X, np.float32, 3)
        nn = np.zeros(nX, np.int32)
        d2 = np.zeros(nX, np.float32)
        self._check(self._L.lsr_stage_nn(self._h, pQ, nQ, pX, nX, C.c_float(r), int(mode),
                                         C.c_void_p(nn.ctypes.data), C.c_void_p(d2.ctypes.data)))
        return nn, d2

    def pose_implicit_grad(self, P, Q, T, dL_dT, eps=0.0375, mu=None, dP=None, dQ=None):
        """Gradient of a loss of the refined pose T with respect to the points
        (lsr_pose_implicit_grad). dL_dT: 4x4 gradient of the loss in T. dP, dQ:
        optional output arrays (both torch CUDA tensors or both None for numpy).
        Returns (dP, dQ, g (6), H (6x6), lambda (6), held pairs)."""
        mu = eps * eps if mu is None else mu
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        Tin = np.ascontiguousarray(np.asarray(T, np.float64).reshape(16))
        G = np.ascontiguousarray(np.asarray(dL_dT, np.float64).reshape(16))
        if dP is None:
            dP, dQ = np.zeros((nP, 3), np.float32), np.zeros((nQ, 3), np.float32)
            pdP, pdQ = C.c_void_p(dP.ctypes.data), C.c_void_p(dQ.ctypes.data)
        else:
            pdP, pdQ = C.c_void_p(dP.data_ptr()), C.c_void_p(dQ.data_ptr())
        g, H, lam, n = np.zeros(6), np.zeros(36), np.zeros(6), C.c_int64(0)
        self._check(self._L.lsr_pose_implicit_grad(self._h, pP, nP, pQ, nQ, C.c_void_p(Tin.ctypes.data),
                                                    C.c_float(eps), C.c_float(mu), C.c_void_p(G.ctypes.data), pdP, pdQ,
                                                    C.c_void_p(g.ctypes.data), C.c_void_p(H.ctypes.data),
                                                    C.c_void_p(lam.ctypes.data), C.byref(n)))
        return dP, dQ, g, H.reshape(6, 6), lam, int(n.value)

    def information_matrix(self, P, Q, T, eps=0.05):
        """Information matrix of eq. (5)-(6) for the pose T (P into Q's frame):
        returns (6x6 float64 array, number of correspondences)."""
        pP, kP, nP = _prep(P, np.float32, 3)
        pQ, kQ, nQ = _prep(Q, np.float32, 3)
        Tin = np.ascontiguousarray(np.asarray(T, np.float64).reshape(16))
        info = np.zeros(36, np.float64)
        n = C.c_int64(0)
        self._check(self._L.lsr_information_matrix(self._h, pP, nP, pQ, nQ, C.c_void_p(Tin.ctypes.data),
                                                   C.c_float(eps), C.c_void_p(info.ctypes.data), C.byref(n)))
        return info.reshape(6, 6), int(n.value)

    def voxel_downsample(self, P, leaf=0.05):
        """Voxel downsampling of Algorithm 1: (m x 3 float32 numpy array of
        voxel means in voxel order)."""
        pP, kP, n = _prep(P, np.float32, 3)
        out = np.zeros((n, 3), np.float32)
        m = C.c_int64(0)
        self._check(self._L.lsr_voxel_downsample(self._h, pP, n, C.c_float(leaf), C.c_void_p(out.ctypes.data), n,
                                                 C.byref(m)))
        return out[:m.value].copy()

    def surfel_correct(self, pos, nrm, t0, tu, T_old, T_new, t_kf, cam):
        """Dense model correction of eq. (7). pos, nrm: n x 3, t0, tu: n (numpy
        or CUDA tensors); T_old, T_new: m x 4 x 4, t_kf: m ascending, cam: 7.
        Returns (pos', nrm', keep, kept) as numpy arrays (or CUDA tensors when
        pos is one)."""
        pp, kp, n = _prep(pos, np.float32, 3)
        pn, kn, _ = _prep(nrm, np.float32, 3)
        p0, k0, _ = _prep(t0, np.float32, 1)
        pu, ku, _ = _prep(tu, np.float32, 1)
        To = np.ascontiguousarray(np.asarray(T_old, np.float64).reshape(-1, 16))
        Tn = np.ascontiguousarray(np.asarray(T_new, np.float64).reshape(-1, 16))
        tk = np.ascontiguousarray(np.asarray(t_kf, np.float32).reshape(-1))
        cm = np.ascontiguousarray(np.asarray(cam, np.float32).reshape(7))
        if _is_torch(pos):
            import torch
            po = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
            no = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
            ko = torch.empty(n, dtype=torch.uint8, device=pos.device)
            ptrs = (C.c_void_p(po.data_ptr()), C.c_void_p(no.data_ptr()), C.c_void_p(ko.data_ptr()))
        else:
            po, no, ko = np.zeros((n, 3), np.float32), np.zeros((n, 3), np.float32), np.zeros(n, np.uint8)
            ptrs = (C.c_void_p(po.ctypes.data), C.c_void_p(no.ctypes.data), C.c_void_p(ko.ctypes.data))
        kept = C.c_int64(0)
        self._check(self._L.lsr_surfel_correct(self._h, n, pp, pn, p0, pu, len(To), C.c_void_p(To.ctypes.data),
                                               C.c_void_p(Tn.ctypes.data), C.c_void_p(tk.ctypes.data),
                                               C.c_void_p(cm.ctypes.data), *ptrs, C.byref(kept)))
        return po, no, ko, int(kept.value)

    # -- objective (device tensors)
    def _obj_args(self, Ps, Qs, xi, T0):
        n = len(Ps)
        arrP = (C.c_void_p * n)(*[p.data_ptr() for p in Ps])
        arrQ = (C.c_void_p * n)(*[q.data_ptr() for q in Qs])
        nP = np.array([p.shape[0] for p in Ps], np.int64)
        nQ = np.array([q.shape[0] for q in Qs], np.int64)
        xi = np.ascontiguousarray(np.asarray(xi, np.float64).reshape(n, 6))
        T0 = np.ascontiguousarray(np.asarray(T0, np.float64).reshape(n, 16))
        return n, arrP, arrQ, nP, nQ, xi, T0

    def objective_fwd(self, Ps, Qs, xi, T0, eps=0.0375, mu=None):
        n, arrP, arrQ, nP, nQ, xi, T0 = self._obj_args(Ps, Qs, xi, T0)
        mu = eps * eps if mu is None else mu
        E = np.zeros(n, np.float64)
        self._check(self._L.lsr_objective_fwd(self._h, n, C.cast(arrP, C.POINTER(C.c_void_p)),
                                              C.c_void_p(nP.ctypes.data), C.cast(arrQ, C.POINTER(C.c_void_p)),
                                              C.c_void_p(nQ.ctypes.data), C.c_void_p(xi.ctypes.data),
                                              C.c_void_p(T0.ctypes.data), C.c_float(eps), C.c_float(mu),
                                              C.c_void_p(E.ctypes.data)))
        return E

    def objective_bwd(self, Ps, Qs, xi, T0, dE, dPs, dQs, eps=0.0375, mu=None):
        n, arrP, arrQ, nP, nQ, xi, T0 = self._obj_args(Ps, Qs, xi, T0)
        mu = eps * eps if mu is None else mu
        dE = np.ascontiguousarray(np.asarray(dE, np.float64).reshape(n))
        arrdP = (C.c_void_p * n)(*[t.data_ptr() for t in dPs])
        arrdQ = (C.c_void_p * n)(*[t.data_ptr() for t in dQs])
        dxi = np.zeros((n, 6), np.float64)
        self._check(self._L.lsr_objective_bwd(self._h, n, C.cast(arrP, C.POINTER(C.c_void_p)),
                                              C.c_void_p(nP.ctypes.data), C.cast(arrQ, C.POINTER(C.c_void_p)),
                                              C.c_void_p(nQ.ctypes.data), C.c_void_p(xi.ctypes.data),
                                              C.c_void_p(T0.ctypes.data), C.c_float(eps), C.c_float(mu),
                                              C.c_void_p(dE.ctypes.data), C.cast(arrdP, C.POINTER(C.c_void_p)),
                                              C.cast(arrdQ, C.POINTER(C.c_void_p)), C.c_void_p(dxi.ctypes.data)))
        return dxi


_default_ctx = {}


def context(device: int = 0) -> Context:
    """A process-wide default context per device (default parameters)."""
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


def register_pair(P, Q, vpP=None, vpQ=None, **params) -> Registration:
    ctx = context()
    if params:
        ctx.set_params(default_params(**params))
    return ctx.register_pair(P, Q, vpP, vpQ)
