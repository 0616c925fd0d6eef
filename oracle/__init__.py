"""FP64 CPU oracle for the LoopSmart global registration hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (``paper_1801_01572_gb300``) never imports it, and the two share no
code: the oracle is plain C (``lsr_oracle.c``) compiled with gcc, wrapped here
with ctypes and numpy.

Every function follows a passage of the paper (Sec. IV, Algorithm 1, eq. (1),
eq. (3)-(5)) or the FPFH definition the paper cites (Rusu et al., ICRA 2009);
the C file states the passage and the reading taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblsr_oracle.so")
_lock = threading.Lock()
_lib = None

D = 33


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("r_normal", C.c_double), ("r_feature", C.c_double), ("eps_inlier", C.c_double),
                ("tau", C.c_double), ("cos_normal", C.c_double), ("min_inlier_ratio", C.c_double),
                ("mu_scale", C.c_double), ("n_hypotheses", C.c_int64), ("refine_iters", C.c_int32),
                ("refine_levels", C.c_int32), ("seed", C.c_uint64), ("pair_id", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("T", C.c_double * 16), ("T_hyp", C.c_double * 16), ("inliers", C.c_int64),
                ("survivors", C.c_int64), ("best_h", C.c_int64), ("hyp_inliers", C.c_int64),
                ("n_normal_ok", C.c_int64), ("fitness", C.c_double), ("hyp_fitness", C.c_double),
                ("status", C.c_int32), ("refine_iters_done", C.c_int32)]


class Diag(C.Structure):
    _fields_ = [("nn_amb", C.c_int64), ("hyp_amb", C.c_int64), ("surv_touch", C.c_int64), ("n_top", C.c_int64),
                ("top_h", C.c_int64 * 16), ("top_count", C.c_int64 * 16), ("top_amb", C.c_int64 * 16), ("top_touch", C.c_int64 * 16),
                ("top_fitness", C.c_double * 16), ("final_amb", C.c_int64)]


DEFAULTS = dict(r_normal=0.05, r_feature=0.125, eps_inlier=0.0375, tau=0.9,
                cos_normal=float(np.cos(np.deg2rad(30.0))), min_inlier_ratio=0.05, mu_scale=1.0,
                n_hypotheses=4_000_000, refine_iters=50, refine_levels=3, seed=0, pair_id=0)


def _P(a, dt):
    return a.ctypes.data_as(C.POINTER(dt)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, ip, up8, u64p = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint8), C.POINTER(C.c_uint64)
            i64, dbl = C.c_int64, C.c_double
            sig = {
                "orc_set_threads": (None, [C.c_int]),
                "orc_get_threads": (C.c_int, []),
                "orc_radius_count_brute": (None, [dp, i64, dp, i64, dbl, ip]),
                "orc_radius_count_grid": (None, [dp, i64, dp, i64, dbl, ip]),
                "orc_eig3": (None, [dp, dp, dp]),
                "orc_normals": (None, [dp, i64, dp, dbl, ip, i64, dp, dp, ip, dp]),
                "orc_pair_features": (C.c_int, [dp, dp, dp, dp, dp]),
                "orc_spfh": (None, [dp, dp, i64, dbl, ip, i64, dbl, dp, ip, ip]),
                "orc_fpfh": (None, [dp, dp, dp, i64, dbl, ip, i64, dp]),
                "orc_match": (None, [dp, i64, dp, i64, i64, ip, i64, ip, dp, dp]),
                "orc_philox4x64_10": (None, [u64p, u64p, u64p]),
                "orc_sample_indices": (None, [C.c_uint64, C.c_uint64, i64, i64, i64, ip]),
                "orc_hypotheses": (None, [dp, i64, dp, i64, ip, up8, up8, i64, C.c_uint64, C.c_uint64, dbl, up8]),
                "orc_kabsch": (None, [dp, dp, i64, dp, dp]),
                "orc_nn_within_grid": (None, [dp, i64, dp, i64, dbl, ip, dp]),
                "orc_nn_within_brute": (None, [dp, i64, dp, i64, dbl, ip, dp]),
                "orc_consensus": (None, [dp, i64, dp, i64, dp, dp, i64, dbl, dbl, ip, dp, ip]),
                "orc_exp_so3": (None, [dp, dp]),
                "orc_apply_xi": (None, [dp, dp, dp]),
                "orc_refine": (C.c_int, [dp, i64, dp, i64, dp, dbl, dbl, C.c_int, dbl, dp]),
                "orc_refine_gnc": (C.c_int, [dp, i64, dp, i64, dp, dbl, dbl, C.c_int, C.c_int, dbl, dp]),
                "orc_gnc_stride": (i64, [i64, C.c_int, C.c_int]),
                "orc_objective": (C.c_double, [dp, i64, dp, i64, dp, dp, dbl, dbl, dp, dp, dp, ip]),
                "orc_information": (None, [dp, i64, dp, i64, dp, dbl, dbl, dp, ip, ip, dp]),
                "orc_register": (C.c_int, [dp, i64, dp, i64, dp, dp, C.POINTER(Params), C.POINTER(Result), dp, dp, ip,
                                          C.POINTER(Diag)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a, shape_last=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_last is not None:
        a = a.reshape(-1, shape_last)
    return a


def _idx(qidx):
    if qidx is None:
        return None, 0
    q = np.ascontiguousarray(np.asarray(qidx, dtype=np.int64))
    return q, len(q)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


# ------------------------------------------------------------------ neighbours
def radius_count_brute(P, X, r):
    P, X = _f64(P, 3), _f64(X, 3)
    out = np.zeros(len(X), np.int64)
    lib().orc_radius_count_brute(_P(P, C.c_double), len(P), _P(X, C.c_double), len(X), r, _P(out, C.c_int64))
    return out


def radius_count_grid(P, X, r):
    P, X = _f64(P, 3), _f64(X, 3)
    out = np.zeros(len(X), np.int64)
    lib().orc_radius_count_grid(_P(P, C.c_double), len(P), _P(X, C.c_double), len(X), r, _P(out, C.c_int64))
    return out


def nn_within(Q, X, r, brute=False):
    Q, X = _f64(Q, 3), _f64(X, 3)
    nn = np.zeros(len(X), np.int64)
    d2 = np.zeros(len(X), np.float64)
    f = lib().orc_nn_within_brute if brute else lib().orc_nn_within_grid
    f(_P(Q, C.c_double), len(Q), _P(X, C.c_double), len(X), r, _P(nn, C.c_int64), _P(d2, C.c_double))
    return nn, d2


def eig3(A):
    A = _f64(A).reshape(9)
    w = np.zeros(3)
    V = np.zeros(9)
    lib().orc_eig3(_P(A, C.c_double), _P(w, C.c_double), _P(V, C.c_double))
    return w, V.reshape(3, 3)


# ------------------------------------------------------------------ normals
def normals(P, vp=(0.0, 0.0, 0.0), r=0.05, qidx=None):
    """Returns (normals nq x 3, curvature nq, count nq, diag nq x 3)."""
    P = _f64(P, 3)
    vp = _f64(vp).reshape(3)
    q, nq = _idx(qidx)
    m = nq if q is not None else len(P)
    nrm, curv = np.zeros((m, 3)), np.zeros(m)
    cnt, diag = np.zeros(m, np.int64), np.zeros((m, 3))
    lib().orc_normals(_P(P, C.c_double), len(P), _P(vp, C.c_double), r, _P(q, C.c_int64), nq,
                      _P(nrm, C.c_double), _P(curv, C.c_double), _P(cnt, C.c_int64), _P(diag, C.c_double))
    return nrm, curv, cnt, diag


# ------------------------------------------------------------------ FPFH
def pair_features(ps, ns, pt, nt):
    a = [_f64(v).reshape(3) for v in (ps, ns, pt, nt)]
    f = np.zeros(3)
    ok = lib().orc_pair_features(*[_P(v, C.c_double) for v in a], _P(f, C.c_double))
    return bool(ok), f


def spfh(P, N, r=0.125, qidx=None, delta=1e-4):
    """Returns (spfh nq x 33, k nq, nclose nq)."""
    P, N = _f64(P, 3), _f64(N, 3)
    q, nq = _idx(qidx)
    m = nq if q is not None else len(P)
    S = np.zeros((m, D))
    k, nc = np.zeros(m, np.int64), np.zeros(m, np.int64)
    lib().orc_spfh(_P(P, C.c_double), _P(N, C.c_double), len(P), r, _P(q, C.c_int64), nq, delta,
                   _P(S, C.c_double), _P(k, C.c_int64), _P(nc, C.c_int64))
    return S, k, nc


def fpfh(P, N, S, r=0.125, qidx=None):
    P, N, S = _f64(P, 3), _f64(N, 3), _f64(S, D)
    q, nq = _idx(qidx)
    m = nq if q is not None else len(P)
    F = np.zeros((m, D))
    lib().orc_fpfh(_P(P, C.c_double), _P(N, C.c_double), _P(S, C.c_double), len(P), r, _P(q, C.c_int64), nq,
                   _P(F, C.c_double))
    return F


# ------------------------------------------------------------------ matching
def match(A, B, qidx=None):
    """Brute-force NN of each row of A among the rows of B: (nn, d1, d2)."""
    A = _f64(A)
    B = _f64(B)
    dim = A.shape[1]
    q, nq = _idx(qidx)
    m = nq if q is not None else len(A)
    nn, d1, d2 = np.zeros(m, np.int64), np.zeros(m), np.zeros(m)
    lib().orc_match(_P(A, C.c_double), len(A), _P(B, C.c_double), len(B), dim, _P(q, C.c_int64), nq,
                    _P(nn, C.c_int64), _P(d1, C.c_double), _P(d2, C.c_double))
    return nn, d1, d2


# ------------------------------------------------------------------ RNG + hypotheses
def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, np.uint64).reshape(2))
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_P(c, C.c_uint64), _P(k, C.c_uint64), _P(out, C.c_uint64))
    return out


def sample_indices(seed, pair, h0, nh, n):
    out = np.zeros((nh, 4), np.int64)
    lib().orc_sample_indices(C.c_uint64(seed), C.c_uint64(pair), h0, nh, n, _P(out, C.c_int64))
    return out


def hypotheses(P, Q, nn, validP, validQ, H, seed, pair, tau=0.9):
    """Per-hypothesis flag: 0 rejected, 1 survives, 2 ambiguous."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    nn = np.ascontiguousarray(np.asarray(nn, np.int64))
    vP = np.ascontiguousarray(np.asarray(validP, np.uint8))
    vQ = np.ascontiguousarray(np.asarray(validQ, np.uint8))
    flag = np.zeros(H, np.uint8)
    lib().orc_hypotheses(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(nn, C.c_int64),
                         _P(vP, C.c_uint8), _P(vQ, C.c_uint8), H, C.c_uint64(seed), C.c_uint64(pair), tau,
                         _P(flag, C.c_uint8))
    return flag


# ------------------------------------------------------------------ pose
def kabsch(p, q):
    p, q = _f64(p, 3), _f64(q, 3)
    R, t = np.zeros(9), np.zeros(3)
    lib().orc_kabsch(_P(p, C.c_double), _P(q, C.c_double), len(p), _P(R, C.c_double), _P(t, C.c_double))
    return R.reshape(3, 3), t


def consensus(P, Q, Rs, ts, eps, band=0.0):
    """Inlier count, sum of squared inlier distances, and near-eps count per pose."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    Rs = _f64(Rs).reshape(-1, 9)
    ts = _f64(ts).reshape(-1, 3)
    nh = len(Rs)
    cnt, amb = np.zeros(nh, np.int64), np.zeros(nh, np.int64)
    sd = np.zeros(nh)
    lib().orc_consensus(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(Rs, C.c_double),
                        _P(ts, C.c_double), nh, eps, band, _P(cnt, C.c_int64), _P(sd, C.c_double), _P(amb, C.c_int64))
    return cnt, sd, amb


def exp_so3(w):
    w = _f64(w).reshape(3)
    R = np.zeros(9)
    lib().orc_exp_so3(_P(w, C.c_double), _P(R, C.c_double))
    return R.reshape(3, 3)


def apply_xi(xi, T):
    xi = _f64(xi).reshape(6)
    T = _f64(T).reshape(16)
    out = np.zeros(16)
    lib().orc_apply_xi(_P(xi, C.c_double), _P(T, C.c_double), _P(out, C.c_double))
    return out.reshape(4, 4)


def refine(P, Q, T, eps_r, mu, iters=30, tol=1e-10):
    P, Q = _f64(P, 3), _f64(Q, 3)
    T = _f64(T).reshape(16)
    out = np.zeros(16)
    n = lib().orc_refine(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(T, C.c_double), eps_r, mu,
                         iters, tol, _P(out, C.c_double))
    return out.reshape(4, 4), int(n)


def refine_gnc(P, Q, T, eps, mu_scale=1.0, levels=3, iters=50, tol=1e-10):
    """Graduated refinement: radii eps * 2^(L-1-l), subsets by caller index."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    T = _f64(T).reshape(16)
    out = np.zeros(16)
    n = lib().orc_refine_gnc(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(T, C.c_double), eps,
                             mu_scale, levels, iters, tol, _P(out, C.c_double))
    return out.reshape(4, 4), int(n)


def gnc_stride(n, level, levels):
    return int(lib().orc_gnc_stride(int(n), int(level), int(levels)))


def information(P, Q, T, eps=0.05, band=0.0):
    """Information matrix of eq. (5)-(6): sum of G_p^T G_p, G_p = [-[p]_x | I],
    over the points p of T P whose NN in Q lies closer than eps. Returns
    (info 6x6, n, namb, amb_max): namb points have their NN distance within
    band of eps, the largest |T p|^2 among them is amb_max."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    T = _f64(T).reshape(16)
    info = np.zeros(36)
    n, namb, amb_max = C.c_int64(0), C.c_int64(0), C.c_double(0.0)
    lib().orc_information(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(T, C.c_double), eps, band,
                          _P(info, C.c_double), C.byref(n), C.byref(namb), C.byref(amb_max))
    return info.reshape(6, 6), n.value, namb.value, amb_max.value


def voxel_downsample(P, leaf):
    """Downsampling of Algorithm 1 (first line): one point per occupied voxel of
    edge leaf, the mean of the points in it. Reading: voxels are aligned to the
    coordinate origin, key = floor(p / leaf) per axis in FP64, and the output
    is ordered by (k_z, k_y, k_x) ascending. Returns (points m x 3 float64,
    counts m)."""
    P = np.asarray(P, np.float64)
    keys = np.floor(P / float(leaf)).astype(np.int64)
    order = np.lexsort((keys[:, 0], keys[:, 1], keys[:, 2]))
    ks = keys[order]
    new = np.ones(len(ks), bool)
    new[1:] = np.any(ks[1:] != ks[:-1], axis=1)
    group = np.cumsum(new) - 1
    m = int(group[-1]) + 1 if len(group) else 0
    sums = np.zeros((m, 3))
    np.add.at(sums, group, P[order])
    counts = np.bincount(group, minlength=m)
    return sums / counts[:, None], counts


def nn_single_cell(Q, X, cell):
    """The O(1) grid lookup of eq. (1) (a speed mode, not exact): each query
    looks only in its own cell, index = floor((x - c) / cell) per axis with c
    the centroid of Q (reading: floor, and "centre" as the centroid), and takes
    the nearest Q point there. Returns (nn index or -1, squared distance or
    inf), ties to the smaller index."""
    Q, X = np.asarray(Q, np.float64), np.asarray(X, np.float64)
    c = Q.mean(axis=0)
    kq = np.floor((Q - c) / cell).astype(np.int64)
    kx = np.floor((X - c) / cell).astype(np.int64)
    table = {}
    for j, k in enumerate(map(tuple, kq)):
        table.setdefault(k, []).append(j)
    nn = np.full(len(X), -1, np.int64)
    d2 = np.full(len(X), np.inf)
    for i, k in enumerate(map(tuple, kx)):
        js = table.get(k)
        if not js:
            continue
        dd = ((Q[js] - X[i]) ** 2).sum(1)
        a = int(np.argmin(dd))
        nn[i], d2[i] = js[a], dd[a]
    return nn, d2


def consensus_single_cell(P, Q, Rs, ts, eps):
    """Consensus of Alg. 1 with the single-cell lookup of eq. (1) as the
    nearest-neighbour search (the paper's speed mode; cell edge = eps on the
    lattice through Q's centroid): per pose [R | t], the points of P whose own
    cell's nearest Q point is closer than eps, and the sum of their squared
    distances. FP64."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    Rs = _f64(Rs).reshape(-1, 3, 3)
    ts = _f64(ts).reshape(-1, 3)
    cnt, sd = np.zeros(len(Rs), np.int64), np.zeros(len(Rs))
    for k, (R, t) in enumerate(zip(Rs, ts)):
        _, d2 = nn_single_cell(Q, P @ R.T + t, eps)
        inl = d2 < eps * eps
        cnt[k], sd[k] = int(inl.sum()), float(d2[inl].sum())
    return cnt, sd


def consensus_normals(P, NP, Q, NQ, Rs, ts, eps, cos_normal, band=0.0):
    """Consensus of Alg. 1 with the normal check applied to every inlier (the
    alternative reading of "normal check moved into hypotheses testing",
    Sec. IV): per pose [R | t], a point p of P counts if its nearest Q point q
    (exact search, ties to the smaller index) is closer than eps and
    cos(R n_p, n_q) >= cos_normal, both normals valid (non-zero). Returns
    (count, sum of squared distances, ambiguous): ambiguous counts the points
    an FP32 evaluation may decide the other way (distance within band of eps,
    cosine within band of the threshold, or a runner-up within band of the
    nearest). FP64."""
    P, Q, NP, NQ = _f64(P, 3), _f64(Q, 3), _f64(NP, 3), _f64(NQ, 3)
    Rs = _f64(Rs).reshape(-1, 3, 3)
    ts = _f64(ts).reshape(-1, 3)
    vP = np.abs(NP).sum(1) > 0
    vQ = np.abs(NQ).sum(1) > 0
    cnt, sd, amb = np.zeros(len(Rs), np.int64), np.zeros(len(Rs)), np.zeros(len(Rs), np.int64)
    for k, (R, t) in enumerate(zip(Rs, ts)):
        X = P @ R.T + t
        j, d2 = nn_within(Q, X, eps + band)
        has = j >= 0
        jj = np.where(has, j, 0)
        cs = ((NP @ R.T) * NQ[jj]).sum(1)
        inl = has & (d2 < eps * eps) & vP & vQ[jj] & (cs >= cos_normal)
        cnt[k], sd[k] = int(inl.sum()), float(d2[inl].sum())
        if band > 0:
            d = np.sqrt(np.where(has, d2, np.inf))
            near = has & ((np.abs(d - eps) < band) | (np.abs(cs - cos_normal) < band))
            amb[k] = int(near.sum())
    return cnt, sd, amb


def _gm(s, mu):
    """Geman-McClure rho(s) = mu s / (mu + s) of eq. (4) and its first two
    derivatives in s."""
    d = mu + s
    return mu * s / d, mu * mu / (d * d), -2.0 * mu * mu / (d * d * d)


def _skew(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def pose_grad_hess(X, Y, T, mu):
    """E(xi) = sum_i rho(|T(xi) x_i - y_i|^2) with the pairs (x_i, y_i) held and
    T(xi) = [Exp(w) | v] T (the left perturbation of the refinement): E, its
    gradient g and its exact Hessian H in xi = (w, v) at xi = 0.

    With z = R x + t, r = z - y, s = |r|^2 and J = [-[z]_x | I]:
      g = sum 2 rho'(s) J^T r,
      H = sum 4 rho''(s) (J^T r)(J^T r)^T + 2 rho'(s) (J^T J + S),
    S the second derivative of r . Exp(w) z at w = 0, nonzero in the rotation
    block only: S_ab = (r_a z_b + r_b z_a) / 2 - (r . z) delta_ab."""
    X, Y = _f64(X, 3), _f64(Y, 3)
    T = np.asarray(T, np.float64)
    Z = X @ T[:3, :3].T + T[:3, 3]
    Rr = Z - Y
    s = (Rr * Rr).sum(1)
    rho, d1, d2 = _gm(s, mu)
    g, H = np.zeros(6), np.zeros((6, 6))
    for z, r, a1, a2 in zip(Z, Rr, d1, d2):
        J = np.hstack([-_skew(z), np.eye(3)])
        Jr = J.T @ r
        g += 2.0 * a1 * Jr
        Sm = np.zeros((6, 6))
        Sm[:3, :3] = 0.5 * (np.outer(r, z) + np.outer(z, r)) - (r @ z) * np.eye(3)
        H += 4.0 * a2 * np.outer(Jr, Jr) + 2.0 * a1 * (J.T @ J + Sm)
    return float(rho.sum()), g, H


def pose_optimum(X, Y, T0, mu, iters=60, tol=1e-15):
    """The pose minimising E over the held pairs, by Newton steps with the exact
    Hessian of pose_grad_hess (each step solves H d = -g and moves T to
    [Exp(d_w) | d_v] T), halving a step that does not lower E. Stops when
    |d| < tol. Returns (T, |g| at the end)."""
    T = np.asarray(T0, np.float64).copy()
    E, g, H = pose_grad_hess(X, Y, T, mu)
    for _ in range(iters):
        d = np.linalg.solve(H, -g)
        step = 1.0
        while True:
            Tn = apply_xi(step * d, T)
            En, gn, Hn = pose_grad_hess(X, Y, Tn, mu)
            if En <= E or step < 1e-6:
                break
            step *= 0.5
        T, E, g, H = Tn, En, gn, Hn
        if np.linalg.norm(step * d) < tol:
            break
    return T, float(np.linalg.norm(g))


def pose_implicit_grad(X, Y, T, mu, dL_dxi):
    """Gradient of a loss L of the optimal pose with respect to the held pairs
    (implicit function theorem at the optimum T, where g = 0): with dL_dxi the
    gradient of L in the left perturbation xi of T, lambda = H^-1 dL_dxi and
    phi_i = lambda . g_i = 2 rho'(s_i) a_i . r_i, a_i = w_l x z_i + v_l,
      dL/dx_i = -R^T dphi_i/dz_i,  dL/dy_i = -dphi_i/dy_i,
      dphi/dz = 4 rho''(s) (a . r) r + 2 rho'(s) (a + r x w_l),
      dphi/dy = -4 rho''(s) (a . r) r - 2 rho'(s) a.
    Returns (dL/dX, dL/dY)."""
    X, Y = _f64(X, 3), _f64(Y, 3)
    T = np.asarray(T, np.float64)
    _, _, H = pose_grad_hess(X, Y, T, mu)
    lam = np.linalg.solve(H, np.asarray(dL_dxi, np.float64).reshape(6))
    wl, vl = lam[:3], lam[3:]
    Z = X @ T[:3, :3].T + T[:3, 3]
    Rr = Z - Y
    s = (Rr * Rr).sum(1)
    _, d1, d2 = _gm(s, mu)
    A = np.cross(wl, Z) + vl
    ar = (A * Rr).sum(1)
    dz = 4.0 * d2[:, None] * ar[:, None] * Rr + 2.0 * d1[:, None] * (A + np.cross(Rr, wl))
    dy = -4.0 * d2[:, None] * ar[:, None] * Rr - 2.0 * d1[:, None] * A
    return -(dz @ T[:3, :3]), -dy


def surfel_correct(pos, nrm, t0, tu, T_old, T_new, t_kf, cam, band=None):
    """Dense model correction of eq. (7), in FP64 with numpy.

    For each surfel (position p, normal n, time stamps t0 < tu), F is the set
    of keyframes f with t0 < t_f < tu that observe the surfel before the
    correction: the point T_f_old^-1 p lies in front of the camera, no farther
    than the maximum depth, and projects inside the image (reading: pinhole
    camera cam = (fx, fy, cx, cy, width, height, max depth), u = fx x / z + cx,
    0 <= u < width, likewise v). With k = |F|,
        p' = (1/k) sum_f T_f_new T_f_old^-1 p,
        n' = normalize((1/k) sum_f R_f_new R_f_old^-1 n),
    and a surfel with k = 0 is removed (keep = False; p, n returned unchanged).
    T_old, T_new: m x 4 x 4 camera-to-world poses; t_kf: m time stamps.
    Returns (p', n', keep); with band = (metres, pixels) also a fourth array,
    border: surfels for which some keyframe of their time window decides
    visibility within that band of a limit (depth 0 or the maximum, an image
    edge), so that an FP32 evaluation may decide it the other way (reporting
    only)."""
    pos, nrm = np.asarray(pos, np.float64), np.asarray(nrm, np.float64)
    t0, tu = np.asarray(t0, np.float64), np.asarray(tu, np.float64)
    T_old, T_new = np.asarray(T_old, np.float64), np.asarray(T_new, np.float64)
    fx, fy, cx, cy, W, H, dmax = (float(v) for v in cam)
    sp = np.zeros_like(pos)
    sn = np.zeros_like(nrm)
    k = np.zeros(len(pos), np.int64)
    border = np.zeros(len(pos), bool)
    for f in range(len(T_old)):
        inv = np.linalg.inv(T_old[f])
        M = T_new[f] @ inv
        xc = pos @ inv[:3, :3].T + inv[:3, 3]
        z = xc[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * xc[:, 0] / z + cx
            v = fy * xc[:, 1] / z + cy
        seen = (t0 < t_kf[f]) & (t_kf[f] < tu) & (z > 0) & (z <= dmax) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
        if band is not None:
            bm, bp = band
            win = (t0 < t_kf[f]) & (t_kf[f] < tu)
            with np.errstate(invalid="ignore"):
                near = (np.abs(z) < bm) | (np.abs(z - dmax) < bm) | (np.abs(u) < bp) | (np.abs(u - W) < bp) | \
                    (np.abs(v) < bp) | (np.abs(v - H) < bp)
            border |= win & near
        k += seen
        sp[seen] += pos[seen] @ M[:3, :3].T + M[:3, 3]
        sn[seen] += nrm[seen] @ M[:3, :3].T
    keep = k > 0
    p_out, n_out = pos.copy(), nrm.copy()
    p_out[keep] = sp[keep] / k[keep, None]
    m = sn[keep] / k[keep, None]
    n_out[keep] = m / np.linalg.norm(m, axis=1, keepdims=True)
    if band is not None:
        return p_out, n_out, keep, border
    return p_out, n_out, keep


def objective(P, Q, xi, T0, eps, mu, grad=True):
    """E and (if grad) dE/dP, dE/dQ, dE/dxi, plus the NN index of each point."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    xi = _f64(xi).reshape(6)
    T0 = _f64(T0).reshape(16)
    nn = np.zeros(len(P), np.int64)
    if grad:
        dP, dQ, dxi = np.zeros((len(P), 3)), np.zeros((len(Q), 3)), np.zeros(6)
    else:
        dP = dQ = dxi = None
    E = lib().orc_objective(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(xi, C.c_double),
                            _P(T0, C.c_double), eps, mu, _P(dP, C.c_double), _P(dQ, C.c_double),
                            _P(dxi, C.c_double), _P(nn, C.c_int64))
    return float(E), dP, dQ, dxi, nn


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def register(P, Q, vpP=(0, 0, 0), vpQ=(0, 0, 0), debug=False, diag=False, **kw):
    """Algorithm 1 end to end, then the robust refinement. Returns a dict.

    diag=True adds what an FP32 implementation may decide the other way
    (reporting only, the result is unchanged): ``nn_amb`` points of P whose
    descriptor NN gap is at most 1e-5, ``hyp_amb`` hypotheses whose
    pre-rejection lies in its band, ``surv_touch`` survivors with a sampled
    point in ``nn_amb``, the 16 best normal-checked hypotheses in selection
    order (``top``: id, count, points within 1e-5 m of eps, whether a sampled
    point is in ``nn_amb``, fitness) and
    ``final_amb`` at the refined pose."""
    P, Q = _f64(P, 3), _f64(Q, 3)
    vpP = _f64(vpP).reshape(3)
    vpQ = _f64(vpQ).reshape(3)
    prm = make_params(**kw)
    res = Result()
    dg = Diag() if diag else None
    fP = np.zeros((len(P), D)) if debug else None
    fQ = np.zeros((len(Q), D)) if debug else None
    nn = np.zeros(len(P), np.int64) if debug else None
    rc = lib().orc_register(_P(P, C.c_double), len(P), _P(Q, C.c_double), len(Q), _P(vpP, C.c_double),
                            _P(vpQ, C.c_double), C.byref(prm), C.byref(res), _P(fP, C.c_double),
                            _P(fQ, C.c_double), _P(nn, C.c_int64), C.byref(dg) if dg is not None else None)
    out = dict(rc=rc, T=np.array(res.T).reshape(4, 4), T_hyp=np.array(res.T_hyp).reshape(4, 4),
               inliers=res.inliers, fitness=res.fitness, status=res.status, survivors=res.survivors,
               best_h=res.best_h, hyp_inliers=res.hyp_inliers, hyp_fitness=res.hyp_fitness,
               n_normal_ok=res.n_normal_ok, refine_iters=res.refine_iters_done)
    if debug:
        out.update(FP=fP, FQ=fQ, nn=nn)
    if diag:
        k = int(dg.n_top)
        out.update(nn_amb=int(dg.nn_amb), hyp_amb=int(dg.hyp_amb), surv_touch=int(dg.surv_touch),
                   final_amb=int(dg.final_amb),
                   top=[dict(h=int(dg.top_h[i]), count=int(dg.top_count[i]), amb=int(dg.top_amb[i]),
                             touch=int(dg.top_touch[i]), fitness=float(dg.top_fitness[i])) for i in range(k)])
    return out
