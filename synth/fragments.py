"""Seeded synthetic fragment pairs.

The paper evaluates on fragment pairs of the augmented ICL-NUIM / Redwood
registration benchmark (Sec. IV, Table I), which are not available here. These
generators stand in for them with the same structure: planar-dominated indoor
surfaces, sensor-scale noise, partial overlap and an unknown rigid motion.

  objects : 6 planar patches, 3 spheres and 2 boxes inside a 2 m cube, points
            drawn uniformly by area (about 2.5 cm spacing at 5,000 points).
  room    : floor, four walls and 20 boxes / cylinders standing on the floor,
            sampled on a 1 cm surface lattice and snapped to a 1 cm voxel grid in
            each fragment's own frame (like a TSDF fragment surface).

The second cloud Q is the scene under a ground-truth pose T (q = T p), sampled
independently of P (its own random sampling or lattice offsets, its own voxel
grid and its own noise). The overlap |P & Q| / |P| is set by a plane sweep
along a random direction. Seeds are 1000 + 100 * config + pair.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CONFIGS = {
    0: dict(kind="objects", n_pairs=1, n_p=5_000, n_q=5_000, sigma=0.002, overlap=0.70, outliers=0.10),
    1: dict(kind="room", n_pairs=1, n_p=150_000, n_q=150_000, sigma=0.003, overlap=0.50, outliers=0.0),
    2: dict(kind="room", n_pairs=256, n_range=(10_000, 120_000), overlap_range=(0.30, 0.80), sigma=0.003,
            outliers=0.0),
    3: dict(kind="room", n_pairs=64, n_p=200_000, n_q=200_000, sigma=0.003, overlap=0.50, outliers=0.0),
    4: dict(kind="room", n_pairs=32, n_p=50_000, n_q=50_000, sigma=0.003, overlap=0.50, outliers=0.0),
}


@dataclass
class FragmentPair:
    P: np.ndarray            # (nP, 3) float32, fragment P in its own frame
    Q: np.ndarray            # (nQ, 3) float32, fragment Q in its own frame
    T: np.ndarray            # (4, 4) float64 ground truth, q = T p
    vpP: np.ndarray          # (3,) viewpoint of P (normals face it)
    vpQ: np.ndarray          # (3,) the same viewpoint in Q's frame
    seed: int
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------- rigid motions
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-uniform rotation from a normalised Gaussian quaternion (Shoemake)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_pose(rng: np.random.Generator, max_t: float = 1.0) -> np.ndarray:
    """Uniform rotation (all angles up to 180 deg) and a translation uniform in a ball."""
    T = np.eye(4)
    T[:3, :3] = random_rotation(rng)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    T[:3, 3] = d * max_t * rng.uniform() ** (1.0 / 3.0)
    return T


def pose_error(Ta: np.ndarray, Tb: np.ndarray) -> tuple[float, float]:
    """(rotation angle of Ra^T Rb in degrees, |ta - tb| in metres)."""
    Ra, Rb = np.asarray(Ta)[:3, :3], np.asarray(Tb)[:3, :3]
    M = Ra.T @ Rb
    c = (np.trace(M) - 1.0) / 2.0
    s = 0.5 * np.linalg.norm([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
    ang = float(np.degrees(np.arctan2(s, c)))
    return ang, float(np.linalg.norm(np.asarray(Ta)[:3, 3] - np.asarray(Tb)[:3, 3]))


def _apply(T, X):
    return X @ T[:3, :3].T + T[:3, 3]


# --------------------------------------------------------------------- surface primitives
class _Rect:
    def __init__(self, c, a1, a2, h1, h2):
        self.c, self.a1, self.a2, self.h1, self.h2 = (np.asarray(c, float), np.asarray(a1, float),
                                                      np.asarray(a2, float), float(h1), float(h2))
        self.area = 4.0 * self.h1 * self.h2

    def random(self, n, rng):
        u = rng.uniform(-self.h1, self.h1, n)
        v = rng.uniform(-self.h2, self.h2, n)
        return self.c + u[:, None] * self.a1 + v[:, None] * self.a2

    def lattice(self, s, rng):
        u = np.arange(-self.h1 + rng.uniform(0, s), self.h1, s)
        v = np.arange(-self.h2 + rng.uniform(0, s), self.h2, s)
        U, V = np.meshgrid(u, v, indexing="ij")
        return self.c + U.reshape(-1, 1) * self.a1 + V.reshape(-1, 1) * self.a2


class _Sphere:
    def __init__(self, c, R):
        self.c, self.R = np.asarray(c, float), float(R)
        self.area = 4.0 * np.pi * self.R ** 2

    def random(self, n, rng):
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return self.c + self.R * d

    def lattice(self, s, rng):
        n = max(8, int(round(self.area / (s * s))))
        k = np.arange(n) + 0.5
        z = 1.0 - 2.0 * k / n
        phi = np.pi * (1.0 + 5 ** 0.5) * k
        r = np.sqrt(1.0 - z * z)
        d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1) @ random_rotation(rng).T
        return self.c + self.R * d


class _Cylinder:
    """Vertical cylinder standing on z = z0: side wall and top disk."""

    def __init__(self, c, r, h):
        self.c, self.r, self.h = np.asarray(c, float), float(r), float(h)
        self.side = 2.0 * np.pi * self.r * self.h
        self.top = np.pi * self.r ** 2
        self.area = self.side + self.top

    def random(self, n, rng):
        on_side = rng.uniform(size=n) < self.side / self.area
        th = rng.uniform(0, 2 * np.pi, n)
        z = np.where(on_side, rng.uniform(0, self.h, n), self.h)
        rr = np.where(on_side, self.r, self.r * np.sqrt(rng.uniform(size=n)))
        return self.c + np.stack([rr * np.cos(th), rr * np.sin(th), z], axis=1)

    def lattice(self, s, rng):
        nth = max(8, int(round(2 * np.pi * self.r / s)))
        th = (np.arange(nth) + rng.uniform()) * (2 * np.pi / nth)
        z = np.arange(rng.uniform(0, s), self.h, s)
        TH, Z = np.meshgrid(th, z, indexing="ij")
        side = np.stack([self.r * np.cos(TH).ravel(), self.r * np.sin(TH).ravel(), Z.ravel()], axis=1)
        u = np.arange(-self.r + rng.uniform(0, s), self.r, s)
        U, V = np.meshgrid(u, u, indexing="ij")
        keep = U ** 2 + V ** 2 <= self.r ** 2
        top = np.stack([U[keep], V[keep], np.full(keep.sum(), self.h)], axis=1)
        return self.c + np.concatenate([side, top], axis=0)


def _box_faces(c, R, half, bottom=True):
    faces = []
    for ax in range(3):
        if not bottom and ax == 2:
            o = [1]
        else:
            o = [-1, 1]
        a1, a2 = [(ax + 1) % 3, (ax + 2) % 3]
        for sgn in o:
            fc = c + sgn * half[ax] * R[:, ax]
            faces.append(_Rect(fc, R[:, a1], R[:, a2], half[a1], half[a2]))
    return faces


def _objects_scene(rng):
    """6 planar patches, 3 spheres, 2 boxes in the cube [-1, 1]^3."""
    prims = []
    for _ in range(6):
        R = random_rotation(rng)
        prims.append(_Rect(rng.uniform(-0.7, 0.7, 3), R[:, 0], R[:, 1], rng.uniform(0.2, 0.3), rng.uniform(0.2, 0.3)))
    for _ in range(3):
        prims.append(_Sphere(rng.uniform(-0.7, 0.7, 3), rng.uniform(0.12, 0.18)))
    for _ in range(2):
        prims.extend(_box_faces(rng.uniform(-0.6, 0.6, 3), random_rotation(rng), rng.uniform(0.1, 0.15, 3)))
    vp = np.array([0.0, -2.5, 1.0])
    return prims, vp


class _Occluded:
    """A primitive with the points inside some vertical footprints removed (floor
    under furniture is not seen by the camera)."""

    def __init__(self, prim, footprints):
        self.prim, self.fp = prim, footprints
        self.area = prim.area

    def _keep(self, X):
        keep = np.ones(len(X), bool)
        for (cx, cy, R, hx, hy, r) in self.fp:
            d = X[:, :2] - [cx, cy]
            if r > 0:
                keep &= (d ** 2).sum(1) > r * r
            else:
                u = d @ R[:2, 0]
                v = d @ R[:2, 1]
                keep &= ~((np.abs(u) < hx) & (np.abs(v) < hy))
        return X[keep]

    def random(self, n, rng):
        return self._keep(self.prim.random(n, rng))

    def lattice(self, s, rng):
        return self._keep(self.prim.lattice(s, rng))


def _room_scene(rng, W=4.0, D=3.5, H=1.5, n_obj=20):
    """Floor, four walls (the band up to H that a fragment's camera sees) and
    n_obj boxes / cylinders: cabinets and shelves against the walls, tables and
    stands in the room; the floor under them is hidden. Furniture is sized so
    that less than half of a fragment lies on the floor and walls, as in the
    cluttered indoor fragments the paper registers. Room size varies by up to
    15% per pair."""
    W *= rng.uniform(0.85, 1.15)
    D *= rng.uniform(0.85, 1.15)
    walls = [_Rect([W / 2, 0.0, H / 2], [1, 0, 0], [0, 0, 1], W / 2, H / 2),
             _Rect([W / 2, D, H / 2], [1, 0, 0], [0, 0, 1], W / 2, H / 2),
             _Rect([0.0, D / 2, H / 2], [0, 1, 0], [0, 0, 1], D / 2, H / 2),
             _Rect([W, D / 2, H / 2], [0, 1, 0], [0, 0, 1], D / 2, H / 2)]
    prims, foot = list(walls), []
    for k in range(n_obj):
        if k % 2 == 0:
            half = np.array([rng.uniform(0.2, 0.6), rng.uniform(0.15, 0.4), rng.uniform(0.2, 0.9)])
            if k % 4 == 0:
                # against a wall (cabinet, shelf), possibly raised off the floor
                side = int(rng.integers(4))
                along = rng.uniform(0.3, (W if side < 2 else D) - 0.3)
                yaw = [0.0, np.pi, np.pi / 2, -np.pi / 2][side]
                x, y = [(along, half[1]), (along, D - half[1]), (half[1], along), (W - half[1], along)][side]
                z = half[2] if rng.uniform() < 0.6 else rng.uniform(0.8, 1.6)
            else:
                yaw = rng.uniform(0, 2 * np.pi)
                x, y, z = rng.uniform(0.5, W - 0.5), rng.uniform(0.5, D - 0.5), half[2]
            R = np.array([[np.cos(yaw), -np.sin(yaw), 0], [np.sin(yaw), np.cos(yaw), 0], [0, 0, 1.0]])
            prims.extend(_box_faces(np.array([x, y, z]), R, half, bottom=z > half[2] + 1e-9))
            if z <= half[2] + 1e-9:
                foot.append((x, y, R, half[0], half[1], 0.0))
        else:
            x, y, r = rng.uniform(0.4, W - 0.4), rng.uniform(0.4, D - 0.4), rng.uniform(0.1, 0.35)
            prims.append(_Cylinder([x, y, 0.0], r, rng.uniform(0.3, 1.4)))
            foot.append((x, y, None, 0.0, 0.0, r))
    prims.insert(0, _Occluded(_Rect([W / 2, D / 2, 0.0], [1, 0, 0], [0, 1, 0], W / 2, D / 2), foot))
    vp = np.array([W / 2, D / 2, 1.2])
    return prims, vp


def _random_area(prims, n, rng):
    areas = np.array([p.area for p in prims])
    counts = rng.multinomial(n, areas / areas.sum())
    X = np.concatenate([p.random(k, rng) for p, k in zip(prims, counts) if k > 0], axis=0)
    return X[rng.permutation(len(X))]


def _lattice(prims, s, rng):
    return np.concatenate([p.lattice(s, rng) for p in prims], axis=0)


def _voxel_snap(X, g):
    """One point per occupied g-voxel (its centre), in the frame of X."""
    k = np.floor(X / g).astype(np.int64)
    k = np.unique(k, axis=0)
    return (k + 0.5) * g


# --------------------------------------------------------------------- pair makers
def _objects_pair(rng, n_p, n_q, sigma, overlap, outliers):
    prims, vp = _objects_scene(rng)
    T = random_pose(rng)
    phi = rng.standard_normal(3)
    d = phi / np.linalg.norm(phi)
    P = _random_area(prims, n_p, rng)
    # Q covers the part of the scene with s >= s_c, which holds `overlap` of P
    sP = P @ d
    s_c = np.quantile(sP, 1.0 - overlap)
    pool = []
    need = n_q
    while need > 0:
        X = _random_area(prims, 4 * n_q, rng)
        X = X[X @ d >= s_c]
        pool.append(X[:need])
        need -= len(pool[-1])
    Qw = np.concatenate(pool, axis=0)
    P = P + rng.normal(0, sigma, P.shape)
    Q = _apply(T, Qw) + rng.normal(0, sigma, Qw.shape)
    n_out = int(round(outliers * n_q))
    if n_out:
        lo, hi = Q.min(0), Q.max(0)
        idx = rng.choice(n_q, n_out, replace=False)
        Q[idx] = rng.uniform(lo, hi, (n_out, 3))
    return P, Q, T, vp, dict(overlap=overlap, n_outliers=n_out)


def _room_pair(rng, n_p, n_q, sigma, overlap, grid=0.01):
    prims, vp = _room_scene(rng)
    T = random_pose(rng)
    # sweep direction oblique to the walls (a sweep along a wall would leave the
    # fragments free to slide along it)
    ang = int(rng.integers(4)) * (np.pi / 2) + np.deg2rad(rng.uniform(25.0, 65.0))
    d = np.array([np.cos(ang), np.sin(ang), 0.0])
    LP = _lattice(prims, grid, rng)           # P's own lattice (world frame)
    LQ = _lattice(prims, grid, rng)           # Q's independent lattice
    sP = np.sort(LP @ d)
    span = n_p + n_q - overlap * n_p
    if span * 1.1 > len(sP):
        raise ValueError(f"scene too small for {n_p}+{n_q} points at overlap {overlap}")
    slack = 1.06
    i0 = int(rng.integers(0, len(sP) - int(span * slack)))
    # P window [a, b], Q window [c, e]; overlap [c, b] holds `overlap` of P
    for _ in range(20):
        a = sP[i0]
        b = sP[min(len(sP) - 1, i0 + int(n_p * slack))]
        c = sP[min(len(sP) - 1, i0 + int(n_p * slack * (1 - overlap)))]
        e = sP[min(len(sP) - 1, i0 + int(n_p * slack * (1 - overlap)) + int(n_q * slack))]
        Pw = LP[(LP @ d >= a) & (LP @ d <= b)]
        Qw = LQ[(LQ @ d >= c) & (LQ @ d <= e)]
        P = _voxel_snap(Pw, grid)
        Q = _voxel_snap(_apply(T, Qw), grid)
        if len(P) >= n_p and len(Q) >= n_q:
            break
        slack *= 1.05
        i0 = max(0, min(i0, len(sP) - int(span * slack) - 1))
    else:  # pragma: no cover - the scene is sized to avoid this
        raise RuntimeError("could not crop enough points")
    P = P[rng.choice(len(P), n_p, replace=False)]
    Q = Q[rng.choice(len(Q), n_q, replace=False)]
    P = P + rng.normal(0, sigma, P.shape)
    Q = Q + rng.normal(0, sigma, Q.shape)
    return P, Q, T, vp, dict(overlap=overlap, n_outliers=0)


def seed_of(config: int, pair: int) -> int:
    return 1000 + 100 * int(config) + int(pair)


def make_pair(config: int = 0, pair: int = 0, seed: int | None = None, n_p: int | None = None,
              n_q: int | None = None, overlap: float | None = None, sigma: float | None = None,
              outliers: float | None = None, kind: str | None = None) -> FragmentPair:
    """One seeded fragment pair of the given configuration (fields can be overridden)."""
    cfg = dict(CONFIGS[int(config)])
    seed = seed_of(config, pair) if seed is None else int(seed)
    rng = np.random.default_rng(seed)
    if "n_range" in cfg:
        lo, hi = cfg["n_range"]
        cfg["n_p"] = int(rng.integers(lo, hi + 1))
        cfg["n_q"] = int(rng.integers(lo, hi + 1))
        cfg["overlap"] = float(rng.uniform(*cfg["overlap_range"]))
    n_p = cfg["n_p"] if n_p is None else int(n_p)
    n_q = cfg["n_q"] if n_q is None else int(n_q)
    overlap = cfg["overlap"] if overlap is None else float(overlap)
    sigma = cfg["sigma"] if sigma is None else float(sigma)
    outliers = cfg.get("outliers", 0.0) if outliers is None else float(outliers)
    kind = cfg["kind"] if kind is None else kind
    if kind == "objects":
        P, Q, T, vp, meta = _objects_pair(rng, n_p, n_q, sigma, overlap, outliers)
    else:
        P, Q, T, vp, meta = _room_pair(rng, n_p, n_q, sigma, overlap)
    meta.update(config=int(config), pair=int(pair), kind=kind, sigma=sigma)
    return FragmentPair(P=np.ascontiguousarray(P, np.float32), Q=np.ascontiguousarray(Q, np.float32), T=T,
                        vpP=vp.astype(np.float64), vpQ=_apply(T, vp[None])[0], seed=seed, meta=meta)


def make_batch(config: int, n_pairs: int | None = None, first: int = 0, **kw) -> list[FragmentPair]:
    n = CONFIGS[int(config)]["n_pairs"] if n_pairs is None else int(n_pairs)
    return [make_pair(config, first + i, **kw) for i in range(n)]
