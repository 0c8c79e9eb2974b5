"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds geometry only: point sets on closed curves or surfaces,
their quadrature-weighted tangents (2D) or outward normals (3D), and loss
weights.  It holds none of the method's arithmetic (no snapping, no kernels,
no sums) and is the one module both the CUDA path's tests/bench and the oracle
take their inputs from.

Workloads (the paper's datasets -- Siddiqi silhouettes, Stanford Dragon -- are
not available, so seeded synthetic shapes of the same kind stand in):

* ``circle``   -- K points evenly spaced on a circle, counter-clockwise,
                  with chord tangents Z_k = Y_{k+1} - Y_k (eq. tangentVec).
* ``stars``    -- several non-intersecting star-shaped polygons sampled
                  evenly by arc length (stand-in for the 2D silhouettes of
                  Sec. 6 Example 3).
* ``torus_sphere`` -- area-uniform samples on a torus plus a concentric
                  sphere, with outward normals times area per sample (stand-in
                  for the 3D point clouds of Sec. 6 Examples 4-5).
* ``jittered_sphere`` -- points on a sphere with isotropic Gaussian jitter
                  (the differentiation workload; no normals).
* ``batch_stars`` -- many independent shapes of uneven grid size and point
                  count.

Every generator takes an explicit seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Shape:
    """One problem instance: a grid (dims, h), tau, points and weights."""
    D: int
    dims: tuple
    h: float
    tau: float
    points: np.ndarray            # K x D world coordinates, float64
    weights: np.ndarray | None    # K x D tangents (2D) / normals (3D), or None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.points.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.dims))


def _closed_chords(P):
    """Z_k = P_{k+1} - P_k with P_{K+1} = P_1 (eq. tangentVec)."""
    return np.roll(P, -1, axis=0) - P


def circle(N=128, K=256, radius=0.3, center=(0.5, 0.5), tau=0.005):
    """K points at angles 2*pi*k/K on a circle (CCW), chord tangents."""
    h = 1.0 / N
    t = 2.0 * np.pi * np.arange(K) / K
    P = np.stack([center[0] + radius * np.cos(t), center[1] + radius * np.sin(t)], 1)
    return Shape(2, (N, N), h, tau, P, _closed_chords(P), name="circle",
                 meta=dict(radius=radius, center=center))


def _star_vertices(rng, nv_lo, nv_hi, r_lo, r_hi):
    nv = int(rng.integers(nv_lo, nv_hi + 1))
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, nv))
    rad = rng.uniform(r_lo, r_hi, nv)
    return ang, rad


def _sample_polygon(V, n):
    """n points evenly spaced by arc length along the closed polygon V (CCW)."""
    E = np.roll(V, -1, axis=0) - V
    L = np.sqrt((E ** 2).sum(1))
    cum = np.concatenate([[0.0], np.cumsum(L)])
    s = np.arange(n) * (cum[-1] / n)
    seg = np.searchsorted(cum, s, side="right") - 1
    seg = np.clip(seg, 0, len(V) - 1)
    u = (s - cum[seg]) / L[seg]
    return V[seg] + u[:, None] * E[seg]


def stars(N=2048, K=40000, n_shapes=8, tau=0.002, seed=2, r_lo=0.03, r_hi=0.15,
          nv_lo=5, nv_hi=12, box=(0.05, 0.95), gap=0.02, center=None):
    """Seeded non-intersecting star-shaped polygons, CCW, sampled by arc length.

    Centres are drawn by rejection so that circumscribed discs (radius r_hi)
    plus ``gap`` do not overlap and stay inside ``box``.  K is split among the
    polygons in proportion to perimeter.  Tangents are chords of consecutive
    samples along each polygon.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    polys, centres, radii = [], [], []
    tries = 0
    while len(polys) < n_shapes:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place star polygons")
        ang, rad = _star_vertices(rng, nv_lo, nv_hi, r_lo, r_hi)
        rmax = float(rad.max())
        if center is not None and n_shapes == 1:
            c = np.asarray(center, float)
        else:
            c = rng.uniform(box[0] + rmax, box[1] - rmax, 2)
            if any(np.hypot(*(c - q)) < rmax + rq + gap for q, rq in zip(centres, radii)):
                continue
        centres.append(c)
        radii.append(rmax)
        polys.append(c + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1))
    per = np.array([np.sqrt(((np.roll(V, -1, 0) - V) ** 2).sum(1)).sum() for V in polys])
    ks = np.floor(K * per / per.sum()).astype(int)
    ks[np.argsort(-(K * per / per.sum() - ks))[: K - ks.sum()]] += 1
    P, Z = [], []
    for V, k in zip(polys, ks):
        S = _sample_polygon(V, int(k))
        P.append(S)
        Z.append(_closed_chords(S))
    return Shape(2, (N, N), h, tau, np.concatenate(P), np.concatenate(Z),
                 name="stars", meta=dict(polygons=polys, counts=ks, seed=seed))


def _sphere_dirs(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def torus_sphere(N=256, K=200000, tau=0.004, seed=3, R=0.25, r=0.1, rs=0.12,
                 center=(0.5, 0.5, 0.5)):
    """Area-uniform samples on a torus (axis z) and a concentric sphere.

    Weights are outward unit normals times (surface area / samples on that
    surface), i.e. n dA quadrature weights for the normal flux of eq. normflux.
    """
    rng = np.random.default_rng(seed)
    c = np.asarray(center, float)
    A_t = 4.0 * np.pi ** 2 * R * r
    A_s = 4.0 * np.pi * rs ** 2
    k_t = int(round(K * A_t / (A_t + A_s)))
    k_s = K - k_t
    # torus: azimuth uniform, tube angle with density proportional to R + r cos(theta)
    th = np.empty(0)
    while th.shape[0] < k_t:
        cand = rng.uniform(0.0, 2.0 * np.pi, 2 * k_t)
        acc = rng.uniform(0.0, R + r, 2 * k_t) < (R + r * np.cos(cand))
        th = np.concatenate([th, cand[acc]])
    th = th[:k_t]
    ph = rng.uniform(0.0, 2.0 * np.pi, k_t)
    Pt = np.stack([(R + r * np.cos(th)) * np.cos(ph), (R + r * np.cos(th)) * np.sin(ph),
                   r * np.sin(th)], 1)
    Nt = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), np.sin(th)], 1)
    ds = _sphere_dirs(rng, k_s)
    P = np.concatenate([Pt + c, rs * ds + c])
    W = np.concatenate([Nt * (A_t / k_t), ds * (A_s / k_s)])
    return Shape(3, (N, N, N), 1.0 / N, tau, P, W, name="torus_sphere",
                 meta=dict(R=R, r=r, rs=rs, center=center, k_torus=k_t, k_sphere=k_s))


def sphere(N=64, K=4000, radius=0.3, center=(0.5, 0.5, 0.5), tau=0.02, seed=7):
    """Area-uniform samples on one sphere with n dA weights."""
    rng = np.random.default_rng(seed)
    d = _sphere_dirs(rng, K)
    P = np.asarray(center, float) + radius * d
    W = d * (4.0 * np.pi * radius ** 2 / K)
    return Shape(3, (N, N, N), 1.0 / N, tau, P, W, name="sphere",
                 meta=dict(radius=radius, center=center))


def jittered_sphere(N=128, K=20000, radius=0.3, sigma=0.01, tau=0.01, seed=5,
                    center=(0.5, 0.5, 0.5)):
    """Points on a sphere plus isotropic N(0, sigma^2) jitter; no normals."""
    rng = np.random.default_rng(seed)
    d = _sphere_dirs(rng, K)
    P = np.asarray(center, float) + radius * d + rng.normal(scale=sigma, size=(K, 3))
    return Shape(3, (N, N, N), 1.0 / N, tau, P, None, name="jittered_sphere",
                 meta=dict(radius=radius, sigma=sigma))


def loss_weights(n_nodes, seed=50):
    """w(X) ~ N(0, 1) per grid node (float64)."""
    return np.random.default_rng(seed).normal(size=n_nodes)


def batch_stars(n=96, seed=4, sides=(256, 384, 512, 768, 1024), k_lo=500, k_hi=20000):
    """Independent shapes: side N uniform over ``sides``, h = 1/N, tau = 2h,
    one star polygon centred at (0.5, 0.5) with radii U[0.15, 0.40] and
    5-12 vertices, K uniform in [k_lo, k_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.choice(sides))
        K = int(rng.integers(k_lo, k_hi + 1))
        s = stars(N=N, K=K, n_shapes=1, tau=2.0 / N, seed=int(rng.integers(1 << 31)),
                  r_lo=0.15, r_hi=0.40, center=(0.5, 0.5))
        s.name = "batch%d" % i
        out.append(s)
    return out


def random_points(D, N, K, tau, seed=11, lo=0.1, hi=0.9, weights=False):
    """K uniform random points in [lo, hi]^D on an N^D grid (h = 1/N)."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(lo, hi, size=(K, D))
    W = rng.normal(size=(K, D)) * (1.0 / N) if weights else None
    return Shape(D, (N,) * D, 1.0 / N, tau, P, W, name="random%dd" % D)


# Named workloads with the sizes the paper-derived configurations use.
def config_c1():
    """2D FP64 slice: 128^2 grid, K=256 points on a circle, tau=0.005."""
    return circle(N=128, K=256, radius=0.3, center=(0.5, 0.5), tau=0.005)


def config_c2(tau=0.002):
    """2D mixed precision: 2048^2 grid, K=40000 on 8 star polygons."""
    return stars(N=2048, K=40000, n_shapes=8, tau=tau, seed=2)


def config_c3():
    """3D mixed precision: 256^3 grid, K=200000 on a torus plus a sphere."""
    return torus_sphere(N=256, K=200000, tau=0.004, seed=3)


def config_c5():
    """3D differentiation: 128^3 grid, K=20000 jittered sphere points."""
    return jittered_sphere(N=128, K=20000, radius=0.3, sigma=0.01, tau=0.01, seed=5)


# ---------------------------------------------------------------- triangle meshes
# Closed, outward-wound (counter-clockwise seen from outside) triangle meshes of
# the Example 5 objects: a sphere, a cube and a capped cylinder.  Geometry only:
# the sources (incentres, normals) are the method's job.

def mesh_sphere(center=(0.5, 0.5, 0.5), r=0.3, n_lat=24, n_lon=48):
    """UV sphere: (V, F) with F int64 vertex indices."""
    c = np.asarray(center, float)
    V = [c + [0, 0, r], c - [0, 0, r]]
    for i in range(1, n_lat):
        th = np.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * np.pi * j / n_lon
            V.append(c + r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]))
    V = np.array(V)

    def ring(i, j):  # vertex of latitude ring i (1 .. n_lat-1), longitude j
        return 2 + (i - 1) * n_lon + (j % n_lon)

    F = []
    for j in range(n_lon):
        F.append([0, ring(1, j), ring(1, j + 1)])
        F.append([1, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)])
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b, cc, d = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            F.append([a, cc, d])
            F.append([a, d, b])
    return V, np.array(F, dtype=np.int64)


def mesh_cube(center=(0.5, 0.5, 0.5), half=0.25, n=8):
    """Cube with each face cut into n x n squares of two triangles."""
    c = np.asarray(center, float)
    V, F = [], []
    for axis in range(3):
        for s in (-1.0, 1.0):
            u, v = [a for a in range(3) if a != axis]
            base = len(V)
            for i in range(n + 1):
                for j in range(n + 1):
                    p = np.zeros(3)
                    p[axis] = s * half
                    p[u] = -half + 2 * half * i / n
                    p[v] = -half + 2 * half * j / n
                    V.append(c + p)
            for i in range(n):
                for j in range(n):
                    a = base + i * (n + 1) + j
                    b, cc, d = a + (n + 1), a + 1, a + (n + 1) + 1
                    # (u, v, axis) right-handed when (axis+1)%3 == u; flip for the -s face
                    tri = [[a, b, d], [a, d, cc]]
                    right = (axis + 1) % 3 == u
                    if (s > 0) != right:
                        tri = [[a, d, b], [a, cc, d]]
                    F.extend(tri)
    return np.array(V), np.array(F, dtype=np.int64)


def mesh_cylinder(center=(0.5, 0.5, 0.5), r=0.2, half_height=0.25, n_theta=48, n_z=12):
    """Capped cylinder along z: side quads and triangle-fan caps."""
    c = np.asarray(center, float)
    V, F = [], []
    for k in range(n_z + 1):
        z = -half_height + 2 * half_height * k / n_z
        for j in range(n_theta):
            t = 2 * np.pi * j / n_theta
            V.append(c + [r * np.cos(t), r * np.sin(t), z])
    for k in range(n_z):
        for j in range(n_theta):
            a = k * n_theta + j
            b = k * n_theta + (j + 1) % n_theta
            cc, d = a + n_theta, b + n_theta
            F.append([a, b, d])
            F.append([a, d, cc])
    bot, top = len(V), len(V) + 1
    V.append(c + [0, 0, -half_height])
    V.append(c + [0, 0, half_height])
    for j in range(n_theta):
        F.append([bot, (j + 1) % n_theta, j])
        F.append([top, n_z * n_theta + j, n_z * n_theta + (j + 1) % n_theta])
    return np.array(V), np.array(F, dtype=np.int64)
