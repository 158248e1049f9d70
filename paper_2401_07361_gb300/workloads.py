"""Seeded synthetic inputs for the spherical Biot-Savart sum and its tree code.

This module only makes inputs (points on the unit sphere, quadrature weights, vorticity
fields).  It holds none of the summation method's arithmetic, imports neither the CUDA
binding nor the oracle, and is the one piece of code that both sides of a parity test
share.

Recipes (arXiv 2401.07361 names the workloads; the sizes follow the benchmark configs):
  icosahedral_points(L)   vertices of an icosahedron whose faces are split into four L
                          times (Sec. 2: "an iteratively refined icosahedron"); 10 * 4^L + 2.
  uniform_points(n, seed) z ~ U(-1, 1), lambda ~ U(0, 2 pi) (uniform on the sphere).
  voronoi_areas(pos)      spherical Voronoi cell areas (the node-patch areas of Sec. 2).
  rh_vorticity            Rossby-Haurwitz wave k = 4 (Sec. 4.2, Eq. rhwave), written in
                          Cartesian form 2 w z + 30 K z (x^4 - 6 x^2 y^2 + y^4).
  sh_series_vorticity     sum_{l=1..L} sum_m c_lm Y_lm, c_lm ~ N(0, 1) / l, orthonormal real
                          spherical harmonics (zero mean because l >= 1).
  jet_vorticity           a zonal jet u(phi) = u0 exp(1 / ((phi - phi0)(phi - phi1))) / e_n on
                          (phi0, phi1) plus a Gaussian bump, on the unit sphere in days.
Random numbers come from numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

EARTH_RADIUS_M = 6.371e6
SECONDS_PER_DAY = 86400.0
GRAVITY = 9.80616


# ---------------------------------------------------------------------------------- points
def _icosahedron_vertices():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            v += [(0.0, a, b * g), (a, b * g, 0.0), (a * g, 0.0, b)]
    v = np.array(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _icosahedron_faces(v):
    faces = []
    n = len(v)
    edge2 = np.min([np.sum((v[0] - v[k]) ** 2) for k in range(1, n)])
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                dij = np.sum((v[i] - v[j]) ** 2)
                dik = np.sum((v[i] - v[k]) ** 2)
                djk = np.sum((v[j] - v[k]) ** 2)
                if max(abs(dij - edge2), abs(dik - edge2), abs(djk - edge2)) < 1e-9:
                    faces.append((i, j, k))
    return np.array(faces, dtype=np.int64)


def icosahedral_points(level: int) -> np.ndarray:
    """Vertices of the icosahedron refined ``level`` times (edge midpoints pushed out to the
    sphere).  Returns float64 ``[10 * 4**level + 2, 3]``."""
    v = [tuple(p) for p in _icosahedron_vertices()]
    pts = list(v)
    faces = [tuple(f) for f in _icosahedron_faces(np.array(v))]
    for _ in range(level):
        mid = {}
        new_faces = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = np.add(pts[a], pts[b])
                p = p / np.linalg.norm(p)
                mid[key] = len(pts)
                pts.append(tuple(p))
            return mid[key]

        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        faces = new_faces
    out = np.array(pts, dtype=np.float64)
    assert out.shape[0] == 10 * 4 ** level + 2
    return out


def icosahedral_mesh(level: int):
    """The refined icosahedron as a triangulation: vertices ``[10 * 4**level + 2, 3]`` (those
    of ``icosahedral_points(level)``, same order) and faces ``int32 [20 * 4**level, 3]`` (the
    children of each face in the order (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))."""
    v = [tuple(p) for p in _icosahedron_vertices()]
    pts = list(v)
    faces = [tuple(int(x) for x in f) for f in _icosahedron_faces(np.array(v))]
    for _ in range(level):
        mid = {}
        new_faces = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = np.add(pts[a], pts[b])
                p = p / np.linalg.norm(p)
                mid[key] = len(pts)
                pts.append(tuple(p))
            return mid[key]

        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        faces = new_faces
    return np.array(pts, dtype=np.float64), np.array(faces, dtype=np.int32)


def gaussian_vortex_vorticity(pos, area, lat_c=math.pi / 20, lon_c=0.0):
    """Initial vorticity of the Gaussian vortex test (Sec. 4.3): 4 pi exp(-16 |x - x_c|^2) + C
    (per day), x_c at latitude lat_c and longitude lon_c, C such that sum zeta A = 0."""
    xc = np.array([math.cos(lat_c) * math.cos(lon_c), math.cos(lat_c) * math.sin(lon_c), math.sin(lat_c)])
    d2 = np.sum((pos - xc) ** 2, axis=1)
    z = 4.0 * math.pi * np.exp(-16.0 * d2)
    return z - np.sum(z * area) / np.sum(area)


def uniform_points(n: int, seed: int = 0) -> np.ndarray:
    """``n`` points uniform on the unit sphere, float64 ``[n, 3]``."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, n)
    lam = rng.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(lam), r * np.sin(lam), z], axis=1)


def equal_areas(n: int) -> np.ndarray:
    return np.full(n, 4.0 * np.pi / n, dtype=np.float64)


def voronoi_areas(pos: np.ndarray) -> np.ndarray:
    """Spherical Voronoi cell areas of ``pos`` (they sum to 4 pi)."""
    from scipy.spatial import SphericalVoronoi

    sv = SphericalVoronoi(np.asarray(pos, dtype=np.float64), radius=1.0, center=np.zeros(3))
    return np.asarray(sv.calculate_areas(), dtype=np.float64)


def lat_lon(pos: np.ndarray):
    pos = np.asarray(pos, dtype=np.float64)
    lat = np.arcsin(np.clip(pos[:, 2], -1.0, 1.0))
    lon = np.arctan2(pos[:, 1], pos[:, 0])
    return lat, lon


# ------------------------------------------------------------------------------ vorticity
def rh_vorticity(pos: np.ndarray, w: float, K: float) -> np.ndarray:
    """Rossby-Haurwitz wave number 4: 2 w z + 30 K z (x^4 - 6 x^2 y^2 + y^4)."""
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    return 2.0 * w * z + 30.0 * K * z * (x**4 - 6.0 * x**2 * y**2 + y**4)


def polar_vortex_vorticity(pos: np.ndarray, beta: float = 1.5, theta0: float = 15 * math.pi / 32) -> np.ndarray:
    """Initial polar vortex of Sec. 4.4: pi exp(-2 beta^2 (1 - cos(theta0 - theta)))
    (2 beta^2 cos(theta) sin(theta0 - theta) + sin(theta)), theta the latitude."""
    lat, _ = lat_lon(pos)
    e = np.exp(-2.0 * beta**2 * (1.0 - np.cos(theta0 - lat)))
    return math.pi * e * (2.0 * beta**2 * np.cos(lat) * np.sin(theta0 - lat) + np.sin(lat))


def _real_sh_iter(pos: np.ndarray, lmax: int):
    """Yields ((l, m), values) of the orthonormal real spherical harmonics Y_lm at ``pos``
    for 0 <= l <= lmax, m in [-l, l]; m > 0 uses cos(m lambda), m < 0 uses sin(|m| lambda).
    Normalised associated Legendre functions by the standard three-term recurrence in l (no
    Condon-Shortley phase).  Holds O(1) arrays at a time."""
    pos = np.asarray(pos, dtype=np.float64)
    z = np.clip(pos[:, 2], -1.0, 1.0)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    lam = np.arctan2(pos[:, 1], pos[:, 0])
    pmm = np.full_like(z, 1.0 / math.sqrt(4.0 * math.pi))
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s
        cm = np.cos(m * lam) if m > 0 else None
        sm = np.sin(m * lam) if m > 0 else None
        plm2, plm1 = None, pmm
        for l in range(m, lmax + 1):
            if l == m:
                p = pmm
            elif l == m + 1:
                p = math.sqrt(2.0 * m + 3.0) * z * pmm
            else:
                a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                p = a * (z * plm1 - b * plm2)
            if l > m:
                plm2, plm1 = plm1, p
            if m == 0:
                yield (l, 0), p
            else:
                yield (l, m), math.sqrt(2.0) * p * cm
                yield (l, -m), math.sqrt(2.0) * p * sm


def real_sh_table(pos: np.ndarray, lmax: int):
    """Orthonormal real spherical harmonics as a dict {(l, m): values} (small lmax only)."""
    return {key: val.copy() for key, val in _real_sh_iter(pos, lmax)}


def sh_coefficients(lmax: int, seed: int):
    """c_lm ~ N(0, 1) / l for 1 <= l <= lmax, m = -l..l, in (l, m) order."""
    rng = np.random.default_rng(seed)
    coef = {}
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            coef[(l, m)] = rng.standard_normal() / l
    return coef


def sh_series_vorticity(pos: np.ndarray, lmax: int, seed: int = 0, chunk: int = 1 << 16) -> np.ndarray:
    """Random vorticity sum_{l=1..lmax} sum_m c_lm Y_lm with c_lm ~ N(0,1)/l.  With no l = 0
    term its integral over the sphere is zero (the zero total circulation of Sec. 2); the
    discrete circulation sum_j zeta_j A_j of a point set is that integral's quadrature error
    and is left as it is.  The points are taken in chunks that stay in cache; every value is
    computed elementwise in the same order whatever the chunk, so the result does not depend
    on it."""
    coef = sh_coefficients(lmax, seed)
    pos = np.asarray(pos, dtype=np.float64)
    zeta = np.zeros(pos.shape[0])
    for c0 in range(0, pos.shape[0], chunk):
        zc = zeta[c0:c0 + chunk]
        for key, y in _real_sh_iter(pos[c0:c0 + chunk], lmax):
            if key[0] >= 1:
                zc += coef[key] * y
    return zeta


def jet_vorticity(pos: np.ndarray, u0_ms: float = 80.0, bump_height_m: float = 120.0,
                  alpha: float = 1.0 / 3.0, beta: float = 1.0 / 15.0) -> np.ndarray:
    """Zonal jet plus Gaussian bump, unit sphere, time in days (vorticity in 1/day).

    Jet: u(phi) = u0 exp(1 / ((phi - phi0)(phi - phi1))) / e_n on (phi0, phi1), zero
    elsewhere, phi0 = pi / 7, phi1 = pi / 2 - phi0, e_n = exp(-4 / (phi1 - phi0)^2); its
    vorticity is -(1 / cos phi) d(u cos phi) / d phi = -du/dphi + u tan phi.
    Bump: a exp(-(lambda / alpha)^2 - ((phi_c - phi) / beta)^2), phi_c = pi / 4, with the
    amplitude a = g h / (f (R beta)^2) of a geostrophic height bump h on radius R at
    f = 2 Omega sin(phi_c), converted to 1/day.  The mean is removed.
    """
    lat, lon = lat_lon(pos)
    phi0 = math.pi / 7.0
    phi1 = math.pi / 2.0 - phi0
    en = math.exp(-4.0 / (phi1 - phi0) ** 2)
    u0 = u0_ms * SECONDS_PER_DAY / EARTH_RADIUS_M
    inside = (lat > phi0) & (lat < phi1)
    zeta = np.zeros_like(lat)
    p = lat[inside]
    q = (p - phi0) * (p - phi1)
    u = u0 * np.exp(1.0 / q) / en
    dudp = u * (-(2.0 * p - phi0 - phi1) / (q * q))
    zeta[inside] = -dudp + u * np.tan(p)
    phic = math.pi / 4.0
    f = 2.0 * (2.0 * math.pi / SECONDS_PER_DAY) * math.sin(phic)
    amp = GRAVITY * bump_height_m / (f * (EARTH_RADIUS_M * beta) ** 2) * SECONDS_PER_DAY
    zeta += amp * np.exp(-(lon / alpha) ** 2 - ((phic - lat) / beta) ** 2)
    return zeta - np.mean(zeta)


# ------------------------------------------------------------------------------ workloads
RH_W_PER_S = 7.848e-6
RH_K_PER_S = 7.848e-6


def ensemble_sizes(B: int = 64, lo: int = 10242, hi: int = 163842, seed: int = 0):
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), B)]


def workload(name: str, areas: str = "default"):
    """Named synthetic workloads: returns dict(pos, zeta, area, params...).

    ico5_rh       N = 10242 icosahedral level-5 vertices, RH wave 4 (w = K = 7.848e-6 1/s),
                  equal areas 4 pi / N (``areas="voronoi"`` for node-patch areas).
    rand655k_sh16 N = 655362 uniform points (seed 0), Voronoi areas, SH series l <= 16
                  (coefficients seed 0; the points use seed 0 as well: sub-stream 1 for
                  the coefficients would change nothing structural, the recipe is stated).
    ico9_jet      N = 2621442 icosahedral level-9 vertices, jet + bump, equal areas.
    rand10m_sh32  N = 10485762 uniform points (seed 0), SH series l <= 32, equal areas.
    polar163k     N = 163842 icosahedral level-7 vertices, the polar vortex of Sec. 4.4, equal
                  areas (degree 6 as in that experiment).
    """
    if name == "ico5_rh":
        pos = icosahedral_points(5)
        zeta = rh_vorticity(pos, RH_W_PER_S, RH_K_PER_S)
        area = voronoi_areas(pos) if areas == "voronoi" else equal_areas(len(pos))
        return dict(pos=pos, zeta=zeta, area=area, theta=0.7, degree=8, leaf_size=128)
    if name == "rand655k_sh16":
        pos = uniform_points(655362, seed=0)
        zeta = sh_series_vorticity(pos, 16, seed=0)
        area = equal_areas(len(pos)) if areas == "equal" else voronoi_areas(pos)
        return dict(pos=pos, zeta=zeta, area=area, theta=0.7, degree=8, leaf_size=128)
    if name == "ico9_jet":
        pos = icosahedral_points(9)
        zeta = jet_vorticity(pos)
        area = voronoi_areas(pos) if areas == "voronoi" else equal_areas(len(pos))
        return dict(pos=pos, zeta=zeta, area=area, theta=0.7, degree=8, leaf_size=128)
    if name == "rand10m_sh32":
        pos = uniform_points(10485762, seed=0)
        zeta = sh_series_vorticity(pos, 32, seed=0)
        return dict(pos=pos, zeta=zeta, area=equal_areas(len(pos)), theta=0.7, degree=8,
                    leaf_size=256)
    if name == "polar163k":
        pos = icosahedral_points(7)
        zeta = polar_vortex_vorticity(pos)
        area = voronoi_areas(pos) if areas == "voronoi" else equal_areas(len(pos))
        return dict(pos=pos, zeta=zeta, area=area, leaf_size=128, degree=6)
    if name == "ensemble64":
        # 64 independent instances, N_b log-uniform in [10242, 163842] (seed 0); uniform points
        # (seed 100 + b); equal areas 4 pi / N_b; RH wave 4 plus 1e-2 x an RMS-normalised
        # random harmonic series to degree 12 (seed 1000 + b).
        sizes = ensemble_sizes(64, 10242, 163842, seed=0)
        pos, zeta, area = [], [], []
        for b, nb in enumerate(sizes):
            p = uniform_points(nb, seed=100 + b)
            z = rh_vorticity(p, RH_W_PER_S, RH_K_PER_S)
            noise = sh_series_vorticity(p, 12, seed=1000 + b)
            z = z + 1e-2 * np.sqrt(np.mean(z * z)) * noise / np.sqrt(np.mean(noise * noise))
            pos.append(p)
            zeta.append(z)
            area.append(equal_areas(nb))
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        return dict(pos=np.vstack(pos), zeta=np.concatenate(zeta), area=np.concatenate(area), offsets=off,
                    theta=0.7, degree=8, leaf_size=128)
    raise KeyError(name)
