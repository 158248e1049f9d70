"""Python face of the plain FP64 CPU oracle (``sts_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs
of ``bench.py`` use it; the CUDA library never does, and this module never imports the
library.  Arrays are numpy float64 / int64, positions row-major ``[n, 3]``.

What each function follows in arXiv 2401.07361:
  direct           the midpoint-rule particle system of Sec. 2 with Eq. altkernel.
  Tree             the refined-icosahedron tree and target-leaf traversal of Sec. 3.
  Tree.velocity    PC (proxy-point form, or the literal alpha-solve) + PP, Sec. 3.3.
  rk4_step         the classical RK4 of Sec. 4 applied to the Sec. 2 system
                   dx_i/dt = u_i, dzeta_i/dt = -2 Omega dz_i/dt.
  rel_l2           the relative l2 error E of Sec. 4.1 (area weighted).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sts_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11"]


def build(force: bool = False) -> str:
    """Compiles ``liboracle.so`` next to its source (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            lib.or_direct.argtypes = [i64, P, P, P, i64, P, P, i32]
            lib.or_tree_build.restype = P
            lib.or_tree_build.argtypes = [i64, P, i32, i32]
            lib.or_tree_free.argtypes = [P]
            lib.or_tree_info.argtypes = [P, P]
            lib.or_tree_export.argtypes = [P] + [P] * 11
            lib.or_tree_lists.argtypes = [P, dbl]
            lib.or_lists_export.argtypes = [P, P, P, P, P]
            lib.or_tree_velocity.argtypes = [P, P, P, dbl, i32, i32, P, P, i32]
            lib.or_tree_clusters.argtypes = [P, P, P, i32, P, P, P, P]
            lib.or_proxy_reference.argtypes = [i32, P, P]
            lib.or_vref_inverse.argtypes = [i32, P]
            lib.or_cluster.argtypes = [P, i32, i64, P, P, P, P, P]
            lib.or_pc_pair.argtypes = [P, i32, i64, P, P, P, P, P]
            lib.or_direct_potential.argtypes = [i64, P, P, P, i64, P, P, i32]
            lib.or_tree_potential.argtypes = [P, P, P, dbl, i32, i32, P, P, i32]
            lib.or_pc_pair_potential.argtypes = [P, i32, i64, P, P, P, P, P]
            lib.or_dual_lists.argtypes = [P, dbl, P]
            lib.or_dual_export.argtypes = [P, i32, P, P]
            lib.or_tree_velocity_dual.argtypes = [P, P, P, dbl, i32, P, P, i32]
            lib.or_icosahedron.argtypes = [P, P]
            lib.or_amr_create.argtypes = [P, i64, i64, i32, C.POINTER(P)]
            lib.or_amr_free.argtypes = [P]
            lib.or_amr_set.argtypes = [P, P, P]
            lib.or_amr_step.argtypes = [P, dbl, dbl, P]
            lib.or_amr_info.argtypes = [P, P]
            lib.or_amr_export.argtypes = [P] + [P] * 10
            lib.or_amr_update.argtypes = [P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def nbasis(d: int) -> int:
    return (d + 1) * (d + 2) // 2


def direct(pos, zeta, area, targets=None, nthreads: int = 0):
    """Direct sum u_i = -(1/4pi) sum_{j != i} (x_i x x_j) zeta_j A_j / (|x_i - x_j|^2 / 2).

    ``targets``: optional original indices; the result then has one row per target.
    """
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    zeta = _f64(zeta, (n,))
    area = _f64(area, (n,))
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    vel = np.zeros((nt, 3))
    _check(_L().or_direct(n, _p(pos), _p(zeta), _p(area), nt, _p(tg), _p(vel), nthreads), "direct")
    return vel


def direct_potential(pos, zeta, area, targets=None, nthreads: int = 0):
    """Direct sum of the stream function psi_i = -(1/4pi) sum_{j != i} log(|x_i - x_j|^2 / 2)
    zeta_j A_j (the Green's function of Sec. 2 as the kernel).  ``targets`` as for direct."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    zeta = _f64(zeta, (n,))
    area = _f64(area, (n,))
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    psi = np.zeros(nt)
    _check(_L().or_direct_potential(n, _p(pos), _p(zeta), _p(area), nt, _p(tg), _p(psi), nthreads),
           "direct potential")
    return psi


class Tree:
    """The icosahedral triangle tree of Sec. 3 over ``pos``."""

    def __init__(self, pos, leaf_size: int = 128, max_level: int = 16):
        self.pos = _f64(pos, (-1, 3))
        self.leaf_size = leaf_size
        self.max_level = max_level
        h = _L().or_tree_build(self.pos.shape[0], _p(self.pos), leaf_size, max_level)
        if not h:
            raise RuntimeError("oracle tree build failed (bad arguments or out of memory)")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_tree_free(h)
            self._h = None

    def info(self):
        a = np.zeros(8, dtype=np.int64)
        _check(_L().or_tree_info(self._h, _p(a)), "info")
        return dict(n=int(a[0]), nodes=int(a[1]), leaves=int(a[2]), depth=int(a[3]),
                    nfar=int(a[4]), nnear=int(a[5]))

    def export(self):
        inf = self.info()
        n, nn, nl = inf["n"], inf["nodes"], inf["leaves"]
        out = dict(
            perm=np.zeros(n, np.int64), level=np.zeros(nn, np.int32), key=np.zeros(nn, np.uint64),
            parent=np.zeros(nn, np.int32), first_child=np.zeros(nn, np.int32),
            nchild=np.zeros(nn, np.int32), start=np.zeros(nn, np.int64), count=np.zeros(nn, np.int64),
            leaf=np.zeros(nn, np.int32), leaves=np.zeros(nl, np.int32), geom=np.zeros((nn, 13)),
        )
        _check(_L().or_tree_export(self._h, *[_p(out[k]) for k in (
            "perm", "level", "key", "parent", "first_child", "nchild", "start", "count", "leaf",
            "leaves", "geom")]), "export")
        return out

    def lists(self, theta: float):
        _check(_L().or_tree_lists(self._h, float(theta)), "lists")
        inf = self.info()
        nl = inf["leaves"]
        out = dict(far_off=np.zeros(nl + 1, np.int64), far_idx=np.zeros(inf["nfar"], np.int32),
                   near_off=np.zeros(nl + 1, np.int64), near_idx=np.zeros(inf["nnear"], np.int32))
        _check(_L().or_lists_export(self._h, _p(out["far_off"]), _p(out["far_idx"]),
                                    _p(out["near_off"]), _p(out["near_idx"])), "lists export")
        return out

    def velocity(self, zeta, area, theta: float = 0.7, degree: int = 8, literal: bool = False,
                 nthreads: int = 0, return_stats: bool = False):
        n = self.pos.shape[0]
        zeta = _f64(zeta, (n,))
        area = _f64(area, (n,))
        vel = np.zeros((n, 3))
        st = np.zeros(2, np.int64)
        _check(_L().or_tree_velocity(self._h, _p(zeta), _p(area), float(theta), int(degree),
                                     int(bool(literal)), _p(vel), _p(st), nthreads), "tree velocity")
        if return_stats:
            return vel, dict(pc=int(st[0]), pp=int(st[1]))
        return vel

    def potential(self, zeta, area, theta: float = 0.7, degree: int = 8, literal: bool = False,
                  nthreads: int = 0, return_stats: bool = False):
        """Tree-code stream function (same lists and proxies as ``velocity``)."""
        n = self.pos.shape[0]
        zeta = _f64(zeta, (n,))
        area = _f64(area, (n,))
        psi = np.zeros(n)
        st = np.zeros(2, np.int64)
        _check(_L().or_tree_potential(self._h, _p(zeta), _p(area), float(theta), int(degree),
                                      int(bool(literal)), _p(psi), _p(st), nthreads), "tree potential")
        if return_stats:
            return psi, dict(pc=int(st[0]), pp=int(st[1]))
        return psi

    def dual_lists(self, theta: float):
        """Pairs of the dual traversal (Sec. 3.4): {"PP"|"PC"|"CP"|"CC": (target nodes,
        source nodes)} in traversal order."""
        cnt = np.zeros(4, np.int64)
        _check(_L().or_dual_lists(self._h, float(theta), _p(cnt)), "dual lists")
        out = {}
        for k, name in enumerate(("PP", "PC", "CP", "CC")):
            t = np.zeros(int(cnt[k]), np.int32)
            s = np.zeros(int(cnt[k]), np.int32)
            _check(_L().or_dual_export(self._h, k, _p(t), _p(s)), "dual export")
            out[name] = (t, s)
        return out

    def velocity_dual(self, zeta, area, theta: float = 0.7, degree: int = 8, nthreads: int = 0,
                      return_stats: bool = False):
        """Tree-code velocity with all four interactions of the dual traversal."""
        n = self.pos.shape[0]
        zeta = _f64(zeta, (n,))
        area = _f64(area, (n,))
        vel = np.zeros((n, 3))
        st = np.zeros(5, np.int64)
        _check(_L().or_tree_velocity_dual(self._h, _p(zeta), _p(area), float(theta), int(degree), _p(vel),
                                          _p(st), nthreads), "dual velocity")
        if return_stats:
            return vel, dict(pp=int(st[0]), pc=int(st[1]), cp=int(st[2]), cc=int(st[3]), down=int(st[4]))
        return vel

    def clusters(self, zeta, area, degree: int):
        n = self.pos.shape[0]
        zeta = _f64(zeta, (n,))
        area = _f64(area, (n,))
        nc = np.zeros(1, np.int64)
        _check(_L().or_tree_clusters(self._h, _p(zeta), _p(area), degree, _p(nc), None, None, None),
               "clusters")
        M = nbasis(degree)
        c = int(nc[0])
        ids = np.zeros(c, np.int32)
        yt = np.zeros((c, M, 3))
        W = np.zeros((c, M))
        _check(_L().or_tree_clusters(self._h, _p(zeta), _p(area), degree, _p(nc), _p(ids), _p(yt),
                                     _p(W)), "clusters")
        return ids, yt, W


class Amr:
    """Adaptive mesh refinement of Appendix A over a particle triangulation (base faces
    ``faces[t0, 3]`` over ``n0`` base particles, at most ``levels`` levels of splitting)."""

    def __init__(self, faces, n0: int, levels: int = 3):
        faces = np.ascontiguousarray(faces, dtype=np.int32)
        self._h = C.c_void_p()
        _check(_L().or_amr_create(_p(faces), faces.shape[0], int(n0), int(levels), C.byref(self._h)), "amr create")
        info = np.zeros(4, np.int64)
        _check(_L().or_amr_info(self._h, _p(info)), "amr info")
        self.n0, self.nv, self.t0, self.nt = (int(x) for x in info)

    def __del__(self):
        if getattr(self, "_h", None):
            _L().or_amr_free(self._h)
            self._h = None

    def set(self, pos0, zeta0):
        _check(_L().or_amr_set(self._h, _p(_f64(pos0, (self.n0, 3))), _p(_f64(zeta0, (self.n0,)))), "amr set")

    def update(self, pos, zeta):
        """Positions and vorticities of the alive vertices (arrays over all vertices)."""
        _check(_L().or_amr_update(self._h, _p(_f64(pos, (self.nv, 3))), _p(_f64(zeta, (self.nv,)))), "amr update")

    def step(self, eps1: float, eps2: float):
        """One refinement pass; returns (splits, merges, alive vertices, leaf triangles)."""
        c = np.zeros(4, np.int64)
        _check(_L().or_amr_step(self._h, float(eps1), float(eps2), _p(c)), "amr step")
        return tuple(int(x) for x in c)

    def export(self):
        nt, nv = self.nt, self.nv
        o = dict(tv=np.zeros((nt, 3), np.int32), tparent=np.zeros(nt, np.int32), tchild=np.zeros(nt, np.int32),
                 tlevel=np.zeros(nt, np.int8), vparent=np.zeros((nv, 2), np.int32), tstate=np.zeros(nt, np.uint8),
                 valive=np.zeros(nv, np.uint8), pos=np.zeros((nv, 3)), zeta=np.zeros(nv), area=np.zeros(nv))
        _check(_L().or_amr_export(self._h, *(_p(o[k]) for k in ("tv", "tparent", "tchild", "tlevel", "vparent",
                                                                 "tstate", "valive", "pos", "zeta", "area"))),
               "amr export")
        return o


def tree_velocity(pos, zeta, area, theta=0.7, degree=8, leaf_size=128, max_level=16, nthreads=0):
    return Tree(pos, leaf_size, max_level).velocity(zeta, area, theta, degree, nthreads=nthreads)


def proxy_reference(d: int):
    """Approximate Fekete points on the reference simplex: (beta[M,3], candidate index[M])."""
    M = nbasis(d)
    beta = np.zeros((M, 3))
    cand = np.zeros(M, np.int32)
    _check(_L().or_proxy_reference(d, _p(beta), _p(cand)), "proxy reference")
    return beta, cand


def vref_inverse(d: int):
    M = nbasis(d)
    out = np.zeros((M, M))
    _check(_L().or_vref_inverse(d, _p(out)), "vref inverse")
    return out


def cluster(verts, d, ys, ws):
    """Proxy points, weights and SBB moments of one source triangle (verts[3,3])."""
    verts = _f64(verts, (3, 3))
    ys = _f64(ys, (-1, 3))
    ws = _f64(ws, (ys.shape[0],))
    M = nbasis(d)
    yt, W, om = np.zeros((M, 3)), np.zeros(M), np.zeros(M)
    _check(_L().or_cluster(_p(verts), d, ys.shape[0], _p(ys), _p(ws), _p(yt), _p(W), _p(om)),
           "cluster")
    return yt, W, om


def pc_pair(verts, d, ys, ws, x):
    """PC interaction of target x with one triangle: (literal alpha-solve, proxy form)."""
    verts = _f64(verts, (3, 3))
    ys = _f64(ys, (-1, 3))
    ws = _f64(ws, (ys.shape[0],))
    x = _f64(x, (3,))
    lit, prx = np.zeros(3), np.zeros(3)
    _check(_L().or_pc_pair(_p(verts), d, ys.shape[0], _p(ys), _p(ws), _p(x), _p(lit), _p(prx)),
           "pc pair")
    return lit, prx


def pc_pair_potential(verts, d, ys, ws, x):
    """The potential's PC interaction of target x with one triangle: (literal alpha-solve,
    proxy form), both without the -1/4pi."""
    verts = _f64(verts, (3, 3))
    ys = _f64(ys, (-1, 3))
    ws = _f64(ws, (ys.shape[0],))
    x = _f64(x, (3,))
    lit, prx = np.zeros(1), np.zeros(1)
    _check(_L().or_pc_pair_potential(_p(verts), d, ys.shape[0], _p(ys), _p(ws), _p(x), _p(lit), _p(prx)),
           "pc pair potential")
    return float(lit[0]), float(prx[0])


def icosahedron():
    V = np.zeros((12, 3))
    F = np.zeros((20, 3), np.int32)
    _L().or_icosahedron(_p(V), _p(F))
    return V, F


def _project(x):
    return x / np.sqrt(np.sum(x * x, axis=1, keepdims=True))


def forcing_ramp(t, Tp=4.0, Tf=15.0):
    """A(t) of the polar-vortex forcing (Sec. 4.4): a half-cosine ramp up over [0, Tp), 1 until
    Tf - Tp, a half-cosine ramp down until Tf, 0 after (and before 0)."""
    t = float(t)
    if t < 0.0 or t >= Tf:
        return 0.0
    if t < Tp:
        return (1.0 - math.cos(t / Tp * math.pi)) / 2.0
    if t < Tf - Tp:
        return 1.0
    return (1.0 - math.cos(math.pi + (t - Tf + Tp) / Tp * math.pi)) / 2.0


def forcing_profile(pos, theta1=math.pi / 3):
    """B(theta) of the forcing (Sec. 4.4), theta the latitude: with r = tan^2 theta1 / tan^2
    theta, B = r exp(1 - r) in the northern hemisphere, 0 in the southern."""
    pos = _f64(pos, (-1, 3))
    lat = np.arcsin(np.clip(pos[:, 2], -1.0, 1.0))
    out = np.zeros(len(pos))
    north = lat > 0.0
    r = math.tan(theta1) ** 2 / np.tan(lat[north]) ** 2
    out[north] = r * np.exp(1.0 - r)
    return out


def forcing(pos, t, k, amplitude, Tp=4.0, Tf=15.0, theta1=math.pi / 3):
    """F_R(x, t) = amplitude k^2 A(t) B(theta) cos(k phi) (Sec. 4.4; the paper's amplitude is
    (3/5) Omega), phi the longitude."""
    pos = _f64(pos, (-1, 3))
    lon = np.arctan2(pos[:, 1], pos[:, 0])
    return amplitude * k * k * forcing_ramp(t, Tp, Tf) * forcing_profile(pos, theta1) * np.cos(k * lon)


def rk4_step(pos, zeta, area, dt, Omega, velocity, project=True, t=0.0, forcing=None):
    """One classical RK4 step of the Sec. 2 system (x, zeta), dzeta/dt = -2 Omega u_z.

    ``velocity(x, zeta, area)`` evaluates u at the stage positions with the stage
    vorticities.  Stage points and the new positions are projected to the sphere
    (x / |x|) when ``project`` is set.  ``forcing(x, t)``: the forced system of Sec. 4.4,
    whose Biot-Savart source strength is (zeta - F_R(x, t)) A at every stage (stage times t,
    t + dt/2, t + dt/2, t + dt); the particle vorticity still follows dzeta/dt = -2 Omega u_z.
    """
    pos = _f64(pos, (-1, 3))
    zeta = _f64(zeta)
    proj = _project if project else (lambda v: v)
    k = []
    xs, zs = pos, zeta
    for c, ts in zip((0.5, 0.5, 1.0, None), (t, t + 0.5 * dt, t + 0.5 * dt, t + dt)):
        u = velocity(xs, zs if forcing is None else zs - forcing(xs, ts), area)
        k.append(u)
        if c is None:
            break
        xs = proj(pos + (c * dt) * u)
        zs = zeta + (c * dt) * (-2.0 * Omega * u[:, 2])
    ksum = (k[0] + 2.0 * k[1]) + (2.0 * k[2] + k[3])
    new_pos = proj(pos + (dt / 6.0) * ksum)
    new_zeta = zeta + (dt / 6.0) * (-2.0 * Omega * ksum[:, 2])
    return new_pos, new_zeta


def rel_l2(v, v_ref, area):
    """E = sqrt(sum |v - v_ref|^2 A / sum |v_ref|^2 A) (Sec. 4.1)."""
    v = np.asarray(v, np.float64).reshape(-1, 3)
    v_ref = np.asarray(v_ref, np.float64).reshape(-1, 3)
    a = np.asarray(area, np.float64).reshape(-1)
    num = np.sum(np.sum((v - v_ref) ** 2, axis=1) * a)
    den = np.sum(np.sum(v_ref ** 2, axis=1) * a)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def rel_max(v, v_ref):
    """max_i |v_i - v_ref_i| / max_i |v_ref_i|."""
    v = np.asarray(v, np.float64).reshape(-1, 3)
    v_ref = np.asarray(v_ref, np.float64).reshape(-1, 3)
    den = np.max(np.linalg.norm(v_ref, axis=1))
    return float(np.max(np.linalg.norm(v - v_ref, axis=1)) / (den if den > 0 else 1.0))
