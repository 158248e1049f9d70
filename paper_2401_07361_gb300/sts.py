"""Python binding of the C ABI in ``include/sts.h`` (``libsts.so``), argument marshalling only.

Every function has the name of the C entry point it calls.  Device arrays are torch CUDA
tensors (float64 unless stated, contiguous); host arrays of the export calls are numpy.
``stream`` is a ``torch.cuda.Stream`` or None for the current stream.  Every non-zero return
code raises ``StsError`` with the library's message.  There is no fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

STS_FP64 = 0
STS_MIXED = 1
STS_OK, STS_ERR_ARG, STS_ERR_CUDA, STS_ERR_CAPACITY, STS_ERR_TIMEOUT, STS_ERR_NONFINITE, STS_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
PHASES = ("build", "sort", "lists", "prep", "upward", "eval", "direct", "cluster")

_lock = threading.Lock()
_lib = None


class StsError(RuntimeError):
    pass


class sts_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("degree", C.c_int32), ("leaf_size", C.c_int32),
                ("max_level", C.c_int32), ("precision", C.c_int32), ("near_fp64_tau", C.c_double)]


class sts_forcing(C.Structure):
    """The vorticity forcing of Sec. 4.4 (see include/sts.h)."""
    _fields_ = [("k", C.c_int32), ("reserved", C.c_int32), ("amplitude", C.c_double), ("Tp", C.c_double),
                ("Tf", C.c_double), ("theta1", C.c_double)]


def forcing(k, amplitude, Tp=4.0, Tf=15.0, theta1=math.pi / 3):
    """sts_forcing for zonal wavenumber k; the paper's amplitude is (3/5) Omega."""
    return sts_forcing(int(k), 0, float(amplitude), float(Tp), float(Tf), float(theta1))


def params(theta=0.7, degree=8, leaf_size=128, max_level=16, precision=STS_MIXED, near_fp64_tau=0.0):
    return sts_params(float(theta), int(degree), int(leaf_size), int(max_level), int(precision),
                      float(near_fp64_tau))


def load(build_if_needed: bool = True):
    """Loads ``libsts.so`` (building it first when sources are newer, if allowed).  The
    environment variable STS_LIBRARY names another build of the same library to load."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("STS_LIBRARY") or _build.LIB
        if build_if_needed and path == _build.LIB and _build.needs_build():
            _build.build()
        if not os.path.exists(path):
            raise StsError(f"libsts.so is missing ({path}); build it with paper_2401_07361_gb300.build")
        lib = C.CDLL(path)
        P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        PP = C.POINTER(sts_params)
        sig = {
            "sts_create": (i32, [C.POINTER(P)]),
            "sts_destroy": (None, [P]),
            "sts_last_error": (C.c_char_p, []),
            "sts_status": (i32, [P, P]),
            "sts_selftest_wait": (i32, [P, i32, P]),
            "sts_direct": (i32, [P, P, P, P, i64, i32, P, P]),
            "sts_direct_targets": (i32, [P, P, P, P, i64, P, i64, i32, P, P]),
            "sts_direct_noalloc": (i32, [P, P, P, i64, i32, P, P]),
            "sts_tree_build": (i32, [P, P, i64, PP, P]),
            "sts_velocity": (i32, [P, P, P, PP, P, P]),
            "sts_potential": (i32, [P, P, P, PP, P, P]),
            "sts_velocity_dual": (i32, [P, P, P, PP, P, P]),
            "sts_dual_export": (i32, [P, i32, P, P, P, P]),
            "sts_velocity_range": (i32, [P, P, P, PP, i64, i64, i32, P, P]),
            "sts_leaf_work": (i32, [P, i32, P, P]),
            "sts_leaf_range": (i32, [P, i64, i64, P, P, P]),
            "sts_unpermute": (i32, [P, P, P, P]),
            "sts_dual_stats": (i32, [P, i32, P, P]),
            "sts_set_traversal": (i32, [P, i32]),
            "sts_amr_init": (i32, [P, P, i64, i64, P, P, i32, P]),
            "sts_amr_step": (i32, [P, dbl, dbl, P, P]),
            "sts_amr_info": (i32, [P, P]),
            "sts_amr_gather": (i32, [P, P, P, P, P, P]),
            "sts_amr_scatter": (i32, [P, P, P, P]),
            "sts_amr_export": (i32, [P] + [P] * 10 + [P]),
            "sts_direct_potential": (i32, [P, P, P, P, i64, i32, P, P]),
            "bve_rk4_step": (i32, [P, P, P, P, i64, dbl, dbl, PP, P]),
            "bve_rk4_step_forced": (i32, [P, P, P, P, i64, dbl, dbl, dbl, C.POINTER(sts_forcing), PP, P]),
            "sts_tree_build_batched": (i32, [P, P, P, i32, PP, P]),
            "bve_rk4_step_batched": (i32, [P, P, P, P, P, i32, dbl, dbl, PP, P]),
            "sts_tree_info": (i32, [P, P, P]),
            "sts_tree_export": (i32, [P] + [P] * 11 + [P]),
            "sts_lists_export": (i32, [P, P, P, P, P, P]),
            "sts_clusters_export": (i32, [P, P, P, P, P]),
            "sts_proxy_reference": (i32, [i32, P, P]),
            "sts_stats": (i32, [P, P, P]),
            "sts_set_timing": (i32, [P, i32]),
            "sts_phase_times": (i32, [P, P, P, i32]),
            "sts_launch_count": (i32, [P]),
            "sts_set_graph": (i32, [P, i32]),
            "sts_tree_velocity": (i32, [P, P, P, P, P, i32, PP, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc, fn):
    if rc != 0:
        msg = load().sts_last_error().decode(errors="replace")
        raise StsError(f"{fn} returned {rc}: {msg}")


def _dev(t, dtype=None, numel=None, name="array"):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise StsError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise StsError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise StsError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise StsError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _host(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------------------- context
def sts_create():
    h = C.c_void_p()
    _check(load().sts_create(C.byref(h)), "sts_create")
    return h


def sts_destroy(ctx):
    if ctx is not None and _lib is not None:
        _lib.sts_destroy(ctx)


def sts_status(ctx, stream=None):
    _check(load().sts_status(ctx, _stream(stream)), "sts_status")


def sts_selftest_wait(ctx, spins, stream=None):
    """Runs the bounded-wait self-test; returns the library's return code (STS_ERR_TIMEOUT
    expected) instead of raising."""
    return int(load().sts_selftest_wait(ctx, int(spins), _stream(stream)))


# ------------------------------------------------------------------------------- compute
def sts_direct(ctx, pos, zeta, area, precision=STS_FP64, vel=None, stream=None):
    import torch

    n = pos.shape[0]
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    _check(load().sts_direct(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                             _dev(area, torch.float64, n, "area"), n, int(precision),
                             _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)), "sts_direct")
    return vel


def sts_direct_targets(ctx, pos, zeta, area, targets, precision=STS_FP64, vel=None, stream=None):
    import torch

    n = pos.shape[0]
    nt = targets.numel()
    if vel is None:
        vel = torch.empty((nt, 3), dtype=torch.float64, device=pos.device)
    _check(load().sts_direct_targets(ctx, _dev(pos, torch.float64, 3 * n, "pos"),
                                     _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                     n, _dev(targets, torch.int64, nt, "targets"), nt, int(precision),
                                     _dev(vel, torch.float64, 3 * nt, "vel"), _stream(stream)),
           "sts_direct_targets")
    return vel


def sts_direct_noalloc(pos, zeta, area, precision=STS_FP64, vel=None, stream=None):
    import torch

    n = pos.shape[0]
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    _check(load().sts_direct_noalloc(_dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                                     _dev(area, torch.float64, n, "area"), n, int(precision),
                                     _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)),
           "sts_direct_noalloc")
    return vel


def sts_tree_build(ctx, pos, p, stream=None):
    import torch

    n = pos.shape[0]
    _check(load().sts_tree_build(ctx, _dev(pos, torch.float64, 3 * n, "pos"), n, C.byref(p), _stream(stream)),
           "sts_tree_build")


def sts_velocity(ctx, zeta, area, p, vel=None, stream=None):
    import torch

    n = zeta.numel()
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=zeta.device)
    _check(load().sts_velocity(ctx, _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                               C.byref(p), _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)),
           "sts_velocity")
    return vel


def sts_velocity_dual(ctx, zeta, area, p, vel=None, stream=None):
    """Tree-code velocity vel[n,3] by the dual traversal (PP, PC, CP, CC) for the tree last
    built in ctx."""
    import torch

    n = zeta.numel()
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=zeta.device)
    _check(load().sts_velocity_dual(ctx, _dev(zeta, torch.float64, n, "zeta"),
                                    _dev(area, torch.float64, n, "area"), C.byref(p),
                                    _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)),
           "sts_velocity_dual")
    return vel


def sts_velocity_range(ctx, zeta, area, p, leaf_begin, leaf_end, out_sorted=False, vel=None, stream=None):
    """Velocities of the targets of depth-first leaves [leaf_begin, leaf_end) only.  With
    out_sorted, returns the compact block of those targets in sorted slot order (one GPU's
    share, see sts_leaf_range); else writes their rows of vel[n,3] (caller's order)."""
    import torch

    n = zeta.numel()
    if vel is None:
        if out_sorted:
            s0, s1 = sts_leaf_range(ctx, leaf_begin, leaf_end, stream)
            vel = torch.empty((s1 - s0, 3), dtype=torch.float64, device=zeta.device)
        else:
            vel = torch.zeros((n, 3), dtype=torch.float64, device=zeta.device)
    _check(load().sts_velocity_range(ctx, _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                     C.byref(p), int(leaf_begin), int(leaf_end), int(bool(out_sorted)),
                                     _dev(vel, torch.float64, vel.numel(), "vel"), _stream(stream)),
           "sts_velocity_range")
    return vel


def sts_leaf_work(ctx, degree, stream=None):
    """Per-leaf PC + PP interactions (numpy int64[nleaves]) of the current target-leaf lists."""
    import numpy as np

    nl = sts_tree_info(ctx, stream)["leaves"]
    work = np.zeros(max(nl, 1), dtype=np.int64)
    _check(load().sts_leaf_work(ctx, int(degree), _host(work), _stream(stream)), "sts_leaf_work")
    return work[:nl]


def sts_leaf_range(ctx, leaf_begin, leaf_end, stream=None):
    """(slot_begin, slot_end) of the targets of depth-first leaves [leaf_begin, leaf_end)."""
    a, b = C.c_int64(0), C.c_int64(0)
    _check(load().sts_leaf_range(ctx, int(leaf_begin), int(leaf_end), C.byref(a), C.byref(b), _stream(stream)),
           "sts_leaf_range")
    return a.value, b.value


def sts_unpermute(ctx, vel_sorted, vel=None, stream=None):
    """vel[perm[t]] = vel_sorted[t]: sorted slot order back to the caller's order."""
    import torch

    n = vel_sorted.shape[0]
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=vel_sorted.device)
    _check(load().sts_unpermute(ctx, _dev(vel_sorted, torch.float64, 3 * n, "vel_sorted"),
                                _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)), "sts_unpermute")
    return vel


DUAL_KINDS = ("PP", "PC", "CP", "CC")


def sts_dual_export(ctx, stream=None):
    """Pairs of the last dual traversal: {"PP"|"PC"|"CP"|"CC": (target nodes, source nodes)},
    sorted by target (leaf or cluster order), then source."""
    out = {}
    for k, name in enumerate(DUAL_KINDS):
        cnt = np.zeros(1, np.int64)
        _check(load().sts_dual_export(ctx, k, _host(cnt), None, None, _stream(stream)), "sts_dual_export")
        t, s = np.zeros(int(cnt[0]), np.int32), np.zeros(int(cnt[0]), np.int32)
        _check(load().sts_dual_export(ctx, k, _host(cnt), _host(t), _host(s), _stream(stream)), "sts_dual_export")
        out[name] = (t, s)
    return out


# ---------------------------------------------------------------------------- adaptive mesh
def sts_amr_init(ctx, faces, pos0, zeta0, levels=3, stream=None):
    """Adaptive mesh over the base triangulation faces[t0, 3] (host) of the particles pos0[n0, 3],
    zeta0[n0] (device)."""
    import torch

    faces = np.ascontiguousarray(faces, dtype=np.int32)
    n0 = pos0.shape[0]
    _check(load().sts_amr_init(ctx, _host(faces), faces.shape[0], n0, _dev(pos0, torch.float64, 3 * n0, "pos0"),
                               _dev(zeta0, torch.float64, n0, "zeta0"), int(levels), _stream(stream)), "sts_amr_init")


def sts_amr_step(ctx, eps1, eps2, stream=None):
    """One refinement pass; returns (splits, merges, particles, leaf triangles)."""
    c = np.zeros(4, np.int64)
    _check(load().sts_amr_step(ctx, float(eps1), float(eps2), _host(c), _stream(stream)), "sts_amr_step")
    return tuple(int(x) for x in c)


def sts_amr_info(ctx):
    a = np.zeros(5, np.int64)
    _check(load().sts_amr_info(ctx, _host(a)), "sts_amr_info")
    return dict(n0=int(a[0]), nv=int(a[1]), t0=int(a[2]), nt=int(a[3]), particles=int(a[4]))


def sts_amr_gather(ctx, stream=None):
    """The particles (device tensors): pos[np, 3], zeta[np], area[np], ids[np]."""
    import torch

    n = sts_amr_info(ctx)["particles"]
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.empty((n, 3), dtype=torch.float64, device=dev)
    zeta = torch.empty(n, dtype=torch.float64, device=dev)
    area = torch.empty(n, dtype=torch.float64, device=dev)
    ids = torch.empty(n, dtype=torch.int64, device=dev)
    _check(load().sts_amr_gather(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                                 _dev(area, torch.float64, n, "area"), _dev(ids, torch.int64, n, "ids"),
                                 _stream(stream)), "sts_amr_gather")
    return pos, zeta, area, ids


def sts_amr_scatter(ctx, pos, zeta, stream=None):
    import torch

    n = pos.shape[0]
    _check(load().sts_amr_scatter(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                                  _stream(stream)), "sts_amr_scatter")


def sts_amr_export(ctx, stream=None):
    i = sts_amr_info(ctx)
    nt, nv = i["nt"], i["nv"]
    o = dict(tv=np.zeros((nt, 3), np.int32), tparent=np.zeros(nt, np.int32), tchild=np.zeros(nt, np.int32),
             tlevel=np.zeros(nt, np.int8), vparent=np.zeros((nv, 2), np.int32), tstate=np.zeros(nt, np.uint8),
             valive=np.zeros(nv, np.uint8), pos=np.zeros((nv, 3)), zeta=np.zeros(nv), area=np.zeros(nv))
    _check(load().sts_amr_export(ctx, *(_host(o[k]) for k in ("tv", "tparent", "tchild", "tlevel", "vparent",
                                                               "tstate", "valive", "pos", "zeta", "area")),
                                 _stream(stream)), "sts_amr_export")
    return o


def sts_set_traversal(ctx, dual=True):
    """Selects the dual traversal (True) or the target-leaf lists (False) for sts_velocity,
    sts_tree_velocity and the RK4 steps."""
    _check(load().sts_set_traversal(ctx, int(bool(dual))), "sts_set_traversal")


def sts_dual_stats(ctx, degree, stream=None):
    a = np.zeros(5, np.int64)
    _check(load().sts_dual_stats(ctx, int(degree), _host(a), _stream(stream)), "sts_dual_stats")
    return dict(pp=int(a[0]), pc=int(a[1]), cp=int(a[2]), cc=int(a[3]), down=int(a[4]))


def sts_potential(ctx, zeta, area, p, psi=None, stream=None):
    """Tree-code stream function psi[n] (FP64) for the tree last built in ctx."""
    import torch

    n = zeta.numel()
    if psi is None:
        psi = torch.empty(n, dtype=torch.float64, device=zeta.device)
    _check(load().sts_potential(ctx, _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                C.byref(p), _dev(psi, torch.float64, n, "psi"), _stream(stream)),
           "sts_potential")
    return psi


def sts_direct_potential(ctx, pos, zeta, area, precision=STS_FP64, psi=None, stream=None):
    """Direct-sum stream function psi[n] (FP64)."""
    import torch

    n = pos.shape[0]
    if psi is None:
        psi = torch.empty(n, dtype=torch.float64, device=pos.device)
    _check(load().sts_direct_potential(ctx, _dev(pos, torch.float64, 3 * n, "pos"),
                                       _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                       n, int(precision), _dev(psi, torch.float64, n, "psi"), _stream(stream)),
           "sts_direct_potential")
    return psi


def bve_rk4_step(ctx, pos, zeta, area, dt, Omega, p, stream=None):
    import torch

    n = pos.shape[0]
    _check(load().bve_rk4_step(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                               _dev(area, torch.float64, n, "area"), n, float(dt), float(Omega), C.byref(p),
                               _stream(stream)), "bve_rk4_step")


def bve_rk4_step_forced(ctx, pos, zeta, area, t, dt, Omega, forcing, p, stream=None):
    """One RK4 step of the forced system of Sec. 4.4 starting at time t (in place)."""
    import torch

    n = pos.shape[0]
    _check(load().bve_rk4_step_forced(ctx, _dev(pos, torch.float64, 3 * n, "pos"),
                                      _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                      n, float(t), float(dt), float(Omega), C.byref(forcing), C.byref(p),
                                      _stream(stream)), "bve_rk4_step_forced")


def _offsets(offsets):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    return off, int(off.shape[0] - 1)


def sts_tree_build_batched(ctx, pos, offsets, p, stream=None):
    import torch

    off, ninst = _offsets(offsets)
    n = pos.shape[0]
    if ninst < 1 or off[-1] != n:
        raise StsError(f"offsets must end at the number of particles ({n}), got {off[-1] if ninst >= 0 else None}")
    _check(load().sts_tree_build_batched(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _host(off), ninst,
                                         C.byref(p), _stream(stream)), "sts_tree_build_batched")


def bve_rk4_step_batched(ctx, pos, zeta, area, offsets, dt, Omega, p, stream=None):
    import torch

    off, ninst = _offsets(offsets)
    n = pos.shape[0]
    if ninst < 1 or off[-1] != n:
        raise StsError(f"offsets must end at the number of particles ({n})")
    _check(load().bve_rk4_step_batched(ctx, _dev(pos, torch.float64, 3 * n, "pos"),
                                       _dev(zeta, torch.float64, n, "zeta"), _dev(area, torch.float64, n, "area"),
                                       _host(off), ninst, float(dt), float(Omega), C.byref(p), _stream(stream)),
           "bve_rk4_step_batched")


# ---------------------------------------------------------------------------- inspection
def sts_tree_info(ctx, stream=None):
    a = np.zeros(8, np.int64)
    _check(load().sts_tree_info(ctx, _host(a), _stream(stream)), "sts_tree_info")
    keys = ("n", "nodes", "leaves", "depth", "nfar", "nnear", "clusters", "tasks")
    return {k: int(v) for k, v in zip(keys, a)}


def sts_tree_export(ctx, stream=None):
    inf = sts_tree_info(ctx, stream)
    n, nn, nl = inf["n"], inf["nodes"], inf["leaves"]
    out = dict(perm=np.zeros(n, np.int64), level=np.zeros(nn, np.int32), key=np.zeros(nn, np.uint64),
               parent=np.zeros(nn, np.int32), first_child=np.zeros(nn, np.int32), nchild=np.zeros(nn, np.int32),
               start=np.zeros(nn, np.int64), count=np.zeros(nn, np.int64), leaf=np.zeros(nn, np.int32),
               leaves=np.zeros(nl, np.int32), geom=np.zeros((nn, 13)))
    _check(load().sts_tree_export(ctx, *[_host(out[k]) for k in ("perm", "level", "key", "parent", "first_child",
                                                                  "nchild", "start", "count", "leaf", "leaves",
                                                                  "geom")], _stream(stream)), "sts_tree_export")
    return out


def sts_lists_export(ctx, stream=None):
    inf = sts_tree_info(ctx, stream)
    nl = inf["leaves"]
    out = dict(far_off=np.zeros(nl + 1, np.int64), far_idx=np.zeros(inf["nfar"], np.int32),
               near_off=np.zeros(nl + 1, np.int64), near_idx=np.zeros(inf["nnear"], np.int32))
    _check(load().sts_lists_export(ctx, _host(out["far_off"]), _host(out["far_idx"]), _host(out["near_off"]),
                                   _host(out["near_idx"]), _stream(stream)), "sts_lists_export")
    return out


def sts_clusters_export(ctx, degree, stream=None):
    inf = sts_tree_info(ctx, stream)
    c = inf["clusters"]
    M = (degree + 1) * (degree + 2) // 2
    ids, yt, W = np.zeros(c, np.int32), np.zeros((c, M, 3)), np.zeros((c, M))
    _check(load().sts_clusters_export(ctx, _host(ids), _host(yt), _host(W), _stream(stream)),
           "sts_clusters_export")
    return ids, yt, W


def sts_proxy_reference(degree):
    M = (degree + 1) * (degree + 2) // 2
    beta, vinv = np.zeros((M, 3)), np.zeros((M, M))
    _check(load().sts_proxy_reference(int(degree), _host(beta), _host(vinv)), "sts_proxy_reference")
    return beta, vinv


def sts_stats(ctx, stream=None):
    a = np.zeros(2, np.int64)
    _check(load().sts_stats(ctx, _host(a), _stream(stream)), "sts_stats")
    return dict(pc=int(a[0]), pp=int(a[1]))


def sts_set_timing(ctx, on=True):
    _check(load().sts_set_timing(ctx, int(bool(on))), "sts_set_timing")


def sts_phase_times(ctx):
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), np.int32)
    _check(load().sts_phase_times(ctx, _host(ms), _host(cnt), len(PHASES)), "sts_phase_times")
    return {k: (float(m), int(c)) for k, m, c in zip(PHASES, ms, cnt)}


def sts_tree_velocity(ctx, pos, zeta, area, p, vel=None, offsets=None, stream=None):
    import torch

    n = pos.shape[0]
    off, ninst = _offsets(offsets if offsets is not None else [0, n])
    if off[-1] != n:
        raise StsError(f"offsets must end at the number of particles ({n})")
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    _check(load().sts_tree_velocity(ctx, _dev(pos, torch.float64, 3 * n, "pos"), _dev(zeta, torch.float64, n, "zeta"),
                                    _dev(area, torch.float64, n, "area"), _host(off), ninst, C.byref(p),
                                    _dev(vel, torch.float64, 3 * n, "vel"), _stream(stream)), "sts_tree_velocity")
    return vel


def sts_set_graph(ctx, on=True):
    _check(load().sts_set_graph(ctx, int(bool(on))), "sts_set_graph")


def sts_launch_count():
    a = np.zeros(1, np.int64)
    _check(load().sts_launch_count(_host(a)), "sts_launch_count")
    return int(a[0])


class Context:
    """Owns one ``sts_ctx`` (freed on close or garbage collection)."""

    def __init__(self):
        self.h = sts_create()

    def close(self):
        if self.h is not None:
            sts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
