"""ctypes binding of ``libsemgb.so`` (the C ABI in ``include/sem.h``).

Every function here has the name of the C entry point it calls and only marshals
arguments: numpy arrays for host pointers, CUDA tensors (or raw integer addresses) for
``*_dev`` pointers. All arithmetic runs in the library. The library is loaded on first use;
if it has not been built, or cannot be loaded, the call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

SEM_OK = 0
ERRORS = {-1: "SEM_EINVAL", -2: "SEM_ENOMEM", -3: "SEM_ECUDA", -4: "SEM_ESTATE", -5: "SEM_ETIMEOUT",
          -6: "SEM_EDIVERGED"}

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name: (restype, argtypes) for every symbol declared in include/sem.h
SIGNATURES = {
    "sem_version": (_I, []),
    "sem_gll": (_I, [_I, _P, _P, _P]),
    "sem_color_elements": (_I, [_I, _I, _I, _P, _P, _P]),
    "sem_patch_plan": (_I, [_I, _I, _I, _P, _P, _P, _P]),
    "sem_geometry": (_I, [_I, _I, _P, _P, _P, _P]),
    "sem_geometry_points": (_I, [_I, _I, _P, _P, _P]),
    "sem_locate_points": (_I, [_I, _P, _I, _P, _P, _P]),
    "sem_point_source_forces": (_I, [_I, _P, _P, _P, _P, _P]),
    "sem_create": (_I, [_P, _I, _I, _P]),
    "sem_destroy": (_I, [_P]),
    "sem_set_option": (_I, [_P, _I, ctypes.c_longlong]),
    "sem_set_mesh": (_I, [_P, _I, _I, _P, _P]),
    "sem_set_mesh_corners": (_I, [_P, _I, _I, _P, _P]),
    "sem_set_material": (_I, [_P, _P, _P, _P]),
    "sem_set_moduli": (_I, [_P, _P, _P, _P]),
    "sem_set_moduli_dev": (_I, [_P, _P, _P, _P]),
    "sem_suggest_dt": (_I, [_P, _D, _P]),
    "sem_set_dt": (_I, [_P, _D]),
    "sem_locate_nodes": (_I, [_P, _I, _P, _P, _P]),
    "sem_node_xyz": (_I, [_P, _I, _P, _P]),
    "sem_set_sources": (_I, [_P, _I, _P, _P, _D, _D]),
    "sem_set_source_nodes": (_I, [_P, _I, _P, _P, _D, _D]),
    "sem_set_receivers": (_I, [_P, _I, _P, _P]),
    "sem_set_receiver_nodes": (_I, [_P, _I, _P]),
    "sem_set_shots": (_I, [_P, _I]),
    "sem_set_shot_sources": (_I, [_P, _I, _P, _P, _P, _D, _D]),
    "sem_set_shot_moment_sources": (_I, [_P, _I, _P, _P, _P, _D, _D]),
    "sem_set_shot_sources_at": (_I, [_P, _I, _P, _P, _P, _P, _D, _D]),
    "sem_set_state": (_I, [_P, _P, _P, _P]),
    "sem_set_state_dev": (_I, [_P, _P, _P, _P]),
    "sem_set_step": (_I, [_P, ctypes.c_longlong]),
    "sem_init_acceleration": (_I, [_P]),
    "sem_get_state": (_I, [_P, _P, _P, _P]),
    "sem_get_state_dev": (_I, [_P, _P, _P, _P]),
    "sem_step": (_I, [_P, _I]),
    "sem_run": (_I, [_P, _I, _P]),
    "sem_run_dev": (_I, [_P, _I, _P]),
    "sem_run_snapshots": (_I, [_P, _I, _P]),
    "sem_run_record_snapshots": (_I, [_P, _I, _P, _P]),
    "sem_check_finite": (_I, [_P]),
    "sem_apply_stiffness": (_I, [_P, _P, _P]),
    "sem_apply_stiffness_strided": (_I, [_P, _P, _P, _I]),
    "sem_node_order": (_I, [_P, _P]),
    "sem_energy": (_I, [_P, _P]),
    "sem_adjoint_begin": (_I, [_P]),
    "sem_adjoint_step": (_I, [_P, _P]),
    "sem_adjoint_accumulate": (_I, [_P, _P, _P, _P]),
    "sem_adjoint_gradients": (_I, [_P, _P, _P, _P]),
    "sem_adjoint_segment": (_I, [_P, _I, _P, _P]),
    "sem_energy_noalloc": (_I, [_P, _I, _P, _P, _P, _P]),
    "sem_sync": (_I, [_P]),
    "sem_autotune": (_I, [_P, _I, _P, _P]),
    "sem_profile_steps": (_I, [_P, _I, _P]),
    "sem_tune_patch_shape": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _I, _I, _P, _P, _P]),
    "sem_group_create": (_I, [_P, _I, _P]),
    "sem_group_destroy": (_I, [_P]),
    "sem_group_step": (_I, [_P, _I]),
    "sem_group_sync": (_I, [_P]),
    "sem_group_last_error": (ctypes.c_char_p, [_P]),
    "sem_group_set_option": (_I, [_P, _I, ctypes.c_longlong]),
    "sem_group_info": (_I, [_P, _P]),
    "sem_info": (_I, [_P, _P]),
    "sem_color_counts": (_I, [_P, _P]),
    "sem_patch_info": (_I, [_P, _P]),
    "sem_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


class SemError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {message}")
        self.code = code


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """The loaded library (raises if it is missing and ``build_if_missing`` is False)."""
    global _lib
    if _lib is None:
        path = os.environ.get("SEMGB_LIBRARY", _build.LIB)  # alternate build of the same sources
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libsemgb is not built ({path} missing); call "
                                   "paper_2606_12850_gb300.build.build() first")
            _build.build()
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(code: int, where: str, ctx=None):
    if code != SEM_OK:
        msg = lib().sem_last_error(ctx.handle if ctx is not None else None)
        raise SemError(code, where, (msg or b"").decode(errors="replace"))


def _host(a, dtype, shape=None):
    """Contiguous numpy array of ``dtype`` (copied only when needed) and its pointer."""
    arr = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and arr.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} values, got {arr.size}")
    return arr, arr.ctypes.data_as(_P)


def _dev(t, nvalues=None, ctx=None):
    """Device address of a contiguous float32 CUDA tensor on the context's GPU (or an int
    address, taken as is). Checked before any library call: a tensor of another dtype would
    be read or written at the wrong byte size, one on another GPU at a foreign address."""
    if t is None:
        return None
    if isinstance(t, int):
        return _P(t)
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch.float32":
        raise TypeError(f"device tensor must be float32, got {t.dtype}")
    if ctx is not None and t.device.index != ctx.device:
        raise ValueError(f"device tensor is on cuda:{t.device.index}, the context on cuda:{ctx.device}")
    if not t.is_contiguous():
        raise ValueError("device tensor must be contiguous")
    if nvalues is not None and t.numel() < nvalues:
        raise ValueError(f"device tensor holds {t.numel()} values, needs {nvalues}")
    return _P(t.data_ptr())


class Ctx:
    """Owner of a ``sem_ctx*``; destroyed with the object."""

    def __init__(self, handle: int, ngll: int):
        self.handle = _P(handle)
        self.ngll = ngll
        self.nglob = 0
        self.nspec = 0
        self.nrec = 0
        self.shots = 1
        self.device = 0

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.sem_destroy(self.handle)
            self.handle = None


def sem_version() -> int:
    return lib().sem_version()


def sem_gll(ngll: int):
    m = max(int(ngll), 1)
    xi, w, h = np.empty(m), np.empty(m), np.empty((m, m))
    _check(lib().sem_gll(ngll, xi.ctypes.data_as(_P), w.ctypes.data_as(_P), h.ctypes.data_as(_P)), "sem_gll")
    return xi, w, h


def sem_color_elements(ibool, ngll: int, nglob: int):
    ib, p = _host(ibool, np.int32)
    if ib.size == 0 or ib.size % ngll ** 3:
        raise ValueError(f"ibool must hold [nspec][{ngll}^3] entries")
    nspec = ib.size // ngll ** 3
    color = np.empty(nspec, dtype=np.int32)
    nc = ctypes.c_int(0)
    _check(lib().sem_color_elements(nspec, ngll, nglob, p, color.ctypes.data_as(_P), ctypes.byref(nc)),
           "sem_color_elements")
    return color, nc.value


def sem_geometry(ctrl, ngll: int):
    """Library geometry of the elements ``ctrl`` [nspec][8][3]: returns xyz [nspec][ngll^3][3],
    dxi_dx [nspec][ngll^3][3][3] ([r][d] = d xi_r / d x_d) and jac [nspec][ngll^3]."""
    c, p = _host(ctrl, np.float64)
    if c.size == 0 or c.size % 24:
        raise ValueError("ctrl must hold [nspec][8][3] corner coordinates")
    nspec = c.size // 24
    n3 = ngll ** 3
    xyz = np.empty((nspec, n3, 3))
    g = np.empty((nspec, n3, 3, 3))
    jac = np.empty((nspec, n3))
    _check(lib().sem_geometry(ngll, nspec, p, xyz.ctypes.data_as(_P), g.ctypes.data_as(_P),
                              jac.ctypes.data_as(_P)), "sem_geometry")
    return xyz, g, jac


def sem_geometry_points(ngll: int, xyz):
    """Host-only geometry from per-point positions xyz [nspec][ngll^3][3]: (dxi_dx
    [nspec][ngll^3][3][3], jac [nspec][ngll^3])."""
    pts, pp = _host(xyz, np.float64)
    n3 = ngll ** 3
    nspec = pts.size // (3 * n3)
    G = np.empty((nspec, n3, 3, 3))
    J = np.empty((nspec, n3))
    _check(lib().sem_geometry_points(int(ngll), nspec, pp, G.ctypes.data_as(_P), J.ctypes.data_as(_P)),
           "sem_geometry_points")
    return G, J


def sem_locate_points(ctrl, xyz):
    """Element (lowest index; -1 outside) and reference coordinates of each point among the
    trilinear elements ``ctrl`` [nspec][8][3]."""
    c, pc = _host(ctrl, np.float64)
    if c.size == 0 or c.size % 24:
        raise ValueError("ctrl must hold [nspec][8][3] corner coordinates")
    pts, pp = _host(np.atleast_2d(xyz), np.float64)
    if pts.size % 3:
        raise ValueError("xyz must hold [npts][3] coordinates")
    n = pts.size // 3
    elem = np.empty(n, dtype=np.int32)
    ref = np.empty((n, 3))
    _check(lib().sem_locate_points(c.size // 24, pc, n, pp, elem.ctypes.data_as(_P), ref.ctypes.data_as(_P)),
           "sem_locate_points")
    return elem, ref


def sem_point_source_forces(ngll: int, ctrl_e, ref, force=None, moment=None):
    """Nodal forces [ngll^3][3] of a point force or a moment tensor at reference coordinates
    ``ref`` of the element with corners ``ctrl_e`` [8][3]."""
    c, pc = _host(ctrl_e, np.float64, (8, 3))
    r, pr = _host(ref, np.float64, (3,))
    f = None if force is None else _host(force, np.float64, (3,))
    m = None if moment is None else _host(moment, np.float64, (6,))
    out = np.empty((ngll ** 3, 3))
    _check(lib().sem_point_source_forces(ngll, pc, pr, f[1] if f else None, m[1] if m else None,
                                         out.ctypes.data_as(_P)), "sem_point_source_forces")
    return out


def sem_create(ngll: int, device: int = 0, stream=None) -> Ctx:
    out = _P()
    s = None
    if stream is not None:
        s = _P(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().sem_create(ctypes.byref(out), ngll, device, s), "sem_create")
    c = Ctx(out.value, ngll)
    c.device = int(device)
    return c


def sem_destroy(ctx: Ctx):
    if ctx.handle is not None:
        _check(lib().sem_destroy(ctx.handle), "sem_destroy")
        ctx.handle = None


SEM_OPT_SWEEP_SLABS = 1
SEM_OPT_CONTRACTION = 2
SEM_OPT_ASSEMBLY = 3
SEM_OPT_SWEEP_STALL_TEST = 4
SEM_OPT_NODE_ORDER = 5
SEM_OPT_FUSED_NEWMARK = 6
SEM_OPT_SHOT_PAIRS = 7
SEM_OPT_PATCH_SHAPE = 8
SEM_GROUP_MODE = 1
SEM_GROUP_STALL_TEST = 2


def sem_set_option(ctx: Ctx, option: int, value: int):
    _check(lib().sem_set_option(ctx.handle, int(option), int(value)), "sem_set_option", ctx)


def sem_set_mesh(ctx: Ctx, ibool, xyz, nglob: int):
    """Mesh from the positions of every local point, xyz [nspec][ngll^3][3]."""
    n3 = ctx.ngll ** 3
    ib, pi = _host(ibool, np.int32)
    if ib.size == 0 or ib.size % n3:
        raise ValueError(f"ibool must hold [nspec][{ctx.ngll}^3] entries")
    nspec = ib.size // n3
    pts, pp = _host(xyz, np.float64, (nspec, n3, 3))
    _check(lib().sem_set_mesh(ctx.handle, nspec, int(nglob), pi, pp), "sem_set_mesh", ctx)
    ctx.nspec, ctx.nglob = nspec, int(nglob)


def sem_set_mesh_corners(ctx: Ctx, ibool, ctrl, nglob: int):
    """Mesh of trilinear hexahedra from their corners, ctrl [nspec][8][3]."""
    n3 = ctx.ngll ** 3
    ib, pi = _host(ibool, np.int32)
    if ib.size == 0 or ib.size % n3:
        raise ValueError(f"ibool must hold [nspec][{ctx.ngll}^3] entries")
    nspec = ib.size // n3
    ct, pc = _host(ctrl, np.float64, (nspec, 8, 3))
    _check(lib().sem_set_mesh_corners(ctx.handle, nspec, int(nglob), pi, pc), "sem_set_mesh_corners", ctx)
    ctx.nspec, ctx.nglob = nspec, int(nglob)


def sem_set_material(ctx: Ctx, rho, vp, vs):
    shape = (ctx.nspec, ctx.ngll ** 3)
    r, pr = _host(rho, np.float32, shape)
    a, pa = _host(vp, np.float32, shape)
    b, pb = _host(vs, np.float32, shape)
    _check(lib().sem_set_material(ctx.handle, pr, pa, pb), "sem_set_material", ctx)


def sem_set_moduli(ctx: Ctx, rho, kappa, mu):
    shape = (ctx.nspec, ctx.ngll ** 3)
    r, pr = _host(rho, np.float32, shape)
    a, pa = _host(kappa, np.float32, shape)
    b, pb = _host(mu, np.float32, shape)
    _check(lib().sem_set_moduli(ctx.handle, pr, pa, pb), "sem_set_moduli", ctx)


def sem_set_moduli_dev(ctx: Ctx, rho, kappa, mu):
    n = ctx.nspec * ctx.ngll ** 3
    _check(lib().sem_set_moduli_dev(ctx.handle, _dev(rho, n, ctx), _dev(kappa, n, ctx), _dev(mu, n, ctx)),
           "sem_set_moduli_dev", ctx)


def sem_suggest_dt(ctx: Ctx, courant: float) -> float:
    out = ctypes.c_double(0.0)
    _check(lib().sem_suggest_dt(ctx.handle, float(courant), ctypes.byref(out)), "sem_suggest_dt", ctx)
    return out.value


def sem_set_dt(ctx: Ctx, dt: float):
    _check(lib().sem_set_dt(ctx.handle, float(dt)), "sem_set_dt", ctx)


def sem_locate_nodes(ctx: Ctx, xyz, surface_z=None) -> np.ndarray:
    pts, pp = _host(np.atleast_2d(xyz), np.float64)
    n = pts.size // 3
    out = np.empty(n, dtype=np.int32)
    z = ctypes.byref(ctypes.c_double(surface_z)) if surface_z is not None else None
    _check(lib().sem_locate_nodes(ctx.handle, n, pp, z, out.ctypes.data_as(_P)), "sem_locate_nodes", ctx)
    return out


def sem_node_xyz(ctx: Ctx, node) -> np.ndarray:
    nd, pn = _host(np.atleast_1d(node), np.int32)
    out = np.empty((nd.size, 3))
    _check(lib().sem_node_xyz(ctx.handle, nd.size, pn, out.ctypes.data_as(_P)), "sem_node_xyz", ctx)
    return out


def sem_set_sources(ctx: Ctx, xyz, force, f0: float, t0: float):
    """Point forces at positions xyz [nsrc][3], snapped to the nearest nodes."""
    pts, pp = _host(np.atleast_2d(xyz), np.float64)
    n = pts.size // 3
    fo, pf = _host(np.atleast_2d(force), np.float64, (n, 3))
    _check(lib().sem_set_sources(ctx.handle, n, pp, pf, float(f0), float(t0)), "sem_set_sources", ctx)


def sem_set_source_nodes(ctx: Ctx, node, force, f0: float, t0: float):
    nd, pn = _host(np.atleast_1d(node), np.int32)
    fo, pf = _host(np.atleast_2d(force), np.float64, (nd.size, 3))
    _check(lib().sem_set_source_nodes(ctx.handle, nd.size, pn, pf, float(f0), float(t0)), "sem_set_source_nodes",
           ctx)


def sem_set_shots(ctx: Ctx, nshots: int):
    _check(lib().sem_set_shots(ctx.handle, int(nshots)), "sem_set_shots", ctx)
    ctx.shots = int(nshots)


def sem_set_shot_sources(ctx: Ctx, shot, node, force, f0: float, t0: float):
    sh, ps = _host(np.atleast_1d(shot), np.int32)
    nd, pn = _host(np.atleast_1d(node), np.int32, (sh.size,))
    fo, pf = _host(np.atleast_2d(force), np.float64, (sh.size, 3))
    _check(lib().sem_set_shot_sources(ctx.handle, sh.size, ps, pn, pf, float(f0), float(t0)),
           "sem_set_shot_sources", ctx)


def sem_set_shot_moment_sources(ctx: Ctx, shot, node, moment, f0: float, t0: float):
    nd, pn = _host(np.atleast_1d(node), np.int32)
    sh, ps = _host(np.atleast_1d(shot), np.int32, (nd.size,))
    mo, pm = _host(np.atleast_2d(moment), np.float64, (nd.size, 6))
    _check(lib().sem_set_shot_moment_sources(ctx.handle, nd.size, ps, pn, pm, float(f0), float(t0)),
           "sem_set_shot_moment_sources", ctx)


def sem_set_shot_sources_at(ctx: Ctx, shot, xyz, force=None, moment=None, f0: float = 10.0, t0: float = 0.12):
    """Sources at arbitrary positions (see sem.h); ``shot`` None applies each in every shot."""
    pts, pp = _host(np.atleast_2d(xyz), np.float64)
    if pts.size % 3:
        raise ValueError("xyz must hold [nsrc][3] coordinates")
    n = pts.size // 3
    sh = None if shot is None else _host(np.atleast_1d(shot), np.int32, (n,))
    fo = None if force is None else _host(np.atleast_2d(force), np.float64, (n, 3))
    mo = None if moment is None else _host(np.atleast_2d(moment), np.float64, (n, 6))
    _check(lib().sem_set_shot_sources_at(ctx.handle, n, sh[1] if sh else None, pp, fo[1] if fo else None,
                                         mo[1] if mo else None, float(f0), float(t0)), "sem_set_shot_sources_at", ctx)


def sem_set_receivers(ctx: Ctx, xyz) -> np.ndarray:
    """Receivers at positions xyz [nrec][3], snapped to the nearest nodes; returns the nodes."""
    pts, pp = _host(np.atleast_2d(xyz), np.float64)
    n = pts.size // 3
    out = np.empty(n, dtype=np.int32)
    _check(lib().sem_set_receivers(ctx.handle, n, pp, out.ctypes.data_as(_P)), "sem_set_receivers", ctx)
    ctx.nrec = n
    return out


def sem_set_receiver_nodes(ctx: Ctx, node):
    nd, pn = _host(np.atleast_1d(node), np.int32)
    _check(lib().sem_set_receiver_nodes(ctx.handle, nd.size, pn), "sem_set_receiver_nodes", ctx)
    ctx.nrec = nd.size


def _state_ptrs(ctx, arrays):
    keep, ptrs = [], []
    for a in arrays:
        if a is None:
            ptrs.append(None)
        else:
            arr, p = _host(a, np.float32, (ctx.shots, ctx.nglob, 3))
            keep.append(arr)
            ptrs.append(p)
    return keep, ptrs


def sem_set_state(ctx: Ctx, u=None, v=None, a=None):
    keep, (pu, pv, pa) = _state_ptrs(ctx, (u, v, a))
    _check(lib().sem_set_state(ctx.handle, pu, pv, pa), "sem_set_state", ctx)


def sem_set_state_dev(ctx: Ctx, u=None, v=None, a=None):
    n = 3 * ctx.nglob * ctx.shots
    _check(lib().sem_set_state_dev(ctx.handle, _dev(u, n, ctx), _dev(v, n, ctx), _dev(a, n, ctx)), "sem_set_state_dev",
           ctx)


def sem_set_step(ctx: Ctx, step: int):
    _check(lib().sem_set_step(ctx.handle, int(step)), "sem_set_step", ctx)


def sem_init_acceleration(ctx: Ctx):
    _check(lib().sem_init_acceleration(ctx.handle), "sem_init_acceleration", ctx)


def sem_get_state(ctx: Ctx, want=(True, True, True)):
    shape = (ctx.nglob, 3) if ctx.shots == 1 else (ctx.shots, ctx.nglob, 3)
    outs = [np.empty(shape, dtype=np.float32) if w else None for w in want]
    ptrs = [o.ctypes.data_as(_P) if o is not None else None for o in outs]
    _check(lib().sem_get_state(ctx.handle, *ptrs), "sem_get_state", ctx)
    return tuple(outs)


def sem_get_state_dev(ctx: Ctx, u=None, v=None, a=None):
    n = 3 * ctx.nglob * ctx.shots
    _check(lib().sem_get_state_dev(ctx.handle, _dev(u, n, ctx), _dev(v, n, ctx), _dev(a, n, ctx)), "sem_get_state_dev",
           ctx)


def sem_step(ctx: Ctx, nsteps: int):
    _check(lib().sem_step(ctx.handle, int(nsteps)), "sem_step", ctx)


def sem_run(ctx: Ctx, nsteps: int, record: bool = True, out=None):
    seis = None
    if record and ctx.nrec:
        shape = (ctx.nrec, 3, nsteps) if ctx.shots == 1 else (ctx.shots, ctx.nrec, 3, nsteps)
        seis = out if out is not None else np.empty(shape, dtype=np.float32)
        if seis.dtype != np.float32 or not seis.flags.c_contiguous or seis.size != int(np.prod(shape)):
            raise ValueError("out must be a contiguous float32 [shots][nrec][3][nsteps] array")
    _check(lib().sem_run(ctx.handle, int(nsteps), seis.ctypes.data_as(_P) if seis is not None else None),
           "sem_run", ctx)
    return seis


def sem_run_dev(ctx: Ctx, nsteps: int, seis_dev=None):
    _check(lib().sem_run_dev(ctx.handle, int(nsteps), _dev(seis_dev, ctx.shots * ctx.nrec * 3 * nsteps, ctx)),
           "sem_run_dev", ctx)


def sem_run_snapshots(ctx: Ctx, nsteps: int, u_dev):
    n = 3 * ctx.nglob * ctx.shots * int(nsteps)
    _check(lib().sem_run_snapshots(ctx.handle, int(nsteps), _dev(u_dev, n, ctx)), "sem_run_snapshots", ctx)


def sem_run_record_snapshots(ctx: Ctx, nsteps: int, seis_dev, u_dev):
    n = 3 * ctx.nglob * ctx.shots * int(nsteps)
    ns = ctx.shots * ctx.nrec * 3 * int(nsteps)
    seis_ptr = _dev(seis_dev, ns, ctx) if seis_dev is not None else None
    _check(lib().sem_run_record_snapshots(ctx.handle, int(nsteps), seis_ptr, _dev(u_dev, n, ctx)),
           "sem_run_record_snapshots", ctx)


def sem_check_finite(ctx: Ctx):
    _check(lib().sem_check_finite(ctx.handle), "sem_check_finite", ctx)


def sem_apply_stiffness(ctx: Ctx, u_dev, f_dev):
    n = 3 * ctx.nglob
    _check(lib().sem_apply_stiffness(ctx.handle, _dev(u_dev, n, ctx), _dev(f_dev, n, ctx)), "sem_apply_stiffness", ctx)


def sem_apply_stiffness_strided(ctx: Ctx, u_dev, f_dev, node_stride: int):
    n = node_stride * ctx.nglob
    _check(lib().sem_apply_stiffness_strided(ctx.handle, _dev(u_dev, n, ctx), _dev(f_dev, n, ctx), int(node_stride)),
           "sem_apply_stiffness_strided", ctx)


def sem_energy(ctx: Ctx):
    out = np.zeros(2)
    _check(lib().sem_energy(ctx.handle, out.ctypes.data_as(_P)), "sem_energy", ctx)
    return float(out[0]), float(out[1])


def sem_energy_noalloc(ctx: Ctx, u_dev, v_dev, f_dev, nglob: int | None = None):
    """Energy sums from caller-owned device arrays with no device allocation (see sem.h)."""
    n = ctx.nglob if nglob is None else int(nglob)
    out = np.zeros(2)
    m = 3 * min(n, ctx.nglob)
    _check(lib().sem_energy_noalloc(ctx.handle, n, _dev(u_dev, m, ctx), _dev(v_dev, m, ctx), _dev(f_dev, m, ctx),
                                    out.ctypes.data_as(_P)), "sem_energy_noalloc", ctx)
    return float(out[0]), float(out[1])


def sem_adjoint_begin(ctx: Ctx):
    _check(lib().sem_adjoint_begin(ctx.handle), "sem_adjoint_begin", ctx)


def sem_adjoint_step(ctx: Ctx, G_dev=None):
    _check(lib().sem_adjoint_step(ctx.handle, _dev(G_dev, 3 * ctx.nrec, ctx)), "sem_adjoint_step", ctx)


def sem_adjoint_accumulate(ctx: Ctx, u_lo, u_mid, u_hi):
    n = 3 * ctx.nglob
    _check(lib().sem_adjoint_accumulate(ctx.handle, _dev(u_lo, n, ctx), _dev(u_mid, n, ctx), _dev(u_hi, n, ctx)),
           "sem_adjoint_accumulate", ctx)


def sem_adjoint_gradients(ctx: Ctx):
    shape = (ctx.nspec, ctx.ngll ** 3)
    outs = [np.empty(shape) for _ in range(3)]
    _check(lib().sem_adjoint_gradients(ctx.handle, *[o.ctypes.data_as(_P) for o in outs]), "sem_adjoint_gradients",
           ctx)
    return tuple(outs)


def sem_adjoint_segment(ctx: Ctx, count: int, G_dev, u_dev):
    _check(lib().sem_adjoint_segment(ctx.handle, int(count), _dev(G_dev, 3 * ctx.nrec * int(count), ctx),
                                     _dev(u_dev, 3 * ctx.nglob * (int(count) + 2), ctx)), "sem_adjoint_segment", ctx)


def sem_autotune(ctx: Ctx, reps: int = 5):
    """Times both contraction forms on this context and keeps the faster; returns
    (ms per sweep [line owners, per point], chosen form 1 or 2)."""
    ms = np.zeros(2)
    choice = ctypes.c_int(0)
    _check(lib().sem_autotune(ctx.handle, int(reps), ms.ctypes.data_as(_P), ctypes.byref(choice)), "sem_autotune", ctx)
    return ms, choice.value


def sem_profile_steps(ctx: Ctx, nsteps: int):
    """Runs nsteps time steps launched one by one with CUDA events around each force sweep;
    returns (mean ms of the sweep per step, mean ms of the rest per step)."""
    ms = np.zeros(2)
    _check(lib().sem_profile_steps(ctx.handle, int(nsteps), ms.ctypes.data_as(_P)), "sem_profile_steps", ctx)
    return float(ms[0]), float(ms[1])


def patch_shape_code(bx: int, by: int, bz: int) -> int:
    """SEM_OPT_PATCH_SHAPE value of a bx x by x bz brick."""
    return int(bx) | (int(by) << 8) | (int(bz) << 16)


def sem_tune_patch_shape(ctx: Ctx, ibool, nglob: int, rho, vp, vs, xyz=None, ctrl=None, reps: int = 5):
    """Times every brick shape this order's patch kernel can take on the given mesh and
    material (per-point positions xyz or trilinear corners ctrl) and sets the fastest for
    the context's next sem_set_mesh; returns [((bx, by, bz), ms per step's sweep)] and the
    chosen (bx, by, bz)."""
    if (xyz is None) == (ctrl is None):
        raise ValueError("give exactly one of xyz (per-point positions) and ctrl (corners)")
    n3 = ctx.ngll ** 3
    ib, pi = _host(ibool, np.int32)
    nspec = ib.size // n3
    if xyz is not None:
        pts, px = _host(xyz, np.float64, (nspec, n3, 3))
        pc = None
    else:
        cts, pc = _host(ctrl, np.float64, (nspec, 8, 3))
        px = None
    mats = [_host(m, np.float32, (nspec, n3)) for m in (rho, vp, vs)]
    cap = 64
    shapes = np.zeros(cap, dtype=np.int32)
    ms = np.zeros(cap)
    count = ctypes.c_int(0)
    _check(lib().sem_tune_patch_shape(ctx.handle, nspec, int(nglob), pi, px, pc, *(m[1] for m in mats), int(reps),
                                      cap, shapes.ctypes.data_as(_P), ms.ctypes.data_as(_P), ctypes.byref(count)),
           "sem_tune_patch_shape", ctx)
    dec = lambda v: (int(v) & 0xFF, (int(v) >> 8) & 0xFF, (int(v) >> 16) & 0xFF)  # noqa: E731
    rows = [(dec(shapes[k]), float(ms[k])) for k in range(min(cap, count.value))]
    return rows, min(rows, key=lambda r: r[1])[0]


class Group:
    """Several contexts stepped together (see sem_group_step in sem.h)."""

    def __init__(self, ctxs):
        self.ctxs = list(ctxs)  # keeps the contexts alive
        arr = (_P * len(self.ctxs))(*[c.handle for c in self.ctxs])
        out = _P()
        code = lib().sem_group_create(ctypes.byref(out), len(self.ctxs), arr)
        if code != SEM_OK:
            raise SemError(code, "sem_group_create", (lib().sem_group_last_error(None) or b"").decode())
        self.handle = out.value

    def _check(self, code, where):
        if code != SEM_OK:
            raise SemError(code, where, (lib().sem_group_last_error(self.handle) or b"").decode())

    def step(self, nsteps: int):
        self._check(lib().sem_group_step(self.handle, int(nsteps)), "sem_group_step")

    def sync(self):
        self._check(lib().sem_group_sync(self.handle), "sem_group_sync")

    def set_option(self, option: int, value: int):
        self._check(lib().sem_group_set_option(self.handle, int(option), int(value)), "sem_group_set_option")

    def info(self) -> dict:
        out = (ctypes.c_int * 2)()
        self._check(lib().sem_group_info(self.handle, out), "sem_group_info")
        return {"persistent": bool(out[0]), "sweep_launches": int(out[1])}

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().sem_group_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def sem_sync(ctx: Ctx):
    _check(lib().sem_sync(ctx.handle), "sem_sync", ctx)


def sem_info(ctx: Ctx) -> dict:
    out = np.zeros(9, dtype=np.int64)
    _check(lib().sem_info(ctx.handle, out.ctypes.data_as(_P)), "sem_info", ctx)
    keys = ("nspec", "nglob", "ngll", "ncolors", "steps", "device_bytes", "shots", "slabs", "launches")
    return {k: int(v) for k, v in zip(keys, out)}


def sem_node_order(ctx: Ctx) -> np.ndarray:
    """perm[i] = caller node of the solver's internal node i."""
    out = np.zeros(ctx.nglob, dtype=np.int32)
    _check(lib().sem_node_order(ctx.handle, out.ctypes.data_as(_P)), "sem_node_order", ctx)
    return out


def sem_patch_info(ctx: Ctx) -> dict:
    out = np.zeros(8, dtype=np.int64)
    _check(lib().sem_patch_info(ctx.handle, out.ctypes.data_as(_P)), "sem_patch_info", ctx)
    keys = ("patches", "colors", "max_nodes", "tables", "bx", "by", "bz", "assembly")
    return {k: int(v) for k, v in zip(keys, out)}


def sem_patch_plan(ngll: int, ibool, nglob: int):
    """Host-only: (patch of every element, colour of every patch, info dict) of the patches
    the library builds for this mesh."""
    ib = np.ascontiguousarray(ibool, dtype=np.int32)
    nspec = ib.size // (ngll ** 3)
    patch_of = np.zeros(nspec, dtype=np.int32)
    color_of = np.full(nspec, -1, dtype=np.int32)
    info = np.zeros(7, dtype=np.int64)
    _check(lib().sem_patch_plan(int(ngll), int(nspec), int(nglob), ib.ctypes.data_as(_P),
                                patch_of.ctypes.data_as(_P), color_of.ctypes.data_as(_P),
                                info.ctypes.data_as(_P)), "sem_patch_plan")
    keys = ("patches", "colors", "max_nodes", "tables", "bx", "by", "bz")
    d = {k: int(v) for k, v in zip(keys, info)}
    return patch_of, color_of[:d["patches"]], d


def sem_color_counts(ctx: Ctx) -> np.ndarray:
    nc = sem_info(ctx)["ncolors"]
    out = np.zeros(nc, dtype=np.int32)
    _check(lib().sem_color_counts(ctx.handle, out.ctypes.data_as(_P)), "sem_color_counts", ctx)
    return out


def sem_last_error(ctx: Ctx | None = None) -> str:
    return (lib().sem_last_error(ctx.handle if ctx is not None else None) or b"").decode(errors="replace")


@dataclass
class Setup:
    """A context set up for a workload: located sources/receivers and the time step."""

    ctx: Ctx
    dt: float
    src_nodes: np.ndarray
    rec_nodes: np.ndarray


def setup_workload(workload, device: int = 0, stream=None, dt: float | None = None,
                   src_nodes=None, rec_nodes=None) -> Setup:
    """Create a context and issue the set-up calls for a ``inputs.Workload`` in order:
    mesh, material, dt (the library's CFL suggestion unless given), node location
    (unless given), sources, receivers, zero state."""
    m = workload.mesh
    ctx = sem_create(m.ngll, device, stream)
    sem_set_mesh_corners(ctx, m.ibool, m.ctrl, m.nglob)
    sem_set_material(ctx, workload.rho, workload.vp, workload.vs)
    if dt is None:
        dt = sem_suggest_dt(ctx, workload.courant)
    sem_set_dt(ctx, dt)
    if src_nodes is None:
        src_nodes = sem_locate_nodes(ctx, workload.source_xyz)
    if rec_nodes is None:
        surf = m.lengths[2] if workload.receiver_surface_only else None
        rec_nodes = sem_locate_nodes(ctx, workload.receiver_xyz, surf)
    sem_set_source_nodes(ctx, src_nodes, workload.source_force, workload.f0, workload.t0)
    sem_set_receiver_nodes(ctx, rec_nodes)
    sem_set_state(ctx)
    return Setup(ctx, dt, np.asarray(src_nodes), np.asarray(rec_nodes))


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


class Solver:
    """Object form of the C ABI for one model on one GPU: owns a context, and each method
    issues the calls of include/sem.h in their required order. Host data are numpy arrays;
    wavefields may also be CUDA tensors (then the *_dev calls are used, with no host copy)."""

    def __init__(self, ngll: int, ibool, ctrl, nglob: int, rho, vp, vs, device: int = 0, stream=None,
                 courant: float = 0.4, dt: float | None = None):
        self.ctx = sem_create(ngll, device, stream)
        sem_set_mesh_corners(self.ctx, ibool, ctrl, nglob)
        sem_set_material(self.ctx, rho, vp, vs)
        self.dt = sem_suggest_dt(self.ctx, courant) if dt is None else float(dt)
        sem_set_dt(self.ctx, self.dt)
        self.top = float(np.max(np.asarray(ctrl)[..., 2]))

    @classmethod
    def from_workload(cls, workload, device: int = 0, stream=None, dt: float | None = None) -> "Solver":
        """A solver for an ``inputs.Workload`` with its sources and receivers located (nearest
        nodes; receivers on the top face when the workload asks for that) and a zero state."""
        m = workload.mesh
        s = cls(m.ngll, m.ibool, m.ctrl, m.nglob, workload.rho, workload.vp, workload.vs, device, stream,
                workload.courant, dt)
        s.set_sources(workload.source_xyz, workload.source_force, workload.f0, workload.t0)
        s.set_receivers(workload.receiver_xyz, surface=workload.receiver_surface_only)
        s.set_state()
        return s

    def locate(self, xyz, surface: bool = False) -> np.ndarray:
        """Nearest global node of each point (on the top face with ``surface``)."""
        return sem_locate_nodes(self.ctx, xyz, self.top if surface else None)

    def set_sources(self, xyz, force=None, f0: float = 10.0, t0: float = 0.12, moment=None,
                    snap: bool = True, shot=None):
        """Point forces (or moment tensors) at xyz [n][3]: on the nearest nodes with ``snap``
        (point forces only), else spread over the element that holds each point."""
        if snap and moment is None:
            nodes = self.locate(xyz)
            if shot is None:
                sem_set_source_nodes(self.ctx, nodes, force, f0, t0)
            else:
                sem_set_shot_sources(self.ctx, shot, nodes, force, f0, t0)
        else:
            sem_set_shot_sources_at(self.ctx, shot, xyz, force=force, moment=moment, f0=f0, t0=t0)

    def set_receivers(self, xyz, surface: bool = False) -> np.ndarray:
        nodes = self.locate(xyz, surface)
        sem_set_receiver_nodes(self.ctx, nodes)
        return nodes

    def set_shots(self, nshots: int):
        sem_set_shots(self.ctx, nshots)

    def set_state(self, u=None, v=None, a=None):
        if any(_is_cuda(x) for x in (u, v, a)):
            sem_set_state_dev(self.ctx, u, v, a)
        else:
            sem_set_state(self.ctx, u, v, a)

    def state(self):
        """(u, v, a) as host arrays."""
        return sem_get_state(self.ctx)

    def step(self, nsteps: int):
        sem_step(self.ctx, nsteps)

    def run(self, nsteps: int, seis_dev=None):
        """Advance and record: host seismograms returned, or into a CUDA tensor."""
        if seis_dev is not None:
            sem_run_dev(self.ctx, nsteps, seis_dev)
            return seis_dev
        return sem_run(self.ctx, nsteps)

    def apply_stiffness(self, u_dev, f_dev):
        sem_apply_stiffness(self.ctx, u_dev, f_dev)

    def energy(self):
        return sem_energy(self.ctx)

    def sync(self):
        sem_sync(self.ctx)
