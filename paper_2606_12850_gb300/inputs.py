"""Seeded synthetic inputs: structured hexahedral meshes, material tables, source and
receiver positions, random wavefields.

This module is shared by the tests, the benchmark and the CUDA path's callers. It holds
none of the spectral-element arithmetic: no GLL points, no Jacobians, no moduli, no mass,
no time stepping. It only lays out integer lattices (the local-to-global map ``ibool``),
the eight corner vertices of each hexahedron, per-point material *inputs* (rho, vp, vs)
and physical positions. Each consumer (the FP64 oracle, the CUDA library) derives
everything else on its own.

Conventions (the CUDA library's ``include/sem.h`` states the same):

* local GLL point index ``p = i + n*j + n*n*k`` with ``n = ngll``; ``i`` runs along xi
  (the x axis of the structured lattice), ``j`` along eta (y), ``k`` along zeta (z);
* ``ibool`` is int32 ``[nspec][ngll**3]``, 0-based, ``i`` fastest;
* element corners ``ctrl`` are float64 ``[nspec][8][3]``; corner ``c = a + 2*b + 4*d``
  sits at reference coordinates ``(xi, eta, zeta) = (2a-1, 2b-1, 2d-1)``;
* elements are numbered ``e = ex + nx*(ey + ny*ez)``;
* global lattice node ``(gx, gy, gz)`` gets index ``gx + Gx*(gy + Gy*gz)`` with
  ``G = n_elem*(ngll-1) + 1`` per axis, or ``n_elem*(ngll-1)`` when periodic
  (the lattice index wraps modulo ``G``).

The workloads follow the paper's experiments (Sec. V-C: homogeneous media, Ricker point
source, stations at the surface) and the configurations the project measures: a
homogeneous 8x8x8 cube of side 1 km at NGLL=5, a three-layer jittered cube of side 4 km
with 256 GLL intervals per side, many shots on a 48^3 layered cube, the layered cube with a
Gaussian velocity anomaly (sensitivity kernels), and the 16^3 layered medium of the
learned surrogate with random moment-tensor sources. Random numbers come from splitmix64
(uniform) and the Box-Muller transform (normal), seeded.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """``count`` successive outputs of the splitmix64 generator (Steele, Lea and Flood,
    OOPSLA 2014) started from ``seed + stream * 2**32``; returns uint64."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    base = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + gamma * idx
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z & _MASK64


def uniform(seed: int, shape, low: float = 0.0, high: float = 1.0, stream: int = 0) -> np.ndarray:
    """Seeded i.i.d. U(low, high) doubles from splitmix64 (top 53 bits)."""
    shape = tuple(np.atleast_1d(shape).tolist()) if not isinstance(shape, tuple) else shape
    count = int(np.prod(shape)) if len(shape) else 1
    bits = splitmix64(seed, count, stream) >> np.uint64(11)
    u01 = bits.astype(np.float64) * (1.0 / 9007199254740992.0)
    return (low + (high - low) * u01).reshape(shape)


def normal(seed: int, shape, stream: int = 0) -> np.ndarray:
    """Seeded i.i.d. N(0, 1) doubles by the Box-Muller transform of two splitmix64 uniforms."""
    shape = tuple(np.atleast_1d(shape).tolist()) if not isinstance(shape, tuple) else shape
    count = int(np.prod(shape)) if len(shape) else 1
    u1 = uniform(seed, (count,), stream=2 * stream + 1)
    u2 = uniform(seed, (count,), stream=2 * stream + 2)
    u1 = np.where(u1 > 0.0, u1, 2.0 ** -53)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)


@dataclass
class HexMesh:
    """A structured conforming hexahedral mesh given as corner vertices plus ``ibool``."""

    nx: int
    ny: int
    nz: int
    ngll: int
    lengths: tuple
    periodic: bool
    ibool: np.ndarray  # int32 [nspec][ngll^3]
    ctrl: np.ndarray  # float64 [nspec][8][3]
    nglob: int
    elem_ijk: np.ndarray  # int64 [nspec][3] lattice position (ex, ey, ez)

    @property
    def nspec(self) -> int:
        return self.ibool.shape[0]

    @property
    def nlocal(self) -> int:
        return self.ibool.size


def structured_hex_mesh(n, ngll: int, length, jitter: float = 0.0, seed: int = 2606,
                        periodic: bool = False) -> HexMesh:
    """Regular lattice of ``nx*ny*nz`` hexahedra over ``[0,Lx]x[0,Ly]x[0,Lz]``.

    ``jitter`` > 0 displaces every interior lattice vertex by i.i.d. U(-jitter*h, jitter*h)
    per axis (h = element edge along that axis); boundary vertices stay put, so the
    domain is still the box. ``periodic`` wraps the global numbering (no jitter allowed:
    corner coordinates stay per element, so a wrapped element keeps its true shape).
    """
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    Lx, Ly, Lz = (length,) * 3 if np.isscalar(length) else tuple(float(v) for v in length)
    if ngll < 2:
        raise ValueError("ngll must be >= 2")
    if periodic and jitter:
        raise ValueError("jitter is only defined for non-periodic meshes")
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    N = ngll - 1

    # vertex lattice, [vz][vy][vx][3]
    vx = np.arange(nx + 1) * hx
    vy = np.arange(ny + 1) * hy
    vz = np.arange(nz + 1) * hz
    verts = np.stack(np.meshgrid(vx, vy, vz, indexing="ij"), axis=-1).transpose(2, 1, 0, 3).copy()
    verts[:, :, -1, 0] = Lx  # exact box faces, no rounding drift
    verts[:, -1, :, 1] = Ly
    verts[-1, :, :, 2] = Lz
    if jitter:
        d = uniform(seed, (nz + 1, ny + 1, nx + 1, 3), -jitter, jitter)
        d *= np.array([hx, hy, hz])
        interior = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        verts[interior] += d[interior]

    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    nspec = nx * ny * nz
    ctrl = np.empty((nspec, 8, 3))
    for c in range(8):
        a, b, d = c & 1, (c >> 1) & 1, (c >> 2) & 1
        ctrl[:, c, :] = verts[ez + d, ey + b, ex + a]

    if periodic:
        Gx, Gy, Gz = nx * N, ny * N, nz * N
    else:
        Gx, Gy, Gz = nx * N + 1, ny * N + 1, nz * N + 1
    kk, jj, ii = np.meshgrid(np.arange(ngll), np.arange(ngll), np.arange(ngll), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()  # p = i + n j + n^2 k order
    gx = (ex[:, None] * N + ii[None, :]) % Gx
    gy = (ey[:, None] * N + jj[None, :]) % Gy
    gz = (ez[:, None] * N + kk[None, :]) % Gz
    ibool = (gx + Gx * (gy + Gy * gz)).astype(np.int32)
    elem_ijk = np.stack([ex, ey, ez], axis=1)
    return HexMesh(nx, ny, nz, ngll, (Lx, Ly, Lz), periodic, ibool, ctrl, Gx * Gy * Gz, elem_ijk)


def bent_map(x: np.ndarray, lengths, amplitude=(0.15, 0.10, 0.12)) -> np.ndarray:
    """A smooth polynomial bending of the box [0,Lx]x[0,Ly]x[0,Lz] onto a curved solid, for
    meshes whose elements are not trilinear: in units of the box, (x, y, z) ->
    (x + a y^2, y + b z^2, z + c x^2) (quadratic in each coordinate, so a GLL interpolant of
    degree >= 2 reproduces it exactly; the Jacobian determinant is 1 + 8 a b c x y z > 0 and
    the image has volume (1 + a b c) Lx Ly Lz). ``x`` is [..., 3] physical coordinates."""
    L = np.asarray(lengths, dtype=np.float64)
    a, b, c = amplitude
    s = np.asarray(x, dtype=np.float64) / L
    out = np.stack([s[..., 0] + a * s[..., 1] ** 2, s[..., 1] + b * s[..., 2] ** 2, s[..., 2] + c * s[..., 0] ** 2],
                   axis=-1)
    return out * L


def per_point(mesh: HexMesh, per_element: np.ndarray) -> np.ndarray:
    """Broadcast a per-element value to every local GLL point, float32 [nspec][ngll^3]."""
    return np.repeat(np.asarray(per_element, dtype=np.float32)[:, None], mesh.ibool.shape[1], axis=1)


@dataclass
class Workload:
    """Everything a run needs, as plain inputs (no derived quantities)."""

    name: str
    mesh: HexMesh
    rho: np.ndarray  # float32 [nspec][ngll^3], kg/m^3
    vp: np.ndarray  # float32, m/s
    vs: np.ndarray  # float32, m/s
    source_xyz: np.ndarray  # float64 [nsrc][3], m
    source_force: np.ndarray  # float64 [nsrc][3], N
    f0: float  # Ricker dominant frequency, Hz
    t0: float  # Ricker delay, s
    receiver_xyz: np.ndarray  # float64 [nrec][3]
    nsteps: int
    courant: float
    receiver_surface_only: bool = False
    extra: dict = field(default_factory=dict)


def homogeneous_cube(n: int = 8, ngll: int = 5, side: float = 1000.0, rho: float = 2500.0,
                     vp: float = 3000.0, vs: float = 1730.0, nsteps: int = 200) -> Workload:
    """Homogeneous cube, free surface on all faces, Ricker 10 Hz +z point force of 1e10 N at
    the centre (a lattice vertex), eight receivers on the top face at x in
    {1,3,5,7}/8 * side and y in {3,5}/8 * side, Courant number 0.4."""
    mesh = structured_hex_mesh(n, ngll, side)
    ones = np.ones(mesh.nspec)
    xs = np.array([1, 3, 5, 7]) * side / 8.0
    ys = np.array([3, 5]) * side / 8.0
    rec = np.array([[x, y, side] for y in ys for x in xs])
    f0 = 10.0
    return Workload(
        name=f"homogeneous cube {n}^3 hex, NGLL={ngll}, {side / 1000:g} km",
        mesh=mesh, rho=per_point(mesh, rho * ones), vp=per_point(mesh, vp * ones),
        vs=per_point(mesh, vs * ones),
        source_xyz=np.array([[side / 2, side / 2, side / 2]]),
        source_force=np.array([[0.0, 0.0, 1.0e10]]), f0=f0, t0=1.2 / f0,
        receiver_xyz=rec, nsteps=nsteps, courant=0.4)


LAYERS = (  # (vp, rho) from the bottom layer up; vs = vp / 1.73
    (5000.0, 3000.0),
    (3500.0, 2600.0),
    (2000.0, 2200.0),
)

# elements per side that keep 256 GLL intervals per side (fixed points per wavelength)
LAYERED_ELEMS = {3: 128, 5: 64, 7: 43, 9: 32}


def layered_cube(ngll: int = 5, n: int | None = None, side: float = 4000.0, jitter: float = 0.1,
                 seed: int = 2606, nsteps: int = 1000, nrec_side: int = 16) -> Workload:
    """Three horizontal layers (vp 5000/3500/2000 m/s from the bottom up, vs = vp/1.73,
    rho 3000/2600/2200 kg/m^3) with interfaces at element layers floor(n/3) and
    floor(2n/3); interior vertices jittered by up to 10 % of the element size; Ricker
    10 Hz +z point force at the centre; ``nrec_side**2`` receivers on the top face at
    ((i+1/2)/m * side, (j+1/2)/m * side), to be snapped to surface nodes by the caller."""
    if n is None:
        n = LAYERED_ELEMS.get(ngll, 64)
    mesh = structured_hex_mesh(n, ngll, side, jitter=jitter, seed=seed)
    ez = mesh.elem_ijk[:, 2]
    layer = np.where(ez < n // 3, 0, np.where(ez < (2 * n) // 3, 1, 2))
    vp_e = np.array([LAYERS[l][0] for l in range(3)])[layer]
    rho_e = np.array([LAYERS[l][1] for l in range(3)])[layer]
    m = nrec_side
    rec = np.array([[(i + 0.5) / m * side, (j + 0.5) / m * side, side]
                    for j in range(m) for i in range(m)])
    f0 = 10.0
    return Workload(
        name=f"three-layer jittered cube {n}^3 hex, NGLL={ngll}, {side / 1000:g} km",
        mesh=mesh, rho=per_point(mesh, rho_e), vp=per_point(mesh, vp_e),
        vs=per_point(mesh, vp_e / 1.73),
        source_xyz=np.array([[side / 2, side / 2, side / 2]]),
        source_force=np.array([[0.0, 0.0, 1.0e10]]), f0=f0, t0=1.2 / f0,
        receiver_xyz=rec, nsteps=nsteps, courant=0.4, receiver_surface_only=True)


def perturbed_layered_cube(n: int = 32, ngll: int = 5, amplitude: float = 0.05, seed: int = 2606,
                           nsteps: int = 800, nrec_side: int = 8, side: float = 4000.0) -> Workload:
    """The three-layer jittered cube with a seeded Gaussian velocity anomaly: vp and vs of
    every element are scaled by 1 + amplitude * exp(-|c - x0|^2 / (2 s^2)), c the mean of
    the element's eight corners, x0 uniform in the middle half of the box (seeded) and
    s = side / 8. ``nrec_side**2`` receivers on the top face. The unperturbed material is
    kept in ``extra["background"]`` as (rho, vp, vs)."""
    w = layered_cube(ngll, n=n, side=side, seed=seed, nsteps=nsteps, nrec_side=nrec_side)
    x0 = uniform(seed, (3,), 0.25 * side, 0.75 * side, stream=13)
    sig = side / 8.0
    c = w.mesh.ctrl.mean(axis=1)
    scale = (1.0 + amplitude * np.exp(-np.sum((c - x0) ** 2, axis=1) / (2.0 * sig * sig))).astype(np.float32)
    w.extra["background"] = (w.rho.copy(), w.vp.copy(), w.vs.copy())
    w.extra["anomaly_centre"] = x0
    w.vp = w.vp * scale[:, None]
    w.vs = w.vs * scale[:, None]
    w.name = f"{w.name}, {100 * amplitude:g}% Gaussian velocity anomaly"
    return w


def surrogate_cube(n: int = 16, ngll: int = 5, nrec_side: int = 8, nsteps: int = 1000, f0: float = 0.5,
                   t0: float = 2.0, side: float = 4000.0) -> Workload:
    """The medium of the learned surrogate: the three-layer jittered cube (side 4 km) with
    ``n`` elements per side, ``nrec_side**2`` surface receivers and a Ricker of dominant
    frequency f0 delayed by t0. At 0.5 Hz the shortest S wavelength spans about seven
    element widths at n = 16, so the traces vary smoothly enough with the source position
    for a few thousand runs to sample them. The source term is set per run."""
    w = layered_cube(ngll, n=n, side=side, nsteps=nsteps, nrec_side=nrec_side)
    w.f0, w.t0 = f0, t0
    w.name = f"{w.name}, {nrec_side * nrec_side} surface receivers, Ricker {f0:g} Hz"
    return w


def surrogate_sources(count: int, side: float, seed: int, margin: float = 0.05) -> tuple:
    """Source positions i.i.d. uniform in [margin, 1 - margin]^3 * side and moment tensors
    (Mxx, Myy, Mzz, Mxy, Mxz, Myz) with i.i.d. N(0, 1) entries scaled to unit Euclidean
    norm. Returns (positions [count][3], moments [count][6])."""
    pos = uniform(seed, (count, 3), margin * side, (1.0 - margin) * side, stream=21)
    m = normal(seed, (count, 6), stream=22)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    return pos, m


def random_field(nglob: int, seed: int, scale: float = 1.0, stream: int = 7) -> np.ndarray:
    """Seeded U(-scale, scale) wavefield, float32 [nglob][3]."""
    return uniform(seed, (nglob, 3), -scale, scale, stream=stream).astype(np.float32)


def shot_positions(nshots: int, side: float, seed: int = 3, margin: float = 0.1) -> np.ndarray:
    """Seeded source positions, i.i.d. uniform in [margin, 1 - margin]^3 * side, [nshots][3]."""
    return uniform(seed, (nshots, 3), margin * side, (1.0 - margin) * side, stream=11)


def batched_layered_cube(n: int = 48, ngll: int = 5, nshots: int = 32, seed: int = 2606,
                         shot_seed: int = 3, nsteps: int = 1000) -> tuple:
    """Many shots on one model: the three-layer jittered cube (side 4 km) with ``n`` elements
    per side and ``nshots`` Ricker +z point forces at seeded random positions (one per shot),
    sharing the 16 x 16 surface receivers. Returns (workload, source positions [nshots][3])."""
    w = layered_cube(ngll, n=n, seed=seed, nsteps=nsteps)
    pos = shot_positions(nshots, w.mesh.lengths[0], shot_seed)
    w.name = f"{w.name}, {nshots} shots"
    w.extra["shot_xyz"] = pos
    return w, pos
