"""Plain FP64 CPU oracle of the spectral-element elastic hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product (the CUDA library and its Python binding)
imports, links or runs this file; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do. It shares no code with the
CUDA path: it computes its own GLL basis, geometry, moduli, mass, forces and time stepping
with numpy in float64, from the paper's definitions, and it takes its inputs from the
neutral generator ``paper_2606_12850_gb300.inputs`` (lattices and positions only).

Every function cites the passage of arXiv 2606.12850 ("High-Order Spectral Element Methods
for Wave Propagation on ARM Multicore CPU with SME") it follows, by section. Where the
paper is silent the reading used is stated in the docstring; these readings are:

* Newmark variant: Sec. I and Sec. V-C give the scheme's order (two) and an explicit scheme
  with a diagonal mass matrix; read as the explicit predictor/corrector with beta = 0,
  gamma = 1/2 (equivalent to central differences in displacement).
* Step n advances u^n -> u^{n+1}; the source acts at t_{n+1} = (n+1) dt, and the record of
  step n is u^{n+1}.
* Ricker wavelet R(tau) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0.
* CFL time step dt = C * min_e(dx_min(e) / vp_max(e)), dx_min the smallest distance between
  neighbouring GLL points of element e along a grid line (Sec. IV-B: the spacing shrinks
  as O(N^-2); Sec. V-C: dt = min(dt_CFL, ...)).
* Isotropic Hooke law with the stiffness tensor of Sec. II-B written with
  lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2, kappa = lambda + 2 mu / 3.
* Material sensitivities (not in the paper): the exact gradient of the discrete scheme
  above, by its discrete adjoint.
* Moment-tensor source at a node (not in the paper): f_I = M grad(psi_I)(x_s) with the
  gradient of the lowest-numbered element that holds the node.
* Sources between nodes (not in the paper): tested against the Lagrange basis of the
  lowest-numbered element holding the point, f_I = F psi_I(x_s) for a point force and
  f_I = M grad(psi_I)(x_s) for a moment tensor.

Array conventions: element-local fields are numpy arrays shaped
``(nspec, ..., k, j, i)`` so that flattening the last three axes gives the local point
index ``p = i + n j + n^2 k`` used by ``ibool``; ``hprime[i, l] = l_l'(xi_i)``.

Parity status: every function here is pinned by a CPU test in ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (see each test's docstring).
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------------------
# 1D basis (Sec. II-B, the spectral element method)
# --------------------------------------------------------------------------------------


def legendre(N: int, x):
    """Legendre polynomial P_N and its derivative at x, by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and P'_N from
    (1 - x^2) P'_N = N (P_{N-1} - x P_N) (with the endpoint values N(N+1)/2 * (+-1)^(N+1))."""
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    if N == 0:
        return np.ones_like(x), np.zeros_like(x)
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    dp = np.empty_like(x)
    interior = np.abs(np.abs(x) - 1.0) > 0.0
    dp[interior] = N * (p_prev[interior] - x[interior] * p[interior]) / (1.0 - x[interior] ** 2)
    end = ~interior
    dp[end] = 0.5 * N * (N + 1) * np.sign(x[end]) ** (N + 1)
    return p, dp


def gll_points_weights(N: int):
    """The N+1 Gauss-Lobatto-Legendre nodes xi_0 < ... < xi_N on [-1, 1] and their weights
    (Sec. II-B). Nodes: -1, 1 and the roots of P'_N, found by Newton's method on P'_N
    started from the Chebyshev-Gauss-Lobatto points. Weights: w_i = 2 / (N (N+1) P_N(xi_i)^2)."""
    if N < 1:
        raise ValueError("polynomial degree N must be >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(100):
        # P'_N and P''_N at the interior nodes: (1-x^2) P'' = 2x P' - N(N+1) P
        p, dp = legendre(N, x[1:-1])
        ddp = (2 * x[1:-1] * dp - N * (N + 1) * p) / (1 - x[1:-1] ** 2)
        step = dp / ddp
        x[1:-1] -= step
        if np.all(np.abs(step) < 1e-16):
            break
    x[0], x[-1] = -1.0, 1.0
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN ** 2)
    return x, w


def lagrange_basis(xi: np.ndarray, x) -> np.ndarray:
    """l_i(x) for the nodes xi, by the product formula of Sec. II-B; returns [len(x), N+1]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(xi)
    out = np.ones((len(x), n))
    for i in range(n):
        for m in range(n):
            if m != i:
                out[:, i] *= (x - xi[m]) / (xi[i] - xi[m])
    return out


def lagrange_derivative_matrix(xi: np.ndarray) -> np.ndarray:
    """hprime[i, l] = l_l'(xi_i): the derivative of the product formula of Sec. II-B,
    l_l'(x) = sum_{m != l} 1/(xi_l - xi_m) prod_{q != l, m} (x - xi_q)/(xi_l - xi_q),
    evaluated at the nodes. This is the 1D differentiation matrix that turns the
    xi-derivative into small matrix products (Sec. II-B)."""
    n = len(xi)
    H = np.zeros((n, n))
    for i in range(n):
        for l in range(n):
            total = 0.0
            for m in range(n):
                if m == l:
                    continue
                term = 1.0 / (xi[l] - xi[m])
                for q in range(n):
                    if q != l and q != m:
                        term *= (xi[i] - xi[q]) / (xi[l] - xi[q])
                total += term
            H[i, l] = total
    return H


class Basis:
    """GLL nodes, weights and derivative matrix for NGLL = N+1 points per direction."""

    def __init__(self, ngll: int):
        self.ngll = ngll
        self.xi, self.w = gll_points_weights(ngll - 1)
        self.hprime = lagrange_derivative_matrix(self.xi)


# --------------------------------------------------------------------------------------
# Geometry: trilinear hexahedra (Sec. II-B: hexahedral elements on the reference cube)
# --------------------------------------------------------------------------------------

_CORNER_SIGNS = np.array([[2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1]
                          for c in range(8)], dtype=np.float64)


def trilinear_shape(xi, eta, zeta):
    """The eight trilinear shape functions N_c and their reference derivatives
    dN_c/d(xi, eta, zeta); corner c sits at (2a-1, 2b-1, 2d-1), c = a + 2b + 4d."""
    s = _CORNER_SIGNS
    fx = 1 + s[:, 0] * xi
    fy = 1 + s[:, 1] * eta
    fz = 1 + s[:, 2] * zeta
    N = fx * fy * fz / 8.0
    dN = np.stack([s[:, 0] * fy * fz, fx * s[:, 1] * fz, fx * fy * s[:, 2]], axis=1) / 8.0
    return N, dN  # [8], [8][3]


def element_geometry(ctrl: np.ndarray, basis: Basis):
    """Physical position, inverse Jacobian and Jacobian determinant at every GLL point of
    every element, from the analytic derivatives of the trilinear map
    x(xi, eta, zeta) = sum_c N_c X_c.

    Returns ``xyz [nspec,3,k,j,i]``, ``dxi_dx [nspec,3(r),3(d),k,j,i]`` with
    dxi_dx[:, r, d] = d xi_r / d x_d, and ``jac [nspec,k,j,i]`` = det(dx/dxi)."""
    n = basis.ngll
    nspec = ctrl.shape[0]
    xyz = np.empty((nspec, 3, n, n, n))
    dxi_dx = np.empty((nspec, 3, 3, n, n, n))
    jac = np.empty((nspec, n, n, n))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                N, dN = trilinear_shape(basis.xi[i], basis.xi[j], basis.xi[k])
                xyz[:, :, k, j, i] = np.einsum("c,ecd->ed", N, ctrl)
                # A[e, d, r] = d x_d / d xi_r
                A = np.einsum("cr,ecd->edr", dN, ctrl)
                jac[:, k, j, i] = np.linalg.det(A)
                dxi_dx[:, :, :, k, j, i] = np.linalg.inv(A)  # inv(A)[r, d] = d xi_r / d x_d
    return xyz, dxi_dx, jac


def isoparametric_geometry(xyz: np.ndarray, basis: Basis):
    """Inverse Jacobian and determinant at every GLL point from the positions of the GLL
    points themselves (Sec. II-B: every element is a map of the reference cube, here the
    map interpolated by the same tensor-product Lagrange basis as the displacement):
    dx_d/dxi_r at a point is the sum over l of l_l'(xi) times x_d at the l-th point of the
    grid line through it along direction r; then numpy's 3x3 inverse and determinant.

    ``xyz [nspec,3,k,j,i]``; returns ``dxi_dx [nspec,3(r),3(d),k,j,i]`` and ``jac
    [nspec,k,j,i]`` as element_geometry does."""
    H = basis.hprime
    A = np.empty(xyz.shape[:2] + (3,) + xyz.shape[2:])  # [e, d, r, k, j, i] = dx_d / dxi_r
    A[:, :, 0] = np.einsum("il,edkjl->edkji", H, xyz)
    A[:, :, 1] = np.einsum("jl,edkli->edkji", H, xyz)
    A[:, :, 2] = np.einsum("kl,edlji->edkji", H, xyz)
    Am = np.moveaxis(A, (1, 2), (4, 5))  # [e, k, j, i, d, r]
    jac = np.linalg.det(Am)
    inv = np.linalg.inv(Am)  # [e, k, j, i, r, d] = dxi_r / dx_d
    return np.moveaxis(inv, (4, 5), (1, 2)), jac


def global_coordinates(xyz: np.ndarray, ibool: np.ndarray, nglob: int) -> np.ndarray:
    """Coordinates of every global node, read from any local point that maps to it."""
    nspec = xyz.shape[0]
    out = np.full((nglob, 3), np.nan)
    out[ibool.reshape(-1)] = xyz.reshape(nspec, 3, -1).transpose(0, 2, 1).reshape(-1, 3)
    return out


# --------------------------------------------------------------------------------------
# Material, mass (Sec. II-B: elastic wave equation, Hooke's law, diagonal mass)
# --------------------------------------------------------------------------------------


def moduli(rho, vp, vs):
    """Isotropic moduli (kappa, mu) from density and wave speeds, in float64:
    mu = rho vs^2, lambda = rho (vp^2 - 2 vs^2), kappa = lambda + 2/3 mu."""
    rho = np.asarray(rho, dtype=np.float64)
    vp = np.asarray(vp, dtype=np.float64)
    vs = np.asarray(vs, dtype=np.float64)
    mu = rho * vs * vs
    lam = rho * (vp * vp - 2.0 * vs * vs)
    return lam + 2.0 * mu / 3.0, mu


def quadrature_weights_3d(basis: Basis) -> np.ndarray:
    """w_i w_j w_k laid out [k, j, i]."""
    w = basis.w
    return w[:, None, None] * w[None, :, None] * w[None, None, :]


def mass_matrix(rho_kji, jac, ibool, nglob, basis: Basis) -> np.ndarray:
    """Diagonal mass from GLL quadrature of the left-hand side of the weak form (Sec. II-B):
    M_I = sum over local points (e, i, j, k) mapped to I of rho J w_i w_j w_k."""
    contrib = rho_kji * jac * quadrature_weights_3d(basis)[None]
    M = np.zeros(nglob)
    np.add.at(M, ibool.reshape(-1), contrib.reshape(-1))
    return M


# --------------------------------------------------------------------------------------
# Stiffness action (Sec. II-B: matrix-free evaluation of -int grad(w) : T)
# --------------------------------------------------------------------------------------


def element_forces(u_e, dxi_dx, jac, kappa, mu, basis: Basis) -> np.ndarray:
    """Matrix-free element internal forces F = -K_e u_e, in the order of Sec. II-B:

    1. reference derivatives of each displacement component along xi, eta, zeta, each a
       batch of small products with the 1D derivative matrix;
    2. physical gradient by the chain rule, du_c/dx_d = sum_r du_c/dxi_r dxi_r/dx_d;
    3. strain and isotropic stress sigma = lambda tr(eps) I + 2 mu eps (Hooke's law);
    4. fluxes t_{r,c} = J sum_d sigma_{cd} dxi_r/dx_d;
    5. the three transposed products with the GLL weights folded in, which evaluate
       -int grad(w) : sigma by GLL quadrature for every test function w.

    ``u_e`` is [nspec, 3, k, j, i]; returns the same shape."""
    H = basis.hprime
    w = basis.w
    du = np.empty(u_e.shape[:2] + (3,) + u_e.shape[2:])  # [e, c, r, k, j, i]
    du[:, :, 0] = np.einsum("il,eckjl->eckji", H, u_e)
    du[:, :, 1] = np.einsum("jl,eckli->eckji", H, u_e)
    du[:, :, 2] = np.einsum("kl,eclji->eckji", H, u_e)
    grad = np.einsum("ecrkji,erdkji->ecdkji", du, dxi_dx)  # du_c/dx_d
    eps = 0.5 * (grad + grad.transpose(0, 2, 1, 3, 4, 5))
    lam = kappa - 2.0 * mu / 3.0
    tr = eps[:, 0, 0] + eps[:, 1, 1] + eps[:, 2, 2]
    sigma = 2.0 * mu[:, None, None] * eps
    for c in range(3):
        sigma[:, c, c] += lam * tr
    t = jac[:, None, None] * np.einsum("ecdkji,erdkji->erckji", sigma, dxi_dx)  # [e, r, c, ...]
    # -sum over quadrature points q of w_q * t_r,c(q) * d l_p / d xi_r (q)
    F = -(np.einsum("k,j,l,li,eckjl->eckji", w, w, w, H, t[:, 0])
          + np.einsum("k,i,l,lj,eckli->eckji", w, w, w, H, t[:, 1])
          + np.einsum("j,i,l,lk,eclji->eckji", w, w, w, H, t[:, 2]))
    return F


def gather(u: np.ndarray, ibool: np.ndarray, n: int) -> np.ndarray:
    """Element-local copy u_e[e, c, k, j, i] = u[ibool[e, p], c] (the global-to-local map)."""
    nspec = ibool.shape[0]
    return u[ibool].reshape(nspec, n, n, n, 3).transpose(0, 4, 1, 2, 3)


def assemble(F_e: np.ndarray, ibool: np.ndarray, nglob: int) -> np.ndarray:
    """Sum element contributions into global nodes: f[ibool[e, p]] += F_e[e, :, p]."""
    nspec = F_e.shape[0]
    f = np.zeros((nglob, 3))
    np.add.at(f, ibool.reshape(-1), F_e.reshape(nspec, 3, -1).transpose(0, 2, 1).reshape(-1, 3))
    return f


class Model:
    """Mesh + material + basis with every derived array the solver needs (all float64).

    The mesh is ``ctrl`` (trilinear corners [nspec][8][3]; geometry by element_geometry) or,
    with ``points`` [nspec][ngll^3][3] (the position of every local point in local point
    order), any element shape (geometry by isoparametric_geometry; ``ctrl`` may then be None
    and is taken from the corner points)."""

    def __init__(self, ibool, ctrl, nglob, rho, vp, vs, ngll, points=None):
        self.basis = Basis(ngll)
        n = ngll
        self.ngll = n
        self.ibool = np.asarray(ibool)
        self.nspec = self.ibool.shape[0]
        self.nglob = int(nglob)
        if points is None:
            self.ctrl = np.asarray(ctrl, dtype=np.float64)
            self.xyz, self.dxi_dx, self.jac = element_geometry(self.ctrl, self.basis)
        else:
            pts = np.asarray(points, dtype=np.float64).reshape(self.nspec, n, n, n, 3)
            self.xyz = np.ascontiguousarray(np.moveaxis(pts, 4, 1))  # [e, 3, k, j, i]
            self.dxi_dx, self.jac = isoparametric_geometry(self.xyz, self.basis)
            N = n - 1
            corner = [(a * N, b * N, d * N) for d in (0, 1) for b in (0, 1) for a in (0, 1)]
            self.ctrl = np.stack([pts[:, k, j, i, :] for (i, j, k) in corner], axis=1) if ctrl is None \
                else np.asarray(ctrl, dtype=np.float64)
        shape = (self.nspec, n, n, n)
        self.rho = np.asarray(rho, dtype=np.float64).reshape(shape)
        self.vp = np.asarray(vp, dtype=np.float64).reshape(shape)
        self.vs = np.asarray(vs, dtype=np.float64).reshape(shape)
        self.kappa, self.mu = moduli(self.rho, self.vp, self.vs)
        self.mass = mass_matrix(self.rho, self.jac, self.ibool, self.nglob, self.basis)
        self._node_xyz = None

    @property
    def node_xyz(self) -> np.ndarray:
        if self._node_xyz is None:
            self._node_xyz = global_coordinates(self.xyz, self.ibool, self.nglob)
        return self._node_xyz

    def forces(self, u: np.ndarray) -> np.ndarray:
        """f = -K u for a global field u [nglob, 3]."""
        u_e = gather(np.asarray(u, dtype=np.float64), self.ibool, self.ngll)
        F = element_forces(u_e, self.dxi_dx, self.jac, self.kappa, self.mu, self.basis)
        return assemble(F, self.ibool, self.nglob)

    def min_spacing_over_vp(self) -> np.ndarray:
        """Per element: smallest distance between neighbouring GLL points along a grid
        line, divided by the largest vp of the element."""
        x = self.xyz
        d = [np.linalg.norm(np.diff(x, axis=ax), axis=1).reshape(self.nspec, -1).min(axis=1)
             for ax in (2, 3, 4)]
        dx = np.minimum(np.minimum(d[0], d[1]), d[2])
        return dx / self.vp.reshape(self.nspec, -1).max(axis=1)

    def cfl_dt(self, courant: float) -> float:
        """dt = C * min_e(dx_min(e) / vp_max(e))."""
        return float(courant * self.min_spacing_over_vp().min())

    def nearest_nodes(self, points, surface_z: float | None = None) -> np.ndarray:
        """Index of the global node nearest to each point (ties: lowest index). With
        ``surface_z`` only nodes whose z lies within 1e-9 * max(1, |surface_z|) of it are
        candidates (nodes on a flat face, up to the rounding of their positions)."""
        pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
        cand = np.arange(self.nglob)
        if surface_z is not None:
            tol = 1e-9 * max(1.0, abs(surface_z))
            cand = cand[np.abs(self.node_xyz[:, 2] - surface_z) <= tol]
        out = np.empty(len(pts), dtype=np.int64)
        for r, p in enumerate(pts):
            d2 = np.sum((self.node_xyz[cand] - p) ** 2, axis=1)
            out[r] = cand[int(np.argmin(d2))]  # argmin returns the first minimum
        return out


# --------------------------------------------------------------------------------------
# Source and time stepping (Sec. I, Sec. V-C)
# --------------------------------------------------------------------------------------


def ricker(t, f0: float, t0: float):
    """Ricker wavelet with dominant frequency f0 delayed by t0 (Sec. V-C names a Ricker
    source): R = (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2."""
    a = (np.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def moment_tensor_forces(model: Model, node: int, moment) -> tuple:
    """Nodal forces of a moment-tensor point source at global node ``node``: the body force
    -M . grad(delta(x - x_s)) tested against the Lagrange basis of Sec. II-B gives, after
    integration by parts, f_I = M grad(psi_I)(x_s). The gradient is taken in the
    lowest-numbered element that holds the node (a GLL node on an element face has one
    one-sided gradient per element; this is the reading used). ``moment`` =
    (Mxx, Myy, Mzz, Mxy, Mxz, Myz). Returns (nodes [m], forces [m, 3]) for the nodes whose
    basis function has a nonzero gradient at x_s."""
    n = model.ngll
    ib = model.ibool.reshape(model.nspec, -1)
    e = int(np.nonzero(np.any(ib == node, axis=1))[0][0])
    p0 = int(np.nonzero(ib[e] == node)[0][0])
    i0, j0, k0 = p0 % n, (p0 // n) % n, p0 // (n * n)
    mxx, myy, mzz, mxy, mxz, myz = (float(v) for v in moment)
    M = np.array([[mxx, mxy, mxz], [mxy, myy, myz], [mxz, myz, mzz]])
    D = model.dxi_dx[e, :, :, k0, j0, i0]  # D[r, d] = d xi_r / d x_d at the source
    H = model.basis.hprime  # H[a, b] = l_b'(xi_a)
    nodes, forces = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                # d psi_(i,j,k) / d xi_r at (xi_i0, xi_j0, xi_k0): psi = l_i(xi) l_j(eta) l_k(zeta)
                dpsi = np.array([H[i0, i] * (j == j0) * (k == k0),
                                 H[j0, j] * (i == i0) * (k == k0),
                                 H[k0, k] * (i == i0) * (j == j0)], dtype=np.float64)
                if not np.any(dpsi):
                    continue
                grad = dpsi @ D  # d psi / d x_d
                nodes.append(int(ib[e, i + n * (j + n * k)]))
                forces.append(M @ grad)
    return np.array(nodes, dtype=np.int64), np.array(forces)


def lagrange_basis_derivative(xi: np.ndarray, x) -> np.ndarray:
    """l_i'(x) at arbitrary points: the product formula of Sec. II-B differentiated by the
    product rule, l_i'(x) = sum_{m != i} 1/(xi_i - xi_m) prod_{q != i, m} (x - xi_q)/(xi_i - xi_q).
    Returns [len(x), N+1]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(xi)
    out = np.zeros((len(x), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (xi[i] - xi[m]))
            for q in range(n):
                if q != i and q != m:
                    term = term * (x - xi[q]) / (xi[i] - xi[q])
            out[:, i] += term
    return out


def locate_point(model: Model, x, tol: float = 1e-9):
    """Element holding a physical point, and the point's reference coordinates. Elements are
    tried in index order, those whose corner bounding box (widened by ``tol`` times its
    largest side) contains x; for each, the trilinear map x(xi) = sum_c N_c(xi) X_c is
    inverted by Newton's method from the element centre, and the first element whose
    solution lies in [-1 - tol, 1 + tol]^3 is taken (so a point on a shared face goes to the
    lowest-numbered element, the same tie rule as node location). Returns (e, xi[3]) with xi
    clipped to [-1, 1]; ValueError if no element holds x."""
    x = np.asarray(x, dtype=np.float64)
    for e in range(model.nspec):
        X = model.ctrl[e]
        lo, hi = X.min(axis=0), X.max(axis=0)
        pad = tol * float(np.max(hi - lo))
        if np.any(x < lo - pad) or np.any(x > hi + pad):
            continue
        ref = np.zeros(3)
        for _ in range(60):
            N, dN = trilinear_shape(*ref)
            A = X.T @ dN  # A[d, r] = d x_d / d xi_r
            step = np.linalg.solve(A, N @ X - x)
            ref = ref - step
            if np.max(np.abs(step)) < 1e-15 or np.max(np.abs(ref)) > 10.0:
                break
        if np.all(np.abs(ref) <= 1.0 + tol):
            return e, np.clip(ref, -1.0, 1.0)
    raise ValueError(f"point {x} lies outside the mesh")


def point_source_forces(model: Model, x_s, force=None, moment=None) -> tuple:
    """Nodal forces of a point source at an arbitrary position x_s (a reading: the paper's
    sources sit on nodes; between nodes the source is tested against the Lagrange basis of
    Sec. II-B of the element that holds x_s, found by locate_point):
      point force F delta(x - x_s)           ->  f_I = F psi_I(x_s),
      moment tensor -M . grad delta(x - x_s)  ->  f_I = M grad psi_I(x_s),
    with psi_(i,j,k) = l_i(xi) l_j(eta) l_k(zeta) at the reference coordinates of x_s and
    grad psi = (d xi / d x)^T grad_xi psi, d xi / d x the inverse of the analytic trilinear
    Jacobian at x_s. Exactly one of ``force`` (Fx, Fy, Fz) and ``moment`` (Mxx, Myy, Mzz,
    Mxy, Mxz, Myz) is given. Returns (e, xi[3], nodes [m], forces [m, 3]) over the element's
    points whose force is not exactly zero."""
    if (force is None) == (moment is None):
        raise ValueError("give exactly one of force and moment")
    e, ref = locate_point(model, x_s)
    n = model.ngll
    xi = model.basis.xi
    L = [lagrange_basis(xi, ref[r])[0] for r in range(3)]
    dL = [lagrange_basis_derivative(xi, ref[r])[0] for r in range(3)]
    _, dN = trilinear_shape(*ref)
    D = np.linalg.inv(model.ctrl[e].T @ dN)  # D[r, d] = d xi_r / d x_d
    if moment is not None:
        mxx, myy, mzz, mxy, mxz, myz = (float(v) for v in moment)
        M = np.array([[mxx, mxy, mxz], [mxy, myy, myz], [mxz, myz, mzz]])
    ib = model.ibool.reshape(model.nspec, -1)
    nodes, forces = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                if force is not None:
                    f = np.asarray(force, dtype=np.float64) * (L[0][i] * L[1][j] * L[2][k])
                else:
                    dpsi = np.array([dL[0][i] * L[1][j] * L[2][k],
                                     L[0][i] * dL[1][j] * L[2][k],
                                     L[0][i] * L[1][j] * dL[2][k]])
                    f = M @ (dpsi @ D)
                if not np.any(f):
                    continue
                nodes.append(int(ib[e, i + n * (j + n * k)]))
                forces.append(f)
    return e, ref, np.array(nodes, dtype=np.int64), np.array(forces)


def newmark_run(model: Model, dt: float, nsteps: int, u0=None, v0=None, a0=None,
                src_nodes=(), src_force=(), f0: float = 10.0, t0: float = 0.12,
                rec_nodes=(), energy: bool = False):
    """Explicit second-order Newmark time stepping with the diagonal mass (Sec. I, II-B,
    V-C), predictor/corrector with beta = 0, gamma = 1/2. For n = 0 .. nsteps-1:

        u^{n+1} = u^n + dt v^n + dt^2/2 a^n
        a^{n+1} = M^{-1} ( -K u^{n+1} + sum_s F_s R(t_{n+1} - t0) delta_{node s} )
        v^{n+1} = v^n + dt/2 (a^n + a^{n+1})

    with t_{n+1} = (n+1) dt. Records u^{n+1} at the receiver nodes after step n.
    With ``energy`` it also returns E^{n+1/2} = 1/2 v_h^T M v_h + 1/2 (u^{n+1})^T K u^n,
    v_h = (u^{n+1} - u^n)/dt, which the scheme conserves exactly without a source.

    Returns (seis [nrec, 3, nsteps], u, v, a[, energies])."""
    ng = model.nglob
    u = np.zeros((ng, 3)) if u0 is None else np.array(u0, dtype=np.float64)
    v = np.zeros((ng, 3)) if v0 is None else np.array(v0, dtype=np.float64)
    a = np.zeros((ng, 3)) if a0 is None else np.array(a0, dtype=np.float64)
    Minv = 1.0 / model.mass
    src_nodes = np.asarray(src_nodes, dtype=np.int64).reshape(-1)
    src_force = np.asarray(src_force, dtype=np.float64).reshape(-1, 3)
    rec_nodes = np.asarray(rec_nodes, dtype=np.int64).reshape(-1)
    seis = np.zeros((len(rec_nodes), 3, nsteps))
    energies = []
    f_prev = model.forces(u) if energy else None
    for n in range(nsteps):
        u_new = u + dt * v + 0.5 * dt * dt * a
        f = model.forces(u_new)
        if energy:
            vh = (u_new - u) / dt
            energies.append(0.5 * np.sum(model.mass[:, None] * vh * vh) - 0.5 * np.sum(u_new * f_prev))
            f_prev = f
        t = (n + 1) * dt
        fs = f.copy()
        for s, g in enumerate(src_nodes):
            fs[g] += src_force[s] * ricker(t, f0, t0)
        a_new = Minv[:, None] * fs
        v = v + 0.5 * dt * (a + a_new)
        u, a = u_new, a_new
        if len(rec_nodes):
            seis[:, :, n] = u[rec_nodes]
    if energy:
        return seis, u, v, a, np.array(energies)
    return seis, u, v, a


def dispersion_error(w, w_theory, axis: int = -1):
    """Waveform error of Sec. V-C-1: int (w - w_theory)^2 dt / int w_theory^2 dt, as printed
    (a ratio of squared norms, no square root). Uniform samples: the dt cancels."""
    w = np.asarray(w, dtype=np.float64)
    wt = np.asarray(w_theory, dtype=np.float64)
    return np.sum((w - wt) ** 2, axis=axis) / np.sum(wt ** 2, axis=axis)


# --------------------------------------------------------------------------------------
# Convenience: a whole run from a neutral workload description
# --------------------------------------------------------------------------------------


def build_model(workload, elems=None) -> Model:
    """Oracle model of a workload; with ``elems`` only those elements are kept (global
    numbering unchanged), which is exact for forces and mass at any node whose
    elements are all included."""
    m = workload.mesh
    sel = slice(None) if elems is None else np.asarray(elems)
    return Model(m.ibool[sel], m.ctrl[sel], m.nglob, workload.rho[sel], workload.vp[sel],
                 workload.vs[sel], m.ngll)


def elements_touching(ibool: np.ndarray, nodes) -> np.ndarray:
    """Indices of the elements whose ibool row contains any of ``nodes``."""
    return np.nonzero(np.isin(ibool, np.asarray(nodes)).any(axis=1))[0]


def locate_workload(model: Model, workload):
    """Source nodes (nearest node) and receiver nodes (nearest surface node when the
    workload asks for surface receivers)."""
    src = model.nearest_nodes(workload.source_xyz)
    surf = workload.mesh.lengths[2] if workload.receiver_surface_only else None
    rec = model.nearest_nodes(workload.receiver_xyz, surface_z=surf)
    return src, rec


def run_workload(workload, nsteps: int | None = None, model: Model | None = None):
    """Oracle solution of a workload from rest: returns dict(seis, u, v, a, dt, src, rec)."""
    model = build_model(workload) if model is None else model
    dt = model.cfl_dt(workload.courant)
    src, rec = locate_workload(model, workload)
    n = workload.nsteps if nsteps is None else nsteps
    seis, u, v, a = newmark_run(model, dt, n, src_nodes=src, src_force=workload.source_force,
                                f0=workload.f0, t0=workload.t0, rec_nodes=rec)
    return dict(seis=seis, u=u, v=v, a=a, dt=dt, src=src, rec=rec, model=model)


# --------------------------------------------------------------------------------------
# Discrete adjoint and material sensitivities (the gradient of a seismogram loss)
# --------------------------------------------------------------------------------------
#
# From a zero state the explicit Newmark scheme above is the leapfrog recursion
#     M (u^{n+1} - 2 u^n + u^{n-1}) + dt^2 (K u^n - f^n) = 0,   n = 1 .. N-1,
# with u^0 = u^1 = 0 and records s^n = R u^n (n = 1 .. N). For a loss L(s) with
# G^n = dL/ds^n, the Lagrangian L - sum_n (lam^n)^T R^n gives the adjoint recursion
#     M (lam^{m-1} - 2 lam^m + lam^{m+1}) + dt^2 K lam^m = R^T G^m,  m = N .. 2,
# with lam^N = lam^{N+1} = 0 (the same symmetric operator run backward in time with the
# receiver residuals as sources), and the gradient
#     dL/dp = - sum_{n=1}^{N-1} (lam^n)^T [ dM/dp (u^{n+1} - 2 u^n + u^{n-1}) + dt^2 dK/dp u^n ].
# Per local point q (weights w_q J_q): dM/drho_q puts w_q J_q on node I(q);
# lam^T dK/dkappa_q u = w_q J_q tr e(lam) tr e(u);
# lam^T dK/dmu_q u = w_q J_q 2 (e(lam) : e(u) - tr e(lam) tr e(u) / 3),
# with e the discrete strain of Sec. II-B at the quadrature point.


def element_strain(u_e, dxi_dx, basis: Basis) -> np.ndarray:
    """Symmetric gradient (strain) of an element-local field at every GLL point, by the same
    reference derivatives and chain rule as element_forces: [nspec, 3, 3, k, j, i]."""
    H = basis.hprime
    du = np.empty(u_e.shape[:2] + (3,) + u_e.shape[2:])
    du[:, :, 0] = np.einsum("il,eckjl->eckji", H, u_e)
    du[:, :, 1] = np.einsum("jl,eckli->eckji", H, u_e)
    du[:, :, 2] = np.einsum("kl,eclji->eckji", H, u_e)
    grad = np.einsum("ecrkji,erdkji->ecdkji", du, dxi_dx)
    return 0.5 * (grad + grad.transpose(0, 2, 1, 3, 4, 5))


def set_moduli(model: Model, rho=None, kappa=None, mu=None) -> Model:
    """A copy of ``model`` with per-point rho, kappa, mu replaced (float64 [nspec, k, j, i]);
    the mass is re-assembled when rho changes."""
    import copy
    m = copy.copy(model)
    if rho is not None:
        m.rho = np.asarray(rho, dtype=np.float64).reshape(model.rho.shape)
        m.mass = mass_matrix(m.rho, m.jac, m.ibool, m.nglob, m.basis)
    if kappa is not None:
        m.kappa = np.asarray(kappa, dtype=np.float64).reshape(model.kappa.shape)
    if mu is not None:
        m.mu = np.asarray(mu, dtype=np.float64).reshape(model.mu.shape)
    return m


def forward_history(model: Model, dt: float, nsteps: int, src_nodes, src_force, f0, t0, rec_nodes):
    """Forward run from rest keeping every displacement: returns (u [nsteps+1, nglob, 3] with
    u[n] = u^n, seis [nrec, 3, nsteps] with seis[..., n-1] = s^n)."""
    ng = model.nglob
    u = np.zeros((ng, 3))
    v = np.zeros((ng, 3))
    a = np.zeros((ng, 3))
    Minv = 1.0 / model.mass
    src_nodes = np.asarray(src_nodes, dtype=np.int64).reshape(-1)
    src_force = np.asarray(src_force, dtype=np.float64).reshape(-1, 3)
    rec_nodes = np.asarray(rec_nodes, dtype=np.int64).reshape(-1)
    hist = np.zeros((nsteps + 1, ng, 3))
    seis = np.zeros((len(rec_nodes), 3, nsteps))
    for n in range(nsteps):
        u_new = u + dt * v + 0.5 * dt * dt * a
        f = model.forces(u_new)
        for s, g in enumerate(src_nodes):
            f[g] += src_force[s] * ricker((n + 1) * dt, f0, t0)
        a_new = Minv[:, None] * f
        v = v + 0.5 * dt * (a + a_new)
        u, a = u_new, a_new
        hist[n + 1] = u
        seis[:, :, n] = u[rec_nodes]
    return hist, seis


def adjoint_gradient(model: Model, dt: float, u_hist: np.ndarray, rec_nodes, G: np.ndarray):
    """Gradient of a loss with dL/ds^n = G[..., n-1] (G [nrec, 3, nsteps]) with respect to
    rho, kappa and mu at every local point, by the discrete adjoint above.
    Returns (g_rho, g_kappa, g_mu), each float64 [nspec, k, j, i]."""
    N = u_hist.shape[0] - 1
    ng = model.nglob
    n = model.ngll
    rec_nodes = np.asarray(rec_nodes, dtype=np.int64).reshape(-1)
    Minv = 1.0 / model.mass
    wJ = model.jac * quadrature_weights_3d(model.basis)[None]
    g_rho = np.zeros_like(model.rho)
    g_kappa = np.zeros_like(model.kappa)
    g_mu = np.zeros_like(model.mu)
    lam_next = np.zeros((ng, 3))  # lam^{m+1}
    lam = np.zeros((ng, 3))       # lam^m
    for m in range(N, 1, -1):
        inj = np.zeros((ng, 3))
        np.add.at(inj, rec_nodes, G[:, :, m - 1])
        lam_prev = 2.0 * lam - lam_next + Minv[:, None] * (dt * dt * model.forces(lam) + inj)
        # gradient term n = m - 1 with lam^{m-1}
        k = m - 1
        lam_e = gather(lam_prev, model.ibool, n)
        u_e = gather(u_hist[k], model.ibool, n)
        acc_e = gather(u_hist[k + 1] - 2.0 * u_hist[k] + u_hist[k - 1], model.ibool, n)
        el = element_strain(lam_e, model.dxi_dx, model.basis)
        eu = element_strain(u_e, model.dxi_dx, model.basis)
        tr_l = el[:, 0, 0] + el[:, 1, 1] + el[:, 2, 2]
        tr_u = eu[:, 0, 0] + eu[:, 1, 1] + eu[:, 2, 2]
        ee = np.einsum("ecdkji,ecdkji->ekji", el, eu)
        g_kappa -= dt * dt * wJ * tr_l * tr_u
        g_mu -= dt * dt * wJ * 2.0 * (ee - tr_l * tr_u / 3.0)
        g_rho -= wJ * np.einsum("eckji,eckji->ekji", lam_e, acc_e)
        lam_next, lam = lam, lam_prev
    return g_rho, g_kappa, g_mu
