"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only *generates inputs*: hexahedral meshes (node coordinates and
corner vertex ids) and initial states given by closed-form flow fields.  It
holds none of the DGSEM arithmetic (no derivative matrices, metrics, fluxes or
time integration), so the oracle and the CUDA library can both be fed from it
without sharing any of the method.

Layouts (the library's public layout):
  * ``xyz[e, k, j, i, c]``  float64, node coordinates at Legendre-Gauss-Lobatto
    (LGL) points, ``i`` runs along the element's local xi direction.
  * ``corner_vid[e, c]``    int64, vertex id of corner ``c = bi + 2 bj + 4 bk``
    where ``bi`` = 0 for ``i = 0`` and 1 for ``i = N``.  Periodic images share
    one id.
  * ``U[e, k, j, i, v]``    float64 conservative state (rho, rho u, rho v,
    rho w, rho e).

Workloads follow the paper's test cases: the Taylor-Green vortex
(Sec. 5.2, Eq. tgv_ic with Version II), a manufactured density wave for
convergence (Sec. 5.1 uses an advected sinusoid), a Sod-type shock tube for the
sub-cell shock capturing of Sec. 2.3, and an isentropic vortex.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "lgl_points", "ROTATIONS", "box_mesh", "prim_to_cons", "tgv_state",
    "density_wave_state", "sod_state", "isentropic_vortex_state", "box_face_bc", "couette_state",
    "uniform_state", "random_perturbation",
]


def lgl_points(N: int) -> np.ndarray:
    """LGL points on [-1, 1] used only to *place* mesh nodes.

    Uses numpy's Legendre-series root finder (a library routine); the DG
    operators themselves are built independently by each implementation.
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def _proper_rotations():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                mats.append(R)
    return mats


#: The 24 proper rotations of the reference cube, as signed permutation matrices.
ROTATIONS = _proper_rotations()
assert len(ROTATIONS) == 24


def box_mesh(N, nel, length=(2 * math.pi,) * 3, origin=(0.0, 0.0, 0.0),
             curved=0.0, seed=None, rotate=None, permute=None, periodic=(True, True, True),
             rotations=None):
    """Box of ``nel = (nx, ny, nz)`` hexahedra at degree ``N``, periodic in the
    directions ``periodic`` marks (all three by default); the other directions
    end in boundary faces (``period`` is 0 there, see ``box_face_bc``).

    ``curved`` displaces every node by ``curved * h * s(x)`` in each Cartesian
    direction, with ``s = sin(2 pi x'/Lx) sin(2 pi y'/Ly) sin(2 pi z'/Lz)`` in
    box-relative coordinates and ``h`` the smallest element edge; ``s`` vanishes
    on the box faces, so the mesh stays periodic and watertight.

    With ``seed`` given, every element's local frame is turned by one of the 24
    proper cube rotations and the element ids are shuffled, both drawn from
    ``numpy.random.Generator(PCG64(seed))``; ``rotate``/``permute`` override the
    two choices separately.  ``rotations`` (E,) sets every element's rotation
    index (into ``ROTATIONS``) explicitly instead.

    Returns a dict with ``N``, ``E``, ``xyz`` (E, n, n, n, 3), ``corner_vid``
    (E, 8), ``period`` (3,), ``rot`` (E,) rotation index, ``canon`` (E,) the
    canonical (ix, iy, iz)-ordered element index of every element, ``nel``,
    ``length`` and ``origin``.
    """
    nx, ny, nz = (int(v) for v in nel)
    if min(nx, ny, nz) < 1:
        raise ValueError("need at least one element per direction")
    Lx, Ly, Lz = (float(v) for v in length)
    ox, oy, oz = (float(v) for v in origin)
    n = N + 1
    E = nx * ny * nz
    xi = lgl_points(N)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    h = min(hx, hy, hz)

    rng = np.random.Generator(np.random.PCG64(seed)) if seed is not None else None
    do_rot = (seed is not None) if rotate is None else bool(rotate)
    do_perm = (seed is not None) if permute is None else bool(permute)
    rot = np.zeros(E, dtype=np.int64)
    if rotations is not None:
        rot = np.asarray(rotations, dtype=np.int64).reshape(E)
        if rot.min() < 0 or rot.max() > 23:
            raise ValueError("rotation indices are 0..23")
        do_rot = True
    elif do_rot:
        r = rng if rng is not None else np.random.Generator(np.random.PCG64(0))
        rot = r.integers(0, 24, size=E)
    if do_perm:
        r = rng if rng is not None else np.random.Generator(np.random.PCG64(0))
        canon = r.permutation(E)
    else:
        canon = np.arange(E)

    # canonical element (ex, ey, ez) for every element index (x fastest)
    ez_all, rem = np.divmod(canon, nx * ny)
    ey_all, ex_all = np.divmod(rem, nx)

    # canonical node coordinates X[e, k, j, i, c]
    ref = (xi + 1.0) / 2.0
    X = np.empty((E, n, n, n, 3))
    X[..., 0] = ox + (ex_all[:, None, None, None] + ref[None, None, None, :]) * hx
    X[..., 1] = oy + (ey_all[:, None, None, None] + ref[None, None, :, None]) * hy
    X[..., 2] = oz + (ez_all[:, None, None, None] + ref[None, :, None, None]) * hz
    if curved != 0.0:
        s = (np.sin(2 * math.pi * (X[..., 0] - ox) / Lx)
             * np.sin(2 * math.pi * (X[..., 1] - oy) / Ly)
             * np.sin(2 * math.pi * (X[..., 2] - oz) / Lz))
        X = X + (curved * h * s)[..., None]

    # canonical corner vertex ids
    cvid = np.empty((E, 8), dtype=np.int64)
    px, py, pz = (bool(v) for v in periodic)
    mx, my, mz = nx + 1, ny + 1, nz + 1  # vertex counts per direction
    for c in range(8):
        bi, bj, bk = c & 1, (c >> 1) & 1, (c >> 2) & 1
        vx = (ex_all + bi) % nx if px else ex_all + bi
        vy = (ey_all + bj) % ny if py else ey_all + bj
        vz = (ez_all + bk) % nz if pz else ez_all + bk
        cvid[:, c] = vx + mx * (vy + my * vz)

    if not do_rot:
        xyz, corner_vid = X, cvid
    else:
        xyz = np.empty_like(X)
        corner_vid = np.empty_like(cvid)
        idx = np.arange(n)
        # local centred index (2i - N) -> canonical centred index via R
        I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")   # I[i,j,k]
        loc = np.stack([2 * I - N, 2 * J - N, 2 * K - N], axis=-1)  # [i,j,k,3]
        for r_id in range(24):
            sel = np.nonzero(rot == r_id)[0]
            if sel.size == 0:
                continue
            R = ROTATIONS[r_id]
            can = (loc @ R.T + N) // 2            # canonical (i', j', k')
            ci, cj, ck = can[..., 0], can[..., 1], can[..., 2]
            # xyz[e, k, j, i] = X[e, k', j', i']
            src = X[sel][:, ck, cj, ci]            # [sel, i, j, k, 3]
            xyz[sel] = np.transpose(src, (0, 3, 2, 1, 4))
            for c in range(8):
                b = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
                cc = (R @ (2 * b - 1) + 1) // 2
                corner_vid[sel, c] = cvid[sel, cc[0] + 2 * cc[1] + 4 * cc[2]]
    return {
        "N": N, "E": E, "xyz": np.ascontiguousarray(xyz),
        "corner_vid": np.ascontiguousarray(corner_vid),
        "period": np.array([Lx if px else 0.0, Ly if py else 0.0, Lz if pz else 0.0]), "rot": rot,
        "canon": canon,
        "nel": (nx, ny, nz), "length": (Lx, Ly, Lz), "origin": (ox, oy, oz),
    }


def ogrid_mesh(N, m=3, k=2, nz=3, length=(1.0, 1.0, 1.0), inner=0.3, curved=0.0, seed=None):
    """An unstructured hexahedral mesh, periodic in x, y and z: the unit square
    split into five blocks (a centre square [a, 1 - a]^2 of m x m cells and
    four trapezoids of m x k cells between it and the square's sides),
    extruded in z over nz layers, scaled to ``length``.  The centre square's
    corners are vertices of three quadrilaterals (edges of three hexahedra),
    and the square's corner, identified periodically, of eight; the cells
    are straight-sided (bilinear), LGL nodes of degree N.  ``curved``
    displaces every node like ``box_mesh`` (sine products that vanish on the
    box faces); with ``seed`` the element ids are shuffled.

    Returns a dict with ``N``, ``E``, ``xyz`` (E, n, n, n, 3), ``corner_vid``
    (E, 8) and ``period``."""
    Lx, Ly, Lz = (float(v) for v in length)
    a = float(inner)
    n = N + 1
    xi = lgl_points(N)
    ref = (xi + 1.0) / 2.0
    g = np.linspace(0.0, 1.0, m + 1)
    rr = np.linspace(0.0, 1.0, k + 1)
    quads = []

    def block(P, ns, nr, us, vs):
        for i in range(ns):
            for j in range(nr):
                quads.append((P(us[i], vs[j]), P(us[i + 1], vs[j]), P(us[i], vs[j + 1]), P(us[i + 1], vs[j + 1])))

    w = 1.0 - 2.0 * a
    block(lambda u, v: (a + w * u, a + w * v), m, m, g, g)                        # centre
    block(lambda s, r: ((1 - r) * s + r * (a + w * s), r * a), m, k, g, rr)        # bottom
    block(lambda s, r: ((1 - r) * s + r * (a + w * s), 1 - r * a), m, k, g, rr)    # top
    block(lambda s, r: (r * a, (1 - r) * s + r * (a + w * s)), m, k, g, rr)        # left
    block(lambda s, r: (1 - r * a, (1 - r) * s + r * (a + w * s)), m, k, g, rr)    # right
    # counter-clockwise corners (positive Jacobian): swap the two local axes otherwise
    fixed = []
    for p00, p10, p01, p11 in quads:
        cross = (p10[0] - p00[0]) * (p01[1] - p00[1]) - (p10[1] - p00[1]) * (p01[0] - p00[0])
        fixed.append((p00, p10, p01, p11) if cross > 0 else (p00, p01, p10, p11))
    Q = len(fixed)
    E = Q * nz
    hz = Lz / nz
    vid2d = {}

    def vid(p):
        key = (round(p[0] % 1.0, 9) % 1.0, round(p[1] % 1.0, 9) % 1.0)
        return vid2d.setdefault(key, len(vid2d))

    X = np.empty((E, n, n, n, 3))
    cvid = np.empty((E, 8), dtype=np.int64)
    for q, (p00, p10, p01, p11) in enumerate(fixed):
        c = np.array([p00, p10, p01, p11], dtype=np.float64)
        ids = [vid(p) for p in (p00, p10, p01, p11)]
        # bilinear map at the LGL nodes: x[j, i] for xi (i) and eta (j)
        U, V = np.meshgrid(ref, ref, indexing="xy")
        xy = ((1 - U) * (1 - V))[..., None] * c[0] + (U * (1 - V))[..., None] * c[1] \
            + ((1 - U) * V)[..., None] * c[2] + (U * V)[..., None] * c[3]
        for lz in range(nz):
            e = q * nz + lz
            X[e, :, :, :, 0] = Lx * xy[None, :, :, 0]
            X[e, :, :, :, 1] = Ly * xy[None, :, :, 1]
            X[e, :, :, :, 2] = (lz + ref)[:, None, None] * hz
            for cc in range(8):
                bi, bj, bk = cc & 1, (cc >> 1) & 1, (cc >> 2) & 1
                cvid[e, cc] = ids[bi + 2 * bj] + len(fixed) * 4 * ((lz + bk) % nz)
    if curved != 0.0:
        h = min(Lx, Ly) * min(a / k, w / m, (1.0 - a) / max(m, k)) if k > 0 else min(Lx, Ly) / m
        h = min(h, hz)
        s = (np.sin(2 * math.pi * X[..., 0] / Lx) * np.sin(2 * math.pi * X[..., 1] / Ly)
             * np.sin(2 * math.pi * X[..., 2] / Lz))
        X = X + (curved * h * s)[..., None]
    if seed is not None:
        perm = np.random.Generator(np.random.PCG64(seed)).permutation(E)
        X, cvid = X[perm], cvid[perm]
    return {"N": N, "E": E, "xyz": np.ascontiguousarray(X), "corner_vid": np.ascontiguousarray(cvid),
            "period": np.array([Lx, Ly, Lz])}


BOX_SIDES = ("x-", "x+", "y-", "y+", "z-", "z+")


def box_face_bc(mesh, side_bc):
    """Boundary-condition row per element face of a ``box_mesh`` box:
    ``side_bc`` maps box sides ("x-", "x+", "y-", "y+", "z-", "z+") to a row
    index k >= 1 (faces inside the box, or on periodic sides, get 0).  Faces
    are found by their centroid (the local frames may be rotated).  Returns
    int32 [E, 6]."""
    N, E = mesh["N"], mesh["E"]
    n = N + 1
    X = mesh["xyz"].reshape(E, n, n, n, 3)  # [e, k, j, i, c]
    faces = [X[:, :, :, 0], X[:, :, :, -1], X[:, :, 0, :], X[:, :, -1, :], X[:, 0], X[:, -1]]
    out = np.zeros((E, 6), dtype=np.int32)
    lo = np.asarray(mesh["origin"], dtype=float)
    hi = lo + np.asarray(mesh["length"], dtype=float)
    tol = 1e-9 * float(np.max(mesh["length"]))
    for f, F in enumerate(faces):
        c = F.reshape(E, -1, 3).mean(axis=1)
        for d in range(3):
            if mesh["period"][d] > 0:
                continue
            for end, name in ((lo[d], BOX_SIDES[2 * d]), (hi[d], BOX_SIDES[2 * d + 1])):
                k = side_bc.get(name, 0)
                if k:
                    out[np.abs(c[:, d] - end) < tol, f] = k
    return out


def couette_state(xyz, U_wall=1.0, h=1.0, T_wall=1.0, p=1.0, mu=0.01, Pr=0.72, gamma=1.4, R=1.0):
    """Compressible plane Couette flow between isothermal no-slip walls at
    y = 0 (at rest) and y = h (moving with U_wall in x), both at T_wall: an
    exact steady solution of the compressible Navier-Stokes equations with
    constant mu and lambda = gamma R mu / ((gamma - 1) Pr): u = U_wall y / h,
    v = w = 0, uniform pressure, T = T_wall + mu U_wall^2 y (h - y) / (2 lambda h^2),
    rho = p / (R T)."""
    y = xyz[..., 1]
    lam = gamma * R * mu / ((gamma - 1.0) * Pr)
    T = T_wall + mu * U_wall ** 2 * y * (h - y) / (2.0 * lam * h * h)
    rho = p / (R * T)
    z = np.zeros_like(y)
    return prim_to_cons(rho, U_wall * y / h, z, z, np.full_like(y, p), gamma)


def prim_to_cons(rho, u, v, w, p, gamma=1.4):
    """Conservative state from density, velocity and pressure (ideal gas)."""
    rho = np.asarray(rho, dtype=np.float64)
    U = np.empty(rho.shape + (5,))
    U[..., 0] = rho
    U[..., 1] = rho * u
    U[..., 2] = rho * v
    U[..., 3] = rho * w
    U[..., 4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return U


def tgv_state(xyz, Ma=0.1, gamma=1.4, R=1.0, version=2, rho0=1.0, U0=1.0, L=1.0):
    """Taylor-Green vortex initial state (Sec. 5.2, Eq. tgv_ic).

    ``p0`` follows from ``Ma = U0 sqrt(rho0 / (gamma p0))``.  Version II holds the
    temperature at ``T0 = p0 / (rho0 R)`` and sets ``rho = p / (R T0)``;
    Version I holds ``rho = rho0``.
    """
    x, y, z = xyz[..., 0] / L, xyz[..., 1] / L, xyz[..., 2] / L
    p0 = rho0 * U0 * U0 / (gamma * Ma * Ma)
    u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = p0 + rho0 * U0 * U0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    if version == 2:
        T0 = p0 / (rho0 * R)
        rho = p / (R * T0)
    else:
        rho = np.full_like(p, rho0)
    return prim_to_cons(rho, u, v, w, p, gamma)


def density_wave_state(xyz, t=0.0, amp=0.2, vel=(1.0, 1.0, 1.0), p=1.0,
                       wavelength=(2.0, 2.0, 2.0), gamma=1.4):
    """Advected density sinusoid: an exact solution of the Euler equations.

    ``rho = 1 + amp sin(2 pi sum_d (x_d - vel_d t) / wavelength_d)``, constant
    velocity and pressure.
    """
    ph = sum(2 * math.pi * (xyz[..., d] - vel[d] * t) / wavelength[d] for d in range(3))
    rho = 1.0 + amp * np.sin(ph)
    ones = np.ones_like(rho)
    return prim_to_cons(rho, vel[0] * ones, vel[1] * ones, vel[2] * ones, p * ones, gamma)


def sod_state(xyz, x_split=1.0, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), gamma=1.4):
    """Sod-type tube along x: ``(rho, u, p)`` = ``left`` for x < x_split, else ``right``.

    On a periodic [0, 2) box the second jump sits at x = 0 (= 2).
    """
    x = xyz[..., 0]
    L = x < x_split
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    z = np.zeros_like(rho)
    return prim_to_cons(rho, u, z, z, p, gamma)


def isentropic_vortex_state(xyz, center, strength=5.0, mean=(1.0, 1.0, 0.0),
                            gamma=1.4, period=None):
    """Isentropic vortex in the x-y plane (inviscid exact translating solution).

    ``delta u = beta/(2 pi) exp((1-r^2)/2) (-(y-yc), x-xc)``,
    ``T = 1 - (gamma-1) beta^2/(8 gamma pi^2) exp(1 - r^2)``, ``rho = T^(1/(gamma-1))``,
    ``p = rho^gamma``.  With ``period`` given the nearest periodic image of
    the centre is used.
    """
    dx = xyz[..., 0] - center[0]
    dy = xyz[..., 1] - center[1]
    if period is not None:
        dx = dx - period[0] * np.round(dx / period[0])
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = dx * dx + dy * dy
    f = strength / (2 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = mean[0] - f * dy
    v = mean[1] + f * dx
    w = mean[2] + np.zeros_like(u)
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return prim_to_cons(rho, u, v, w, p, gamma)


def mms_state(xyz, t=0.0, A=0.1, a=1.0):
    """The manufactured solution of Sec. 5.1 (Eq. mms) at the points xyz and
    time t: with phi = 2 pi (x + y + z - a t), density and the three momentum
    components 2 + A sin(phi), total energy (2 + A sin(phi))^2 (the bold u of
    Eq. mms read as the momentum).  Period 1 in x, y and z."""
    X = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    r = 2.0 + A * np.sin(2 * math.pi * (X[:, 0] + X[:, 1] + X[:, 2] - a * t))
    U = np.stack([r, r, r, r, r * r], axis=-1)
    return U.reshape(np.asarray(xyz).shape[:-1] + (5,))


def uniform_state(shape, rho=1.2, vel=(0.3, -0.2, 0.1), p=2.0, gamma=1.4):
    """A constant state (free-stream) of the given leading shape."""
    ones = np.ones(shape)
    return prim_to_cons(rho * ones, vel[0] * ones, vel[1] * ones, vel[2] * ones, p * ones, gamma)


def random_perturbation(U, scale, seed):
    """``U`` times ``1 + scale * r`` with ``r`` uniform in [-1, 1] from ``PCG64(seed)``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return U * (1.0 + scale * rng.uniform(-1.0, 1.0, size=U.shape))


def rotation_pair_meshes(N, curved=0.1):
    """Meshes that put every ordered pair of the 24 cube rotations across a
    face: 3^3 periodic boxes whose centre element (canonical index 13) is
    turned by rotation a and its six face neighbours by 6 k .. 6 k + 5
    (k = 0..3), for a = 0..23 (96 meshes).  The other elements take a fixed
    spread of rotations.  Yields (a, neighbour rotations, mesh)."""
    nbrs = (12, 14, 10, 16, 4, 22)
    for a in range(24):
        for k in range(4):
            rot = (np.arange(27) * 7 + a) % 24
            rot[13] = a
            for j, e in enumerate(nbrs):
                rot[e] = 6 * k + j
            yield a, tuple(6 * k + j for j in range(6)), box_mesh(N, (3, 3, 3), curved=curved, rotations=rot)
