"""Pins for the oracle's point-wise fluxes (Sec. 2.1 Eq. nse; the two-point flux of
Sec. 2.2 Nonlinear Stability; the Riemann solvers of FillFlux, App. A).

Checks: hand-computed states (tests/golden/point_fluxes.txt), consistency
f*(a, a) = f(a), symmetry of the two-point flux, Roe's exact upwinding for
supersonic states and exact resolution of a stationary contact, rotational
invariance and the mirror property f*(L, R, n) = -f*(R, L, -n), and physical
invariants of the viscous flux (no stress under rigid rotation or pure
dilatation, frame invariance, Fourier heat flux with lambda = cp mu / Pr).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300.workloads import prim_to_cons

GOLD = os.path.join(os.path.dirname(__file__), "golden", "point_fluxes.txt")


def cons(rho, u, v, w, p, g=1.4):
    return prim_to_cons(np.array(rho), u, v, w, p, g)


def rot_matrix(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rotate_state(U, R):
    V = U.copy()
    V[1:4] = R @ U[1:4]
    return V


def load_golden():
    rows = []
    with open(GOLD) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            rows.append((parts[0], np.array(parts[1:6], float), np.array(parts[6:11], float),
                         np.array(parts[11:14], float), np.array(parts[14:19], float)))
    return rows


def test_golden_point_fluxes():
    rows = load_golden()
    assert len(rows) >= 4
    for kind, UL, UR, n, f in rows:
        got = O.point_flux(kind, UL, UR, n)
        np.testing.assert_allclose(got, f, rtol=1e-12, atol=1e-12, err_msg=kind)


@pytest.mark.parametrize("kind", ["roe", "lf", "kep"])
def test_consistency(kind):
    U = cons(1.3, 0.4, -0.2, 0.7, 2.1)
    n = np.array([0.3, -0.5, 0.8])
    if kind != "kep":
        n = n / np.linalg.norm(n)
    f = O.point_flux(kind, U, U, n)
    np.testing.assert_allclose(f, O.point_flux("euler", U, U, n), rtol=1e-14, atol=1e-14)


def test_kep_symmetric_and_kinetic_energy_form():
    UL = cons(1.3, 0.4, -0.2, 0.7, 2.1)
    UR = cons(0.8, -0.1, 0.5, 0.2, 1.4)
    m = np.array([0.3, -0.5, 0.8])
    fa = O.point_flux("kep", UL, UR, m)
    fb = O.point_flux("kep", UR, UL, m)
    np.testing.assert_allclose(fa, fb, rtol=1e-15)
    # momentum flux = mass flux times the mean velocity plus the mean pressure;
    # mass flux = mean density times mean normal velocity (Pirozzoli's form)
    uL, uR = UL[1:4] / UL[0], UR[1:4] / UR[0]
    ubar = (uL + uR) / 2
    rbar = (UL[0] + UR[0]) / 2
    assert abs(fa[0] - rbar * ubar @ m) < 1e-14
    pL = 0.4 * (UL[4] - 0.5 * UL[0] * uL @ uL)
    pR = 0.4 * (UR[4] - 0.5 * UR[0] * uR @ uR)
    np.testing.assert_allclose(fa[1:4], fa[0] * ubar + (pL + pR) / 2 * m, rtol=1e-14, atol=1e-15)


def test_roe_supersonic_is_upwind():
    """All Roe wave speeds positive -> f* = f(U_L) exactly (Roe property)."""
    n = np.array([1.0, 0.0, 0.0])
    UL = cons(1.0, 3.0, 0.2, -0.1, 1.0)
    UR = cons(0.7, 2.6, 0.1, 0.3, 0.8)
    f = O.point_flux("roe", UL, UR, n)
    np.testing.assert_allclose(f, O.point_flux("euler", UL, UL, n), rtol=1e-13, atol=1e-13)
    # and leftward supersonic -> f(U_R)
    UL2 = cons(1.0, -3.0, 0.2, -0.1, 1.0)
    UR2 = cons(0.7, -2.6, 0.1, 0.3, 0.8)
    f2 = O.point_flux("roe", UL2, UR2, n)
    np.testing.assert_allclose(f2, O.point_flux("euler", UR2, UR2, n), rtol=1e-13, atol=1e-13)
    # oblique normal, rotated frame
    R = rot_matrix(7)
    nr = R @ n
    f3 = O.point_flux("roe", rotate_state(UL, R), rotate_state(UR, R), nr)
    g = O.point_flux("euler", rotate_state(UL, R), rotate_state(UL, R), nr)
    np.testing.assert_allclose(f3, g, rtol=1e-13, atol=1e-13)


def test_roe_stationary_contact():
    """u = 0, equal pressure, density jump: Roe returns (0, p n, 0) (no dissipation)."""
    n = np.array([0.6, 0.0, 0.8])
    p = 1.7
    f = O.point_flux("roe", cons(1.0, 0, 0, 0, p), cons(0.2, 0, 0, 0, p), n)
    np.testing.assert_allclose(f, [0, p * n[0], p * n[1], p * n[2], 0], atol=1e-14)
    # a moving contact with tangential slip is still resolved exactly by Roe:
    # flux equals the upwind (left) state's flux for u_n > 0
    n = np.array([1.0, 0, 0])
    UL = cons(1.0, 0.3, 0.5, 0.0, 1.0)
    UR = cons(0.4, 0.3, -0.2, 0.1, 1.0)
    f = O.point_flux("roe", UL, UR, n)
    ref = O.point_flux("euler", UL, UL, n)
    assert abs(f[0] - ref[0]) < 1e-13   # mass flux is upwinded


@pytest.mark.parametrize("kind", ["roe", "lf"])
def test_rotation_and_mirror(kind):
    UL = cons(1.1, 0.3, -0.4, 0.2, 1.9)
    UR = cons(0.6, -0.2, 0.1, 0.5, 0.7)
    n = np.array([0.2, 0.9, -0.3])
    n /= np.linalg.norm(n)
    f = O.point_flux(kind, UL, UR, n)
    # mirror: swapping sides and flipping the normal flips the flux
    np.testing.assert_allclose(O.point_flux(kind, UR, UL, -n), -f, rtol=1e-13, atol=1e-14)
    # rotational invariance
    R = rot_matrix(3)
    fr = O.point_flux(kind, rotate_state(UL, R), rotate_state(UR, R), R @ n)
    np.testing.assert_allclose(fr[[0, 4]], f[[0, 4]], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(fr[1:4], R @ f[1:4], rtol=1e-13, atol=1e-14)


def test_lf_dissipates():
    """LF adds -lambda_max/2 (U_R - U_L) to the central flux with lambda_max >= |u_n| + c."""
    UL = cons(1.0, 0.0, 0, 0, 1.0)
    UR = cons(0.125, 0.0, 0, 0, 0.1)
    n = np.array([1.0, 0, 0])
    f = O.point_flux("lf", UL, UR, n)
    central = (O.point_flux("euler", UL, UL, n) + O.point_flux("euler", UR, UR, n)) / 2
    d = central - f
    lam = d[[0, 4]] / ((UR - UL)[[0, 4]] / 2)
    np.testing.assert_allclose(lam, np.sqrt(1.4), rtol=1e-14)


def _g(ux=0, uy=0, uz=0, vx=0, vy=0, vz=0, wx=0, wy=0, wz=0, Tx=0, Ty=0, Tz=0):
    return np.array([[ux, uy, uz], [vx, vy, vz], [wx, wy, wz], [Tx, Ty, Tz]], float)


def test_viscous_flux_invariants():
    prm = O.params(mu=0.3, Pr=0.72)
    U = cons(1.2, 0.3, -0.1, 0.2, 1.5)
    n = np.array([0.3, -0.7, 0.4])
    # rigid rotation: antisymmetric velocity gradient -> no stress
    f = O.point_visc(U, _g(uy=0.5, vx=-0.5, uz=-0.2, wx=0.2, vz=0.9, wy=-0.9), n, prm)
    np.testing.assert_allclose(f, 0, atol=1e-15)
    # pure dilatation (Stokes hypothesis: zero bulk viscosity) -> no stress
    f = O.point_visc(U, _g(ux=0.7, vy=0.7, wz=0.7), n, prm)
    np.testing.assert_allclose(f, 0, atol=1e-15)
    # Fourier heat flux: energy component = lambda grad T . n, lambda = cp mu / Pr,
    # cp = gamma R / (gamma - 1) = 3.5 for R = 1
    gT = np.array([0.2, -0.4, 0.9])
    f = O.point_visc(U, _g(Tx=gT[0], Ty=gT[1], Tz=gT[2]), n, prm)
    np.testing.assert_allclose(f[:4], 0, atol=1e-15)
    assert abs(f[4] - 3.5 * 0.3 / 0.72 * gT @ n) < 1e-14
    # simple shear u = s y: tau_xy = mu s; flux through n: momentum (mu s n_y, mu s n_x, 0)
    s = 0.8
    f = O.point_visc(U, _g(uy=s), n, prm)
    u = U[1:4] / U[0]
    np.testing.assert_allclose(f, [0, 0.3 * s * n[1], 0.3 * s * n[0], 0,
                                   0.3 * s * (u[0] * n[1] + u[1] * n[0])], atol=1e-15)


def test_viscous_flux_frame_invariance():
    prm = O.params(mu=0.05)
    rng = np.random.Generator(np.random.PCG64(11))
    U = cons(1.2, 0.3, -0.1, 0.2, 1.5)
    G = rng.normal(size=(4, 3))
    n = rng.normal(size=3)
    R = rot_matrix(5)
    f = O.point_visc(U, G, n, prm)
    # rotate: velocity u' = R u, grad' of u' = R (grad u) R^T, grad' T = R grad T
    Ur = rotate_state(U, R)
    Gr = np.zeros_like(G)
    Gr[:3] = R @ G[:3] @ R.T
    Gr[3] = R @ G[3]
    fr = O.point_visc(Ur, Gr, R @ n, prm)
    np.testing.assert_allclose(fr[[0, 4]], f[[0, 4]], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(fr[1:4], R @ f[1:4], rtol=1e-13, atol=1e-14)


def _state_at_T(T, rho=1.3, u=(0.3, -0.2, 0.5), R=1.0, gamma=1.4):
    return prim_to_cons(np.array(rho), np.array(u[0]), np.array(u[1]), np.array(u[2]),
                        np.array(rho * R * T), gamma)


def test_sutherland_viscous_flux_special_cases():
    """Sutherland's law (Eq. sutherland) through the whole viscous flux: at
    T = T_ref it gives mu_ref; it grows like sqrt(T) for T >> T_ref and like
    T^(3/2) for T << T_ref; the heat flux follows mu (constant Pr)."""
    rng = np.random.default_rng(3)
    g = rng.normal(size=(4, 3))
    nv = np.array([0.3, -0.8, 0.5])
    Tref = 0.7
    const = O.params(mu=2e-3)
    suth = O.params(mu=2e-3, sutherland=True, T_ref=Tref)

    def ratio(T):
        U = _state_at_T(T)
        fs, fc = O.point_visc(U, g, nv, suth), O.point_visc(U, g, nv, const)
        r = fs[1:] / fc[1:]
        assert np.allclose(r, r[0], rtol=1e-13, atol=0)  # stress and heat flux scale alike
        return r[0]

    assert abs(ratio(Tref) - 1.0) < 1e-14
    # T >> T_ref: mu(4T) / mu(T) -> 2
    assert abs(ratio(4e6 * Tref) / ratio(1e6 * Tref) - 2.0) < 1e-6
    # T << T_ref: mu(T) -> (1.4042 / 0.4042) (T/T_ref)^(3/2)
    th = 1e-8
    assert abs(ratio(th * Tref) / (1.4042 / 0.4042 * th ** 1.5) - 1.0) < 1e-6
    # the Euler part has no viscous flux: the mass component is zero
    assert O.point_visc(_state_at_T(2.0), g, nv, suth)[0] == 0.0
