"""Pins of the oracle's boundary conditions (walls, slip walls, prescribed
states), by states the discrete operator must hold exactly:

* compressible plane Couette flow (linear velocity, quadratic temperature,
  uniform pressure) between isothermal no-slip walls is an exact steady
  solution of the Navier-Stokes equations whose fields the DG space holds
  exactly for N >= 2, so the operator must vanish to round-off;
* the same with an adiabatic moving upper wall (its own exact profile);
* a uniform stream parallel to slip walls, and a uniform stream through
  prescribed-state boundaries equal to it, on curved rotated meshes;
* mass (all walls) and total energy (walls at rest, adiabatic) are conserved
  by the discrete operator in a wall-bounded box;
* closed forms of the boundary terms on affine elements: the residual of a
  uniform state against another prescribed state, and the lifted gradients
  at slip walls crossed by a normal velocity."""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

GAM, R, PR = 1.4, 1.0, 0.72


def _weights(N):
    x, w, *_ = O.ops(N)
    return np.einsum("i,j,k->kji", w, w, w).reshape(-1)


def _channel(N, nel=(3, 4, 3), seed=7, curved=0.0):
    return W.box_mesh(N, nel, length=(2.0, 1.0, 2.0), origin=(0.0, 0.0, 0.0),
                      periodic=(True, False, True), seed=seed, curved=curved)


@pytest.mark.parametrize("N,Rg", [(2, R), (3, R), (5, R), (3, 2.5)])
def test_couette_between_isothermal_walls_is_a_discrete_steady_state(N, Rg):
    """With a gas constant other than 1 the wall temperatures are consistent
    with the inner state only through T = p / (rho R)."""
    m = _channel(N)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
    mu, Uw, Tw = 0.02, 0.7, 1.3 / Rg
    bcs = [(1, 0.0, 0.0, 0.0, Tw), (1, Uw, 0.0, 0.0, Tw)]
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=bcs)
    U = W.couette_state(m["xyz"], U_wall=Uw, T_wall=Tw, p=0.9, mu=mu, R=Rg).reshape(m["E"], -1, 5)
    Ut = M.rhs(U, O.params(mu=mu, R=Rg))
    # terms of size p / h ~ 3 and mu U / h^2 ~ 0.2 cancel to round-off
    assert np.abs(Ut).max() < 1e-12, np.abs(Ut).max(axis=(0, 1))
    # a wrong wall temperature is seen
    bad = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(1, 0.0, 0.0, 0.0, Tw + 0.1 / Rg), bcs[1]])
    assert np.abs(bad.rhs(U, O.params(mu=mu, R=Rg))).max() > 1e-3


def test_couette_with_an_adiabatic_moving_wall():
    """Isothermal wall at rest at y = 0, adiabatic wall moving with U at y = h:
    T = T_w + mu U^2 (h y - y^2 / 2) / (lambda h^2)."""
    N = 3
    m = _channel(N)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
    mu, Uw, Tw, p = 0.02, 0.7, 1.3, 0.9
    lam = GAM * R * mu / ((GAM - 1) * PR)
    y = m["xyz"][..., 1]
    T = Tw + mu * Uw ** 2 * (y - 0.5 * y * y) / lam
    z = np.zeros_like(y)
    U = W.prim_to_cons(p / (R * T), Uw * y, z, z, np.full_like(y, p)).reshape(m["E"], -1, 5)
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(1, 0.0, 0.0, 0.0, Tw), (2, Uw, 0.0, 0.0)])
    assert np.abs(M.rhs(U, O.params(mu=mu))).max() < 1e-12


@pytest.mark.parametrize("N", [3, 4])
def test_uniform_stream_along_slip_walls_and_through_prescribed_states(N):
    m = _channel(N, curved=0.1, seed=8)
    shape = (m["E"], (N + 1) ** 3)
    # along slip walls: the stream is parallel to them
    U = W.uniform_state(shape, rho=1.1, vel=(0.4, 0.0, -0.3), p=2.0)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 1})
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(3,)])
    for prm in (O.params(mu=0.01), O.params(viscous=False, riemann="lf")):
        Ut = M.rhs(U, prm)
        assert np.abs(Ut).max() < 1e-12 * 10, np.abs(Ut).max()
    # through prescribed-state boundaries equal to the stream (any direction)
    U2 = W.uniform_state(shape, rho=1.1, vel=(0.4, 0.5, -0.3), p=2.0)
    M2 = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(4, *U2[0, 0])])
    for prm in (O.params(mu=0.01), O.params(riemann="lf")):
        assert np.abs(M2.rhs(U2, prm)).max() < 1e-12 * 10


def _euler_flux_y(U):
    rho, mx, my, mz, E = U
    v = my / rho
    p = (GAM - 1) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)
    return np.array([my, mx * v, my * v + p, mz * v, (E + p) * v])


@pytest.mark.parametrize("N,kind", [(3, "roe"), (4, "lf")])
def test_boundary_residual_of_a_uniform_state_against_a_prescribed_state(N, kind):
    """Uniform inner stream U_in, prescribed state U_ext != U_in at y = 0 and
    U_in at y = 1, inviscid, affine elements.  Every volume term and inner
    face cancels, so only the nodes on y = 0 move, by the weak form's surface
    term: J Ut = -(s / w_0) (f*(U_in, U_ext; n) - F(U_in) . n), n = -y the
    outward normal; on a box element of height h_y, s / J = 2 / h_y.  f* is
    the point Riemann flux pinned by the hand-computed values."""
    m = _channel(N)
    shape = (m["E"], (N + 1) ** 3)
    U = W.uniform_state(shape, rho=1.1, vel=(0.4, 0.3, -0.2), p=2.0)
    Ue = W.uniform_state((1, 1), rho=1.3, vel=(0.1, 0.6, 0.25), p=2.4)[0, 0]
    fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(4, *Ue), (4, *U[0, 0])])
    prm = O.params(viscous=False, riemann=kind)
    Ut = M.rhs(U, prm)
    w0 = O.ops(N)[1][0]
    hy = 1.0 / 4
    fs = O.point_flux(kind, U[0, 0], Ue, np.array([0.0, -1.0, 0.0]), prm)
    want = -(2 / hy) / w0 * (fs + _euler_flux_y(U[0, 0]))
    y = m["xyz"].reshape(m["E"], -1, 3)[..., 1]
    on = np.abs(y) < 1e-12
    assert on.sum() == 3 * 3 * (N + 1) ** 2
    scale = np.abs(want).max()
    assert np.abs(Ut[on] - want).max() < 1e-12 * scale, (Ut[on][:2], want)
    assert np.abs(Ut[~on]).max() < 1e-12 * scale


@pytest.mark.parametrize("N", [2, 3])
def test_slip_wall_lifting_value_is_the_tangential_velocity(N):
    """A uniform stream with a normal velocity v at slip walls y = 0 and y = 1:
    the lifting value there is the tangential velocity, so the lifted
    gradients of the constant field are zero except dv/dy at the wall nodes,
    which is (q* - q) . n s / (J w_0) = +v 2 / (h_y w_0) at y = 0 and the
    opposite at y = 1."""
    m = _channel(N)
    shape = (m["E"], (N + 1) ** 3)
    v = 0.3
    U = W.uniform_state(shape, rho=1.1, vel=(0.4, v, -0.2), p=2.0)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 1})
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(3,)])
    _, g = M.rhs(U, O.params(mu=0.01), with_grad=True)
    w0 = O.ops(N)[1][0]
    want = v * 2 / (1.0 / 4) / w0
    y = m["xyz"].reshape(m["E"], -1, 3)[..., 1]
    lo, hi = np.abs(y) < 1e-12, np.abs(y - 1) < 1e-12
    assert np.abs(g[lo][:, 1, 1] - want).max() < 1e-12 * want
    assert np.abs(g[hi][:, 1, 1] + want).max() < 1e-12 * want
    rest = g.copy()
    rest[lo | hi, 1, 1] = 0
    assert np.abs(rest).max() < 1e-12 * want


def test_mass_and_energy_conserved_in_a_walled_box():
    N = 3
    m = _channel(N, curved=0.1, seed=9)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(2, 0.0, 0.0, 0.0), (3,)])
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5), 1e-2, 3)
    Ut = M.rhs(U, O.params(mu=0.01))
    _, J = M.metrics()
    wq = _weights(N)[None, :, None] * J[..., None]
    tot = (wq * Ut).sum(axis=(0, 1))
    scale = (wq * np.abs(Ut)).sum(axis=(0, 1))
    assert abs(tot[0]) <= 1e-13 * scale[0] and abs(tot[4]) <= 1e-13 * scale[4], tot / scale
    # momentum is not conserved: the walls exert forces
    assert abs(tot[2]) > 1e-6 * scale[2]


def test_open_faces_need_a_boundary_condition():
    m = _channel(3)
    with pytest.raises(ValueError):
        O.Mesh(3, m["xyz"], m["period"])
    fb = W.box_face_bc(m, {"y-": 1, "y+": 1})
    fb[0, 0] = 1  # a condition on a face that has a partner
    with pytest.raises(ValueError):
        O.Mesh(3, m["xyz"], m["period"], face_bc=fb, bcs=[(3,)])


def test_outflow_at_the_stream_pressure_keeps_a_uniform_stream():
    """Prescribed state upstream, pressure outflow downstream at the stream's
    own pressure: the outer states equal the inner ones, the stream stays."""
    N = 3
    m = _channel(N, curved=0.1, seed=12)
    U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.2, vel=(0.1, 0.6, 0.2), p=3.0)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(4, *U[0, 0]), (5, 3.0)])
    for prm in (O.params(mu=0.01), O.params(riemann="lf", viscous=False)):
        assert np.abs(M.rhs(U, prm)).max() < 1e-11
    # another outflow pressure is seen at the outflow side only
    M2 = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(4, *U[0, 0]), (5, 2.5)])
    Ut = M2.rhs(U, O.params(mu=0.01))
    assert np.abs(Ut).max() > 1e-2


def test_sponge_source():
    """A uniform state has no DG residual: the sponge alone sets Ut =
    -sigma (U - U_base); over LSERK steps every node relaxes like
    U_base + (U - U_base) exp(-sigma t) (fourth order in time)."""
    N = 3
    m = W.box_mesh(N, (3, 3, 3), curved=0.1, seed=13)
    n3 = (N + 1) ** 3
    U = W.uniform_state((m["E"], n3), rho=1.1, vel=(0.3, -0.2, 0.1), p=2.0)
    Ub = W.uniform_state((m["E"], n3), rho=1.0, vel=(0.0, 0.0, 0.0), p=2.0)
    M = O.Mesh(N, m["xyz"], m["period"])
    prm = O.params(mu=0.01)
    sigma = np.full((m["E"], n3), 0.8)
    M.set_sponge(sigma, Ub)
    Ut = M.rhs(U, prm)
    assert np.abs(Ut - (-sigma[..., None] * (U - Ub))).max() < 1e-13
    dt, steps = 0.05, 20
    Uk, t, _ = M.step(U, prm, steps, dt=dt)
    exact = Ub + (U - Ub) * np.exp(-0.8 * t)
    assert np.abs(Uk - exact).max() < 1e-8
    M.set_sponge(None)
    assert np.abs(M.rhs(U, prm)).max() < 1e-11
