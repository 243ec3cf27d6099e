"""Pins of the oracle's manufactured-solution source (Sec. 5.1, Eq. mms) and of
the convergence test the paper runs with it:

* the source against Q = U_t + div F_c - div F_v of the manufactured state,
  derived symbolically here from the Navier-Stokes fluxes (Eq. nse, stress,
  Fourier law), inviscid and viscous, for two advection speeds;
* the stage times: ten LSERK steps of a pure source (a uniform state whose
  residual is zero would not see it) are checked through the convergence
  test below, which fails when the source is taken at the wrong time;
* convergence of the split form on LGL nodes and of the standard form on GL
  nodes towards the manufactured solution at the design order N + 1;
* the source is written for a constant viscosity: Sutherland's law is refused.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W


def _symbolic_source(A, a, mu, viscous, gamma=1.4, Rg=1.0, Pr=0.72):
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t", real=True)
    X = (x, y, z)
    phi = 2 * sp.pi * (x + y + z - a * t)
    rho = 2 + A * sp.sin(phi)
    mom = (rho, rho, rho)
    E = rho ** 2
    vel = [m / rho for m in mom]
    p = (gamma - 1) * (E - sp.Rational(1, 2) * sum(m * v for m, v in zip(mom, vel)))
    T = p / (rho * Rg)
    lam = gamma * Rg * mu / ((gamma - 1) * Pr)
    div = sum(sp.diff(vel[i], X[i]) for i in range(3))
    tau = [[mu * (sp.diff(vel[i], X[j]) + sp.diff(vel[j], X[i])) - (sp.Rational(2, 3) * mu * div if i == j else 0)
            for j in range(3)] for i in range(3)]
    U = [rho, *mom, E]
    Fc = [[mom[d] for d in range(3)]]
    for i in range(3):
        Fc.append([mom[i] * vel[d] + (p if i == d else 0) for d in range(3)])
    Fc.append([(E + p) * vel[d] for d in range(3)])
    Fv = [[0, 0, 0]] + [[tau[i][d] for d in range(3)] for i in range(3)]
    Fv.append([sum(tau[d][k] * vel[k] for k in range(3)) + lam * sp.diff(T, X[d]) for d in range(3)])
    Q = []
    for k in range(5):
        q = sp.diff(U[k], t) + sum(sp.diff(Fc[k][d] - (Fv[k][d] if viscous else 0), X[d]) for d in range(3))
        Q.append(sp.lambdify((x, y, z, t), q, "numpy"))
    return Q


@pytest.mark.parametrize("viscous,a", [(False, 1.0), (True, 1.0), (True, 0.3)])
def test_source_against_symbolic_derivation(viscous, a):
    A, mu = 0.1, 0.05
    Q = _symbolic_source(A, a, mu, viscous)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, size=(50, 3))
    for t in (0.0, 0.37):
        prm = O.params(mu=mu, viscous=viscous, source=1, source_A=A, source_a=a)
        got = O.mms_source(pts, t, prm)
        ref = np.stack([np.broadcast_to(q(pts[:, 0], pts[:, 1], pts[:, 2], t), (len(pts),)) for q in Q], axis=-1)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(got - ref).max(axis=0)


def _mms_error(N, nel, gauss, T=0.1, steps_per_el=8, viscous=True, mu=0.01):
    m = W.box_mesh(N, (nel,) * 3, length=(2.0, 2.0, 2.0), origin=(-1, -1, -1), curved=0.05, seed=2)
    M = O.Mesh(N, m["xyz"], m["period"], gauss=gauss)
    X = M.nodes()
    prm = O.params(mu=mu, viscous=viscous, source=1)
    n = steps_per_el * nel
    U, t, _ = M.step(W.mms_state(X, 0.0), prm, n, dt=T / n)
    ex = W.mms_state(X, t)
    x, w, *_ = O.ops(N, gauss=gauss)
    _, J = M.metrics()
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    return math.sqrt((wq * (U[..., 0] - ex[..., 0]) ** 2).sum() / wq.sum())


@pytest.mark.parametrize("gauss", [False, True])
def test_manufactured_solution_converges_at_design_order(gauss):
    """Sec. 5.1: the design order N + 1 for the split form on LGL nodes and the
    standard form on GL nodes (here N = 2, two meshes of 2^3 and 4^3 curved
    elements on [-1, 1]^3, viscous)."""
    N = 2
    e = [_mms_error(N, nel, gauss) for nel in (2, 4)]
    rate = math.log2(e[0] / e[1])
    assert rate > N + 0.5, (e, rate)


def test_source_needs_constant_viscosity():
    m = W.box_mesh(2, (3, 3, 3))
    M = O.Mesh(2, m["xyz"], m["period"])
    with pytest.raises(RuntimeError):
        M.rhs(W.mms_state(m["xyz"].reshape(m["E"], -1, 3)), O.params(source=1, sutherland=True))
