"""Pins of the oracle's standard DGSEM on Gauss-Legendre nodes (Sec. 2.2,
Eq. dgsem with lhat+-_i = l_i(+-1) / w_i; Sec. 5.1 runs this scheme's
convergence test):

* the GL nodes and weights against their closed forms at N = 1, 2, 3, and the
  quadrature's exactness up to degree 2N + 1 (and not 2N + 2);
* the face interpolation vectors reproduce polynomials up to degree N at
  +-1, and the weak operator satisfies the summation-by-parts identity
  Dhat = D - (l(+1) l(+1)^T - l(-1) l(-1)^T) / w that the GL quadrature
  makes exact;
* the solution-node coordinates and metrics of an affine mesh against the
  affine map;
* free-stream preservation on curved, rotated meshes (the metrics are the
  LGL curl-form polynomials evaluated at the GL nodes);
* discrete conservation, and convergence of R(U) to the exact
  -div(F_c - F_v) of a smooth state;
* convergence of an advected density wave at the design order N + 1;
* uniform streams along slip walls and through prescribed states, and the
  Couette residual falling with N (the face values are interpolated
  conservative states, so the LGL scheme's exact discrete steady state is
  only approached);
* shock capturing is refused on GL nodes.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from test_oracle_dg import _symbolic_rhs


def _weights(N):
    x, w, *_ = O.ops(N, gauss=True)
    return np.einsum("i,j,k->kji", w, w, w).reshape(-1)


def test_gauss_nodes_and_weights_closed_forms():
    x, w, *_ = O.ops(1, gauss=True)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15, rtol=0)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15, rtol=0)
    x, w, *_ = O.ops(2, gauss=True)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15, rtol=0)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15, rtol=0)
    x, w, *_ = O.ops(3, gauss=True)
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    assert np.allclose(x, [-b, -a, a, b], atol=1e-15, rtol=0)
    wa, wb = (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36
    assert np.allclose(w, [wb, wa, wa, wb], atol=1e-15, rtol=0)


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_gauss_quadrature_exact_to_degree_2N_plus_1(N):
    x, w, *_ = O.ops(N, gauss=True)
    for k in range(2 * N + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14, k
    k = 2 * N + 2
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_face_interpolation_and_summation_by_parts(N):
    x, w, D, Dh, _, _ = O.ops(N, gauss=True)
    Lp, Lm = O.face_interp(N, gauss=True)
    for k in range(N + 1):
        assert abs(Lp @ x ** k - 1.0) < 1e-12
        assert abs(Lm @ x ** k - (-1.0) ** k) < 1e-12
    # symmetric nodes: l_i(-1) = l_{N-i}(+1)
    assert np.allclose(Lm, Lp[::-1], atol=1e-13, rtol=0)
    # D differentiates polynomials up to degree N exactly
    for k in range(1, N + 1):
        assert np.allclose(D @ x ** k, k * x ** (k - 1), atol=1e-11 * N * N, rtol=0)
    sbp = D - (np.outer(Lp, Lp) - np.outer(Lm, Lm)) / w[:, None]
    assert np.allclose(Dh, sbp, atol=1e-11 * N * N, rtol=0), np.abs(Dh - sbp).max()


def test_affine_mesh_nodes_and_metrics():
    N = 3
    h = 2 * math.pi / 3
    m = W.box_mesh(N, (3, 3, 3))
    M = O.Mesh(N, m["xyz"], m["period"], gauss=True)
    X = M.nodes()
    xg, *_ = O.ops(N, gauss=True)
    # every element is an axis-aligned cube (some with rotated local frames):
    # its solution nodes are the cube's corner plus h (x_GL + 1) / 2 per axis
    ref = np.sort((xg + 1) * h / 2)
    for e in range(m["E"]):
        lo = m["xyz"].reshape(m["E"], -1, 3)[e].min(axis=0)
        for c in range(3):
            got = np.unique(np.round(X[e, :, c] - lo[c], 12))
            assert np.allclose(got, np.round(ref, 12), atol=1e-12), (e, c)
    Ja, J = M.metrics()
    assert np.allclose(J, (h / 2) ** 3, rtol=1e-13)
    assert np.allclose(np.abs(Ja).sum(axis=(2, 3)), 3 * (h / 2) ** 2, rtol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 5])
@pytest.mark.parametrize("riemann,viscous", [("roe", False), ("roe", True), ("lf", True)])
def test_free_stream_preservation(N, riemann, viscous):
    m = W.box_mesh(N, (3, 3, 2), curved=0.1, seed=20240419)
    M = O.Mesh(N, m["xyz"], m["period"], gauss=True)
    U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=3.0)
    Ut = M.rhs(U, O.params(riemann=riemann, viscous=viscous))
    assert np.abs(Ut).max() < 2e-13, np.abs(Ut).max()
    # the LGL geometry interpolated, not re-sampled: a curved mesh's GL nodes
    # are not those of the LGL scheme
    assert not np.allclose(M.nodes(), m["xyz"].reshape(M.nodes().shape))


@pytest.mark.parametrize("viscous", [False, True])
def test_conservation(viscous):
    N = 3
    m = W.box_mesh(N, (3, 3, 3), curved=0.1, seed=4)
    M = O.Mesh(N, m["xyz"], m["period"], gauss=True)
    U = W.random_perturbation(W.tgv_state(M.nodes(), Ma=0.3).reshape(m["E"], -1, 5), 1e-2, 5)
    Ut = M.rhs(U, O.params(mu=0.01, viscous=viscous))
    _, J = M.metrics()
    wq = _weights(N)[None, :, None] * J[..., None]
    tot = (wq * Ut).sum(axis=(0, 1))
    scale = (wq * np.abs(Ut)).sum(axis=(0, 1))
    assert np.all(np.abs(tot) <= 1e-13 * scale), tot / scale


@pytest.mark.parametrize("viscous", [False, True])
def test_consistency_with_exact_divergence(viscous):
    N = 3
    mu = 0.05
    prim, exact = _symbolic_rhs(mu, viscous=viscous)
    prm = O.params(mu=mu, viscous=viscous)
    errs = []
    for nel in (4, 8):
        m = W.box_mesh(N, (nel,) * 3, curved=0.05, seed=nel)
        M = O.Mesh(N, m["xyz"], m["period"], gauss=True)
        X = M.nodes()
        xx, yy, zz = X[..., 0], X[..., 1], X[..., 2]
        r, u, v, w, p = (np.broadcast_to(f(xx, yy, zz), xx.shape) for f in prim)
        Ut = M.rhs(W.prim_to_cons(r, u, v, w, p), prm)
        ref = np.stack([np.broadcast_to(f(xx, yy, zz), xx.shape) for f in exact], axis=-1)
        errs.append(np.abs(Ut - ref).max(axis=(0, 1)) / np.abs(ref).max(axis=(0, 1)))
    errs = np.array(errs)
    assert np.all(errs[1] < 0.02), errs
    assert np.all(errs[1] < errs[0] / 2 ** (N - 1)), errs


def test_density_wave_convergence():
    """Advected density sinusoid (exact Euler solution): the L2 error falls at
    about the design order N + 1 (Sec. 5.1 reports the design order for the
    standard scheme on GL nodes)."""
    N = 3
    prm = O.params(viscous=False, riemann="roe")
    T = 0.2
    errs = []
    for nel in (4, 8):
        m = W.box_mesh(N, (nel,) * 3, length=(2.0, 2.0, 2.0), origin=(-1, -1, -1), curved=0.05, seed=1)
        M = O.Mesh(N, m["xyz"], m["period"], gauss=True)
        X = M.nodes()
        U0 = W.density_wave_state(X, t=0.0).reshape(m["E"], -1, 5)
        nsteps = 20 * nel
        U, _, _ = M.step(U0, prm, nsteps, dt=T / nsteps)
        ex = W.density_wave_state(X, t=T).reshape(m["E"], -1, 5)
        _, J = M.metrics()
        wq = _weights(N)[None, :] * J
        errs.append(math.sqrt((wq * (U[..., 0] - ex[..., 0]) ** 2).sum() / wq.sum()))
    rate = math.log2(errs[0] / errs[1])
    assert rate > N + 0.5, (errs, rate)


def _channel(N, seed=7, curved=0.0):
    return W.box_mesh(N, (3, 4, 3), length=(2.0, 1.0, 2.0), origin=(0.0, 0.0, 0.0),
                      periodic=(True, False, True), seed=seed, curved=curved)


@pytest.mark.parametrize("N", [3, 4])
def test_uniform_stream_along_slip_walls_and_through_prescribed_states(N):
    m = _channel(N, curved=0.1, seed=8)
    shape = (m["E"], (N + 1) ** 3)
    fb = W.box_face_bc(m, {"y-": 1, "y+": 1})
    U = W.uniform_state(shape, rho=1.1, vel=(0.4, 0.0, -0.3), p=2.0)
    M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=[(3,)], gauss=True)
    for prm in (O.params(mu=0.01), O.params(viscous=False, riemann="lf")):
        assert np.abs(M.rhs(U, prm)).max() < 1e-12
    U2 = W.uniform_state(shape, rho=1.1, vel=(0.4, 0.5, -0.3), p=2.0)
    fb2 = W.box_face_bc(m, {"y-": 1, "y+": 2})
    M2 = O.Mesh(N, m["xyz"], m["period"], face_bc=fb2, bcs=[(4, *U2[0, 0]), (5, 2.0)], gauss=True)
    for prm in (O.params(mu=0.01), O.params(riemann="lf")):
        assert np.abs(M2.rhs(U2, prm)).max() < 1e-12


def test_couette_residual_falls_with_N():
    mu, Uw, Tw = 0.02, 0.7, 1.3
    bcs = [(1, 0.0, 0.0, 0.0, Tw), (1, Uw, 0.0, 0.0, Tw)]
    res = []
    for N in (2, 4, 6):
        m = _channel(N)
        fb = W.box_face_bc(m, {"y-": 1, "y+": 2})
        M = O.Mesh(N, m["xyz"], m["period"], face_bc=fb, bcs=bcs, gauss=True)
        U = W.couette_state(M.nodes(), U_wall=Uw, T_wall=Tw, p=0.9, mu=mu).reshape(m["E"], -1, 5)
        res.append(np.abs(M.rhs(U, O.params(mu=mu))).max())
    assert res[0] < 1e-2 and res[1] < res[0] / 10 and res[2] < res[1] / 10, res


def test_shock_capturing_is_refused():
    m = W.box_mesh(2, (2, 2, 2))
    M = O.Mesh(2, m["xyz"], m["period"], gauss=True)
    U = W.uniform_state((m["E"], 27))
    with pytest.raises(RuntimeError):
        M.rhs(U, O.params(shock=True))
