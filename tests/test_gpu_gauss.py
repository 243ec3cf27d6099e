"""Standard DGSEM on Gauss-Legendre nodes on the GPU against the oracle
(Eq. dgsem with lhat+-_i = l_i(+-1) / w_i; the scheme of Sec. 5.1's GL
convergence test): solution-node coordinates and metrics, the right-hand side
(inviscid and viscous, Roe and LF, ragged meshes, N = 1..7, boundary
conditions, sponge), lifted gradients and face fluxes, ten LSERK steps, the
time step and kinetic energy, FP32-bulk, free streams, the refused
combinations, and sampled elements of the 24^3-element N = 7 mesh.

Bounds as for the LGL path: coordinates and metrics within a few ulp of the
extended-precision oracle; floating point against the long-double oracle
within max(1e-12, 3 x the FP64 oracle's own error) per conservative
variable; FP32-bulk within 2e-4 of max |Ut|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import parity_check, gpu_or_skip, mesh, oracle_params, parity_bound, rel_err

pytestmark = pytest.mark.gpu


def _oracle(m, quad=False, **kw):
    return O.Mesh(m["N"], m["xyz"], m["period"], quad=quad, face_bc=m.get("face_bc"), bcs=m.get("bcs"),
                  gauss=True, **kw)


def _state(m, Ma=0.5, seed=5):
    X = _oracle(m).nodes()
    U = W.tgv_state(X, Ma=Ma).reshape(m["E"], -1, 5)
    return W.random_perturbation(U, 1e-3, seed)


@pytest.mark.parametrize("N", [1, 3, 7])
def test_node_coordinates_and_metrics(N):
    torch, dg = gpu_or_skip()
    m = mesh(N, (3, 3, 4))
    s = dg.Solver(m, nodes="gauss")
    M = _oracle(m)
    X, oX = s.node_coords(), M.nodes()
    assert np.abs(X - oX).max() <= 1e-14 * np.abs(oX).max()
    Ja, J = s.debug("metrics")
    oJa, oJ = M.metrics()
    assert np.abs(Ja - oJa).max() <= 1e-14 * np.abs(oJa).max()
    assert np.abs(J - oJ).max() <= 1e-14 * np.abs(oJ).max()
    # LGL contexts report their input nodes
    s2 = dg.Solver(m)
    assert np.array_equal(s2.node_coords(), m["xyz"].reshape(m["E"], -1, 3))


CASES = [
    (3, (4, 4, 4), 0.1, dict()),
    (7, (3, 4, 3), 0.1, dict()),
    (5, (3, 3, 3), 0.5, dict(riemann="lf")),
    (4, (3, 3, 3), 1.0, dict(viscous=0)),
    (2, (3, 4, 5), 0.5, dict(mu=0.01)),
    (1, (3, 3, 4), 0.5, dict()),
    (6, (3, 3, 3), 0.5, dict(mu=0.01, sutherland=1, T_ref=1.0)),
]


@pytest.mark.parametrize("N,nel,Ma,kw", CASES)
def test_rhs_parity(N, nel, Ma, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel)
    s = dg.Solver(m, nodes="gauss", **kw)
    U = _state(m, Ma=Ma)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = _oracle(m, quad=True).rhs(U, prm)
    o64 = _oracle(m).rhs(U, prm)
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)


def test_gradients_and_face_fluxes():
    torch, dg = gpu_or_skip()
    N = 4
    m = mesh(N, (3, 3, 3))
    s = dg.Solver(m, nodes="gauss", mu=0.01)
    U = _state(m)
    s.rhs(torch.from_numpy(U).cuda())
    torch.cuda.synchronize()
    g = s.debug("grad")
    fs = s.debug("fstar")
    _, og, ofs = _oracle(m, quad=True).rhs(U, oracle_params(s.params), with_grad=True, with_fstar=True)
    assert np.abs(g - og).max() <= 1e-12 * np.abs(og).max()
    assert np.abs(fs - ofs).max() <= 1e-12 * np.abs(ofs).max()


BCS = {
    "walls": [(1, 0.0, 0.0, 0.0, 1.2), (1, 0.6, 0.0, 0.1, 1.0)],
    "adiabatic+slip": [(2, 0.3, 0.0, 0.0), (3,)],
    "inflow+outflow": [(4, 1.1, 0.3, 0.2, -0.1, 6.0), (5, 2.2)],
}


def _channel(N, bcs, nel=(3, 4, 3), seed=31):
    m = W.box_mesh(N, nel, length=(2.0, 1.0, 2.0), origin=(0.0, 0.0, 0.0),
                   periodic=(True, False, True), seed=seed, curved=0.1)
    m["face_bc"] = W.box_face_bc(m, {"y-": 1, "y+": 2})
    m["bcs"] = BCS[bcs]
    return m


@pytest.mark.parametrize("N,bcs,kw", [
    (3, "walls", dict()),
    (5, "adiabatic+slip", dict(riemann="lf")),
    (4, "inflow+outflow", dict()),
    (3, "inflow+outflow", dict(viscous=0)),
])
def test_boundary_conditions(N, bcs, kw):
    torch, dg = gpu_or_skip()
    m = _channel(N, bcs)
    s = dg.Solver(m, nodes="gauss", **kw)
    U = W.random_perturbation(W.tgv_state(_oracle(m).nodes(), Ma=0.5).reshape(m["E"], -1, 5), 1e-2, 3)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = _oracle(m, quad=True).rhs(U, prm)
    bound, floor = parity_bound(_oracle(m).rhs(U, prm), ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sponge(prec):
    torch, dg = gpu_or_skip()
    N = 3
    m = mesh(N, (3, 3, 3))
    n3 = (N + 1) ** 3
    s = dg.Solver(m, nodes="gauss", precision=dg.FP64 if prec == "fp64" else dg.FP32_BULK)
    U = _state(m)
    Ub = W.uniform_state((m["E"], n3), rho=1.0, vel=(0.0, 0.0, 0.0), p=2.0)
    sigma = np.random.default_rng(2).uniform(0.0, 2.0, size=(m["E"], n3))
    s.set_sponge(sigma, Ub)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    M = _oracle(m)
    M.set_sponge(sigma, Ub)
    ref = M.rhs(U, oracle_params(s.params))
    err = rel_err(Ut, ref)
    assert np.all(err <= (1e-12 if prec == "fp64" else 2e-4)), err


def test_ten_steps_parity():
    torch, dg = gpu_or_skip()
    N = 3
    m = W.box_mesh(N, (4, 4, 4), curved=0.1, seed=9)
    s = dg.Solver(m, nodes="gauss", cfl=0.5)
    M = _oracle(m)
    U0 = W.tgv_state(M.nodes()).reshape(m["E"], -1, 5)
    s.set_state(U0)
    dt0 = s.time_step()
    s.step(10)
    U, t = s.get_state()
    prm = oracle_params(s.params)
    odt, _ = M.dt(U0, prm)
    assert abs(dt0 - odt) <= 1e-14 * odt
    Uo, to, _ = M.step(U0, prm, 10)
    assert abs(t - to) <= 1e-13 * to
    assert np.abs(U - Uo).max() / np.abs(Uo).max() <= 1e-10
    k = s.kinetic()
    ok = M.kinetic(U)
    assert abs(k[0] - ok[0]) <= 1e-12 * ok[0] and abs(k[2] - ok[2]) <= 1e-12 * ok[2]


def test_free_stream_and_conservation():
    torch, dg = gpu_or_skip()
    N = 5
    m = mesh(N, (3, 3, 3))
    for prec, tol in ((dg.FP64, 1e-12), (dg.FP32_BULK, 1e-5)):
        s = dg.Solver(m, nodes="gauss", precision=prec, mu=0.01)
        U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=3.0)
        Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
        assert np.abs(Ut).max() <= tol * 10.0, (prec, np.abs(Ut).max())
    s = dg.Solver(m, nodes="gauss", mu=0.01)
    U = _state(m, seed=8)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    x, w, *_ = O.ops(N, gauss=True)
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)
    _, J = s.debug("metrics")
    tot = (wq[None, :, None] * J[..., None] * Ut).sum(axis=(0, 1))
    scale = (wq[None, :, None] * J[..., None] * np.abs(Ut)).sum(axis=(0, 1))
    assert np.all(np.abs(tot) <= 1e-13 * scale), tot / scale


@pytest.mark.parametrize("N,nel,Ma,kw", [(3, (4, 4, 4), 0.1, dict()), (7, (3, 4, 3), 0.1, dict()),
                                        (4, (3, 3, 3), 0.5, dict(riemann="lf", viscous=0))])
def test_fp32_bulk_against_oracle(N, nel, Ma, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel)
    s = dg.Solver(m, nodes="gauss", precision=dg.FP32_BULK, **kw)
    U = _state(m, Ma=Ma)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    ref = _oracle(m).rhs(U, oracle_params(s.params))
    assert np.all(rel_err(Ut, ref) <= 2e-4), rel_err(Ut, ref)


def test_refused_combinations():
    torch, dg = gpu_or_skip()
    m = mesh(3, (3, 3, 3))
    with pytest.raises(dg.DgError) as ex:
        dg.Solver(m, nodes="gauss", shock_capturing=1)
    assert ex.value.code == dg.DG_ERR_ARG
    s = dg.Solver(m, nodes="gauss")
    with pytest.raises(dg.DgError) as ex:
        s.set_params(shock_capturing=1)
    assert ex.value.code == dg.DG_ERR_ARG
    s = dg.Solver(m, nodes="gauss")
    s.set_state(_state(m))
    with pytest.raises(dg.DgError) as ex:
        s.autotune()
    assert ex.value.code == dg.DG_ERR_STATE
    with pytest.raises(dg.DgError):
        dg.Solver(m, nodes=2)


def test_full_size_sampled_elements():
    """The 24^3-element curved, renumbered and rotated N = 7 mesh (7.08 M DOF)
    on GL nodes, as the benchmark runs it: Ut of sampled elements against the
    oracle, which forms only what those elements need."""
    torch, dg = gpu_or_skip()
    N = 7
    m = W.box_mesh(N, (24, 24, 24), curved=0.1, seed=20240419)
    s = dg.Solver(m, nodes="gauss")
    rng = np.random.Generator(np.random.PCG64(1))
    pick = rng.choice(m["E"], size=12, replace=False)
    want = np.zeros(m["E"], bool)
    want[pick] = True
    M = _oracle(m, quad=True, metric_mask=want)
    U = W.tgv_state(M.nodes()).reshape(m["E"], -1, 5)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = M.rhs(U, prm, want=want)
    o64 = _oracle(m, metric_mask=want).rhs(U, prm, want=want)
    bound, floor = parity_bound(o64[want], ref[want])
    err = rel_err(Ut[want], ref[want])
    parity_check(err, bound, floor)
    assert np.isfinite(Ut).all()


@pytest.mark.parametrize("nodes", ["gauss", "lgl"])
@pytest.mark.parametrize("N", [3, 5])
def test_density_wave_convergence(nodes, N):
    """Sec. 5.1's convergence test with both schemes (standard DGSEM on GL
    nodes, split form on LGL nodes) on the GPU: an advected density sinusoid
    (an exact Euler solution) on curved meshes; the L2 error falls at about
    the design order N + 1."""
    torch, dg = gpu_or_skip()
    T = 0.2
    errs = []
    for nel in (4, 8):
        m = W.box_mesh(N, (nel,) * 3, length=(2.0, 2.0, 2.0), origin=(-1, -1, -1), curved=0.05, seed=1)
        s = dg.Solver(m, nodes=nodes, viscous=0)
        X = s.node_coords()
        s.set_state(W.density_wave_state(X, t=0.0).reshape(m["E"], -1, 5))
        nsteps = 20 * nel
        s.step(nsteps, dt=T / nsteps)
        U, t = s.get_state()
        ex = W.density_wave_state(X, t=T).reshape(m["E"], -1, 5)
        x, w, *_ = O.ops(N, gauss=nodes == "gauss")
        _, J = s.debug("metrics")
        wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
        errs.append(np.sqrt((wq * (U[..., 0] - ex[..., 0]) ** 2).sum() / wq.sum()))
    rate = np.log2(errs[0] / errs[1])
    assert rate > N + 0.5, (errs, rate)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_taylor_green_run_stays_stable_at_the_default_cfl(precision):
    """The time-step rule (CFL 0.9, (N + 1)^2 scaling) keeps the standard
    scheme on GL nodes stable: 400 steps of the Taylor-Green vortex (Re 1600,
    Ma 0.1, to t ~ 0.13) on 8^3 curved elements at N = 7 stay finite, conserve mass
    (to FP64 rounding; FP32-bulk to 1e-9) and dissipate kinetic energy."""
    torch, dg = gpu_or_skip()
    N = 7
    m = mesh(N, (8, 8, 8))
    s = dg.Solver(m, nodes="gauss", precision=dg.FP64 if precision == "fp64" else dg.FP32_BULK)
    U0 = W.tgv_state(s.node_coords()).reshape(m["E"], -1, 5)
    s.set_state(U0)
    k0 = s.kinetic()
    s.step(400)
    U, t = s.get_state()
    assert np.isfinite(U).all() and t > 0.1
    k1 = s.kinetic()
    assert k1[0] < k0[0] and k1[1] < 0
    x, w, *_ = O.ops(N, gauss=True)
    _, J = s.debug("metrics")
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    mass0, mass1 = (wq * U0[..., 0]).sum(), (wq * U[..., 0]).sum()
    # FP32-bulk: the surface and volume terms cancel in FP32 arithmetic
    assert abs(mass1 - mass0) <= (1e-12 if precision == "fp64" else 1e-9) * mass0
