"""GPU parity: libdg (hand-written sm_103a kernels, called through the C ABI)
against the CPU oracle on the same seeded inputs.

Bounds: integer maps bit-exact; floating point against the long-double oracle
within max(1e-12, 3 x the FP64 oracle's own error), per conservative variable
(the FP64 rounding floor of the operator exceeds 1e-12 at Ma = 0.1 and
N >= 3, so an FP64 implementation is held to the floor FP64 allows);
10 LSERK steps within 1e-10 relative of the oracle's 10 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import parity_check, gpu_or_skip, mesh, oracle_params, parity_bound, rel_err, rk_stage_weight_sum

pytestmark = pytest.mark.gpu


def _solver(dg, m, **kw):
    return dg.Solver(m, **kw)


@pytest.mark.parametrize("N,nel,seed", [(2, (3, 4, 5), 3), (3, (4, 4, 4), 20240419), (7, (3, 3, 4), 7)])
def test_maps_bit_exact(N, nel, seed):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel, seed=seed)
    s = _solver(dg, m)
    nbr, nodes = s.debug("maps")
    on, of, om, onode = O.Mesh(N, m["xyz"], m["period"]).connectivity()
    np.testing.assert_array_equal(nbr[..., 0], on)
    np.testing.assert_array_equal(nbr[..., 1], of)
    np.testing.assert_array_equal(nbr[..., 2], om)
    np.testing.assert_array_equal(nodes, onode)


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_metrics(N):
    torch, dg = gpu_or_skip()
    m = mesh(N, (3, 3, 4))
    s = _solver(dg, m)
    Ja, J = s.debug("metrics")
    oJa, oJ = O.Mesh(N, m["xyz"], m["period"]).metrics()
    # both are rounded from extended precision: a few ulp apart at most
    assert np.abs(Ja - oJa).max() <= 1e-14 * np.abs(oJa).max()
    assert np.abs(J - oJ).max() <= 1e-14 * np.abs(oJ).max()


CASES = [
    # N, elements, Ma, params
    (3, (4, 4, 4), 0.1, dict()),                                  # TGV 4^3 N=3, Roe + BR1
    (7, (3, 4, 3), 0.1, dict()),                                  # N=7 curved, rotated, ragged
    (5, (3, 3, 3), 0.5, dict(riemann="lf")),                      # LF, viscous
    (4, (3, 3, 3), 1.0, dict(viscous=0)),                         # Euler, Roe
    (2, (3, 4, 5), 0.5, dict(mu=0.01)),                           # ragged, low N
    (1, (3, 3, 4), 0.5, dict()),                                  # N = 1
]


@pytest.mark.parametrize("N,nel,Ma,kw", CASES)
def test_rhs_parity(N, nel, Ma, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel)
    s = _solver(dg, m, **kw)
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=Ma).reshape(m["E"], -1, 5), 1e-3, 5)
    Ud = torch.from_numpy(U).cuda()
    Ut = s.rhs(Ud).cpu().numpy()
    prm = oracle_params(s.params)
    ref = O.Mesh(N, m["xyz"], m["period"], quad=True).rhs(U, prm)
    o64 = O.Mesh(N, m["xyz"], m["period"]).rhs(U, prm)
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)
    if Ma >= 0.5:
        assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("N,nel", [(1, (3, 4, 5)), (2, (3, 4, 5)), (3, (3, 3, 7)), (4, (3, 3, 7))])
@pytest.mark.parametrize("kw", [dict(mu=0.01), dict(mu=0.01, riemann="lf", shock_capturing=1, alpha_force=0.4),
                                dict(viscous=0, riemann="lf", shock_capturing=1)])
def test_partial_last_block(N, nel, kw):
    """Element counts that leave the last thread block of the element kernels
    partly filled (several elements share a block at N <= 4)."""
    torch, dg = gpu_or_skip()
    m = mesh(N, nel)
    s = _solver(dg, m, **kw)
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5), 1e-2, 8)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref, oal = O.Mesh(N, m["xyz"], m["period"], quad=True).rhs(U, prm, with_alpha=True)
    o64 = O.Mesh(N, m["xyz"], m["period"]).rhs(U, prm)
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)
    if s.params.shock_capturing:
        al = s.debug("alpha")
        assert np.abs(al - oal).max() <= 1e-12


def test_gradients_and_face_fluxes():
    torch, dg = gpu_or_skip()
    N = 4
    m = mesh(N, (3, 3, 3))
    s = _solver(dg, m, mu=0.01)
    U = W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5)
    s.rhs(torch.from_numpy(U).cuda())
    torch.cuda.synchronize()
    g = s.debug("grad")
    fs = s.debug("fstar")
    prm = oracle_params(s.params)
    _, og, ofs = O.Mesh(N, m["xyz"], m["period"], quad=True).rhs(U, prm, with_grad=True, with_fstar=True)
    assert np.abs(g - og).max() <= 1e-12 * np.abs(og).max()
    assert np.abs(fs - ofs).max() <= 1e-12 * np.abs(ofs).max()


def test_ten_steps_parity():
    """Taylor-Green vortex, 4^3 elements, N = 3, Roe + BR1, LSERK4 with the CFL
    rule, 10 steps (the plain FP64 configuration)."""
    torch, dg = gpu_or_skip()
    N = 3
    m = W.box_mesh(N, (4, 4, 4))
    s = _solver(dg, m)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    s.set_state(U0)
    dt0 = s.time_step()
    s.step(10)
    U, t = s.get_state()
    prm = oracle_params(s.params)
    M = O.Mesh(N, m["xyz"], m["period"])
    odt, _ = M.dt(U0, prm)
    assert abs(dt0 - odt) <= 1e-14 * odt
    Uo, to, _ = M.step(U0, prm, 10)
    assert abs(t - to) <= 1e-13 * to
    err = np.abs(U - Uo).max() / np.abs(Uo).max()
    assert err <= 1e-10, err
    # and against the slow quad oracle on a few steps of a fixed dt
    Uq, _, _ = O.Mesh(N, m["xyz"], m["period"], quad=True).step(U0, prm, 2, dt=odt)
    s.set_state(U0)
    s.step(2, dt=odt)
    U2, _ = s.get_state()
    assert rel_err(U2, Uq).max() <= 1e-12


def test_time_step_reports_without_stepping():
    """dg_time_step reports the CFL step of the current state and changes
    nothing, also after fixed-dt steps."""
    torch, dg = gpu_or_skip()
    N = 3
    m = W.box_mesh(N, (4, 4, 4))
    s = _solver(dg, m)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    s.set_state(U0)
    prm = oracle_params(s.params)
    M = O.Mesh(N, m["xyz"], m["period"])
    dt1 = s.time_step()
    assert s.time_step() == dt1
    assert abs(dt1 - M.dt(U0, prm)[0]) <= 1e-14 * dt1
    s.step(1, dt=dt1 / 3)
    U1, t1 = s.get_state()
    assert t1 == dt1 / 3
    dt2 = s.time_step()
    assert abs(dt2 - M.dt(U1, prm)[0]) <= 1e-14 * dt2
    assert s.get_state()[1] == t1


def test_advance_equals_stepping_to_the_end_time():
    """dg_advance: CFL steps with the last one clipped on the device, bitwise
    the same as stepping from the host with the reported CFL steps."""
    torch, dg = gpu_or_skip()
    N = 3
    m = W.box_mesh(N, (4, 4, 4), curved=0.1)
    U0 = W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5)
    t_end = 0.037
    a = _solver(dg, m)
    a.set_state(U0)
    ta, ka = a.advance(t_end)
    Ua, _ = a.get_state()
    assert ta == t_end and ka >= 3
    b = _solver(dg, m)
    b.set_state(U0)
    t, k = 0.0, 0
    while t < t_end:
        dt = min(b.time_step(), t_end - t)
        b.step(1, dt=dt)
        t = b.get_state()[1] if dt < t_end - t else t_end
        k += 1
    Ub, _ = b.get_state()
    assert k == ka
    np.testing.assert_array_equal(Ua, Ub)
    # advancing again to the same time does nothing; a cap on the steps stops early
    assert a.advance(t_end) == (t_end, 0)
    a.set_state(U0)
    t2, k2 = a.advance(t_end, max_steps=2)
    assert k2 == 2 and t2 < t_end


@pytest.mark.parametrize("kw", [dict(), dict(riemann="lf", viscous=0),
                                dict(shock_capturing=1, alpha_force=0.5, riemann="lf")])
def test_free_stream_and_conservation(kw):
    torch, dg = gpu_or_skip()
    N = 7
    m = mesh(N, (3, 3, 3))
    s = _solver(dg, m, **kw)
    U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=3.0)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    _, J = s.debug("metrics")
    x, w, _, _, Ds, _ = O.ops(N)
    F = 3.0 + 1.1 * 0.25 + 3.0 * 3.5
    assert np.abs(Ut).max() < 1e-14 * F * np.abs(Ds).sum(axis=1).max() / J.min()
    # conservation on a perturbed TGV state
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 0.02, 3)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :, None] * J[..., None]
    tot = (wq * Ut).sum(axis=(0, 1))
    scale = (wq * np.abs(Ut)).sum(axis=(0, 1))
    assert np.all(np.abs(tot) <= 1e-13 * scale), tot / scale


@pytest.mark.parametrize("alpha_force", [0.3, -1.0])
def test_shock_capturing_parity(alpha_force):
    """Sod-type tube state (the shock-capturing configuration's initial jump,
    smoothed over one element so the indicator sees a range of values)."""
    torch, dg = gpu_or_skip()
    N = 5
    nx = 8
    h = 2.0 / nx
    m = W.box_mesh(N, (nx, 3, 3), length=(2.0, 3 * h, 3 * h), curved=0.05, seed=9)
    s = _solver(dg, m, viscous=0, riemann="lf", shock_capturing=1, alpha_force=alpha_force)
    U = W.sod_state(m["xyz"]).reshape(m["E"], -1, 5)
    U = W.random_perturbation(U, 1e-3, 2)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    al = s.debug("alpha")
    prm = oracle_params(s.params)
    ref, oal = O.Mesh(N, m["xyz"], m["period"], quad=True).rhs(U, prm, with_alpha=True)
    o64 = O.Mesh(N, m["xyz"], m["period"]).rhs(U, prm)
    if alpha_force < 0:
        assert oal.max() > 0 and (oal == 0).any()
        np.testing.assert_array_equal(al > 0, oal > 0)
        assert np.abs(al - oal).max() <= 1e-12
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)


def test_full_size_sampled_elements():
    """The 24^3-element curved, renumbered and rotated N = 7 mesh (7.08 M DOF),
    in the launch configuration the benchmark times: Ut of sampled elements
    against the oracle, which forms only what those elements need."""
    torch, dg = gpu_or_skip()
    N = 7
    m = W.box_mesh(N, (24, 24, 24), curved=0.1, seed=20240419)
    s = _solver(dg, m)
    U = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(1))
    pick = rng.choice(m["E"], size=12, replace=False)
    want = np.zeros(m["E"], bool)
    want[pick] = True
    prm = oracle_params(s.params)
    ref = O.Mesh(N, m["xyz"], m["period"], quad=True, metric_mask=want).rhs(U, prm, want=want)
    o64 = O.Mesh(N, m["xyz"], m["period"], metric_mask=want).rhs(U, prm, want=want)
    bound, floor = parity_bound(o64[want], ref[want])
    err = rel_err(Ut[want], ref[want])
    parity_check(err, bound, floor)
    assert np.isfinite(Ut).all()


def test_state_transfer_through_pinned_and_pageable_host_memory():
    """dg_set_state / dg_get_state convert the layout straight from and into
    pinned host buffers (no staging copy) and through a device staging copy
    for pageable ones: both give the same state, bit for bit."""
    torch, dg = gpu_or_skip()
    N = 3
    m = mesh(N, (3, 4, 3))
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, 9)
    pinned_in = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
    pinned_out = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
    pinned_in.numpy()[...] = U
    s = dg.Solver(m)
    s.set_state(pinned_in.numpy(), t=0.5)
    Up, t = s.get_state(pinned_out.numpy())
    assert t == 0.5
    np.testing.assert_array_equal(pinned_out.numpy(), U)
    s.step(2, dt=1e-3)
    A, _ = s.get_state(pinned_out.numpy())
    B, _ = s.get_state()  # pageable
    np.testing.assert_array_equal(A, B)
    s2 = dg.Solver(m)
    s2.set_state(U.copy(), t=0.5)  # pageable
    s2.step(2, dt=1e-3)
    np.testing.assert_array_equal(s2.get_state()[0], B)


def test_other_low_storage_schemes():
    """dg_set_rk: the five-stage table passed explicitly reproduces the default
    bit for bit; a three-stage scheme (Williamson's RK3) over ten CFL steps
    matches the oracle with the same scheme; bad tables are refused."""
    torch, dg = gpu_or_skip()
    from test_oracle_dg import RK3_WILLIAMSON
    N = 3
    m = W.box_mesh(N, (4, 4, 4), curved=0.1, seed=3)
    U0 = W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5)
    a = _solver(dg, m)
    a.set_state(U0)
    a.step(3)
    b = _solver(dg, m)
    b.set_rk(*O.rk_coeffs())
    b.set_state(U0)
    b.step(3)
    np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
    s = _solver(dg, m, cfl=0.5)
    s.set_rk(*RK3_WILLIAMSON)
    s.set_state(U0)
    s.step(10)
    U, t = s.get_state()
    prm = oracle_params(s.params)
    Uo, to, _ = O.Mesh(N, m["xyz"], m["period"]).step(U0, prm, 10, rk=RK3_WILLIAMSON)
    assert abs(t - to) <= 1e-13 * to
    assert np.abs(U - Uo).max() / np.abs(Uo).max() <= 1e-10
    with pytest.raises(dg.DgError) as ex:  # A[0] must be 0
        s.set_rk([0.1, -0.5], [0.5, 0.5], [0.0, 0.5])
    assert ex.value.code == dg.DG_ERR_ARG
    z = np.zeros(1)
    with pytest.raises(dg.DgError) as ex:  # no stages
        dg._check(dg.load().dg_set_rk(s._h, 0, O._dp(z), O._dp(z), O._dp(z)))
    assert ex.value.code == dg.DG_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fourteen_stage_scheme(prec):
    """The library's built-in fourteen-stage scheme (its own copy of the
    published table) over ten CFL steps against the oracle stepping with the
    oracle's copy, on the compressible Taylor-Green set-up of Sec. 5.2
    (Ma 1.25, Sutherland's law); FP64 within 1e-10 of the oracle, FP32-bulk
    within 1e-5 times the scheme's stage-weight sum (1e-5: a state moved by
    ten steps of FP32-rounded fluxes, for a scheme whose weights are all
    positive; the fourteen-stage scheme amplifies each stage's rounding by
    up to sum |b_i| = 98.6, measured 1.3e-5 against 2.4e-7 for the five-stage
    scheme on this set-up)."""
    torch, dg = gpu_or_skip()
    N = 3
    m = W.box_mesh(N, (4, 4, 4), curved=0.1, seed=14, length=(2 * np.pi,) * 3)
    U0 = W.tgv_state(m["xyz"], Ma=1.25).reshape(m["E"], -1, 5)
    p0 = 1.0 / (1.4 * 1.25 ** 2)
    s = _solver(dg, m, precision=dg.FP64 if prec == "fp64" else dg.FP32_BULK, sutherland=1, T_ref=p0,
                cfl=1.5, dfl=3.0)
    s.set_rk_scheme(dg.RK_NDB14)
    s.set_state(U0)
    s.step(10)
    U, t = s.get_state()
    Uo, to, _ = O.Mesh(N, m["xyz"], m["period"]).step(U0, oracle_params(s.params), 10, rk=O.rk14_coeffs())
    assert abs(t - to) <= (1e-13 if prec == "fp64" else 1e-6) * to
    tol = 1e-10 if prec == "fp64" else 1e-5 * rk_stage_weight_sum(*O.rk14_coeffs()[:2])
    assert np.abs(U - Uo).max() / np.abs(Uo).max() <= tol
    with pytest.raises(dg.DgError) as ex:
        s.set_rk_scheme(7)
    assert ex.value.code == dg.DG_ERR_ARG


@pytest.mark.parametrize("nodes", ["lgl", "gauss"])
def test_unstructured_ogrid_mesh(nodes):
    """The five-block O-grid mesh (edges with three, four and eight elements
    around them): maps bit-exact against the oracle's coordinate matching,
    the right-hand side within the parity bound, FP32-bulk within 2e-4."""
    torch, dg = gpu_or_skip()
    N = 4
    m = W.ogrid_mesh(N, m=3, k=2, nz=3, length=(2 * np.pi,) * 3, curved=0.1, seed=5)
    gauss = nodes == "gauss"
    s = _solver(dg, m, nodes=nodes)
    nbr, nodemap = s.debug("maps")
    on, of, om, onode = O.Mesh(N, m["xyz"], m["period"]).connectivity()
    np.testing.assert_array_equal(nbr[..., 0], on)
    np.testing.assert_array_equal(nbr[..., 1], of)
    np.testing.assert_array_equal(nbr[..., 2], om)
    np.testing.assert_array_equal(nodemap, onode)
    M = O.Mesh(N, m["xyz"], m["period"], gauss=gauss)
    U = W.random_perturbation(W.tgv_state(M.nodes(), Ma=0.5).reshape(m["E"], -1, 5), 1e-3, 2)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = O.Mesh(N, m["xyz"], m["period"], quad=True, gauss=gauss).rhs(U, prm)
    bound, floor = parity_bound(M.rhs(U, prm), ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)
    s32 = _solver(dg, m, nodes=nodes, precision=dg.FP32_BULK)
    assert np.all(rel_err(s32.rhs(torch.from_numpy(U).cuda()).cpu().numpy(), ref) <= 2e-4)


@pytest.mark.parametrize("kw", [dict(R=2.5, gamma=1.3, Pr=0.7, mu=0.01),
                                dict(R=287.0, gamma=1.4, Pr=0.71, mu=0.01, sutherland=1, T_ref=1.0 / 287.0),
                                dict(R=2.5, gamma=1.3, viscous=0, riemann="lf")])
def test_gas_constants_other_than_the_defaults(kw):
    """A gas constant R != 1 (temperature T = p / (rho R), Sutherland's law
    in T, the heat conductivity gamma R mu / ((gamma - 1) Pr)), another
    gamma and Prandtl number: the right-hand side within the parity bound,
    the CFL time step within 1e-14, ten steps within 1e-10, FP32-bulk within
    2e-4."""
    torch, dg = gpu_or_skip()
    N = 4
    m = mesh(N, (3, 3, 4))
    s = _solver(dg, m, **kw)
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.5, gamma=kw["gamma"], R=kw["R"]).reshape(m["E"], -1, 5),
                              1e-3, 6)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = O.Mesh(N, m["xyz"], m["period"], quad=True).rhs(U, prm)
    M = O.Mesh(N, m["xyz"], m["period"])
    bound, floor = parity_bound(M.rhs(U, prm), ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)
    s.set_state(U)
    odt, _ = M.dt(U, prm)
    assert abs(s.time_step() - odt) <= 1e-14 * odt
    s.step(10)
    U10, _ = s.get_state()
    Uo, _, _ = M.step(U, prm, 10)
    assert np.abs(U10 - Uo).max() / np.abs(Uo).max() <= 1e-10
    s32 = _solver(dg, m, precision=dg.FP32_BULK, **kw)
    assert np.all(rel_err(s32.rhs(torch.from_numpy(U).cuda()).cpu().numpy(), ref) <= 2e-4)


def test_maps_for_every_rotation_pair():
    """All 24 x 24 ordered pairs of element rotations across a face (96 meshes
    of 3^3 elements, the centre element against its six neighbours): the
    device maps, built from corner ids, equal the oracle's coordinate
    matching bit for bit."""
    torch, dg = gpu_or_skip()
    N = 2
    for a, bs, m in W.rotation_pair_meshes(N):
        s = _solver(dg, m)
        nbr, nodes = s.debug("maps")
        on, of, om, onode = O.Mesh(N, m["xyz"], m["period"]).connectivity()
        np.testing.assert_array_equal(nbr[..., 0], on, err_msg=str((a, bs)))
        np.testing.assert_array_equal(nbr[..., 1], of, err_msg=str((a, bs)))
        np.testing.assert_array_equal(nbr[..., 2], om, err_msg=str((a, bs)))
        np.testing.assert_array_equal(nodes, onode, err_msg=str((a, bs)))
        s.close()


def test_kinetic_energy_against_oracle_and_reproducible():
    """dg_kinetic (Sec. 5.2: E_k, its exact rate from the right-hand side, the
    volume) against the oracle on LGL nodes, and bitwise the same on repeated
    calls and in a second context of the same state (a fixed grid and a
    fixed order of summation)."""
    torch, dg = gpu_or_skip()
    N = 5
    m = mesh(N, (4, 3, 3), seed=12)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, 4)
    a = _solver(dg, m)
    a.set_state(U0)
    k1 = a.kinetic()
    k2 = a.kinetic()
    b = _solver(dg, m)
    b.set_state(U0)
    k3 = b.kinetic()
    assert tuple(k1) == tuple(k2) == tuple(k3)
    M = O.Mesh(N, m["xyz"], m["period"])
    prm = oracle_params(a.params)
    ok = M.kinetic(U0, M.rhs(U0, prm))
    assert abs(k1[0] - ok[0]) <= 1e-12 * abs(ok[0])
    assert abs(k1[2] - ok[2]) <= 1e-12 * abs(ok[2])
    # the rate is a small difference of O(1) terms: against the magnitude of its terms
    scale = abs(ok[0]) * np.abs(M.rhs(U0, prm)).max() / np.abs(U0).max()
    assert abs(k1[1] - ok[1]) <= 1e-9 * scale
