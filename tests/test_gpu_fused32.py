"""The two-kernel FP32-bulk stage (FillFlux per side node, everything else per
element; csrc/dg_fused32.cuh) against the CPU oracle and against the
four-kernel FP32-bulk stage, and the bookkeeping of its face data.

Bounds: FP32 arithmetic on shifted primitives (unit round-off 6e-8), so one
right-hand side within 2e-4 (max norm per variable, relative to max |Ut|) of
the oracle, as for the four-kernel stage; the two forms differ only in FP32
rounding order (the BR1 face gradient is completed from a partial viscous
flux and the neighbours' halves of q*), so their right-hand sides agree
within 2e-5, and after 10 steps their states differ by no more than either
differs from the FP64 oracle (and below 1e-7 of the state; the state stays
FP64, the two-kernel stage keeps its RK register in FP32); the face data
that a step leaves behind equal
those formed from scratch, so interrupted and uninterrupted step sequences
are bitwise equal.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import gpu_or_skip, mesh, oracle_params, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # N, elements, Ma, params
    (3, (4, 4, 4), 0.1, dict()),                                     # TGV, Roe + BR1
    (7, (3, 4, 3), 0.1, dict()),                                     # N = 7, curved, rotated, ragged
    (5, (3, 3, 3), 0.5, dict(riemann="lf")),                         # LF, viscous
    (4, (3, 3, 3), 1.0, dict(viscous=0)),                            # Euler
    (2, (3, 4, 5), 0.3, dict(mu=0.01)),                              # odd node count, strong viscosity
    (1, (3, 3, 4), 0.5, dict()),                                     # N = 1: every node an edge node
    (6, (3, 3, 3), 0.5, dict(sutherland=1, mu=0.005)),               # Sutherland's law
    (5, (6, 3, 3), 0.5, dict(riemann="lf", shock_capturing=1, viscous=0)),  # FV blending
]


def _pair(dg, m, kw):
    a = dg.Solver(m, precision=dg.FP32_BULK, **kw)
    b = dg.Solver(m, precision=dg.FP32_BULK, **kw)
    b.set_config(stage_form=1)
    assert a.stage_form() == 2 and b.stage_form() == 4
    return a, b


@pytest.mark.parametrize("N,nel,Ma,kw", CASES)
def test_rhs_against_oracle_and_four_kernel_stage(N, nel, Ma, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel, seed=100 + N)
    a, b = _pair(dg, m, kw)
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=Ma).reshape(m["E"], -1, 5), 1e-3, N)
    Ud = torch.from_numpy(U).cuda()
    Ua = a.rhs(Ud).cpu().numpy()
    Ub = b.rhs(Ud).cpu().numpy()
    ref = O.Mesh(N, m["xyz"], m["period"]).rhs(U, oracle_params(a.params))
    assert np.all(rel_err(Ua, ref) <= 2e-4), rel_err(Ua, ref)
    assert np.all(rel_err(Ua, Ub) <= 2e-5), rel_err(Ua, Ub)
    # the face fluxes, face by face, and the lifted gradients node by node
    np.testing.assert_allclose(a.debug("fstar"), b.debug("fstar"), rtol=0,
                               atol=2e-5 * np.abs(b.debug("fstar")).max())
    if a.params.viscous:
        ga, gb = a.debug("grad"), b.debug("grad")
        assert np.abs(ga).max() > 0
        np.testing.assert_allclose(ga, gb, rtol=0, atol=2e-5 * np.abs(gb).max())


def test_free_stream():
    torch, dg = gpu_or_skip()
    N = 7
    m = mesh(N, (3, 3, 3))
    s = dg.Solver(m, precision=dg.FP32_BULK)
    assert s.stage_form() == 2
    U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=71.4)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    _, J = s.debug("metrics")
    _, _, _, _, Ds, _ = O.ops(N)
    F = 1.1 * 0.25 + 71.4 + 71.4 * 3.5
    assert np.abs(Ut).max() < 1e-5 * F * np.abs(Ds).sum(axis=1).max() / J.min()


@pytest.mark.parametrize("N,kw", [(3, dict()), (7, dict()), (5, dict(riemann="lf", shock_capturing=1, viscous=0))])
def test_ten_steps_against_four_kernel_stage_and_oracle(N, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, (4, 3, 3), seed=7 * N)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, N)
    a, b = _pair(dg, m, kw)
    a.set_state(U0)
    dt = a.time_step()
    out = []
    for s in (a, b):
        s.set_state(U0)
        s.step(10, dt=dt)
        out.append(s.get_state()[0])
    Uo, _, _ = O.Mesh(N, m["xyz"], m["period"]).step(U0, oracle_params(a.params), 10, dt=dt)
    # the two FP32 forms differ by FP32 rounding of the fluxes: no more than
    # the four-kernel stage's own distance from the FP64 oracle, and below
    # 1e-7 of the state (measured: 1.3e-8 at N = 3)
    d_forms = np.abs(out[0] - out[1]).max()
    assert d_forms <= np.abs(out[1] - Uo).max(), (d_forms, np.abs(out[1] - Uo).max())
    assert d_forms <= 1e-7 * np.abs(Uo).max()
    assert rel_err(out[0], Uo).max() <= 1e-4


def test_interrupted_steps_equal_uninterrupted_ones():
    """The face data a step leaves behind are the state's: a sequence broken
    by calls that overwrite the face arrays (dg_rhs of another state,
    dg_kinetic, dg_autotune, a configuration change) continues bitwise as if
    nothing happened."""
    torch, dg = gpu_or_skip()
    N = 4
    m = mesh(N, (3, 4, 3), seed=11)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, 2)
    other = torch.from_numpy(W.random_perturbation(U0, 1e-2, 9)).cuda()
    a = dg.Solver(m, precision=dg.FP32_BULK)
    a.set_state(U0)
    dt = a.time_step()
    a.step(6, dt=dt)
    ref = a.get_state()[0]
    b = dg.Solver(m, precision=dg.FP32_BULK)
    b.set_state(U0)
    b.step(2, dt=dt)
    b.rhs(other)
    b.step(1, dt=dt)
    b.kinetic()
    b.step(1, dt=dt)
    b.autotune()
    b.set_config(**dict(b.config(), side_block=128))
    b.step(2, dt=dt)
    np.testing.assert_array_equal(b.get_state()[0], ref)


@pytest.mark.parametrize("N", [2, 7])
def test_cfl_steps_take_the_radii_of_the_last_stage(N):
    """Two-kernel CFL steps take their time step from the radii that the
    previous step's last stage reduced for the state it wrote (the face-data
    pass reduces them for a new state): each step's dt equals, bit for bit,
    the CFL time step that the reduction kernel forms from the state in
    memory (dg_time_step); CFL step sequences broken by dg_time_step,
    dg_rhs of another state, dg_kinetic and a configuration change continue
    bitwise as if nothing happened; a non-finite state is reported."""
    torch, dg = gpu_or_skip()
    m = mesh(N, (3, 4, 3), seed=40 + N)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, N)
    a = dg.Solver(m, precision=dg.FP32_BULK)
    assert a.stage_form() == 2
    a.set_state(U0)
    t = 0.0
    for _ in range(4):
        dt = a.time_step()
        a.step(1)
        t_new = a.get_state()[1]
        assert t_new == t + dt
        t = t_new
    ref, t_ref = a.get_state()
    other = torch.from_numpy(W.random_perturbation(U0, 1e-2, 9)).cuda()
    b = dg.Solver(m, precision=dg.FP32_BULK)
    b.set_state(U0)
    b.step(1)
    b.time_step()
    b.step(1)
    b.rhs(other)
    b.kinetic()
    b.step(1)
    b.set_config(**dict(b.config(), side_block=128))
    b.step(1)
    U, tb = b.get_state()
    assert tb == t_ref
    np.testing.assert_array_equal(U, ref)
    bad = U0.copy()
    bad[1, 3, 4] = np.nan
    b.set_state(bad)
    with pytest.raises(dg.DgError) as err:
        b.step(1, sync=True)
    assert err.value.code == dg.DG_ERR_NONFINITE
    b.set_state(U0)
    b.step(1)
    assert np.isfinite(b.get_state()[0]).all()


def test_profile_step_matches_graph_steps():
    torch, dg = gpu_or_skip()
    N = 5
    m = mesh(N, (3, 3, 4), seed=5)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    a = dg.Solver(m, precision=dg.FP32_BULK)
    a.set_state(U0)
    a.step(3)
    b = dg.Solver(m, precision=dg.FP32_BULK)
    b.set_state(U0)
    prof = b.profile_step(3)
    np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
    assert prof["lift"][1] == 0 and prof["volume"][1] == 15 and prof["surf_flux"][1] == 15


def test_stage_form_selection():
    torch, dg = gpu_or_skip()
    m = mesh(3, (3, 3, 3))
    assert dg.Solver(m, precision=dg.FP32_BULK).stage_form() == 2
    assert dg.Solver(m).stage_form() == 4
    assert dg.Solver(m, precision=dg.FP32_BULK, nodes="gauss").stage_form() == 4
    s = dg.Solver(m)
    s.set_params(precision=dg.FP32_BULK)
    assert s.stage_form() == 2
    s.set_config(stage_form=1)
    assert s.stage_form() == 4


@pytest.mark.parametrize("N", [3, 7])
def test_persistent_launch_equals_per_kernel_launches(N):
    """One persistent launch per step (side and element phases of every stage
    separated by grid-wide barriers) runs the same per-side and per-element
    arithmetic as one launch per kernel and stage: bitwise equal steps, with
    the default scheme and with the 14-stage one."""
    torch, dg = gpu_or_skip()
    m = mesh(N, (4, 3, 5), seed=70 + N)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, N)
    for scheme in ("ck5", "ndb14"):
        out = []
        for persistent in (0, 1):
            s = dg.Solver(m, precision=dg.FP32_BULK)
            s.set_config(persistent=persistent)
            s.set_rk_scheme(scheme)
            s.set_state(U0)
            s.step(4)
            out.append(s.get_state())
            s.close()
        assert out[0][1] == out[1][1]
        np.testing.assert_array_equal(out[0][0], out[1][0])


def test_persistent_waits_give_up():
    """Failure detection without a GPU fault: a persistent step launch whose
    grid-wide barriers wait for a participant that never comes gives up after
    its bounded wait and reports DG_ERR_TIMEOUT; the state is untouched and
    the context steps on as if nothing happened."""
    torch, dg = gpu_or_skip()
    N = 3
    m = mesh(N, (4, 4, 4), seed=5)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    a = dg.Solver(m, precision=dg.FP32_BULK)
    a.set_config(persistent=1)
    a.set_state(U0)
    assert a.selftest_wait_timeout(2000) == dg.DG_ERR_TIMEOUT
    U, t = a.get_state()                       # no timeout left behind
    np.testing.assert_array_equal(U, U0.reshape(U.shape))
    a.step(3)
    b = dg.Solver(m, precision=dg.FP32_BULK)
    b.set_state(U0)
    b.step(3)
    np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
