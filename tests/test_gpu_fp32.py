"""FP32-bulk mode: flux, volume and surface arithmetic in FP32 (on shifted
primitives), state, RK register, metrics and reductions in FP64, against the
FP64 oracle and the FP64 path.

Bounds (FP32 unit round-off is 6e-8; the operator sums O(N^2) terms per node):
  * one right-hand side: max-norm error per variable <= 2e-4 of max |Ut|;
  * free stream: |Ut| <= 1e-5 of the flux scale;
  * after 40 LSERK steps of the Taylor-Green vortex: kinetic-energy
    dissipation rate within 1e-5 relative of the FP64 path (the precision
    target), and the L2 state error within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import gpu_or_skip, mesh, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,nel,Ma,kw", [
    (3, (4, 4, 4), 0.1, dict()),
    (7, (3, 4, 3), 0.1, dict()),
    (5, (3, 3, 3), 0.5, dict(riemann="lf")),
    (2, (3, 4, 5), 0.3, dict(mu=0.01)),
    (5, (6, 3, 3), 0.5, dict(riemann="lf", shock_capturing=1, viscous=0)),
])
def test_fp32_rhs_against_oracle(N, nel, Ma, kw):
    torch, dg = gpu_or_skip()
    m = mesh(N, nel)
    s = dg.Solver(m, precision=dg.FP32_BULK, **kw)
    U = W.random_perturbation(W.tgv_state(m["xyz"], Ma=Ma).reshape(m["E"], -1, 5), 1e-3, 5)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    ref = O.Mesh(N, m["xyz"], m["period"]).rhs(U, oracle_params(s.params))
    err = rel_err(Ut, ref)
    assert np.all(err <= 2e-4), err


def test_fp32_free_stream():
    torch, dg = gpu_or_skip()
    N = 7
    m = mesh(N, (3, 3, 3))
    s = dg.Solver(m, precision=dg.FP32_BULK)
    U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=71.4)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    _, J = s.debug("metrics")
    _, _, _, _, Ds, _ = O.ops(N)
    F = 1.1 * 0.25 + 71.4 + 71.4 * 3.5
    assert np.abs(Ut).max() < 1e-5 * F * np.abs(Ds).sum(axis=1).max() / J.min()


def test_fp32_time_integration_against_fp64():
    """Taylor-Green vortex Re = 1600, Ma = 0.1, 6^3 curved elements at N = 5,
    40 steps at the CFL step of the initial state, FP32-bulk against FP64."""
    torch, dg = gpu_or_skip()
    N = 5
    m = mesh(N, (6, 6, 6))
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    out = {}
    for prec in (dg.FP64, dg.FP32_BULK):
        s = dg.Solver(m, precision=prec)
        s.set_state(U0)
        dt = s.time_step() if prec == dg.FP64 else out[dg.FP64][2]
        s.step(40, dt=dt)
        U, t = s.get_state()
        out[prec] = (U, s.kinetic(), dt, t)
    U64, k64, _, t64 = out[dg.FP64]
    U32, k32, _, t32 = out[dg.FP32_BULK]
    assert t32 == t64
    rate_err = abs(k32[1] - k64[1]) / abs(k64[1])
    assert rate_err <= 1e-5, rate_err
    assert abs(k32[0] - k64[0]) <= 1e-10 * abs(k64[0])
    l2 = np.sqrt(((U32 - U64) ** 2).sum() / (U64 ** 2).sum())
    assert l2 <= 1e-5, l2
    mom = np.sqrt(((U32[..., 1:4] - U64[..., 1:4]) ** 2).sum() / (U64[..., 1:4] ** 2).sum())
    assert mom <= 1e-5, mom


def test_precision_switch_keeps_state():
    torch, dg = gpu_or_skip()
    N = 3
    m = mesh(N, (4, 4, 4))
    s = dg.Solver(m)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    s.set_state(U0)
    a = s.rhs().cpu().numpy()
    s.set_params(precision=dg.FP32_BULK)
    b = s.rhs().cpu().numpy()
    s.set_params(precision=dg.FP64)
    c = s.rhs().cpu().numpy()
    np.testing.assert_array_equal(a, c)
    assert rel_err(b, a).max() < 2e-4


def test_arrays_follow_the_parameters():
    """A context holds the working arrays of its own precision only; switching
    the precision (or turning shock capturing on) with dg_set_params forms
    the missing ones, and the results equal those of a context created with
    those parameters, bit for bit."""
    torch, dg = gpu_or_skip()
    N = 4
    m = mesh(N, (3, 3, 4))
    U = torch.from_numpy(W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, 4)).cuda()
    s = dg.Solver(m)
    b64 = s.sizes()["bytes"]
    r64 = s.rhs(U).cpu().numpy()
    s.set_params(precision=dg.FP32_BULK)
    assert s.sizes()["bytes"] > b64
    r32 = s.rhs(U).cpu().numpy()
    f32 = dg.Solver(m, precision=dg.FP32_BULK)
    assert f32.sizes()["bytes"] < s.sizes()["bytes"]
    np.testing.assert_array_equal(r32, f32.rhs(U).cpu().numpy())
    s.set_params(precision=dg.FP64)
    np.testing.assert_array_equal(s.rhs(U).cpu().numpy(), r64)
    s.set_params(shock_capturing=1, alpha_force=0.3, riemann="lf")
    ref = dg.Solver(m, shock_capturing=1, alpha_force=0.3, riemann="lf")
    np.testing.assert_array_equal(s.rhs(U).cpu().numpy(), ref.rhs(U).cpu().numpy())
