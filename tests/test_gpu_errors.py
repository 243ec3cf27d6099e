"""Error behaviour of the C ABI as include/dg.h states it: invalid sizes and
parameters are refused with DG_ERR_ARG, meshes whose faces do not pair up with
DG_ERR_MESH, stepping before a state is set with DG_ERR_STATE, and a state
that turns non-finite is reported by DG_ERR_NONFINITE (no GPU fault on any of
them: the library checks on the host or flags on the device)."""
import ctypes as C

import numpy as np
import pytest

from paper_2404_12703_gb300 import workloads as W

from gpu_util import gpu_or_skip

pytestmark = pytest.mark.gpu


def _code(dg, fn, *args, **kw):
    try:
        fn(*args, **kw)
    except dg.DgError as e:
        return e.code
    return 0


def test_bad_sizes_and_parameters():
    torch, dg = gpu_or_skip()
    m = W.box_mesh(3, (3, 3, 3))
    assert _code(dg, dg.Solver, m, None, None) == 0
    bad_N = dict(m, N=8)
    assert _code(dg, dg.Solver, bad_N) == dg.DG_ERR_ARG
    empty = dict(m, xyz=m["xyz"][:0], corner_vid=m["corner_vid"][:0])
    assert _code(dg, dg.Solver, empty) == dg.DG_ERR_ARG
    for kw in (dict(gamma=1.0), dict(mu=-1.0), dict(Pr=0.0), dict(cfl=0.0), dict(riemann=7),
               dict(precision=5), dict(sutherland=1, T_ref=0.0)):
        assert _code(dg, dg.Solver, m, None, None, **kw) == dg.DG_ERR_ARG, kw


def test_meshes_whose_faces_do_not_pair_up():
    torch, dg = gpu_or_skip()
    # two elements across a periodic direction: distinct faces share all corners
    two = W.box_mesh(3, (2, 3, 3))
    assert _code(dg, dg.Solver, two) == dg.DG_ERR_MESH
    # an open face: one element's corner ids renumbered apart from the rest
    m = W.box_mesh(3, (3, 3, 3))
    cv = m["corner_vid"].copy()
    cv[5] = cv[5] + 10 ** 9
    assert _code(dg, dg.Solver, dict(m, corner_vid=cv)) == dg.DG_ERR_MESH
    # a face with a repeated corner id
    cv = m["corner_vid"].copy()
    cv[0, 1] = cv[0, 0]
    assert _code(dg, dg.Solver, dict(m, corner_vid=cv)) == dg.DG_ERR_MESH


def test_state_errors():
    torch, dg = gpu_or_skip()
    m = W.box_mesh(3, (3, 3, 3))
    s = dg.Solver(m)
    assert _code(dg, s.step, 1) == dg.DG_ERR_STATE
    assert _code(dg, s.advance, 0.1) == dg.DG_ERR_STATE
    U = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    s.set_state(U)
    assert _code(dg, s.advance, -1.0) == dg.DG_ERR_ARG
    assert _code(dg, s.step, -1) == dg.DG_ERR_ARG
    bad = U.copy()
    bad[4, 7, 0] = np.nan
    s.set_state(bad)
    s.step(1)
    assert _code(dg, s.get_state) == dg.DG_ERR_NONFINITE
    s.set_state(bad)
    assert _code(dg, s.step, 1, sync=True) == dg.DG_ERR_NONFINITE   # dg_step with t_out reports it too
    # a finite state clears the flag
    s.set_state(U)
    s.step(1)
    Ug, t = s.get_state()
    assert np.isfinite(Ug).all() and t > 0


def test_step_reports_the_time_reached():
    """dg_step with t_out synchronises and returns the time dg_get_state reads;
    zero steps return the current time."""
    torch, dg = gpu_or_skip()
    m = W.box_mesh(3, (3, 3, 3))
    s = dg.Solver(m)
    s.set_state(W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5), t=0.25)
    assert s.step(0, sync=True) == 0.25
    t1 = s.step(3, sync=True)
    assert t1 > 0.25 and s.get_state()[1] == t1
    assert s.step(2, dt=1e-3, sync=True) == t1 + 1e-3 + 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_equals_an_uninterrupted_run(prec):
    """Checkpoint / resume: 10 steps, the state and time read out, the context
    destroyed, a new one created from the checkpoint, 10 more steps: bitwise
    equal to 20 uninterrupted steps in FP64 (CFL steps, so the time step is
    recomputed from the restored state).  FP32-bulk takes the reference state
    of its shifted primitives from the state it is given, so a resumed run
    shifts about another state and agrees to FP32 rounding of the fluxes
    (below 1e-7 of the state after 10 steps; measured 2.3e-8), not bit for bit."""
    torch, dg = gpu_or_skip()
    precision = dg.FP64 if prec == "fp64" else dg.FP32_BULK
    m = W.box_mesh(4, (3, 4, 3), curved=0.1, seed=8)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1e-3, 3)
    a = dg.Solver(m, precision=precision)
    a.set_state(U0)
    a.step(20)
    U20, t20 = a.get_state()
    b = dg.Solver(m, precision=precision)
    b.set_state(U0)
    b.step(10)
    U10, t10 = b.get_state()
    b.close()
    c = dg.Solver(m, precision=precision)
    c.set_state(U10, t=t10)
    c.step(10)
    Uc, tc = c.get_state()
    if prec == "fp64":
        assert tc == t20
        np.testing.assert_array_equal(Uc, U20)
    else:
        assert abs(tc - t20) <= 1e-6 * t20
        assert np.abs(Uc - U20).max() <= 1e-7 * np.abs(U20).max()
