"""Serving (continuous batching): cases of different meshes and degrees share
batched launches; each result must be the same alone and in the mix (bitwise:
the per-element arithmetic does not depend on the other cases of a launch),
equal the standalone solver over the same time-step sequence, and the loop
must admit waiting cases as pool memory frees up."""
import math
import time

import numpy as np
import pytest

from paper_2404_12703_gb300 import workloads as W

from gpu_util import gpu_or_skip

pytestmark = pytest.mark.gpu


def tgv_case(N, nel, seed):
    m = W.box_mesh(N, nel, curved=0.1, seed=seed)
    return m, W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5), 1.0 / 1600.0


def vortex_case(N, nel, seed):
    L = 10.0
    m = W.box_mesh(N, nel, length=(L, L, L), curved=0.05, seed=seed)
    U = W.isentropic_vortex_state(m["xyz"], center=(L / 2, L / 2), strength=5.0, period=m["period"])
    return m, U.reshape(m["E"], -1, 5), 0.0


CASES = [("tgv", 3, (4, 4, 4), 1), ("vortex", 5, (3, 4, 3), 2), ("tgv", 3, (3, 4, 5), 3),
         ("vortex", 7, (3, 3, 3), 4), ("tgv", 5, (3, 3, 4), 5)]


def make(kind, N, nel, seed):
    return (tgv_case if kind == "tgv" else vortex_case)(N, nel, seed)


POOLS = {3: 400, 5: 200, 7: 64}


def test_alone_and_in_the_mix_are_bitwise_equal():
    torch, dg = gpu_or_skip()
    t_end = 0.06
    built = [make(*c) for c in CASES]
    alone = []
    for m, U0, mu in built:
        srv = dg.Server(POOLS, max_cases=8)
        tk = srv.submit(m, U0, t_end, mu=mu)
        U, st = srv.wait(tk)
        srv.close()
        assert st["t_final"] == t_end and st["nonfinite"] == 0 and st["steps"] >= 3
        alone.append(U)
    srv = dg.Server(POOLS, max_cases=8)
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]
    for tk, Ua in zip(tickets, alone):
        U, st = srv.wait(tk)
        np.testing.assert_array_equal(U, Ua)
    s = srv.stats()
    assert s["finished"] == len(CASES) and s["resident"] == 0
    srv.close()


def test_server_matches_standalone_solver():
    """Same time-step sequence (CFL steps, the last one clipped at t_end)."""
    torch, dg = gpu_or_skip()
    m, U0, mu = make("tgv", 3, (4, 4, 4), 1)
    t_end = 0.05
    srv = dg.Server(POOLS, max_cases=4)
    U, st = srv.wait(srv.submit(m, U0, t_end, mu=mu))
    srv.close()
    K = int(st["steps"])
    s = dg.Solver(m, mu=mu)
    s.set_state(U0)
    s.step(K - 1)
    _, t = s.get_state()
    s.step(1, dt=t_end - t)
    Us, ts = s.get_state()
    assert abs(ts - t_end) < 1e-15
    assert np.abs(U - Us).max() <= 1e-14 * np.abs(Us).max()


def test_admission_waits_for_memory_and_overlaps():
    """A pool that holds two of the cases at a time: the others queue, are
    admitted as cases retire, and a case submitted while others run starts
    before they finish."""
    torch, dg = gpu_or_skip()
    built = [make("tgv", 3, (4, 4, 4), s) for s in range(5)]
    srv = dg.Server({3: 140}, max_cases=8)       # 64 elements per case: two fit
    t_end = 0.05
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built[:4]]
    time.sleep(0.05)
    late = srv.submit(*built[4][:2], t_end, mu=built[4][2])
    stats = [srv.wait(tk)[1] for tk in tickets + [late]]
    waits = [st["queue_wait"] for st in stats]
    assert max(waits) > 0.0
    assert sum(1 for w in waits if w > 1e-3) >= 2    # some cases had to wait for memory
    for st in stats:
        assert st["t_final"] == t_end and st["nonfinite"] == 0
    # a too-large case is refused at submission
    big = W.box_mesh(3, (6, 6, 6))
    with pytest.raises(dg.DgError):
        srv.submit(big, W.tgv_state(big["xyz"]).reshape(big["E"], -1, 5), 0.01)
    srv.close()


def test_fp32_bulk_serving_close_to_fp64():
    torch, dg = gpu_or_skip()
    m, U0, mu = make("vortex", 5, (3, 4, 3), 2)
    out = {}
    for prec in (dg.FP64, dg.FP32_BULK):
        srv = dg.Server(POOLS, max_cases=4, precision=prec)
        out[prec] = srv.wait(srv.submit(m, U0, 0.1, mu=mu))[0]
        srv.close()
    err = np.sqrt(((out[dg.FP32_BULK] - out[dg.FP64]) ** 2).sum() / (out[dg.FP64] ** 2).sum())
    assert err < 1e-5


def test_resident_dof_cap_admits_in_order():
    """With max_resident_dof equal to one case's DOF, three cases submitted at
    once run one after the other, in submission order, with unchanged results."""
    torch, dg = gpu_or_skip()
    built = [make("tgv", 3, (4, 4, 4), s) for s in (11, 12, 13)]
    dof = built[0][0]["E"] * 4 ** 3
    t_end = 0.03
    free = dg.Server(POOLS, max_cases=8)
    ref = [free.wait(free.submit(m, U0, t_end, mu=mu))[0] for m, U0, mu in built]
    free.close()
    srv = dg.Server(POOLS, max_cases=8, max_resident_dof=dof)
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]
    out = [srv.wait(tk) for tk in tickets]
    srv.close()
    for (U, st), Ur in zip(out, ref):
        np.testing.assert_array_equal(U, Ur)
        assert st["t_final"] == t_end
    waits = [st["queue_wait"] for _, st in out]
    services = [st["service_time"] for _, st in out]
    # each case is admitted only once the previous one has taken its last step
    # (its service time also covers copying its state out, after that)
    assert waits[0] < waits[1] < waits[2]
    assert waits[1] >= 0.5 * services[0]
    assert waits[2] >= waits[1] + 0.5 * services[1]


def test_fp32_bulk_alone_and_in_the_mix_are_bitwise_equal():
    """FP32-bulk cases carry their own reference state, so their results too
    do not depend on the other cases of a launch."""
    torch, dg = gpu_or_skip()
    t_end = 0.04
    built = [make(*c) for c in CASES[:3]]
    alone = []
    for m, U0, mu in built:
        srv = dg.Server(POOLS, max_cases=8, precision=dg.FP32_BULK)
        alone.append(srv.wait(srv.submit(m, U0, t_end, mu=mu))[0])
        srv.close()
    srv = dg.Server(POOLS, max_cases=8, precision=dg.FP32_BULK)
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]
    for tk, Ua in zip(tickets, alone):
        np.testing.assert_array_equal(srv.wait(tk)[0], Ua)
    srv.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_priority_policy_keeps_results_and_serves_oldest_first(prec):
    """With priority_dof of one DOF only the oldest resident case advances in
    each batched step (the others sit it out with their state unchanged): the
    results are bitwise those of the free-for-all mix, and the cases finish
    one after another in submission order."""
    torch, dg = gpu_or_skip()
    precision = dg.FP64 if prec == "fp64" else dg.FP32_BULK
    t_end = 0.04
    built = [make(*c) for c in CASES[:4]]
    free = dg.Server(POOLS, max_cases=8, precision=precision)
    ref = [free.wait(tk)[0] for tk in [free.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]]
    free.close()
    srv = dg.Server(POOLS, max_cases=8, precision=precision, priority_dof=1)
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]
    out = [srv.wait(tk) for tk in tickets]
    stats = srv.stats()
    srv.close()
    for (U, st), Ur in zip(out, ref):
        np.testing.assert_array_equal(U, Ur)
        assert st["t_final"] == t_end and st["nonfinite"] == 0
    # one case at a time: the batched steps add up to the cases' own steps
    # (plus at most one step per case for the hand-over)
    own = sum(st["steps"] for _, st in out)
    assert own <= stats["steps"] <= own + 2 * len(out) + 2, (own, stats["steps"])
    # and they finish in submission order
    ends = [st["time_to_solution"] for _, st in out]
    assert all(ends[i] < ends[i + 1] for i in range(len(ends) - 1)), ends


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_a_nonfinite_case_is_isolated(prec):
    """Fault isolation, made on the host: a NaN planted in one submitted case's
    initial state.  The CFL reduction flags that case only; it retires at
    once with the non-finite flag, and the three other cases of the mix end
    bitwise equal to their runs alone."""
    torch, dg = gpu_or_skip()
    precision = dg.FP64 if prec == "fp64" else dg.FP32_BULK
    t_end = 0.04
    built = [make(*c) for c in CASES[:4]]
    alone = []
    for m, U0, mu in built:
        srv = dg.Server(POOLS, max_cases=8, precision=precision)
        alone.append(srv.wait(srv.submit(m, U0, t_end, mu=mu))[0])
        srv.close()
    bad = 1
    mix = [(m, U0.copy(), mu) for m, U0, mu in built]
    mix[bad][1][2, 5, 0] = np.nan
    srv = dg.Server(POOLS, max_cases=8, precision=precision)
    tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in mix]
    for i, tk in enumerate(tickets):
        U, st = srv.wait(tk)
        if i == bad:
            assert st["nonfinite"] == 1 and st["t_final"] < t_end
        else:
            assert st["nonfinite"] == 0 and st["t_final"] == t_end
            np.testing.assert_array_equal(U, alone[i])
    srv.close()


def test_fp32_bulk_persistent_pools_match_per_kernel_pools():
    """Serving pools that run each step's stages as one persistent launch give
    the per-kernel pools' results bit for bit."""
    torch, dg = gpu_or_skip()
    t_end = 0.05
    built = [make(*c) for c in CASES]
    out = []
    for persistent in (0, 1):
        srv = dg.Server(POOLS, max_cases=8, precision=dg.FP32_BULK, persistent=persistent)
        tickets = [srv.submit(m, U0, t_end, mu=mu) for m, U0, mu in built]
        out.append([srv.wait(tk)[0] for tk in tickets])
        srv.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
