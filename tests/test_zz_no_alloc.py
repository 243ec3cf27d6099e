"""The allocation-free kinetic-energy entry point, dg_kinetic_noalloc.

It exists for callers that cannot call cudaMalloc (their device memory is
handed out in advance by their own arena or pool, or they must not take the
implicit device synchronisation that an allocation can cause).  It keeps its
scratch in a fixed device array inside the library, so this test checks that
it gives the same numbers as the allocating path, dg_kinetic, on two calls in
a row (the second call reuses the scratch the first one left behind), and that
an element count beyond its fixed capacity is refused.

The file name sorts last so that a stop-at-first-failure run has already run
every other test; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_12703_gb300 import workloads as W

from gpu_util import gpu_or_skip

pytestmark = pytest.mark.gpu


def _compare(torch, dg, m, N, nodes, s, U, calls=2):
    """dg_kinetic_noalloc through the C ABI against dg_kinetic of solver s on
    state U, on `calls` calls in a row."""
    s.set_state(U)
    ref = np.array(s.kinetic())                        # allocating path: E_k, dE_k/dt, |Omega|
    Ud = torch.from_numpy(U).cuda()
    Ut = s.rhs(Ud)                                     # the same right-hand side dg_kinetic uses
    _, J = s.debug("metrics")
    Jd = torch.from_numpy(J).cuda()
    lib = dg.load()
    for call in range(calls):
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.dg_kinetic_noalloc(N, nodes, m["E"], ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(Jd.data_ptr()),
                                    ctypes.c_void_p(Ut.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == dg.DG_OK, lib.dg_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same quantities, different summation order: round-off level agreement
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0]), (call, got, ref)
        assert abs(got[1] - ref[1]) <= 1e-12 * max(abs(ref[1]), 1e-300) + 1e-15, (call, got, ref)
        assert abs(got[2] - ref[2]) <= 1e-12 * ref[2], (call, got, ref)
    return ref, Ud, Jd


@pytest.mark.parametrize("N,nodes", [(5, "lgl"), (3, "lgl"), (5, "gauss"), (2, "gauss")])
def test_kinetic_noalloc_matches_dg_kinetic(N, nodes):
    torch, dg = gpu_or_skip()
    m = W.box_mesh(N, (4, 3, 5), curved=0.1, seed=31)
    nd = dg.NODES_GAUSS if nodes == "gauss" else dg.NODES_LGL
    s = dg.Solver(m, mu=0.01, nodes=nodes)
    xyz = s.node_coords() if nodes == "gauss" else m["xyz"]
    U = W.random_perturbation(W.tgv_state(xyz, Ma=0.3).reshape(m["E"], -1, 5), 1e-2, 4)
    ref, Ud, Jd = _compare(torch, dg, m, N, nd, s, U)
    # without Ut the rate is zero and the energy unchanged
    out = dg.kinetic_noalloc(N, Ud, Jd, nodes=nd)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[1] == 0.0 and abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])


def test_kinetic_noalloc_at_its_element_limit():
    """262,144 elements (64^3 at N = 1): the largest input the scratch holds."""
    torch, dg = gpu_or_skip()
    N = 1
    m = W.box_mesh(N, (64, 64, 64), curved=0.1, seed=3)
    assert m["E"] == 262144
    s = dg.Solver(m, mu=0.01)
    U = W.tgv_state(m["xyz"], Ma=0.3).reshape(m["E"], -1, 5)
    _compare(torch, dg, m, N, dg.NODES_LGL, s, U)


def test_kinetic_noalloc_refuses_oversized_input():
    torch, dg = gpu_or_skip()
    lib = dg.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.dg_kinetic_noalloc(3, dg.NODES_LGL, 262145, p, p, None, p, None)
    assert st == dg.DG_ERR_ARG
    assert b"262144" in lib.dg_last_error()
    assert lib.dg_kinetic_noalloc(9, dg.NODES_LGL, 10, p, p, None, p, None) == dg.DG_ERR_ARG
    assert lib.dg_kinetic_noalloc(3, 2, 10, p, p, None, p, None) == dg.DG_ERR_ARG
