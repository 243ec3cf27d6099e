"""The manufactured-solution source of Sec. 5.1 on the GPU against the oracle:
the right-hand side with the source at a given time (both node sets,
inviscid and viscous, two advection speeds), ten LSERK steps with the source
taken at the stage times, FP32-bulk, and the refused combination with
Sutherland's law.  Bounds as in the parity tests."""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import parity_check, gpu_or_skip, oracle_params, parity_bound, rel_err

pytestmark = pytest.mark.gpu


def _mesh(N, nel=(3, 3, 4)):
    return W.box_mesh(N, nel, length=(2.0, 2.0, 2.0), origin=(-1.0, -1.0, -1.0), curved=0.1, seed=4)


def _oracle(m, nodes, quad=False):
    return O.Mesh(m["N"], m["xyz"], m["period"], quad=quad, gauss=nodes == "gauss")


@pytest.mark.parametrize("nodes", ["lgl", "gauss"])
@pytest.mark.parametrize("N,kw", [(3, dict()), (5, dict(viscous=0, source_a=0.5)), (4, dict(riemann="lf", mu=0.02))])
def test_rhs_with_source(nodes, N, kw):
    torch, dg = gpu_or_skip()
    m = _mesh(N)
    s = dg.Solver(m, nodes=nodes, source=dg.SOURCE_MMS, **kw)
    X = s.node_coords()
    t = 0.37
    U = W.random_perturbation(W.mms_state(X, t), 1e-3, 2)
    s.set_state(U, t=t)
    Ut = s.rhs().cpu().numpy()
    prm = oracle_params(s.params)
    ref = _oracle(m, nodes, quad=True).rhs(U, prm, t=t)
    o64 = _oracle(m, nodes).rhs(U, prm, t=t)
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)
    # the source matters at this size
    assert np.abs(ref - _oracle(m, nodes).rhs(U, oracle_params(dg.default_params(**{**kw, "source": 0})))).max() > 1e-3


@pytest.mark.parametrize("nodes", ["lgl", "gauss"])
def test_ten_steps_with_source(nodes):
    torch, dg = gpu_or_skip()
    N = 3
    m = _mesh(N, (3, 3, 3))
    s = dg.Solver(m, nodes=nodes, mu=0.01, source=dg.SOURCE_MMS)
    X = s.node_coords()
    U0 = W.mms_state(X, 0.0)
    s.set_state(U0)
    dt = 2e-3
    s.step(10, dt=dt)
    U, t = s.get_state()
    Uo, to, _ = _oracle(m, nodes).step(U0, oracle_params(s.params), 10, dt=dt)
    assert abs(t - to) <= 1e-14
    assert np.abs(U - Uo).max() / np.abs(Uo).max() <= 1e-10


def test_fp32_bulk_with_source():
    torch, dg = gpu_or_skip()
    N = 4
    m = _mesh(N)
    s = dg.Solver(m, precision=dg.FP32_BULK, mu=0.01, source=dg.SOURCE_MMS)
    X = s.node_coords()
    U = W.mms_state(X, 0.2)
    s.set_state(U, t=0.2)
    Ut = s.rhs().cpu().numpy()
    ref = _oracle(m, "lgl").rhs(U, oracle_params(s.params), t=0.2)
    assert np.all(rel_err(Ut, ref) <= 2e-4), rel_err(Ut, ref)


def test_source_refused_with_sutherland():
    torch, dg = gpu_or_skip()
    with pytest.raises(dg.DgError) as ex:
        dg.Solver(_mesh(2), source=dg.SOURCE_MMS, sutherland=1)
    assert ex.value.code == dg.DG_ERR_ARG


def _mms_l2(dg, N, nel, nodes, T=0.2, cfl=0.2):
    m = W.box_mesh(N, (nel,) * 3, length=(2.0, 2.0, 2.0), origin=(-1.0, -1.0, -1.0), curved=0.05, seed=2)
    s = dg.Solver(m, nodes=nodes, mu=0.01, cfl=cfl, source=dg.SOURCE_MMS)
    X = s.node_coords()
    s.set_state(W.mms_state(X, 0.0))
    t, _ = s.advance(T)
    U, _ = s.get_state()
    _, J = s.debug("metrics")
    w = s.quadrature_weights()
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    return np.sqrt((wq * (U[..., 0] - W.mms_state(X, t)[..., 0]) ** 2).sum() / wq.sum())


@pytest.mark.parametrize("nodes", ["lgl", "gauss"])
@pytest.mark.parametrize("N,levels,cfl", [(3, (8, 16), 0.2), (5, (6, 12), 0.1)])
def test_manufactured_solution_design_order(nodes, N, levels, cfl):
    """Sec. 5.1's convergence test on the GPU (the split form on LGL nodes and
    the standard form on GL nodes): the L2 density error at t = 0.2 on two
    nested curved meshes falls at the design order N + 1 or faster."""
    torch, dg = gpu_or_skip()
    e = [_mms_l2(dg, N, nel, nodes, cfl=cfl) for nel in levels]
    rate = np.log2(e[0] / e[1])
    assert rate > N + 0.5, (e, rate)
