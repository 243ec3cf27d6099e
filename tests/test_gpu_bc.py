"""Boundary conditions on the GPU against the oracle: wall-bounded channels
(curved, rotated, renumbered elements) with isothermal and adiabatic no-slip
walls, slip walls and prescribed states; maps bit-exact, the right-hand side
within the parity bound, Couette flow a discrete steady state, ten steps,
FP32-bulk, and the error cases."""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import parity_check, gpu_or_skip, oracle_params, parity_bound, rel_err

pytestmark = pytest.mark.gpu

BCS = {
    "walls": [(1, 0.0, 0.0, 0.0, 1.2), (1, 0.6, 0.0, 0.1, 1.0)],
    "adiabatic+slip": [(2, 0.3, 0.0, 0.0), (3,)],
    "state": [(4, 1.1, 0.3, 0.2, -0.1, 6.0), (4, 0.9, 0.2, 0.1, 0.0, 5.5)],
    "inflow+outflow": [(4, 1.1, 0.3, 0.2, -0.1, 6.0), (5, 2.2)],
}


def _channel(N, nel=(3, 4, 3), seed=31, curved=0.1, bcs="walls"):
    m = W.box_mesh(N, nel, length=(2.0, 1.0, 2.0), origin=(0.0, 0.0, 0.0),
                   periodic=(True, False, True), seed=seed, curved=curved)
    m["face_bc"] = W.box_face_bc(m, {"y-": 1, "y+": 2})
    m["bcs"] = BCS[bcs]
    return m


def _oracle(m, quad=False):
    return O.Mesh(m["N"], m["xyz"], m["period"], quad=quad, face_bc=m["face_bc"], bcs=m["bcs"])


def _state(m, seed=3):
    U = W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5)
    return W.random_perturbation(U, 1e-2, seed)


def test_maps_bit_exact():
    torch, dg = gpu_or_skip()
    m = _channel(3)
    s = dg.Solver(m)
    nbr, nodes = s.debug("maps")
    on, of, om, onode = _oracle(m).connectivity()
    np.testing.assert_array_equal(nbr[..., 0], on)
    np.testing.assert_array_equal(nbr[..., 1], of)
    np.testing.assert_array_equal(nbr[..., 2], om)
    np.testing.assert_array_equal(nodes, onode)
    assert (on < 0).sum() == 2 * 3 * 3


@pytest.mark.parametrize("N,bcs,kw", [
    (3, "walls", dict()),
    (5, "walls", dict(riemann="lf", sutherland=1, T_ref=1.0)),
    (4, "adiabatic+slip", dict()),
    (3, "state", dict()),
    (5, "state", dict(riemann="lf")),
    (3, "adiabatic+slip", dict(viscous=0)),
    (3, "walls", dict(shock_capturing=1, alpha_force=0.3)),
    (3, "inflow+outflow", dict()),
    (5, "inflow+outflow", dict(riemann="lf", viscous=0)),
])
def test_rhs_parity(N, bcs, kw):
    torch, dg = gpu_or_skip()
    m = _channel(N, bcs=bcs)
    s = dg.Solver(m, **kw)
    U = _state(m)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    ref = _oracle(m, quad=True).rhs(U, prm)
    o64 = _oracle(m).rhs(U, prm)
    bound, floor = parity_bound(o64, ref)
    err = rel_err(Ut, ref)
    parity_check(err, bound, floor)


@pytest.mark.parametrize("N,Rg", [(2, 1.0), (3, 1.0), (5, 1.0), (3, 2.5)])
def test_couette_is_a_discrete_steady_state(N, Rg):
    torch, dg = gpu_or_skip()
    mu, Uw, Tw = 0.02, 0.7, 1.3 / Rg
    m = _channel(N, curved=0.0)
    m["bcs"] = [(1, 0.0, 0.0, 0.0, Tw), (1, Uw, 0.0, 0.0, Tw)]
    s = dg.Solver(m, mu=mu, R=Rg)
    U = W.couette_state(m["xyz"], U_wall=Uw, T_wall=Tw, p=0.9, mu=mu, R=Rg).reshape(m["E"], -1, 5)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    assert np.abs(Ut).max() < 1e-12, np.abs(Ut).max(axis=(0, 1))
    # and stays put over steps
    s.set_state(U)
    s.step(20)
    U20, _ = s.get_state()
    assert np.abs(U20 - U).max() < 1e-12


def test_ten_steps_parity():
    torch, dg = gpu_or_skip()
    N = 3
    m = _channel(N)
    s = dg.Solver(m)
    U0 = _state(m)
    s.set_state(U0)
    s.step(10)
    U, t = s.get_state()
    prm = oracle_params(s.params)
    Uo, to, _ = _oracle(m).step(U0, prm, 10)
    assert abs(t - to) <= 1e-13 * to
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_fp32_bulk_against_oracle():
    torch, dg = gpu_or_skip()
    for bcs in ("walls", "adiabatic+slip", "state", "inflow+outflow"):
        m = _channel(4, bcs=bcs)
        s = dg.Solver(m, precision=dg.FP32_BULK)
        U = _state(m)
        Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
        ref = _oracle(m).rhs(U, oracle_params(s.params))
        assert np.all(rel_err(Ut, ref) <= 2e-4), (bcs, rel_err(Ut, ref))


def test_boundary_errors():
    torch, dg = gpu_or_skip()
    m = _channel(3)
    no_bc = dict(m, face_bc=None)
    with pytest.raises(dg.DgError) as e:
        dg.Solver(no_bc)
    assert e.value.code == dg.DG_ERR_MESH
    fb = m["face_bc"].copy()
    inner = np.argwhere(fb == 0)[0]
    fb[inner[0], inner[1]] = 1
    with pytest.raises(dg.DgError) as e:
        dg.Solver(dict(m, face_bc=fb))
    assert e.value.code == dg.DG_ERR_MESH
    with pytest.raises(dg.DgError) as e:
        dg.Solver(dict(m, bcs=[(7,), (3,)]))
    assert e.value.code == dg.DG_ERR_ARG
    srv = dg.Server({3: 200}, max_cases=2)
    with pytest.raises(dg.DgError):
        srv.submit(m, _state(m), 0.01)
    srv.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sponge_parity(prec):
    torch, dg = gpu_or_skip()
    N = 4
    m = _channel(N, bcs="inflow+outflow")
    p = dg.FP64 if prec == "fp64" else dg.FP32_BULK
    s = dg.Solver(m, precision=p)
    U = _state(m)
    y = m["xyz"].reshape(m["E"], -1, 3)[..., 1]
    sigma = 5.0 * np.clip(y - 0.6, 0.0, None) ** 2           # a zone near the outflow
    Ub = W.uniform_state(U.shape[:2], rho=1.0, vel=(0.0, 0.3, 0.0), p=2.0)
    s.set_sponge(sigma, Ub)
    Ut = s.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    prm = oracle_params(s.params)
    Mq = _oracle(m, quad=True)
    Mq.set_sponge(sigma, Ub)
    ref = Mq.rhs(U, prm)
    if p == dg.FP64:
        M64 = _oracle(m)
        M64.set_sponge(sigma, Ub)
        bound, floor = parity_bound(M64.rhs(U, prm), ref)
        parity_check(rel_err(Ut, ref), bound, floor)
    else:
        assert np.all(rel_err(Ut, ref) <= 2e-4)
    # removing the sponge gives the plain operator back, bitwise
    plain = dg.Solver(m, precision=p).rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    s.set_sponge(None)
    np.testing.assert_array_equal(s.rhs(torch.from_numpy(U).cuda()).cpu().numpy(), plain)
