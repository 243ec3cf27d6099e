"""The launch-configuration autotuner (dg_autotune / dg_set_config).

* every launch variant of every degree gives the same steps: elements per
  block and side block sizes bitwise (they change no arithmetic), the FP64
  volume kernel's per-node mapping within the parity bound of the long-double
  oracle (it sums the split-form terms in another order);
* the tuner returns a valid configuration, times the variants that exist and
  leaves the state unchanged;
* invalid configurations are refused."""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

from gpu_util import parity_check, gpu_or_skip, mesh, oracle_params, parity_bound, rel_err

pytestmark = pytest.mark.gpu


def _variants(N, fp64, form=0):
    """Launch configurations (lift and volume elements per block, mapping, side
    block, stage form, prefetch, launch form).  FP32-bulk form 0 is the
    two-kernel stage on these periodic meshes (elements per block of its
    element kernel, side block, L2 prefetch on or off); form 1 the
    four-kernel stage; the launch form stays per kernel (the persistent form
    has its own tests)."""
    n3 = (N + 1) ** 3
    D = 1 if n3 >= 256 else 256 // n3
    lifts = [D] + ([2 * D] if 2 * D * n3 <= 1024 else [])
    vols = [D] + ([2 * D] if 2 * D * n3 <= 512 else [])
    maps = [1, 0] if fp64 else [0]
    if not fp64 and form == 0:
        return [(D, ve, 0, sb, 0, pf, 0) for ve in vols for sb in (256, 128) for pf in (1, 0)]
    return [(le, ve, pr, sb, form, 1, 0) for le in lifts for ve in vols for pr in maps for sb in (256, 128)]


def _two_steps(s, U0, dt):
    s.set_state(U0)
    s.step(2, dt=dt)
    return s.get_state()[0]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_every_variant_gives_the_same_steps(N):
    torch, dg = gpu_or_skip()
    m = mesh(N, (3, 3, 4), seed=40 + N)
    U0 = W.random_perturbation(W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5), 1e-3, N)
    for prec, form in ((dg.FP64, 0), (dg.FP32_BULK, 0), (dg.FP32_BULK, 1)):
        s = dg.Solver(m, precision=prec)
        s.set_config(*_variants(N, prec == dg.FP64, form)[0])
        assert s.stage_form() == (2 if (prec == dg.FP32_BULK and form == 0) else 4)
        s.set_state(U0)
        dt = s.time_step()
        ref = _two_steps(s, U0, dt)  # the form's default configuration
        for cfg in _variants(N, prec == dg.FP64, form):
            s.set_config(*cfg)
            U = _two_steps(s, U0, dt)
            default_mapping = cfg[2] == (1 if prec == dg.FP64 else 0)
            if default_mapping:
                np.testing.assert_array_equal(U, ref, err_msg=str(cfg))
            else:
                prm = oracle_params(s.params)
                q = O.Mesh(N, m["xyz"], m["period"], quad=True).step(U0, prm, 2, dt=dt)[0]
                o64 = O.Mesh(N, m["xyz"], m["period"]).step(U0, prm, 2, dt=dt)[0]
                bound, floor = parity_bound(o64, q)
                parity_check(rel_err(U, q), bound, floor)
        s.close()


def test_autotune_keeps_the_state_and_picks_a_variant():
    torch, dg = gpu_or_skip()
    N = 5
    m = mesh(N, (4, 4, 4), seed=50)
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    for prec in (dg.FP64, dg.FP32_BULK):
        s = dg.Solver(m, precision=prec)
        s.set_state(U0)
        cfg, ms = s.autotune()
        U, t = s.get_state()
        np.testing.assert_array_equal(U, U0)
        assert t == 0.0
        valid = {v for v in _variants(N, prec == dg.FP64)}
        assert tuple(cfg.values()) in valid, cfg
        assert ms["vol_D"] > 0 and ms["side_256"] > 0
        # the two-kernel FP32-bulk stage has no separate lifting kernel
        assert (ms["lift_D"] is not None) == (prec == dg.FP64)
        assert (ms["vol_D_other_mapping"] is not None) == (prec == dg.FP64)
        assert s.config() == cfg
        # tuned steps agree with the oracle
        dt = s.time_step()
        U2 = _two_steps(s, U0, dt)
        prm = oracle_params(s.params)
        q = O.Mesh(N, m["xyz"], m["period"], quad=True).step(U0, prm, 2, dt=dt)[0]
        if prec == dg.FP64:
            o64 = O.Mesh(N, m["xyz"], m["period"]).step(U0, prm, 2, dt=dt)[0]
            bound, floor = parity_bound(o64, q)
            parity_check(rel_err(U2, q), bound, floor)
        else:
            # FP32-bulk steps: the state changes by O(dt |Ut|) per step, with
            # FP32-rounded fluxes (the near-zero z-momentum sets the largest
            # per-variable relative error)
            assert rel_err(U2, q).max() < 1e-4
        s.close()


def test_invalid_configurations_are_refused():
    torch, dg = gpu_or_skip()
    m = mesh(7, (3, 3, 3))
    s = dg.Solver(m)
    for cfg in [(3, 0, -1, 0), (0, 2, -1, 0), (0, 0, 2, 0), (0, 0, -1, 64), (0, 0, -1, 0, 2), (0, 0, -1, 0, 0, 3),
                (0, 0, -1, 0, 0, 1, 2)]:
        with pytest.raises(dg.DgError) as ei:
            s.set_config(*cfg)
        assert ei.value.code == dg.DG_ERR_ARG
    s32 = dg.Solver(m, precision=dg.FP32_BULK)
    with pytest.raises(dg.DgError):
        s32.set_config(0, 0, 1, 0)
