"""Helpers for the GPU parity tests: building libdg once, feeding the same seeded
inputs to the CUDA path and the oracle, and the error norms with their bounds."""
import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W

_built = False


def gpu_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    global _built
    if not _built:
        from paper_2404_12703_gb300 import build
        build.build()
        _built = True
    from paper_2404_12703_gb300 import dg
    dg.load()
    return torch, dg


def oracle_params(dgp):
    """Oracle parameter vector equal to a dg.Params."""
    return O.params(gamma=dgp.gamma, R=dgp.R, Pr=dgp.Pr, mu=dgp.mu, riemann=dgp.riemann,
                    viscous=dgp.viscous, shock=dgp.shock_capturing, alpha_min=dgp.alpha_min,
                    alpha_max=dgp.alpha_max, cfl=dgp.cfl, dfl=dgp.dfl, alpha_force=dgp.alpha_force,
                    sutherland=dgp.sutherland, T_ref=dgp.T_ref, source=dgp.source, source_A=dgp.source_A,
                    source_a=dgp.source_a)


def rel_err(a, ref):
    """max-norm error per conservative variable, relative to max |ref| of that variable."""
    a = np.asarray(a).reshape(-1, 5)
    ref = np.asarray(ref).reshape(-1, 5)
    scale = np.abs(ref).max(axis=0)
    scale[scale == 0] = 1.0
    return np.abs(a - ref).max(axis=0) / scale


def parity_bound(oracle_fp64, oracle_ld, floor_factor=3.0, base=1e-12):
    """Per-variable bound: 1e-12, or floor_factor times the FP64 oracle's own
    rounding error against the long-double oracle when that floor is higher
    (the stated 1e-12 sits below FP64's floor at low Mach number and high N)."""
    floor = rel_err(oracle_fp64, oracle_ld)
    return np.maximum(base, floor_factor * floor), floor


def parity_check(err, bound, floor):
    """Asserts err <= bound per variable with a message that gives the ratio
    of the GPU error to the FP64 floor (the FP64 oracle's own error against
    the long-double one); with DG_PARITY_LOG set, appends that ratio, the
    error and the floor of the calling test as one JSON line to that file."""
    import inspect
    import json
    import os
    floor = np.asarray(floor, dtype=float)
    err = np.asarray(err, dtype=float)
    ratio = np.where(floor > 0, err / np.where(floor > 0, floor, 1.0), 0.0)
    path = os.environ.get("DG_PARITY_LOG")
    if path:
        test = os.environ.get("PYTEST_CURRENT_TEST", inspect.stack()[1].function).split(" ")[0]
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "ratio_max": float(ratio.max()), "err": err.tolist(),
                                "floor": floor.tolist()}) + "\n")
    assert np.all(err <= bound), {"err": err, "bound": bound, "floor": floor, "gpu_to_floor": ratio}


def rk_stage_weight_sum(A, B):
    """sum_i |b_i| over the Butcher weights of a 2N-storage scheme
    (dU_j = A_j dU_{j-1} + dt L_j, U_j = U_{j-1} + B_j dU_j): stage i's
    right-hand side enters the step with b_i = sum_{j >= i} B_j prod_{k=i+1..j} A_k,
    so a rounding error in each stage's right-hand side reaches the state
    amplified by up to this sum (1 when every b_i >= 0)."""
    s = len(A)
    b = [sum(B[j] * float(np.prod(A[i + 1:j + 1])) for j in range(i, s)) for i in range(s)]
    return float(np.sum(np.abs(b)))


def mesh(N, nel, curved=0.1, seed=20240419, **kw):
    return W.box_mesh(N, nel, curved=curved, seed=seed, **kw)
