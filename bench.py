"""Benchmark: DOF-updates per second per RK stage of the DGSEM time step.

Default workload (one GPU): Taylor-Green vortex Re = 1600, Ma = 0.1 on the
24^3-element curved hexahedral mesh (nodes displaced by 0.1 h sin products,
element ids and local frames permuted from seed 20240419), N = 7 (7,077,888
DOF), KEP split form + Roe + BR1, five-stage LSERK4 with the CFL rule, FP64.
A step is one full time step (CFL reduction + 5 stages of the whole operator).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (a
plain FP64 C restatement of the same method, test infrastructure) on a bounded
sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage (FP64 vs FP32-bulk) and % HBM roofline; serving p50/p99"
UNIT = "DOF-updates/s"
STAGES = 5
N_DEG = 7
NEL = 24
SEED = 20240419

# Algorithmic cost per DOF per RK stage at N = 7 (FP64), counting an FMA as two
# flops: split-form KEP volume with pair symmetry 567, conservative BR1 lifting
# 612, viscous fluxes and their volume term 324, surface Riemann + BR1 fluxes
# 131, ConsToPrim / SurfInt / ApplyJac / RK 50.
FLOPS_PER_DOF = {"volume": 567 + 324 + 30, "lift": 612, "surf_flux": 131, "surf_prims": 10, "cfl": 10}
# Algorithmic bytes per DOF per stage of the minimal two-phase method (FP64):
# 8 (30 + 204 / (N + 1)).
BYTES_PER_DOF = 8 * (30 + 204 / (N_DEG + 1))
# DRAM bytes per DOF of one k_volume<7,1> launch, from the ncu capture summarised
# in profiles/k_volume_tgv12_N7_fp64.md (12^3 mesh; the traffic scales with
# the DOF count).  Set to None whenever the kernel changes until re-measured.
VOLUME_TRAFFIC_BYTES_PER_DOF = 332.02
# FP32-bulk, four-kernel stage: algorithmic bytes per DOF of one volume-kernel
# launch (reads U 40, FP32 metrics 40, FP32 lifted gradients 48, dU 40, surface
# fluxes ~8; writes U 40, dU 40)
VOLUME32_BYTES_PER_DOF = 40 + 40 + 48 + 40 + 8 + 40 + 40
# FP32-bulk, two-kernel stage (the default on periodic meshes), per DOF at
# N = 7, with 6 / (N + 1) = 0.75 element face nodes and 0.375 side nodes per
# DOF.  Element kernel: reads U 40, the FP32 RK register 20, FP32 metrics
# 40, the lifting's volume sums 48, q* 0.75 x 16, side normals 0.75 x 12,
# f* 0.75 x 20; writes U 40, the register 20, the lifting's volume sums of
# the updated state 48, face traces 0.75 x 32 and partial viscous fluxes
# 0.75 x 16 (the sums, 96 B, in viscous runs such as the benchmark's TGV).
# The last stage of a step also reduces the next time step's spectral radii
# from the state and metrics it holds (no further bytes), so the CFL
# reduction kernel does not read the state again.
# Side kernel, per side
# node: reads two traces 64, two partial viscous fluxes 32, side geometry 28;
# writes f* 20 and q* 16 (the edge and corner nodes' re-reads of neighbouring
# traces are not counted).
FACE_NODES_PER_DOF = 6 / (N_DEG + 1)
FELEM32_BYTES_PER_DOF = (40 + 20 + 40 + 48 + FACE_NODES_PER_DOF * (16 + 12 + 20) + 40 + 20 + 48
                         + FACE_NODES_PER_DOF * (32 + 16))
FFLUX32_BYTES_PER_DOF = FACE_NODES_PER_DOF / 2 * (64 + 32 + 28 + 20 + 16)
# a whole stage of the minimal two-phase method with the RK register and the
# metrics in FP64 and the face traces in FP32: 342 B at N = 7 (the budget the
# whole-step HBM fraction is quoted against)
BYTES32_PER_DOF = 342.0
# DRAM bytes per DOF of one launch of the FP32-bulk dominant kernel (ncu); None
# whenever the kernel changes until re-measured
VOLUME32_TRAFFIC_BYTES_PER_DOF = 284.5
# Standard DGSEM on Gauss-Legendre nodes, algorithmic flops per DOF and stage
# (n = N + 1, FMA = 2 flops).  Lifting: D-hat line sums 72 n, metric products
# 36, both faces of three lines 144, 1/J 12, ProlongToFace of the twelve
# gradient components 144.  Volume: D-hat line sums 30 n, three contravariant
# Euler and viscous fluxes 114, stress and heat flux 40, SurfInt 60,
# ApplyJac and RK 25.
GL_FLOPS_PER_DOF = {"lift": 72 * (N_DEG + 1) + 336, "volume": 30 * (N_DEG + 1) + 239}


def workload_desc(nel=NEL):
    E = nel ** 3
    dof = E * (N_DEG + 1) ** 3
    return {
        "workload": f"TGV Re=1600 Ma=0.1 on a {nel}^3-element curved hex mesh (0.1 h sin-product node "
                    f"displacement, element ids and local frames permuted from seed {SEED}), N={N_DEG}, "
                    f"{dof} DOF, KEP split form + Roe + BR1, LSERK4 (5 stages) with CFL 0.9",
        "elements": E, "N": N_DEG, "dof": dof, "precision": "FP64",
        "l2": f"inputs larger than L2 (state {dof * 40 / 1e6:.0f} MB, metrics {dof * 80 / 1e6:.0f} MB "
              f"per GPU); no flush",
    }


def max_over_ranks(x, world, device):
    """The largest of the ranks' values (the job's time is its slowest rank)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replicas_value(units_per_step, ms_step, world):
    """Whole-job throughput of `world` replicas, each doing units_per_step
    per step, timed by the slowest rank."""
    return world * units_per_step / (ms_step * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"dg_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                try:
                    power.append(float(parts[3]))
                except ValueError:
                    pass
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w": statistics.median(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 ALU peak of a GB300, derived from unit counts and clocks: 152 SMs x
# 2 FP64 FMA lanes per SM per clock x 2 flop x 2.07 GHz = 1.26 TFLOP/s (the
# nominal 1.25 TFLOP/s FP64 figure of the part).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def cpu_oracle_sample(steps, nel=6, seed=SEED):
    """The oracle (plain FP64 C, single thread) on a bounded sample of the same
    workload: a nel^3 curved, permuted mesh at N = 7, `steps` LSERK steps."""
    import oracle as O
    from paper_2404_12703_gb300 import workloads as W
    m = W.box_mesh(N_DEG, (nel,) * 3, curved=0.1, seed=seed)
    M = O.Mesh(N_DEG, m["xyz"], m["period"])
    U = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    prm = O.params()
    dof = m["E"] * (N_DEG + 1) ** 3
    times = []
    t = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        U, t, _ = M.step(U, prm, 1, t=t)
        times.append(time.perf_counter() - t0)
    return dof, times


def _oracle_replica(args):
    """One process of the all-cores oracle measurement: builds its sample,
    takes `warmup` untimed steps, waits at the barrier, then steps it
    (returns the stepping time)."""
    steps, nel, seed, barrier = args[:4]
    warmup = args[4] if len(args) > 4 else 0
    import oracle as O
    from paper_2404_12703_gb300 import workloads as W
    m = W.box_mesh(N_DEG, (nel,) * 3, curved=0.1, seed=seed)
    M = O.Mesh(N_DEG, m["xyz"], m["period"])
    U = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    prm = O.params()
    t = 0.0
    if warmup:
        U, t, _ = M.step(U, prm, warmup)
    barrier.wait(timeout=300)
    t0 = time.perf_counter()
    M.step(U, prm, steps, t=t)
    return time.perf_counter() - t0


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_oracle_all_cores(steps=2, nel=4, seed=SEED, warmup=0):
    """The oracle as it stands on every usable host core: one independent
    replica of the sample per core (spawned processes, so nothing is forked
    from a process that holds a CUDA context), all released together by a
    barrier; aggregate DOF-updates/s over the slowest replica's time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(cores)
        with ctx.Pool(cores) as pool:
            times = pool.map_async(_oracle_replica, [(steps, nel, seed, barrier, warmup)] * cores,
                                   chunksize=1).get(timeout=900)
    dof = nel ** 3 * (N_DEG + 1) ** 3
    value = cores * dof * STAGES * steps / max(times)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{cores} independent replicas (one process per core) of {nel}^3 elements of the same "
                      f"curved N=7 TGV workload ({dof} DOF each), {steps} LSERK steps each, single-threaded "
                      f"FP64 C per process; the oracle is not parallelised within a mesh"}


SERVING_SIZES = (4, 8, 12, 16)
SERVING_T_END = 0.02


def serving_cases(n_cases, seed=5):
    """Seeded stream of cases (a shortened version of the serving workload):
    mesh n^3 with n from {4, 8, 12, 16}, N from {3, 5, 7}, half Taylor-Green
    vortex (Re 1600, Ma 0.1, viscous), half isentropic vortex (inviscid,
    strength 5, mean flow (1, 1, 0)), each to t_end = 0.02."""
    from paper_2404_12703_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cases):
        nel = int(rng.choice(SERVING_SIZES))
        N = int(rng.choice([3, 5, 7]))
        if rng.random() < 0.5:
            m = W.box_mesh(N, (nel,) * 3, curved=0.1, seed=1000 + i)
            U = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
            mu, kind = 1.0 / 1600.0, "tgv"
        else:
            L = 10.0
            m = W.box_mesh(N, (nel,) * 3, length=(L, L, L), curved=0.05, seed=1000 + i)
            U = W.isentropic_vortex_state(m["xyz"], center=(L / 2, L / 2), strength=5.0,
                                          period=m["period"]).reshape(m["E"], -1, 5)
            mu, kind = 0.0, "vortex"
        out.append({"mesh": m, "U0": U, "mu": mu, "kind": kind, "N": N, "nel": nel, "t_end": SERVING_T_END})
    return out


SERVING_POOLS = {3: 16 ** 3 * 6, 5: 16 ** 3 * 6, 7: 16 ** 3 * 4}


# FIFO-capped policy: strict arrival order while the resident DOF stay within
# one 16^3 N = 7 case
SERVING_CAP_DOF = 16 ** 3 * 8 ** 3
# priority policy: every case is admitted when it fits; each batched step
# advances the oldest cases within 3 M DOF (first fit) and the rest sit it
# out (a budget about 1.4 times the largest case, chosen by a sweep over
# 1 M - 4.5 M DOF on this stream: it gave the lowest p50 and a lower p99 than
# free batching)
SERVING_PRIORITY_DOF = 3_000_000


def fifo_latencies(arrivals, service):
    """One server, first in first out (Lindley's recursion): case k starts at
    max(its arrival, the previous case's end).  Returns each case's time to
    solution (end - arrival) and the makespan (the last end)."""
    free_at, lat = 0.0, []
    for a, s in zip(arrivals, service):
        free_at = max(float(a), free_at) + float(s)
        lat.append(free_at - float(a))
    return lat, free_at


def serve_all(dg, cases, precision, arrivals, max_resident_dof=0, priority_dof=0, persistent=0):
    """Submits the cases at the given arrival times (s after the start) to one
    server; returns time-to-solution per case, makespan and server stats."""
    srv = dg.Server(SERVING_POOLS, max_cases=64, precision=precision, max_resident_dof=max_resident_dof,
                    priority_dof=priority_dof, persistent=persistent)
    t0 = time.perf_counter()
    tickets = []
    for a, c in zip(arrivals, cases):
        while time.perf_counter() - t0 < a:
            time.sleep(0.0005)
        tickets.append(srv.submit(c["mesh"], c["U0"], c["t_end"], mu=c["mu"]))
    lat = []
    for tk in tickets:
        _, st = srv.wait(tk, with_state=False)
        lat.append(st["time_to_solution"])
    makespan = time.perf_counter() - t0
    sstats = srv.stats()
    srv.close()
    return lat, makespan, sstats


def serving_bench(dg, n_cases, precision):
    """Continuous batching against the same cases run one by one through the
    standalone solver (dg_advance: the same CFL steps, the last one clipped at
    the end time)."""
    import torch
    cases = serving_cases(n_cases)
    dofs = [c["mesh"]["E"] * (c["N"] + 1) ** 3 for c in cases]
    # a case's service one by one: from the solver's creation (mesh set-up:
    # metrics, face data) to its final state, as a served case's time to
    # solution runs from its submission (set-up included) to its result;
    # the advance alone is kept beside it
    service, advance_only = [], []
    seq_dofstage = 0.0
    for c, dof in zip(cases, dofs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv = dg.Solver(c["mesh"], mu=c["mu"], precision=precision)
        sv.set_state(c["U0"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, steps = sv.advance(c["t_end"])
        sv.get_state()
        t2 = time.perf_counter()
        service.append(t2 - t0)
        advance_only.append(t2 - t1)
        seq_dofstage += dof * STAGES * steps
        sv.close()
    mean_service = sum(service) / len(service)
    rate = 0.9 / mean_service
    rng = np.random.Generator(np.random.PCG64(5))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(cases)))
    arrivals -= arrivals[0]
    # the one-by-one queue: same arrivals, FIFO, measured service times
    seq_lat, seq_makespan = fifo_latencies(arrivals, service)
    lat, makespan, sstats = serve_all(dg, cases, precision, arrivals)
    lat_c, makespan_c, sstats_c = serve_all(dg, cases, precision, arrivals, SERVING_CAP_DOF)
    lat_p, makespan_p, sstats_p = serve_all(dg, cases, precision, arrivals, 0, SERVING_PRIORITY_DOF)
    # closed system: every case submitted at once (capacity, not arrivals)
    _, sat_makespan, sat_stats = serve_all(dg, cases, precision, np.zeros(len(cases)))
    persist = None
    if precision == dg.FP32_BULK:
        # the same with each pool's stages in one persistent launch per step
        _, pm, pst = serve_all(dg, cases, precision, np.zeros(len(cases)), persistent=1)
        persist = {"makespan_s": pm, "dof_updates_per_s": pst["dof_stage_updates"] / pm,
                   "step_device_s": pst["step_device_s"]}
    p = lambda v, q: float(np.percentile(np.asarray(v), q))
    return {
        "workload": f"{len(cases)} cases (seeded PCG64(5)): n^3 meshes n in {{{','.join(map(str, SERVING_SIZES))}}}, "
                    f"N in {{3,5,7}}, "
                    f"half TGV (Re 1600, Ma 0.1), half isentropic vortex (inviscid), each to t = {SERVING_T_END}; "
                    f"Poisson arrivals at 0.9 x the one-by-one service rate ({rate:.2f}/s); "
                    + ("the 200 cases of the serving configuration, " if len(cases) == 200 else
                       f"the first {len(cases)} of the serving configuration's 200 cases, ")
                    + "each run to t = 0.02 instead of t = 1 (shortened)",
        "precision": "FP64" if precision == dg.FP64 else "FP32-bulk",
        "p50_s": p(lat, 50), "p99_s": p(lat, 99),
        "dof_updates_per_s": sstats["dof_stage_updates"] / makespan, "makespan_s": makespan,
        "fifo_capped": {"max_resident_dof": SERVING_CAP_DOF, "p50_s": p(lat_c, 50), "p99_s": p(lat_c, 99),
                        "dof_updates_per_s": sstats_c["dof_stage_updates"] / makespan_c, "makespan_s": makespan_c},
        "priority": {"priority_dof": SERVING_PRIORITY_DOF, "p50_s": p(lat_p, 50), "p99_s": p(lat_p, 99),
                     "dof_updates_per_s": sstats_p["dof_stage_updates"] / makespan_p, "makespan_s": makespan_p},
        "one_by_one": {"p50_s": p(seq_lat, 50), "p99_s": p(seq_lat, 99),
                       "dof_updates_per_s": seq_dofstage / seq_makespan, "makespan_s": seq_makespan,
                       "mean_service_s": mean_service,
                       "service": "solver creation (mesh set-up) + set_state + advance + get_state",
                       "busy_dof_updates_per_s": seq_dofstage / sum(service),
                       "mean_advance_only_s": sum(advance_only) / len(advance_only),
                       "busy_advance_only_dof_updates_per_s": seq_dofstage / sum(advance_only)},
        "all_at_once": {"makespan_s": sat_makespan,
                        "dof_updates_per_s": sat_stats["dof_stage_updates"] / sat_makespan,
                        "vs_one_by_one_busy": sum(service) / sat_makespan,
                        "vs_one_by_one_advance_only": sum(advance_only) / sat_makespan,
                        "step_device_s": sat_stats["step_device_s"],
                        "host_s": {k: sat_stats[k] for k in ("capture_host_s", "setup_host_s", "insert_host_s")}},
        "all_at_once_persistent": persist,
        "batched_steps": sstats["steps"], "graph_captures": sstats["captures"],
    }


def shock_tube_bench(dg, torch, stream):
    """Sod tube, 64 x 8 x 8 Cartesian elements on the periodic [0,2] x [0,1/4]^2
    box, N = 5 (884,736 DOF), inviscid, LF fluxes, indicator + FV sub-cell
    blending with alpha in [0, 0.5], CFL steps to t = 0.2; L1 density error
    against the exact Riemann solution on 0.5 < x < 1.5."""
    from paper_2404_12703_gb300 import workloads as W
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from exact_solutions import sod_exact
    N, t_end = 5, 0.2
    m = W.box_mesh(N, (64, 8, 8), length=(2.0, 0.25, 0.25), origin=(0.0, 0.0, 0.0))
    dof = m["E"] * (N + 1) ** 3
    U0 = W.sod_state(m["xyz"]).reshape(m["E"], -1, 5)
    out = {}
    for name, prec in (("fp64", dg.FP64), ("fp32_bulk", dg.FP32_BULK)):
        s = dg.Solver(m, stream=stream, viscous=0, riemann="lf", shock_capturing=1, precision=prec)
        s.set_state(U0)
        s.advance(0.002)  # warm-up (graph capture)
        s.set_state(U0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t, steps = s.advance(t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        U, _ = s.get_state()
        alpha = s.debug("alpha")
        _, J = s.debug("metrics")
        X = m["xyz"].reshape(m["E"], -1, 3)[..., 0]
        sel = (X > 0.5) & (X < 1.5)
        ex = sod_exact(X[sel], t_end, x0=1.0)
        xg = W.lgl_points(N)
        PN = np.polynomial.legendre.legval(xg, [0] * N + [1])
        w = 2.0 / (N * (N + 1) * PN ** 2)  # LGL quadrature weights
        wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
        l1 = float((wq[sel] * np.abs(U[..., 0][sel] - ex[:, 0])).sum() / wq[sel].sum())
        out[name] = {"steps": steps, "t_final": t, "ms_total": ms, "ms_per_step": ms / max(steps, 1),
                     "dof_updates_per_s": dof * STAGES * steps / (ms * 1e-3), "l1_rho_err": l1,
                     "blended_elements": int((alpha > 0).sum()), "alpha_max": float(alpha.max()),
                     "finite": bool(np.isfinite(U).all())}
        s.close()
    return {"workload": "Sod tube 64x8x8 elements, N=5 (884,736 DOF), [0,2]x[0,1/4]^2 periodic, inviscid, LF, "
                        "indicator + FV blending alpha in [0,0.5], CFL 0.9 to t = 0.2", **out}


# CFL number of the 14-stage scheme in the compressible Taylor-Green run:
# the run stays stable to t = 3 for every CFL number from 1.6 to 4.0; its
# stability region reaches 18.5 on the negative real axis and 6.1 on the
# imaginary axis (the five-stage scheme: 4.7 and 3.3)
NDB14_CFL = 3.2


def compressible_bench(dg, torch, stream):
    """Compressible Taylor-Green vortex (Ma 1.25, Re 1600, Version II
    initialisation) on 8^3 Cartesian elements at N = 7 (64^3 DOF, the paper's
    coarsest resolution): Sutherland's law with T_ref = T0, Roe fluxes,
    indicator + FV blending (alpha <= 0.5), CFL steps to t = 3 with E_k,
    its rate and the blended elements every 0.5, in both precisions, with the
    five-stage scheme at CFL 0.9 and the paper's 14-stage scheme at CFL
    NDB14_CFL."""
    from paper_2404_12703_gb300 import workloads as W
    Ma, N, t_end, t_out = 1.25, 7, 3.0, 0.5
    m = W.box_mesh(N, (8, 8, 8))
    dof = m["E"] * (N + 1) ** 3
    U0 = W.tgv_state(m["xyz"], Ma=Ma).reshape(m["E"], -1, 5)
    out = {}
    runs = (("fp64", dg.FP64, "ck5", 0.9), ("fp32_bulk", dg.FP32_BULK, "ck5", 0.9),
            ("fp64_ndb14", dg.FP64, "ndb14", NDB14_CFL), ("fp32_bulk_ndb14", dg.FP32_BULK, "ndb14", NDB14_CFL))
    for name, prec, scheme, cfl in runs:
        s = dg.Solver(m, stream=stream, sutherland=1, T_ref=1.0 / (1.4 * Ma ** 2), shock_capturing=1,
                      precision=prec, cfl=cfl, dfl=cfl)
        s.set_rk_scheme(scheme)
        stages = 14 if scheme == "ndb14" else 5
        s.set_state(U0)
        s.advance(0.01)  # warm-up (graph capture)
        s.set_state(U0)
        ek0 = s.kinetic()[0]
        ms, steps, hist = 0.0, 0, []
        for tk in np.arange(1, int(round(t_end / t_out)) + 1) * t_out:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t, k = s.advance(float(tk))
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            steps += k
            ek, rate, _ = s.kinetic()
            al = s.debug("alpha")
            hist.append({"t": t, "ek": ek, "dissipation_rate": -rate, "blended_elements": int((al > 0).sum()),
                         "alpha_max": float(al.max())})
        U, _ = s.get_state()
        out[name] = {"scheme": scheme, "stages": stages, "cfl": cfl, "steps": steps, "t_final": t,
                     "rhs_evaluations": steps * stages, "ms_per_step": ms / max(steps, 1), "ms_total": ms,
                     "dof_updates_per_s": dof * stages * steps / (ms * 1e-3), "ek0": ek0, "history": hist,
                     "finite": bool(np.isfinite(U).all())}
        s.close()
    for p in ("fp64", "fp32_bulk"):
        a, b = out[p], out[p + "_ndb14"]
        out[p + "_ndb14"]["ek_diff_vs_ck5"] = max(abs(x["ek"] - y["ek"]) for x, y in zip(a["history"], b["history"]))
    return {"workload": f"compressible TGV Ma 1.25 Re 1600, 8^3 Cartesian elements, N = 7 ({dof} DOF), "
                        "Sutherland's law, Roe, indicator + FV blending alpha <= 0.5, to t = 3: LSERK4 (5 stages, "
                        f"CFL 0.9) and the 14-stage scheme of the paper's application run (CFL {NDB14_CFL})", **out}


def channel_bench(dg, torch, stream):
    """Wall-bounded channel: 16 x 8 x 16 curved elements at N = 7 (1,048,576
    DOF) on [0, 4] x [0, 1] x [0, 4], periodic in x and z, isothermal no-slip
    walls at y = 0 (at rest) and y = 1 (moving), Couette flow plus a seeded
    perturbation, 20 CFL steps in both precisions; the walls' lifting values
    and fluxes run in the surface kernels."""
    from paper_2404_12703_gb300 import workloads as W
    N, mu = 7, 1e-3
    m = W.box_mesh(N, (16, 8, 16), length=(4.0, 1.0, 4.0), origin=(0.0, 0.0, 0.0),
                   periodic=(True, False, True), curved=0.1, seed=11)
    m["face_bc"] = W.box_face_bc(m, {"y-": 1, "y+": 2})
    m["bcs"] = [(1, 0.0, 0.0, 0.0, 1.0), (1, 1.0, 0.0, 0.0, 1.0)]
    dof = m["E"] * (N + 1) ** 3
    U0 = W.random_perturbation(W.couette_state(m["xyz"], U_wall=1.0, T_wall=1.0, p=10.0, mu=mu)
                               .reshape(m["E"], -1, 5), 1e-3, 11)
    out = {}
    for name, prec in (("fp64", dg.FP64), ("fp32_bulk", dg.FP32_BULK)):
        s = dg.Solver(m, stream=stream, mu=mu, precision=prec)
        s.set_state(U0)
        s.step(3)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(20)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        U, t = s.get_state()
        out[name] = {"ms_per_step": ms, "dof_updates_per_s": dof * STAGES / (ms * 1e-3), "t": t,
                     "finite": bool(np.isfinite(U).all())}
        s.close()
    return {"workload": f"channel 16x8x16 curved elements, N = 7 ({dof} DOF), isothermal no-slip walls "
                        f"(one moving), Couette + perturbation, Re = 1000, 20 steps", **out}


def gauss_bench(dg, torch, stream, nel=NEL, steps=20):
    """The standard DGSEM on Gauss-Legendre nodes (Sec. 5.1's GL scheme) on the
    main workload's mesh (curved, renumbered, rotated, N = 7), Taylor-Green
    vortex at Ma = 0.1 sampled at the GL nodes, CFL steps in both precisions,
    with each kernel kind's share of the step."""
    from paper_2404_12703_gb300 import workloads as W
    N = 7
    m = W.box_mesh(N, (nel,) * 3, curved=0.1, seed=SEED)
    dof = m["E"] * (N + 1) ** 3
    out = {}
    U0 = None
    for name, prec in (("fp64", dg.FP64), ("fp32_bulk", dg.FP32_BULK)):
        s = dg.Solver(m, stream=stream, precision=prec, nodes="gauss")
        if U0 is None:
            U0 = W.tgv_state(s.node_coords()).reshape(m["E"], -1, 5)
        s.set_state(U0)
        s.step(3)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        U, t = s.get_state()
        prof = s.profile_step(3)
        tot = sum(v[0] for v in prof.values())
        out[name] = {"ms_per_step": ms, "dof_updates_per_s": dof * STAGES / (ms * 1e-3), "t": t,
                     "finite": bool(np.isfinite(U).all()),
                     "kernel_share": {k: v[0] / tot for k, v in prof.items()}}
        if prec == dg.FP64:
            # the lifting kernel dominates: its algorithmic FLOP/s against the FP64 ALU peak
            lift_ms = prof["lift"][0] / max(prof["lift"][1], 1)
            ach = GL_FLOPS_PER_DOF["lift"] * dof / (lift_ms * 1e-3) / 1e12
            vol_ms = prof["volume"][0] / max(prof["volume"][1], 1)
            out[name]["roofline"] = {"kernel": "k_lift_gl<7,double>", "bound": "alu", "achieved": ach,
                                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                                     "flops_per_dof": GL_FLOPS_PER_DOF["lift"], "ms_per_launch": lift_ms,
                                     "volume_ms_per_launch": vol_ms,
                                     "volume_frac": GL_FLOPS_PER_DOF["volume"] * dof / (vol_ms * 1e-3) / 1e12
                                     / FP64_PEAK_TFLOPS}
        s.close()
    return {"workload": f"TGV Re 1600 Ma 0.1 on {nel}^3 curved elements, N = 7 ({dof} DOF), standard DGSEM "
                        f"on Gauss-Legendre nodes, {steps} CFL steps", **out}


# Measured device memory per DOF of the paper's solver (Sec. 4.3, Tab.
# memory_requirements), KiB, for N = 1..7
PAPER_KIB_PER_DOF = {1: 1.457, 2: 1.188, 3: 1.049, 4: 0.996, 5: 0.942, 6: 0.895, 7: 0.869}


def memory_per_dof(dg, stream, nel=8):
    """Device bytes per DOF of one context (state, RK register, scratch,
    metrics in both precisions, lifted gradients, side arrays; LGL nodes,
    FP64) for N = 1..7 on an nel^3 periodic mesh, against the paper's table,
    and the largest N = 7 problem that would fit this GPU's memory."""
    import torch
    from paper_2404_12703_gb300 import workloads as W
    out = {}
    for N in range(1, 8):
        m = W.box_mesh(N, (nel,) * 3, seed=3)
        s = dg.Solver(m, stream=stream)
        dof = m["E"] * (N + 1) ** 3
        kib = s.sizes()["bytes"] / dof / 1024.0
        out[str(N)] = {"kib_per_dof": kib, "paper_kib_per_dof": PAPER_KIB_PER_DOF[N]}
        s.close()
    total = torch.cuda.get_device_properties(0).total_memory
    out["max_dof_N7_this_gpu"] = int(0.95 * total / (out["7"]["kib_per_dof"] * 1024.0))
    return out


def mms_error(dg, torch, stream, N, nel, nodes, T=0.2, cfl=0.2, mu=0.01):
    """L2 density error at time T of the manufactured solution of Sec. 5.1 on
    [-1, 1]^3 (nel^3 curved elements, periodic), viscous, started from its
    interpolant, CFL steps ending exactly on T."""
    from paper_2404_12703_gb300 import workloads as W
    m = W.box_mesh(N, (nel,) * 3, length=(2.0, 2.0, 2.0), origin=(-1.0, -1.0, -1.0), curved=0.05, seed=2)
    s = dg.Solver(m, stream=stream, nodes=nodes, mu=mu, cfl=cfl, source=dg.SOURCE_MMS)
    X = s.node_coords()
    s.set_state(W.mms_state(X, 0.0))
    t, steps = s.advance(T)
    U, _ = s.get_state()
    ex = W.mms_state(X, t)
    Ja, J = s.debug("metrics")
    w = s.quadrature_weights()
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    err = float(np.sqrt((wq * (U[..., 0] - ex[..., 0]) ** 2).sum() / wq.sum()))
    s.close()
    return err, steps


def convergence_study(dg, torch, stream, degrees=(2, 3, 4, 5, 6, 7), T=0.2):
    """Sec. 5.1's convergence test on the GPU: the manufactured solution with
    both schemes (split form on LGL nodes, standard form on GL nodes), L2
    density errors on nested meshes and the experimental orders."""
    out = {}
    for nodes in ("lgl", "gauss"):
        rows = {}
        for N in degrees:
            # a periodic direction needs three elements at least
            levels = (4, 8, 16, 32) if N <= 3 else ((4, 8, 16) if N == 4 else (3, 6, 12))
            cfl = 0.2 if N <= 4 else 0.1  # keeps the RK4 error below the spatial one
            errs = []
            for nel in levels:
                e, steps = mms_error(dg, torch, stream, N, nel, nodes, T=T, cfl=cfl)
                errs.append({"elements": nel ** 3, "l2_rho": e, "steps": steps})
            for i in range(1, len(errs)):
                errs[i]["eoc"] = float(np.log2(errs[i - 1]["l2_rho"] / errs[i]["l2_rho"]))
            rows[str(N)] = errs
        out[nodes] = rows
    return {"workload": f"manufactured solution of Sec. 5.1 (A = 0.1, a = 1, mu = 0.01) on [-1,1]^3 curved "
                        f"periodic meshes, to t = {T}, CFL 0.2 (N <= 4) or 0.1", **out}


def eps_from_gradients(g, wq, mu_ratio, mu0):
    """Sec. 5.2's solenoidal and dilatational dissipation rates, with rho_0 =
    U_0 = L = 1 (Re = 1 / mu_0), from velocity gradients g[..., a, b] =
    d u_a / d x_b at the nodes, the quadrature weights times J (wq) and the
    viscosity ratio mu(T) / mu_0 at the nodes."""
    d = np.asarray(g)[..., :3, :]
    wx = d[..., 2, 1] - d[..., 1, 2]
    wy = d[..., 0, 2] - d[..., 2, 0]
    wz = d[..., 1, 0] - d[..., 0, 1]
    div = d[..., 0, 0] + d[..., 1, 1] + d[..., 2, 2]
    vol = wq.sum()
    eps_s = mu0 * (wq * mu_ratio * (wx * wx + wy * wy + wz * wz)).sum() / vol
    eps_d = 4.0 / 3.0 * mu0 * (wq * mu_ratio * div * div).sum() / vol
    return float(eps_s), float(eps_d)


def dissipation_rates(s, torch):
    """eps_S and eps_D of a solver's current state from the library's BR1
    lifted velocity gradients (one dg_rhs of the state, then the gradient
    copy); the viscosity ratio follows Sutherland's law when it is on."""
    torch.cuda.synchronize()
    s.rhs()
    g = s.debug("grad")
    _, J = s.debug("metrics")
    w = s.quadrature_weights()
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    prm = s.params
    ratio = np.ones_like(J)
    if prm.sutherland:
        U, _ = s.get_state()
        rho = U[..., 0]
        p = (prm.gamma - 1) * (U[..., 4] - 0.5 * (U[..., 1] ** 2 + U[..., 2] ** 2 + U[..., 3] ** 2) / rho)
        th = p / (rho * prm.R) / prm.T_ref
        ratio = 1.4042 * th ** 1.5 / (th + 0.4042)
    return eps_from_gradients(g, wq, ratio, prm.mu)


def tgv_validation(dg, torch, t_end=10.0, every=0.5, levels=(16, 24)):
    """The Taylor-Green vortex of Sec. 5.2 (Re 1600, Ma 0.1, version II) on
    curved, permuted meshes at N = 7, FP32-bulk, CFL steps to t_end: the
    kinetic energy and its exact dissipation rate at every output time, and
    the peak of -dE_k/dt.  (The paper compares with reference data that is
    not part of this repository; the curves here are reported as computed.)"""
    from paper_2404_12703_gb300 import workloads as W
    out = {}
    stream = torch.cuda.Stream()
    for nel in levels:
        m = W.box_mesh(N_DEG, (nel,) * 3, curved=0.1, seed=SEED)
        s = dg.Solver(m, stream=stream, precision=dg.FP32_BULK)
        s.set_state(W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5))
        rows = []
        k = s.kinetic()
        eps = dissipation_rates(s, torch)
        rows.append({"t": 0.0, "E_k": k[0], "minus_dEk_dt": -k[1], "eps_S": eps[0], "eps_D": eps[1], "steps": 0})
        steps = 0
        wall = 0.0
        for i in range(1, int(round(t_end / every)) + 1):
            t0 = time.perf_counter()
            t, ns = s.advance(i * every)
            wall += time.perf_counter() - t0
            steps += ns
            k = s.kinetic()
            eps = dissipation_rates(s, torch)
            rows.append({"t": t, "E_k": k[0], "minus_dEk_dt": -k[1], "eps_S": eps[0], "eps_D": eps[1],
                         "steps": steps})
        U, _ = s.get_state()
        peak = max(rows, key=lambda r: r["minus_dEk_dt"])
        out[f"{nel}^3"] = {"dof": m["E"] * (N_DEG + 1) ** 3, "wall_s": wall, "finite": bool(np.isfinite(U).all()),
                           "peak_minus_dEk_dt": peak["minus_dEk_dt"], "peak_t": peak["t"], "history": rows}
        s.close()
    return {"workload": f"TGV Re 1600 Ma 0.1 (version II), curved permuted meshes, N = 7, FP32-bulk, to t = {t_end}",
            **out}


def run_long(args):
    """FP32-bulk against FP64 over a long Taylor-Green run: 32^3 Cartesian
    elements at N = 5 (7,077,888 DOF), Re 1600, Ma 0.1, both precisions from
    the same state with the same fixed time step (the CFL step of the initial
    state, adjusted to land on every output time), to t_end.  Prints one JSON
    line with E_k and its exact dissipation rate at each output time and the
    L2 state difference at the end."""
    import torch
    from paper_2404_12703_gb300 import build as B
    from paper_2404_12703_gb300 import dg
    from paper_2404_12703_gb300 import workloads as W
    B.build()
    dg.load()
    N, nel = 5, 32
    m = W.box_mesh(N, (nel,) * 3)
    dof = m["E"] * (N + 1) ** 3
    U0 = W.tgv_state(m["xyz"]).reshape(m["E"], -1, 5)
    stream = torch.cuda.Stream()
    s64 = dg.Solver(m, stream=stream)
    s32 = dg.Solver(m, stream=stream, precision=dg.FP32_BULK)
    for s in (s64, s32):
        s.set_state(U0)
    every = args.long_every
    per = int(np.ceil(every / s64.time_step()))
    dt = every / per
    rows, ms = [], {"fp64": 0.0, "fp32_bulk": 0.0}
    t = 0.0
    n_out = int(round(args.long_run / every))
    for k in range(1, n_out + 1):
        for name, s in (("fp64", s64), ("fp32_bulk", s32)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(per, dt=dt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[name] += e0.elapsed_time(e1)
        t = k * every
        k64, k32 = s64.kinetic(), s32.kinetic()
        e64, e32 = dissipation_rates(s64, torch), dissipation_rates(s32, torch)
        rows.append({"t": t, "ek_fp64": k64[0], "ek_fp32": k32[0], "rate_fp64": -k64[1], "rate_fp32": -k32[1],
                     "rate_rel_err": abs(k32[1] - k64[1]) / abs(k64[1]),
                     "ek_rel_err": abs(k32[0] - k64[0]) / abs(k64[0]),
                     "eps_S_fp64": e64[0], "eps_S_fp32": e32[0], "eps_S_rel_err": abs(e32[0] - e64[0]) / abs(e64[0]),
                     "eps_D_fp64": e64[1], "eps_D_fp32": e32[1]})
        print(json.dumps({"progress": rows[-1]}), flush=True)
    U64, _ = s64.get_state()
    U32, _ = s32.get_state()
    steps = per * n_out
    line = {"workload": f"Taylor-Green vortex Re 1600 Ma 0.1, {nel}^3 Cartesian elements, N = {N} ({dof} DOF), "
                        f"FP32-bulk vs FP64 from the same state, fixed dt = {dt:.6g} ({steps} steps) to t = {t}",
            "rows": rows, "max_rate_rel_err": max(r["rate_rel_err"] for r in rows),
            "max_eps_S_rel_err": max(r["eps_S_rel_err"] for r in rows),
            "l2_state_rel_err": float(np.sqrt(((U32 - U64) ** 2).sum() / (U64 ** 2).sum())),
            "finite": bool(np.isfinite(U32).all() and np.isfinite(U64).all()),
            "ms_per_step": {k: v / steps for k, v in ms.items()},
            "dof_updates_per_s": {k: dof * STAGES * steps / (v * 1e-3) for k, v in ms.items()}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """The oracle (plain FP64 C) on the host's cores: one independent replica
    of a 6^3-element sample of the workload per usable core, `warmup` untimed
    and `steps` timed LSERK steps each; the aggregate over the slowest
    replica.  Ranks other than 0 exit without work."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    nel = 6
    dof = nel ** 3 * (N_DEG + 1) ** 3
    try:
        allc = cpu_oracle_all_cores(steps=args.steps, nel=nel, warmup=args.warmup)
        value, cores = allc["value"], allc["cores"]
        ms_step = 1e3 * cores * dof * STAGES / value
        sample = (f"{cores} independent replicas (one process per core) of {nel}^3 elements of the same curved "
                  f"N=7 TGV workload ({dof} DOF each), {args.warmup} untimed and {args.steps} timed LSERK steps "
                  f"each, single-threaded FP64 C per process; aggregate over the slowest replica")
    except Exception as ex:  # the single-process measurement, with the reason
        dof, times = cpu_oracle_sample(args.warmup + args.steps, nel=nel)
        timed = times[args.warmup:]
        value = dof * STAGES * len(timed) / sum(timed)
        cores, ms_step = 1, 1e3 * sum(timed) / len(timed)
        sample = (f"{nel}^3 elements of the same curved N=7 TGV workload ({dof} DOF), one LSERK step per bench "
                  f"step, one process (all cores unavailable: {type(ex).__name__}: {ex})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_desc(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2404_12703_gb300 import build as B
    from paper_2404_12703_gb300 import dg
    from paper_2404_12703_gb300 import workloads as W
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    dg.load()

    nel = args.nel
    m = W.box_mesh(N_DEG, (nel,) * 3, curved=0.1, seed=SEED)
    E = m["E"]
    dof = E * (N_DEG + 1) ** 3
    U0 = W.tgv_state(m["xyz"]).reshape(E, -1, 5)
    stream = torch.cuda.Stream()
    solver = dg.Solver(m, stream=stream)
    solver.set_state(U0)
    # launch configuration chosen by the library's autotuner on this workload
    tune64 = solver.autotune()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up (also captures the step graph)
    solver.step(args.warmup)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = dg.launch_count()
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        solver.step(args.steps)
        ev1.record(stream)
        barrier()
    launches = dg.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, "cuda")
    ms_step = ms / args.steps
    value = replicas_value(dof * STAGES, ms_step, world)
    Ufinal, tfinal = solver.get_state()
    finite = bool(np.isfinite(Ufinal).all())

    # per-kernel device time over the same number of steps, eagerly launched
    # with CUDA events on the solver's stream
    prof = solver.profile_step(args.steps)
    tot_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms_per_launch": (v[0] / v[1] if v[1] else None), "launches": v[1],
                   "share": (v[0] / tot_ms if tot_ms else None)} for k, v in prof.items()}
    vol_ms = kernels["volume"]["ms_per_launch"]
    vol_flops = FLOPS_PER_DOF["volume"] * dof
    achieved_tf = vol_flops / (vol_ms * 1e-3) / 1e12
    peaks, peak_src = measured_peaks()
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP64_PEAK_TFLOPS,
                "traffic": (VOLUME_TRAFFIC_BYTES_PER_DOF * dof if VOLUME_TRAFFIC_BYTES_PER_DOF else None),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                "12^3 capture scaled by DOF)",
                "kernel": "k_volume<7,1> (split-form KEP volume integral + viscous volume term + SurfInt "
                          "+ ApplyJac + RK update)",
                "peak_source": "FP64 FMA peak derived from unit counts and clocks (152 SM x 2 DFMA/clk x "
                               "2 flop x 2.07 GHz)",
                "hbm": {"algorithmic_bytes_per_dof": BYTES_PER_DOF,
                        "achieved_gbs": BYTES_PER_DOF * dof * STAGES / (ms_step * 1e-3) / 1e9,
                        "peak_gbs": peaks.get("hbm_gbs"), "peak_source": peak_src}}
    roofline["hbm"]["frac"] = roofline["hbm"]["achieved_gbs"] / roofline["hbm"]["peak_gbs"]
    # the FP64 rates this GPU reaches in the library's own probes (dg_peak_probe):
    # independent FMA chains, DMMA (mma.sync m8n8k4) chains, and both from the
    # same warps; FP32 FMA for the FP32-bulk path's ALU ceiling
    with Clocks(local) as pclk:
        probe = {name: dg.peak_probe(kind, iters)[0] / 1e12
                 for name, kind, iters in (("fp64_fma", dg.PEAK_FP64_FMA, 16384),
                                           ("fp64_mma", dg.PEAK_FP64_MMA, 4096),
                                           ("fp64_fma_and_mma", dg.PEAK_FP64_BOTH, 4096),
                                           ("fp32_fma", dg.PEAK_FP32_FMA, 131072))}
    probe["clocks"] = pclk.summary()
    probe["unit"] = "TFLOP/s"
    roofline["probe"] = probe
    roofline["frac_of_probe"] = achieved_tf / probe["fp64_fma"]
    total_flops = sum(FLOPS_PER_DOF.values()) * dof * STAGES
    roofline["whole_step_fp64_frac"] = total_flops / (ms_step * 1e-3) / 1e12 / FP64_PEAK_TFLOPS

    # end to end through the public API with host buffers: per step, upload the
    # state from pinned host memory, advance one step, read the state back
    pinned_in = torch.from_numpy(U0.reshape(-1)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    Uh_in = pinned_in.numpy()
    Uh_out = pinned_out.numpy()
    e2e_steps = max(1, min(args.steps, 5))
    solver.set_state(Uh_in)
    solver.step(1)
    solver.get_state(Uh_out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(Uh_in)
        solver.step(1)
        solver.get_state(Uh_out)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    nbytes = dof * 5 * 8

    # FP32-bulk on the same workload: flux/volume/surface arithmetic in FP32,
    # state, RK register, metrics and reductions in FP64
    fp32 = None
    if not args.no_fp32:
        s32 = dg.Solver(m, stream=stream, precision=dg.FP32_BULK)
        s32.set_state(U0)
        tune32 = s32.autotune()
        s32.step(args.warmup)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        s32.step(args.steps)
        e1.record(stream)
        barrier()
        ms32 = e0.elapsed_time(e1) / args.steps
        ms32 = max_over_ranks(ms32, world, "cuda")
        prof32 = s32.profile_step(args.steps)
        tot32 = sum(v[0] for v in prof32.values())
        k32 = {k: {"ms_per_launch": (v[0] / v[1] if v[1] else None), "launches": v[1],
                   "share": (v[0] / tot32 if tot32 else None)} for k, v in prof32.items()}
        vol32 = k32["volume"]["ms_per_launch"]
        form32 = s32.stage_form()
        if form32 == 2:
            kname = "k_felem<7,1> (two-kernel FP32-bulk stage: lifting, KEP volume, viscous volume, SurfInt, " \
                    "ApplyJac, RK update, next stage's face data)"
            vbytes = FELEM32_BYTES_PER_DOF
            k32["surf_flux"]["algorithmic_bytes_per_dof"] = FFLUX32_BYTES_PER_DOF
            sf = k32["surf_flux"]["ms_per_launch"]
            k32["surf_flux"]["hbm_frac"] = FFLUX32_BYTES_PER_DOF * dof / (sf * 1e-3) / 1e9 / peaks.get("hbm_gbs")
        else:
            kname, vbytes = "k_volume<7,1,float>", VOLUME32_BYTES_PER_DOF
        k32["volume"]["algorithmic_bytes_per_dof"] = vbytes
        # the four-kernel stage on the same workload, for comparison
        s32.set_config(**dict(s32.config(), stage_form=1))
        s32.set_state(U0)
        s32.step(args.warmup)
        barrier()
        e0.record(stream)
        s32.step(args.steps)
        e1.record(stream)
        barrier()
        ms32_four = e0.elapsed_time(e1) / args.steps
        s32.set_config(**dict(s32.config(), stage_form=0))
        # accuracy against the FP64 path: same initial state, same fixed dt,
        # `steps` steps each; kinetic-energy dissipation rate and L2 state error
        solver.set_state(U0)
        dt_fix = solver.time_step()
        solver.step(args.steps, dt=dt_fix)
        s32.set_state(U0)
        s32.step(args.steps, dt=dt_fix)
        U64, _ = solver.get_state()
        U32, _ = s32.get_state()
        kin64 = solver.kinetic()
        kin32 = s32.kinetic()
        fp32 = {
            "value": world * dof * STAGES / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
            "speedup_vs_fp64": ms_step / ms32, "dtype": "f32 arithmetic, f64 state/RK/metrics/reductions",
            "autotune": {"config": tune32[0], "variant_ms": tune32[1]},
            "kernels": k32,
            "stage_form": form32,
            "four_kernel_stage_ms_per_step": ms32_four,
            "roofline": {"bound": "hbm", "kernel": kname,
                         "achieved": vbytes * dof / (vol32 * 1e-3) / 1e9,
                         "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": vbytes * dof / (vol32 * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
                         "traffic": (VOLUME32_TRAFFIC_BYTES_PER_DOF * dof if VOLUME32_TRAFFIC_BYTES_PER_DOF
                                     else None),
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_dof": vbytes},
            "whole_step_hbm_frac": BYTES32_PER_DOF * dof * STAGES / (ms32 * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
            "accuracy_vs_fp64": {
                "steps": args.steps, "dt": dt_fix,
                "ke_dissipation_rate_rel_err": abs(kin32[1] - kin64[1]) / abs(kin64[1]),
                "ke_rel_err": abs(kin32[0] - kin64[0]) / abs(kin64[0]),
                "l2_state_rel_err": float(np.sqrt(((U32 - U64) ** 2).sum() / (U64 ** 2).sum())),
            },
        }
        s32.close()

    shock = None
    if not args.no_shock and rank == 0:
        shock = shock_tube_bench(dg, torch, stream)

    comp = chan = gauss = memory = None
    if not args.no_shock and rank == 0:
        comp = compressible_bench(dg, torch, stream)
        chan = channel_bench(dg, torch, stream)
        gauss = gauss_bench(dg, torch, stream, nel=nel)
        memory = memory_per_dof(dg, stream)

    serving = None
    if not args.no_serving and rank == 0:
        serving = {"fp64": serving_bench(dg, args.serving_cases, dg.FP64)}
        if not args.no_fp32:
            serving["fp32_bulk"] = serving_bench(dg, args.serving_cases_fp32, dg.FP32_BULK)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the host's cores: one independent replica per usable
        # core (the headline cpu_baseline), and one replica alone
        cdof, ctimes = cpu_oracle_sample(2, nel=4)
        single = {"value": cdof * STAGES * len(ctimes) / sum(ctimes), "unit": UNIT, "cores": 1, "kind": "oracle",
                  "sample": f"4^3 elements of the same curved N=7 TGV workload ({cdof} DOF), 2 LSERK steps, "
                            f"single-threaded FP64 C"}
        try:
            cpu = cpu_oracle_all_cores()
            cpu["single_core"] = single
        except Exception as ex:  # all cores unavailable: the single-core figure, with the reason
            cpu = dict(single, cpu_model=cpu_model(), all_cores={"unavailable": f"{type(ex).__name__}: {ex}"})

    if rank == 0:
        clocks = clk.summary()
        # energy per DOF and stage (Sec. 4.2: EPID = P_rank PID), from the median
        # board power sampled during the timed region (no cooling share)
        pw = clocks.get("power_w")
        epid = {"power_w": pw, "j_per_dof_stage": (pw / (value / world) if pw else None),
                "paper_a100_j_per_dof_stage": 2.05e-6,
                "note": "board power of this GPU; the paper's figure is Rotor 37 on A100 with 448 W per GPU "
                        "including cooling"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_desc(nel),
            "pid_s": 1.0 / (value / world), "finite": finite, "t_end": tfinal,
            "gpu_launches": launches, "kernels": kernels, "roofline": roofline,
            "autotune": {"config": tune64[0], "variant_ms": tune64[1]},
            "e2e": {"value": world * dof * STAGES / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
            "clocks": clocks, "epid": epid, "cpu_baseline": cpu, "fp32_bulk": fp32, "shock_tube": shock, "compressible_tgv": comp,
            "channel": chan, "gauss_nodes": gauss, "memory": memory,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-bulk measurement")
    ap.add_argument("--serving-cases-fp32", type=int, default=200,
                    help="cases of the FP32-bulk serving stream (the configuration's 200 by default)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-cases", type=int, default=48)
    ap.add_argument("--no-shock", action="store_true", help="skip the shock-tube measurement")
    ap.add_argument("--nel", type=int, default=NEL,
                    help="elements per direction (24 is the benchmark workload; smaller for profiling)")
    ap.add_argument("--long-run", type=float, default=0.0,
                    help="instead of the benchmark: FP32-bulk vs FP64 Taylor-Green run (32^3, N = 5) to this time")
    ap.add_argument("--long-every", type=float, default=0.25, help="output interval of --long-run")
    ap.add_argument("--gauss-only", action="store_true",
                    help="run only the Gauss-Legendre-node measurement (--nel, --steps) and print it")
    ap.add_argument("--tgv-validation", type=float, default=0.0,
                    help="run only the Taylor-Green validation (16^3 and 24^3, N = 7, FP32-bulk) to this time")
    ap.add_argument("--convergence", action="store_true",
                    help="run only the manufactured-solution convergence study of Sec. 5.1 and print it")
    args = ap.parse_args()
    if args.tgv_validation > 0:
        import torch
        from paper_2404_12703_gb300 import build as B
        from paper_2404_12703_gb300 import dg
        B.build()
        dg.load()
        print(json.dumps(tgv_validation(dg, torch, t_end=args.tgv_validation)), flush=True)
        return 0
    if args.convergence:
        import torch
        from paper_2404_12703_gb300 import build as B
        from paper_2404_12703_gb300 import dg
        B.build()
        dg.load()
        print(json.dumps(convergence_study(dg, torch, torch.cuda.Stream())), flush=True)
        return 0
    if args.gauss_only:
        import torch
        from paper_2404_12703_gb300 import build as B
        from paper_2404_12703_gb300 import dg
        B.build()
        dg.load()
        stream = torch.cuda.Stream()
        print(json.dumps(gauss_bench(dg, torch, stream, nel=args.nel, steps=max(args.steps, 1))), flush=True)
        return 0
    if args.long_run > 0:
        return run_long(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
