"""Host logic of the benchmark that needs no GPU: the one-by-one FIFO queue
the serving measurement compares against, and the seeded serving stream."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fifo_queue_closed_forms():
    # no waiting: arrivals further apart than the service times
    lat, end = bench.fifo_latencies([0.0, 5.0, 10.0], [1.0, 2.0, 3.0])
    assert lat == [1.0, 2.0, 3.0] and end == 13.0
    # a backlog: arrivals every second, two seconds of service each ->
    # case k waits k seconds, time to solution 2 + k
    lat, end = bench.fifo_latencies(np.arange(6.0), [2.0] * 6)
    assert lat == [2.0 + k for k in range(6)] and end == 12.0
    # everything at t = 0: the k-th case ends at the sum of the first k services
    svc = [0.5, 1.5, 0.25, 2.0]
    lat, end = bench.fifo_latencies([0.0] * 4, svc)
    assert np.allclose(lat, np.cumsum(svc)) and end == sum(svc)


def test_fifo_queue_against_an_event_simulation():
    rng = np.random.default_rng(2)
    arr = np.cumsum(rng.exponential(1.0, 200))
    svc = rng.exponential(0.9, 200)
    lat, end = bench.fifo_latencies(arr, svc)
    # event view: the server is busy from each start to each end, never overlapping
    starts = arr + np.asarray(lat) - svc
    assert np.all(starts >= arr - 1e-12)
    assert np.all(starts[1:] >= (starts + svc)[:-1] - 1e-9)
    # a case starts late only if the server was busy when it arrived
    late = starts > arr + 1e-12
    assert np.all(np.abs(starts[1:][late[1:]] - (starts + svc)[:-1][late[1:]]) < 1e-9)
    assert abs(end - (starts[-1] + svc[-1])) < 1e-9


def test_serving_stream_is_seeded_and_in_range():
    a = bench.serving_cases(6)
    b = bench.serving_cases(6)
    for x, y in zip(a, b):
        assert x["nel"] == y["nel"] and x["N"] == y["N"] and x["kind"] == y["kind"]
        np.testing.assert_array_equal(x["U0"], y["U0"])
        assert x["nel"] in bench.SERVING_SIZES and x["N"] in (3, 5, 7)
        assert x["t_end"] == bench.SERVING_T_END
        assert x["U0"].shape == (x["nel"] ** 3, (x["N"] + 1) ** 3, 5)
        assert (x["mu"] > 0) == (x["kind"] == "tgv")


def test_dissipation_rates_from_gradients_match_the_oracle():
    """The benchmark's eps_S / eps_D arithmetic (applied to the library's
    lifted gradients on the GPU) against the oracle's, fed the oracle's own
    gradients: equal to round-off, on a state with vorticity and dilatation."""
    import oracle as O
    from paper_2404_12703_gb300 import workloads as W
    N, mu = 5, 0.01
    m = W.box_mesh(N, (3, 3, 3), curved=0.1, seed=3)
    M = O.Mesh(N, m["xyz"], m["period"])
    X = m["xyz"].reshape(m["E"], -1, 3)
    ph = np.sin(X @ np.ones(3))
    U = W.prim_to_cons(1 + 0.1 * ph, ph, 0.5 * np.cos(X[..., 0]), -0.3 * ph, np.full_like(ph, 5.0))
    prm = O.params(mu=mu)
    _, g = M.rhs(U, prm, with_grad=True)
    _, J = M.metrics()
    w = O.ops(N)[1]
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * J
    got = bench.eps_from_gradients(g, wq, np.ones_like(J), mu)
    want = M.dissipation(U, prm)
    assert abs(got[0] - want[0]) < 1e-13 * want[0] and abs(got[1] - want[1]) < 1e-13 * want[1], (got, want)
