"""Pins for the oracle's mesh handling: connectivity (unstructured neighbours with
orientation, Sec. 2.2 and App. A ProlongToFace/SurfInt) and curl-form metrics
(Sec. 2.2, Mapping the Equations).

Independent references: node coordinates (matched again here in numpy), the
closed-form metric of an affine map, the analytic cofactor matrix of the
curved mapping, and the exact volume of the periodic box.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_12703_gb300 import workloads as W


def face_nodes(n, f):
    """(p, q) -> (i, j, k) of local face f, in the face frame used by the oracle."""
    d, end = f // 2, (n - 1) * (f % 2)
    out = np.zeros((n * n, 3), int)
    for q in range(n):
        for p in range(n):
            ijk = [p, q]
            ijk.insert(d, end)
            out[p + n * q] = ijk
    return out


@pytest.mark.parametrize("N,nel,curved,seed", [
    (2, (2, 3, 2), 0.0, None), (3, (3, 4, 5), 0.1, 7), (4, (2, 2, 3), 0.1, 20240419)])
def test_connectivity_by_coordinates(N, nel, curved, seed):
    m = W.box_mesh(N, nel, curved=curved, seed=seed)
    M = O.Mesh(N, m["xyz"], m["period"])
    nbr_e, nbr_f, master, node = M.connectivity()
    E, n = m["E"], N + 1
    L = m["period"]
    X = m["xyz"].reshape(E, n, n, n, 3)  # [e, k, j, i]
    for e in range(E):
        for f in range(6):
            e2, f2 = nbr_e[e, f], nbr_f[e, f]
            assert nbr_e[e2, f2] == e and nbr_f[e2, f2] == f
            assert master[e, f] + master[e2, f2] == 1
            assert master[e, f] == int(e * 6 + f < e2 * 6 + f2)
            a = face_nodes(n, f)
            b = face_nodes(n, f2)
            for pq in range(n * n):
                i, j, k = a[pq]
                i2, j2, k2 = b[node[e, f, pq]]
                d = X[e, k, j, i] - X[e2, k2, j2, i2]
                d = d - L * np.round(d / L)
                assert np.abs(d).max() < 1e-10
                assert node[e2, f2, node[e, f, pq]] == pq


def test_metrics_affine_rotated_elements():
    """Cartesian box with different h per direction and rotated element frames:
    J = det(dx/dxi) and J a^i = J grad(xi_i), closed form per element."""
    N = 3
    m = W.box_mesh(N, (2, 3, 4), length=(1.0, 2.0, 0.5), seed=5)
    M = O.Mesh(N, m["xyz"], m["period"])
    Ja, J = M.metrics()
    n = N + 1
    X = m["xyz"].reshape(m["E"], n, n, n, 3)
    for e in range(m["E"]):
        A = np.stack([(X[e, 0, 0, N] - X[e, 0, 0, 0]) / 2,
                      (X[e, 0, N, 0] - X[e, 0, 0, 0]) / 2,
                      (X[e, N, 0, 0] - X[e, 0, 0, 0]) / 2], axis=1)   # A[c, d] = dx_c/dxi_d
        detA = np.linalg.det(A)
        Ainv = np.linalg.inv(A)
        np.testing.assert_allclose(J[e], detA, rtol=1e-13)
        for i in range(3):
            np.testing.assert_allclose(Ja[e, :, i, :], np.broadcast_to(detA * Ainv[i], (n ** 3, 3)),
                                       atol=1e-13 * abs(detA))


@pytest.mark.parametrize("N", [3, 5])
def test_metrics_converge_to_analytic_cofactor(N):
    """Curved map x = X + eps h s(X) (1,1,1): the curl-form metrics approach the
    exact cofactor matrix det(F) F^{-1} of F = dx/dxi as N grows (interpolation
    error), which fixes the index/sign/transposition conventions."""
    L = 2 * math.pi
    nel = 3
    eps = 0.1
    h = L / nel
    errs = []
    for NN in (N, N + 2):
        m = W.box_mesh(NN, (nel,) * 3, curved=eps)
        M = O.Mesh(NN, m["xyz"], m["period"])
        Ja, J = M.metrics()
        n = NN + 1
        xi = W.lgl_points(NN)
        # undeformed node positions X (canonical, no rotation)
        E = m["E"]
        ez, rem = np.divmod(np.arange(E), nel * nel)
        ey, ex = np.divmod(rem, nel)
        ref = (xi + 1) / 2
        Xg = np.empty((E, n, n, n, 3))
        Xg[..., 0] = (ex[:, None, None, None] + ref[None, None, None, :]) * h
        Xg[..., 1] = (ey[:, None, None, None] + ref[None, None, :, None]) * h
        Xg[..., 2] = (ez[:, None, None, None] + ref[None, :, None, None]) * h
        k = 2 * math.pi / L
        sx, sy, sz = (np.sin(k * Xg[..., c]) for c in range(3))
        cx, cy, cz = (np.cos(k * Xg[..., c]) for c in range(3))
        grad_s = np.stack([k * cx * sy * sz, k * sx * cy * sz, k * sx * sy * cz], axis=-1)
        F = np.eye(3) + eps * h * np.ones(3)[:, None] * grad_s[..., None, :]   # [..., c, d'] dx_c/dX_d'
        F = F * (h / 2)                                                      # dX/dxi = h/2
        det = np.linalg.det(F)
        cof = det[..., None, None] * np.linalg.inv(F)                        # [..., i, c]
        Jr = Ja.reshape(E, n, n, n, 3, 3)
        errs.append(np.abs(Jr - cof).max() / np.abs(cof).max())
        np.testing.assert_allclose(J.reshape(E, n, n, n), det, rtol=0.05)
    # degree-N interpolation error: small, and shrinking fast with N
    assert errs[0] < 0.1
    assert errs[1] < errs[0] / 4, errs


@pytest.mark.parametrize("N,curved,seed", [(3, 0.1, 3), (7, 0.1, 20240419)])
def test_discrete_metric_identities(N, curved, seed):
    """sum_d D_d (J a^d) = 0 node-wise (what makes free-stream preservation
    possible), on a curved, rotated, renumbered mesh."""
    m = W.box_mesh(N, (3, 3, 3), curved=curved, seed=seed)
    M = O.Mesh(N, m["xyz"], m["period"])
    Ja, J = M.metrics()
    _, _, D, *_ = O.ops(N)
    n = N + 1
    Jr = Ja.reshape(m["E"], n, n, n, 3, 3)   # [e, k, j, i, d, c]
    res = (np.einsum("ia,ekjac->ekjic", D, Jr[..., 0, :])
           + np.einsum("ja,ekaic->ekjic", D, Jr[..., 1, :])
           + np.einsum("ka,eajic->ekjic", D, Jr[..., 2, :]))
    scale = np.abs(D).sum(axis=1).max() * np.abs(Ja).max()
    assert np.abs(res).max() < 4e-15 * scale * n


def test_total_volume():
    """Sum of w_i w_j w_k J over all elements = box volume (exact on affine
    elements; curved elements within the quadrature error)."""
    for curved, tol in ((0.0, 1e-13), (0.1, 1e-6)):
        N = 5
        m = W.box_mesh(N, (3, 3, 3), length=(1.0, 2.0, 3.0), curved=curved, seed=2)
        M = O.Mesh(N, m["xyz"], m["period"])
        _, J = M.metrics()
        x, w, *_ = O.ops(N)
        wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)
        vol = (J * wq).sum()
        assert abs(vol - 6.0) < tol * 6.0


def test_rejects_unmatched_mesh():
    m = W.box_mesh(2, (2, 2, 2))
    with pytest.raises(ValueError):
        O.Mesh(2, m["xyz"], np.array([0.0, 0.0, 0.0]))  # no periodicity -> open faces


def test_unstructured_ogrid_mesh():
    """The five-block O-grid mesh (centre square and four trapezoids, periodic
    in x, y and z): every face pairs up, edges have three, four or eight
    elements around them (not only the four of a box), and the operator keeps
    free streams to round-off and conserves on it, with both node sets."""
    from collections import Counter
    N = 3
    m = W.ogrid_mesh(N, m=3, k=2, nz=3, curved=0.1, seed=5)
    cnt = Counter()
    for cv in m["corner_vid"]:
        for c in range(4):
            cnt[tuple(sorted((cv[c], cv[c + 4])))] += 1
    valences = set(cnt.values())
    assert {3, 4, 8} <= valences, valences
    for gauss in (False, True):
        M = O.Mesh(N, m["xyz"], m["period"], gauss=gauss)
        nbr_e, _, _, _ = M.connectivity()
        assert (nbr_e >= 0).all()
        U = W.uniform_state((m["E"], (N + 1) ** 3), rho=1.1, vel=(0.4, -0.3, 0.25), p=3.0)
        Ut = M.rhs(U, O.params(mu=0.01))
        _, J = M.metrics()
        assert np.abs(Ut).max() < 1e-14 * 300.0 / J.min(), np.abs(Ut).max()
        x, w, *_ = O.ops(N, gauss=gauss)
        wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :, None] * J[..., None]
        U2 = W.random_perturbation(W.tgv_state(M.nodes() * 2 * np.pi, Ma=0.3).reshape(m["E"], -1, 5), 1e-2, 3)
        Ut2 = M.rhs(U2, O.params(mu=0.01))
        tot = (wq * Ut2).sum(axis=(0, 1))
        scale = (wq * np.abs(Ut2)).sum(axis=(0, 1))
        assert np.all(np.abs(tot) <= 1e-13 * scale), tot / scale


def test_every_rotation_pair_across_a_face():
    """All 24 x 24 ordered pairs of element rotations meet across a face (the
    centre element of a 3^3 box against its six neighbours, 96 meshes): the
    coordinate matching pairs every face node with the node at the same
    point, and the operator equals the unrotated one mapped back."""
    N = 2
    n = N + 1
    base = W.box_mesh(N, (3, 3, 3), curved=0.1)
    prm = O.params(mu=0.01)
    Ub = W.tgv_state(base["xyz"], Ma=0.5).reshape(base["E"], -1, 5)
    Ut_b = O.Mesh(N, base["xyz"], base["period"]).rhs(Ub, prm).reshape(base["E"], n, n, n, 5)
    scale = np.abs(Ut_b).max(axis=(0, 1, 2, 3))
    idx = np.arange(n)
    I, Jj, K = np.meshgrid(idx, idx, idx, indexing="ij")
    loc = np.stack([2 * I - N, 2 * Jj - N, 2 * K - N], axis=-1)
    seen = set()
    for a, bs, m in W.rotation_pair_meshes(N):
        seen.update((a, b) for b in bs)
        M = O.Mesh(N, m["xyz"], m["period"])
        nbr_e, nbr_f, master, node = M.connectivity()
        X = m["xyz"].reshape(m["E"], n, n, n, 3)
        e = 13
        for f in range(6):
            e2, f2 = nbr_e[e, f], nbr_f[e, f]
            fa, fb = face_nodes(n, f), face_nodes(n, f2)
            for pq in range(n * n):
                i, j, k = fa[pq]
                i2, j2, k2 = fb[node[e, f, pq]]
                d = X[e, k, j, i] - X[e2, k2, j2, i2]
                d = d - m["period"] * np.round(d / m["period"])
                assert np.abs(d).max() < 1e-10, (a, bs, f)
        Ut = M.rhs(W.tgv_state(m["xyz"], Ma=0.5).reshape(m["E"], -1, 5), prm).reshape(m["E"], n, n, n, 5)
        for el in (13, 12, 14, 10, 16, 4, 22):
            R = W.ROTATIONS[m["rot"][el]]
            can = (loc @ R.T + N) // 2
            mapped = Ut_b[m["canon"][el]][can[..., 2], can[..., 1], can[..., 0]]
            got = np.transpose(Ut[el], (2, 1, 0, 3))
            assert np.all(np.abs(got - mapped).max(axis=(0, 1, 2)) <= 1e-12 * scale), (a, bs, el)
    assert len(seen) == 24 * 24


def _corner_xyz(m):
    n = m["N"] + 1
    X = m["xyz"].reshape(m["E"], n, n, n, 3)   # [e, k, j, i]
    out = np.empty((m["E"], 8, 3))
    for c in range(8):
        i, j, k = (c & 1) * (n - 1), ((c >> 1) & 1) * (n - 1), ((c >> 2) & 1) * (n - 1)
        out[:, c] = X[:, k, j, i]
    return out


@pytest.mark.parametrize("make", ["rotation_pairs", "random", "ogrid"])
def test_corner_ids_agree_with_corner_coordinates(make):
    """The corner ids the library pairs faces by name the same point wherever
    they occur (up to the periodic shifts), and distinct ids distinct points:
    the generated meshes (explicit rotations, random rotations and
    renumbering, the O-grid) give the device and the oracle's coordinate
    matching the same topology."""
    if make == "rotation_pairs":
        meshes = [m for _, _, m in W.rotation_pair_meshes(2)][::7]
    elif make == "random":
        meshes = [W.box_mesh(3, (3, 4, 5), curved=0.1, seed=s) for s in (1, 2, 3)]
    else:
        meshes = [W.ogrid_mesh(3, m=3, k=2, nz=3, curved=0.1, seed=5)]
    for m in meshes:
        P = np.asarray(m["period"], dtype=float)
        C = _corner_xyz(m).reshape(-1, 3)
        ids = m["corner_vid"].reshape(-1)
        first = {}
        for v, x in zip(ids, C):
            if v in first:
                d = x - first[v]
                d = np.where(P > 0, d - P * np.round(d / np.where(P > 0, P, 1)), d)
                assert np.abs(d).max() < 1e-9
            else:
                first[v] = x
        pts = np.array(list(first.values()))
        key = np.where(P > 0, np.mod(pts, np.where(P > 0, P, 1)), pts)
        key = np.round(key * 1e6).astype(np.int64)
        key = np.where(P > 0, np.mod(key, np.round(np.where(P > 0, P, 1) * 1e6).astype(np.int64)), key)
        assert len({tuple(r) for r in key}) == len(first)
