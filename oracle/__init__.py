"""Python loader for the plain FP64 CPU oracle (``dg_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it never calls the CUDA library.

Parity status of each function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants and worked examples (see each test's docstring); no
function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DG_ORACLE_SOURCE / DG_ORACLE_BUILD point the loader at another copy of the
# source and build folder: the test that plants mistakes in a copy of the
# oracle and checks that its pins catch each one uses them
_SRC = os.environ.get("DG_ORACLE_SOURCE") or os.path.join(_HERE, "dg_oracle.c")
_OUT = os.environ.get("DG_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS = {}

#: parameter vector layout shared with dg_oracle.c's read_params()
PARAM_KEYS = ("gamma", "R", "Pr", "mu", "riemann", "viscous", "shock",
              "alpha_min", "alpha_max", "cfl", "dfl", "alpha_force", "sutherland", "T_ref",
              "source", "source_A", "source_a")


def build(quad: bool = True, force: bool = False) -> None:
    """Compile the oracle (and its long-double twin) with gcc."""
    os.makedirs(_OUT, exist_ok=True)
    jobs = [("liboracle.so", [])]
    if quad:
        jobs.append(("liboracle_q.so", ["-DORC_QUAD"]))
    procs = []
    for name, extra in jobs:
        out = os.path.join(_OUT, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
               "-ffp-contract=off", *extra, "-o", out + ".tmp", _SRC, "-lm"]
        procs.append((subprocess.Popen(cmd), out))
    for p, out in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed")
        os.replace(out + ".tmp", out)


def _lib(quad: bool = False):
    key = "q" if quad else "d"
    with _LOCK:
        if key in _LIBS:
            return _LIBS[key]
        build(quad=quad)
        lib = C.CDLL(os.path.join(_OUT, "liboracle_q.so" if quad else "liboracle.so"))
        pre = "orcq_" if quad else "orc_"
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)

        def fn(name, res, args):
            f = getattr(lib, pre + name)
            f.restype = res
            f.argtypes = args
            return f

        api = {
            "ops": fn("ops", C.c_int, [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp]),
            "mesh_new": fn("mesh_new", C.c_void_p, [C.c_int, C.c_int, C.c_long, dp, dp, C.c_void_p, C.c_void_p,
                                                    C.c_int, C.c_void_p, ip]),
            "node_xyz": fn("node_xyz", None, [C.c_void_p, dp]),
            "mesh_free": fn("mesh_free", None, [C.c_void_p]),
            "set_sponge": fn("set_sponge", None, [C.c_void_p, C.c_void_p, C.c_void_p]),
            "connectivity": fn("connectivity", None, [C.c_void_p, ip, ip, ip, ip]),
            "metrics": fn("metrics", None, [C.c_void_p, dp, dp]),
            "rhs": fn("rhs", C.c_int, [C.c_void_p, dp, dp, C.c_double, dp, C.c_void_p, dp, dp, dp]),
            "mms_source": fn("mms_source", None, [dp, C.c_long, dp, C.c_double, dp]),
            "dt": fn("dt", C.c_double, [C.c_void_p, dp, dp, ip]),
            "step": fn("step", C.c_int, [C.c_void_p, dp, dp, C.c_int, C.c_double, dp, dp, C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
            "kinetic": fn("kinetic", None, [C.c_void_p, dp, dp, dp]),
            "dissipation": fn("dissipation", C.c_int, [C.c_void_p, dp, dp, dp]),
            "point_flux": fn("point_flux", None, [dp, C.c_int, dp, dp, dp, dp]),
            "point_visc": fn("point_visc", None, [dp, dp, dp, dp, dp]),
            "indicator": fn("indicator", C.c_double, [C.c_int, dp, dp, dp]),
            "lserk_ode": fn("lserk_ode", C.c_double, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                                      C.c_void_p, C.c_void_p, C.c_void_p]),
            "rk_coeffs": fn("rk_coeffs", None, [dp, dp, dp]),
            "rk14_coeffs": fn("rk14_coeffs", None, [dp, dp, dp]),
        }
        _LIBS[key] = api
        return api


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(gamma=1.4, R=1.0, Pr=0.72, mu=1.0 / 1600.0, riemann="roe", viscous=True,
           shock=False, alpha_min=1e-3, alpha_max=0.5, cfl=0.9, dfl=0.9,
           alpha_force=-1.0, sutherland=False, T_ref=1.0, source=0, source_A=0.1,
           source_a=1.0) -> np.ndarray:
    """Flat parameter vector in the oracle's layout.  ``alpha_force >= 0`` makes
    every element blend with that alpha instead of the indicator's (tests).
    ``sutherland``: mu(T) by Sutherland's law, ``mu`` being its value at T_ref.
    ``source = 1``: the manufactured-solution source of Sec. 5.1 with amplitude
    ``source_A`` and advection speed ``source_a``."""
    r = {"roe": 0, "lf": 1}[riemann] if isinstance(riemann, str) else int(riemann)
    return np.array([gamma, R, Pr, mu, r, int(bool(viscous)), int(bool(shock)),
                     alpha_min, alpha_max, cfl, dfl, alpha_force, int(bool(sutherland)), T_ref,
                     int(source), source_A, source_a], dtype=np.float64)


def mms_source(x, t, prm):
    """The manufactured-solution source Q(x, t) [n][5] at points x [n][3]."""
    x = np.ascontiguousarray(np.reshape(x, (-1, 3)), dtype=np.float64)
    Q = np.zeros((x.shape[0], 5))
    _lib()["mms_source"](_dp(_f64(prm)), x.shape[0], _dp(x), float(t), _dp(Q))
    return Q


def ops(N: int, quad: bool = False, gauss: bool = False):
    """Nodes x, weights w, D, Dhat, Dsplit and the inverse Legendre Vandermonde
    of the LGL (default) or Gauss-Legendre (``gauss``) node set."""
    return _ops_all(N, quad, gauss)[:6]


def face_interp(N: int, gauss: bool = False, quad: bool = False):
    """(l_i(+1), l_i(-1)): the Lagrange basis of the node set at the element ends."""
    return _ops_all(N, quad, gauss)[6:]


def _ops_all(N, quad, gauss):
    n = N + 1
    out = [np.zeros(n), np.zeros(n)] + [np.zeros((n, n)) for _ in range(4)] + [np.zeros(n), np.zeros(n)]
    if _lib(quad)["ops"](N, int(bool(gauss)), *[_dp(a) for a in out]) != 0:
        raise ValueError("bad N")
    return tuple(out)


def point_flux(kind: str, UL, UR, nvec, prm=None):
    """Two-state flux: kind in {'roe', 'lf', 'kep', 'euler'} (euler uses UL only)."""
    k = {"roe": 0, "lf": 1, "kep": 2, "euler": 3}[kind]
    f = np.zeros(5)
    prm = params() if prm is None else prm
    _lib()["point_flux"](_dp(_f64(prm)), k, _dp(_f64(UL)), _dp(_f64(UR)), _dp(_f64(nvec)), _dp(f))
    return f


def point_visc(U, g, nvec, prm=None):
    """Viscous flux F_v(U, g) . nvec; g[q, x] = d(u, v, w, T)_q / dx_x."""
    f = np.zeros(5)
    prm = params() if prm is None else prm
    _lib()["point_visc"](_dp(_f64(prm)), _dp(_f64(U)), _dp(_f64(np.reshape(g, 12))), _dp(_f64(nvec)), _dp(f))
    return f


def indicator(N, Uelem, prm=None):
    """Blending factor alpha and modal energy ratio E of one element's state."""
    Ev = np.zeros(1)
    prm = params(shock=True) if prm is None else prm
    a = _lib()["indicator"](N, _dp(_f64(prm)), _dp(_f64(np.reshape(Uelem, (-1, 5)))), _dp(Ev))
    return a, float(Ev[0])


def _rk_args(rk):
    """(ns, A, B, C pointers) of an optional 2N-storage scheme (A, B, C)."""
    if rk is None:
        return 0, None, None, None, None
    A, B, Cc = (np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in rk)
    keep = (A, B, Cc)
    return len(A), A.ctypes.data, B.ctypes.data, Cc.ctypes.data, keep


def lserk_ode(kind: int, lam: float, y0: float, dt: float, n_steps: int, rk=None) -> float:
    """Integrate y' = lam y (kind 0) or y' = -y^2 + cos t (kind 1) with the
    five-stage LSERK scheme, or the 2N-storage scheme rk = (A, B, c)."""
    ns, a, b, c, keep = _rk_args(rk)
    return _lib()["lserk_ode"](kind, lam, y0, dt, n_steps, ns, a, b, c)


def rk_coeffs():
    A, B, Cc = np.zeros(5), np.zeros(5), np.zeros(5)
    _lib()["rk_coeffs"](_dp(A), _dp(B), _dp(Cc))
    return A, B, Cc


def rk14_coeffs():
    """(A, B, c) of the fourteen-stage fourth-order 2N-storage scheme of
    Niegemann, Diehl and Busch (the scheme of the paper's application run);
    pass it as rk= to Mesh.step and lserk_ode."""
    A, B, Cc = np.zeros(14), np.zeros(14), np.zeros(14)
    _lib()["rk14_coeffs"](_dp(A), _dp(B), _dp(Cc))
    return A, B, Cc


class Mesh:
    """Oracle view of one mesh: connectivity, metrics and the DG operator."""

    def __init__(self, N, xyz, period, quad=False, metric_mask=None, face_bc=None, bcs=None, gauss=False):
        """``metric_mask``: optional boolean mask over elements; metrics are then
        formed only for those elements and their face neighbours (use the same
        mask as ``want`` in ``rhs``).  ``face_bc``: [E, 6] boundary-condition row
        per face (0: a face with a partner; k >= 1: row k - 1 of ``bcs``);
        ``bcs``: rows of (type, 8 parameters), type 1 isothermal no-slip wall
        (u_w, v_w, w_w, T_w), 2 adiabatic no-slip wall (u_w, v_w, w_w), 3 slip
        wall, 4 prescribed state (5 conservative values), 5 pressure outflow (p_out).
        ``gauss``: the standard DGSEM on Gauss-Legendre nodes instead of the split
        form on LGL nodes; ``xyz`` stays the LGL-node geometry and ``nodes()``
        returns the solution-node coordinates."""
        self.N = int(N)
        self.n = self.N + 1
        xyz = _f64(xyz)
        self.E = xyz.shape[0]
        self.quad = quad
        self._api = _lib(quad)
        st = C.c_int(0)
        mask = None
        if metric_mask is not None:
            mask = np.ascontiguousarray(np.asarray(metric_mask, dtype=np.uint8))
        fb = bcv = None
        nbc = 0
        if face_bc is not None:
            fb = np.ascontiguousarray(np.asarray(face_bc, dtype=np.int32).reshape(-1))
            bcv = np.zeros((len(bcs), 9))
            for k, row in enumerate(bcs):
                bcv[k, :len(row)] = row
            nbc = len(bcs)
        self.gauss = bool(gauss)
        self._h = self._api["mesh_new"](self.N, int(self.gauss), self.E, _dp(xyz.reshape(-1)), _dp(_f64(period)),
                                        mask.ctypes.data if mask is not None else None,
                                        fb.ctypes.data if fb is not None else None, nbc,
                                        bcv.ctypes.data if bcv is not None else None, C.byref(st))
        self.status = st.value
        if self.status != 0:
            self.close()
            raise ValueError(f"oracle mesh construction failed ({self.status})")

    def set_sponge(self, sigma=None, base=None):
        """Sponge zone: the source -sigma (U - base) at every node (sigma
        [E, n^3], base [E, n^3, 5]); None removes it."""
        if sigma is None:
            self._api["set_sponge"](self._h, None, None)
            return
        self._sg = np.ascontiguousarray(_f64(sigma).reshape(-1))
        self._sb = np.ascontiguousarray(_f64(base).reshape(-1))
        self._api["set_sponge"](self._h, self._sg.ctypes.data, self._sb.ctypes.data)

    def close(self):
        if getattr(self, "_h", None):
            self._api["mesh_free"](self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _state(self, U):
        U = _f64(U).reshape(self.E, self.n ** 3, 5)
        return np.ascontiguousarray(U)

    def connectivity(self):
        E, n2 = self.E, self.n ** 2
        nbr_e = np.zeros((E, 6), np.int32)
        nbr_f = np.zeros((E, 6), np.int32)
        master = np.zeros((E, 6), np.int32)
        node = np.zeros((E, 6, n2), np.int32)
        self._api["connectivity"](self._h, _ip(nbr_e), _ip(nbr_f), _ip(master), _ip(node))
        return nbr_e, nbr_f, master, node

    def nodes(self):
        """Coordinates of the solution nodes [E][n^3][3]."""
        X = np.zeros((self.E, self.n ** 3, 3))
        self._api["node_xyz"](self._h, _dp(X))
        return X

    def metrics(self):
        Ja = np.zeros((self.E, self.n ** 3, 3, 3))
        J = np.zeros((self.E, self.n ** 3))
        self._api["metrics"](self._h, _dp(Ja), _dp(J))
        return Ja, J

    def rhs(self, U, prm, want=None, with_alpha=False, with_grad=False, with_fstar=False, t=0.0):
        """Ut = R(U) (+ the source at time t) in the public layout [E][n^3][5].  ``want`` is an optional
        boolean mask over elements (other elements' Ut are returned as 0).
        Optional extras: alpha [E], lifted gradients [E][n^3][4][3] and the
        surface flux times s-hat on master faces [E][6][n^2][5] (zero on slave
        faces), face node p + n q in the master's face frame."""
        U = self._state(U)
        Ut = np.zeros_like(U)
        mask = None
        if want is not None:
            mask = np.ascontiguousarray(np.asarray(want, dtype=np.uint8))
            assert mask.shape == (self.E,)
        alpha = np.zeros(self.E) if with_alpha else None
        grad = np.zeros((self.E, self.n ** 3, 4, 3)) if with_grad else None
        fstar = np.zeros((self.E, 6, self.n ** 2, 5)) if with_fstar else None
        st = self._api["rhs"](self._h, _dp(_f64(prm)), _dp(U), float(t), _dp(Ut),
                              mask.ctypes.data if mask is not None else None,
                              _dp(alpha) if alpha is not None else None,
                              _dp(grad) if grad is not None else None,
                              _dp(fstar) if fstar is not None else None)
        if st != 0:
            raise RuntimeError(f"oracle rhs failed ({st})")
        out = [Ut]
        if with_alpha:
            out.append(alpha)
        if with_grad:
            out.append(grad)
        if with_fstar:
            out.append(fstar)
        return out[0] if len(out) == 1 else tuple(out)

    def dt(self, U, prm):
        bad = C.c_int(0)
        d = self._api["dt"](self._h, _dp(_f64(prm)), _dp(self._state(U)), C.byref(bad))
        return d, bool(bad.value)

    def step(self, U, prm, n_steps, dt=0.0, t=0.0, rk=None):
        """Advance n_steps LSERK steps (the five-stage scheme, or the 2N-storage
        scheme rk = (A, B, c)); returns (U, t, last dt)."""
        U = self._state(U).copy()
        tt = np.array([t], dtype=np.float64)
        dl = np.zeros(1)
        ns, a, b, c, keep = _rk_args(rk)
        st = self._api["step"](self._h, _dp(_f64(prm)), _dp(U), int(n_steps), float(dt), _dp(tt), _dp(dl),
                               ns, a, b, c)
        if st != 0:
            raise RuntimeError(f"oracle step failed ({st})")
        return U, float(tt[0]), float(dl[0])

    def dissipation(self, U, prm):
        """(eps_S, eps_D): the solenoidal and dilatational dissipation rates of
        Sec. 5.2 from the lifted velocity gradients (rho_0 = U_0 = L = 1,
        Re = 1 / mu); viscous parameters only."""
        out = np.zeros(2)
        st = self._api["dissipation"](self._h, _dp(_f64(prm)), _dp(self._state(U)), _dp(out))
        if st != 0:
            raise RuntimeError(f"oracle dissipation failed ({st})")
        return tuple(out)

    def kinetic(self, U, Ut=None):
        """(E_k, dE_k/dt, |Omega|)."""
        out = np.zeros(3)
        self._api["kinetic"](self._h, _dp(self._state(U)),
                             _dp(self._state(Ut)) if Ut is not None else None, _dp(out))
        return tuple(out)
