"""Thin Python binding of libdg's C ABI (``include/dg.h``).

Argument marshalling only: every step of the DG operator and the time
integration runs in libdg's CUDA kernels.  PyTorch supplies device memory and
the current CUDA stream.  There is no CPU fallback: if libdg.so cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")
_lock = threading.Lock()
_lib = None

DG_OK, DG_ERR_ARG, DG_ERR_MESH, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NONFINITE, DG_ERR_TIMEOUT, DG_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
DG_PENDING = 1
ROE, LF = 0, 1
FP64, FP32_BULK = 0, 1
DEBUG_METRICS, DEBUG_MAPS, DEBUG_GRAD, DEBUG_FSTAR, DEBUG_ALPHA = 0, 1, 2, 3, 4

#: every symbol include/dg.h declares
SERVE_EXPORTS = ("dg_server_default_config", "dg_server_create", "dg_submit", "dg_poll", "dg_server_stats",
                 "dg_server_destroy")
EXPORTS = SERVE_EXPORTS + ("dg_default_params", "dg_init_mesh", "dg_set_stream", "dg_set_params", "dg_set_state",
           "dg_get_state", "dg_rhs", "dg_step", "dg_advance", "dg_autotune", "dg_set_config", "dg_get_config",
           "dg_set_sponge", "dg_node_coords", "dg_quadrature_weights", "dg_selftest_convert",
           "dg_set_rk", "dg_set_rk_scheme", "dg_stage_form", "dg_selftest_wait_timeout",
           "dg_profile_step", "dg_time_step", "dg_kinetic", "dg_debug", "dg_sizes",
           "dg_destroy", "dg_error_string", "dg_last_error", "dg_launch_count", "dg_kinetic_noalloc",
           "dg_peak_probe")


class DgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdg error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("R", C.c_double), ("Pr", C.c_double), ("mu", C.c_double),
                ("riemann", C.c_int), ("viscous", C.c_int), ("shock_capturing", C.c_int),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("cfl", C.c_double),
                ("dfl", C.c_double), ("precision", C.c_int), ("alpha_force", C.c_double),
                ("sutherland", C.c_int), ("T_ref", C.c_double), ("source", C.c_int), ("source_A", C.c_double),
                ("source_a", C.c_double)]


SOURCE_NONE, SOURCE_MMS = 0, 1
RK_CK5, RK_NDB14 = 0, 1


class MeshDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("n_elems", C.c_int64), ("corner_vid", C.POINTER(C.c_int64)),
                ("xyz", C.POINTER(C.c_double)), ("face_bc", C.POINTER(C.c_int)), ("n_bc", C.c_int),
                ("bc", C.POINTER(C.c_double)), ("nodes", C.c_int)]


NODES_LGL, NODES_GAUSS = 0, 1


BC_WALL_ISOTHERMAL, BC_WALL_ADIABATIC, BC_SLIP, BC_STATE, BC_OUTFLOW = 1, 2, 3, 4, 5


def _bc_arrays(mesh):
    """(face_bc int32 [E*6], bc float64 [n_bc*9]) of a mesh dict with optional
    ``face_bc`` [E, 6] and ``bcs`` (rows of type + up to 8 parameters)."""
    if mesh.get("face_bc") is None:
        return None, None, 0
    fb = np.ascontiguousarray(np.asarray(mesh["face_bc"], dtype=np.int32).reshape(-1))
    rows = mesh.get("bcs") or []
    bc = np.zeros((max(len(rows), 1), 9))
    for k, r in enumerate(rows):
        bc[k, :len(r)] = r
    return fb, np.ascontiguousarray(bc.reshape(-1)), len(rows)


class ServerConfig(C.Structure):
    _fields_ = [("gamma", C.c_double), ("R", C.c_double), ("Pr", C.c_double), ("dfl", C.c_double),
                ("precision", C.c_int), ("max_cases", C.c_int), ("pool_elems", C.c_int64 * 8),
                ("max_resident_dof", C.c_int64), ("priority_dof", C.c_int64), ("persistent", C.c_int)]


class CaseDesc(C.Structure):
    _fields_ = [("mesh", MeshDesc), ("U0", C.POINTER(C.c_double)), ("t_end", C.c_double), ("mu", C.c_double),
                ("riemann", C.c_int), ("cfl", C.c_double)]


def load(path: str | None = None):
    """Load libdg.so (build it first with ``paper_2404_12703_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdg.so not found at {p}: run paper_2404_12703_gb300.build.build() first")
        lib = C.CDLL(p)
        vp = C.c_void_p
        dp = C.POINTER(C.c_double)
        sig = {
            "dg_default_params": (None, [C.POINTER(Params)]),
            "dg_init_mesh": (C.c_int, [C.POINTER(vp), C.POINTER(MeshDesc), C.POINTER(Params), vp]),
            "dg_set_stream": (C.c_int, [vp, vp]),
            "dg_node_coords": (C.c_int, [vp, vp, C.c_int]),
            "dg_quadrature_weights": (C.c_int, [vp, dp]),
            "dg_selftest_convert": (C.c_int, [vp, vp, vp, C.c_int64, vp]),
            "dg_set_rk": (C.c_int, [vp, C.c_int, dp, dp, dp]),
            "dg_set_rk_scheme": (C.c_int, [vp, C.c_int]),
            "dg_set_params": (C.c_int, [vp, C.POINTER(Params)]),
            "dg_set_state": (C.c_int, [vp, vp, C.c_int, C.c_double]),
            "dg_get_state": (C.c_int, [vp, vp, C.c_int, dp]),
            "dg_rhs": (C.c_int, [vp, vp, vp]),
            "dg_step": (C.c_int, [vp, C.c_int, C.c_double, dp]),
            "dg_advance": (C.c_int, [vp, C.c_double, C.c_int64, dp, C.POINTER(C.c_int64)]),
            "dg_autotune": (C.c_int, [vp, C.POINTER(C.c_int), dp]),
            "dg_set_sponge": (C.c_int, [vp, vp, vp]),
            "dg_set_config": (C.c_int, [vp, C.POINTER(C.c_int)]),
            "dg_get_config": (C.c_int, [vp, C.POINTER(C.c_int)]),
            "dg_stage_form": (C.c_int, [vp]),
            "dg_selftest_wait_timeout": (C.c_int, [vp, C.c_uint]),
            "dg_profile_step": (C.c_int, [vp, C.c_int, C.c_double, dp, C.POINTER(C.c_int64)]),
            "dg_time_step": (C.c_int, [vp, dp]),
            "dg_kinetic": (C.c_int, [vp, dp]),
            "dg_debug": (C.c_int, [vp, C.c_int, vp, vp]),
            "dg_sizes": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]),
            "dg_destroy": (None, [vp]),
            "dg_error_string": (C.c_char_p, [C.c_int]),
            "dg_last_error": (C.c_char_p, []),
            "dg_launch_count": (C.c_int64, []),
            "dg_kinetic_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int64, vp, vp, vp, vp, vp]),
            "dg_peak_probe": (C.c_int, [C.c_int, C.c_int, dp, dp, vp]),
            "dg_server_default_config": (None, [C.POINTER(ServerConfig)]),
            "dg_server_create": (C.c_int, [C.POINTER(vp), C.POINTER(ServerConfig)]),
            "dg_submit": (C.c_int, [vp, C.POINTER(CaseDesc), C.POINTER(C.c_int64)]),
            "dg_poll": (C.c_int, [vp, C.c_int64, vp, dp]),
            "dg_server_stats": (C.c_int, [vp, dp]),
            "dg_server_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(code):
    if code != DG_OK:
        lib = load()
        raise DgError(code, lib.dg_last_error().decode())
    return code


def default_params(**kw) -> Params:
    p = Params()
    load().dg_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "riemann" and isinstance(v, str):
            v = {"roe": ROE, "lf": LF}[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "fp32": FP32_BULK}[v]
        setattr(p, k, v)
    return p


def kinetic_noalloc(N, U, J, Ut=None, out=None, stream=None, nodes=0):
    """E_k, dE_k/dt and |Omega| of a caller-owned device state without any device
    allocation inside the library (for callers that cannot allocate: see
    dg_kinetic_noalloc in include/dg.h).  U: CUDA float64 [E, n^3, 5];
    J: CUDA float64 [E, n^3]; Ut: like U or None; out: CUDA float64 [3] or None
    (then a tensor is allocated here, by PyTorch, not by the library); nodes:
    NODES_LGL or NODES_GAUSS, the node set of the state.  Every buffer must sit
    on the current CUDA device, whose scratch the library uses."""
    import torch
    if not 1 <= int(N) <= 7:
        raise DgError(DG_ERR_ARG, "N must be in 1..7")
    if int(nodes) not in (NODES_LGL, NODES_GAUSS):
        raise DgError(DG_ERR_ARG, "nodes must be NODES_LGL or NODES_GAUSS")
    E = J.shape[0]
    n3 = (int(N) + 1) ** 3
    _device_buf(J, E * n3, "J")
    _device_buf(U, E * n3 * 5, "U")
    if Ut is not None:
        _device_buf(Ut, E * n3 * 5, "Ut")
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=U.device)
    _device_buf(out, 3, "out")
    cur = torch.cuda.current_device()
    for name, t in (("U", U), ("J", J), ("Ut", Ut), ("out", out)):
        if t is not None and t.device.index != cur:
            raise DgError(DG_ERR_ARG, f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    _check(load().dg_kinetic_noalloc(int(N), int(nodes), int(E), C.c_void_p(U.data_ptr()),
                                     C.c_void_p(J.data_ptr()), C.c_void_p(Ut.data_ptr() if Ut is not None else 0),
                                     C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


PEAK_FP64_FMA, PEAK_FP64_MMA, PEAK_FP64_BOTH, PEAK_FP32_FMA = 0, 1, 2, 3


def peak_probe(kind, iters=4096, stream=None):
    """(FLOP/s, ms) of the arithmetic peak probe `kind` (see dg_peak_probe)."""
    r, t = C.c_double(), C.c_double()
    _check(load().dg_peak_probe(int(kind), int(iters), C.byref(r), C.byref(t), _stream_ptr(stream)))
    return r.value, t.value


def convert_check(x, stream=None):
    """The library's integer-pipe conversions applied to a CUDA float64 tensor:
    (binary32 values, those values back in binary64)."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64:
        raise DgError(DG_ERR_ARG, "x: a CUDA float64 tensor is required")
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    back = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _check(load().dg_selftest_convert(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(back.data_ptr()), x.numel(), _stream_ptr(stream)))
    return out, back


def launch_count() -> int:
    return int(load().dg_launch_count())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _device_buf(t, numel, name, dtype="float64"):
    """Checks a tensor handed to the C ABI as a raw device pointer: a CUDA
    tensor of the given dtype, C-contiguous, with exactly numel values (the
    library reads and writes that many).  Raises DgError (DG_ERR_ARG)
    otherwise, like the library's own size checks."""
    import torch
    want = getattr(torch, dtype)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != want:
        raise DgError(DG_ERR_ARG, f"{name}: a CUDA {dtype} tensor is required")
    if not t.is_contiguous():
        raise DgError(DG_ERR_ARG, f"{name}: the tensor must be contiguous")
    if t.numel() != numel:
        raise DgError(DG_ERR_ARG, f"{name}: {t.numel()} values, expected {numel}")
    return t


def _mesh_arrays(xyz, cvid, N):
    """Checks the sizes of a mesh's node coordinates [E][(N+1)^3][3] and
    corner ids [E][8] before the library reads them."""
    E = int(xyz.shape[0]) if xyz.ndim else 0
    if xyz.size != E * (N + 1) ** 3 * 3:
        raise DgError(DG_ERR_ARG, f"xyz: {xyz.size} values, expected E (N+1)^3 3 = {E * (N + 1) ** 3 * 3}")
    if cvid.size != E * 8:
        raise DgError(DG_ERR_ARG, f"corner_vid: {cvid.size} values, expected 8 E = {8 * E}")


def _host_buf(a, numel, name):
    """Checks a host array handed to the C ABI: float64, C-contiguous, numel values."""
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise DgError(DG_ERR_ARG, f"{name}: a C-contiguous float64 array is required")
    if a.size != numel:
        raise DgError(DG_ERR_ARG, f"{name}: {a.size} values, expected {numel}")
    return a


class Solver:
    """One mesh on the current CUDA device, with its state.

    ``mesh`` is a dict with ``N``, ``xyz`` [E][n][n][n][3] (or [E][n^3][3]) and
    ``corner_vid`` [E][8] as produced by ``workloads.box_mesh``.  ``nodes``:
    "lgl" (split-form DGSEM, the default) or "gauss" (standard DGSEM on
    Gauss-Legendre nodes; ``xyz`` stays the LGL-node geometry and
    ``node_coords()`` gives the solution nodes).
    """

    def __init__(self, mesh, params: Params | None = None, stream=None, nodes="lgl", **kw):
        lib = load()
        self._lib = lib
        self.N = int(mesh["N"])
        self.n = self.N + 1
        xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        cvid = np.ascontiguousarray(mesh["corner_vid"], dtype=np.int64)
        self.E = int(xyz.shape[0])
        _mesh_arrays(xyz, cvid, self.N)
        self.params = params if params is not None else default_params(**kw)
        fb, bc, nbc = _bc_arrays(mesh)
        self._bc_keep = (fb, bc)
        desc = MeshDesc(self.N, self.E, cvid.ctypes.data_as(C.POINTER(C.c_int64)),
                        xyz.ctypes.data_as(C.POINTER(C.c_double)),
                        fb.ctypes.data_as(C.POINTER(C.c_int)) if fb is not None else None, nbc,
                        bc.ctypes.data_as(C.POINTER(C.c_double)) if bc is not None else None,
                        {"lgl": NODES_LGL, "gauss": NODES_GAUSS}[nodes] if isinstance(nodes, str) else int(nodes))
        self.nodes = desc.nodes
        h = C.c_void_p()
        _check(lib.dg_init_mesh(C.byref(h), C.byref(desc), C.byref(self.params), _stream_ptr(stream)))
        self._h = h

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self):
        N, E, S, b = C.c_int(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.dg_sizes(self._h, C.byref(N), C.byref(E), C.byref(S), C.byref(b)))
        return {"N": N.value, "E": E.value, "S": S.value, "bytes": b.value}

    def quadrature_weights(self):
        """1D quadrature weights of the solution nodes (LGL or Gauss-Legendre)."""
        w = (C.c_double * 8)()
        _check(self._lib.dg_quadrature_weights(self._h, w))
        return np.array(list(w)[:self.n])

    def node_coords(self):
        """Coordinates of the solution nodes [E][n^3][3] (numpy, float64)."""
        X = np.zeros((self.E, self.n ** 3, 3))
        _check(self._lib.dg_node_coords(self._h, C.c_void_p(X.ctypes.data), 0))
        return X

    def set_stream(self, stream=None):
        _check(self._lib.dg_set_stream(self._h, _stream_ptr(stream)))

    def set_params(self, params: Params | None = None, **kw):
        """Replaces the parameters (a Params, or keyword changes to the current
        ones); on an error the solver keeps its current parameters."""
        if params is None:
            params = Params()
            C.pointer(params)[0] = self.params  # a copy of the current parameters
            for k, v in kw.items():
                if k == "riemann" and isinstance(v, str):
                    v = {"roe": ROE, "lf": LF}[v]
                if k == "precision" and isinstance(v, str):
                    v = {"fp64": FP64, "fp32": FP32_BULK}[v]
                setattr(params, k, v)
        _check(self._lib.dg_set_params(self._h, C.byref(params)))
        self.params = params

    # -- state ----------------------------------------------------------------
    def set_state(self, U, t=0.0):
        """U: torch CUDA tensor or numpy array, float64, shape [E, n^3, 5] (any view)."""
        size = self.E * self.n ** 3 * 5
        if isinstance(U, np.ndarray):
            Uh = _host_buf(np.ascontiguousarray(U, dtype=np.float64), size, "U")
            _check(self._lib.dg_set_state(self._h, C.c_void_p(Uh.ctypes.data), 0, float(t)))
        else:
            _device_buf(U, size, "U")
            _check(self._lib.dg_set_state(self._h, C.c_void_p(U.data_ptr()), 1, float(t)))

    def get_state(self, out=None):
        """Returns (U, t).  ``out`` may be a CUDA tensor (device copy), a host
        numpy array of E * n^3 * 5 float64 (e.g. backed by pinned memory), or
        None (a new numpy array)."""
        t = C.c_double()
        size = self.E * self.n ** 3 * 5
        if out is None or isinstance(out, np.ndarray):
            U = np.empty((self.E, self.n ** 3, 5)) if out is None else _host_buf(out, size, "out")
            _check(self._lib.dg_get_state(self._h, C.c_void_p(U.ctypes.data), 0, C.byref(t)))
            return U, t.value
        _device_buf(out, size, "out")
        _check(self._lib.dg_get_state(self._h, C.c_void_p(out.data_ptr()), 1, C.byref(t)))
        return out, t.value

    # -- operator and time stepping --------------------------------------------
    def rhs(self, U=None, out=None):
        """Ut = R(U) on the device.  U: CUDA float64 tensor [E, n^3, 5] or None
        (the solver's own state).  Returns a CUDA tensor."""
        import torch
        size = self.E * self.n ** 3 * 5
        if U is not None:
            _device_buf(U, size, "U")
        if out is None:
            out = torch.empty((self.E, self.n ** 3, 5), dtype=torch.float64, device="cuda")
        _device_buf(out, size, "out")
        up = C.c_void_p(U.data_ptr()) if U is not None else C.c_void_p(0)
        _check(self._lib.dg_rhs(self._h, up, C.c_void_p(out.data_ptr())))
        return out

    def step(self, n_steps=1, dt=0.0, sync=False):
        """n_steps LSERK steps (dt <= 0: CFL steps).  Asynchronous and returns
        None; with sync=True the call waits and returns the time reached."""
        if not sync:
            _check(self._lib.dg_step(self._h, int(n_steps), float(dt), None))
            return None
        t = C.c_double()
        _check(self._lib.dg_step(self._h, int(n_steps), float(dt), C.byref(t)))
        return t.value

    def advance(self, t_end, max_steps=1 << 62):
        """CFL steps to exactly t_end (the last one clipped on the device);
        returns (time reached, steps taken)."""
        t = C.c_double()
        k = C.c_int64()
        _check(self._lib.dg_advance(self._h, float(t_end), int(max_steps), C.byref(t), C.byref(k)))
        return t.value, k.value

    def set_rk(self, A=None, B=None, c=None):
        """The 2N-storage low-storage RK scheme of step / advance (A[0] = 0);
        no arguments restore the default five-stage scheme."""
        if A is None:
            _check(self._lib.dg_set_rk(self._h, 0, None, None, None))
            return
        A, B, c = (np.ascontiguousarray(np.asarray(v, dtype=np.float64)).reshape(-1) for v in (A, B, c))
        if not A.size == B.size == c.size:
            raise DgError(DG_ERR_ARG, "A, B and c need one entry per stage each")
        dpt = C.POINTER(C.c_double)
        _check(self._lib.dg_set_rk(self._h, A.size, A.ctypes.data_as(dpt), B.ctypes.data_as(dpt),
                                   c.ctypes.data_as(dpt)))

    def set_rk_scheme(self, scheme):
        """A built-in scheme: RK_CK5 (the default five-stage one) or RK_NDB14
        (the fourteen-stage one of the paper's application run)."""
        if isinstance(scheme, str):
            scheme = {"ck5": RK_CK5, "ndb14": RK_NDB14}[scheme]
        _check(self._lib.dg_set_rk_scheme(self._h, int(scheme)))

    def set_sponge(self, sigma=None, U_base=None):
        """Sponge source -sigma (U - U_base): sigma [E, n^3] >= 0, U_base
        [E, n^3, 5] (host arrays); None removes it."""
        if sigma is None:
            _check(self._lib.dg_set_sponge(self._h, None, None))
            return
        sg = _host_buf(np.ascontiguousarray(sigma, dtype=np.float64), self.E * self.n ** 3, "sigma")
        ub = _host_buf(np.ascontiguousarray(U_base, dtype=np.float64), 5 * sg.size, "U_base")
        _check(self._lib.dg_set_sponge(self._h, C.c_void_p(sg.ctypes.data), C.c_void_p(ub.ctypes.data)))

    CONFIG_KEYS = ("lift_epb", "vol_epb", "vol_pairs", "side_block", "stage_form", "prefetch", "persistent")
    TUNE_KEYS = ("lift_D", "lift_2D", "vol_D", "vol_D_other_mapping", "vol_2D", "vol_2D_other_mapping",
                 "side_256", "side_128")

    def autotune(self):
        """Times the stage kernels' launch variants on the current state and
        keeps the fastest; returns (config, per-variant ms)."""
        cfg = (C.c_int * 7)()
        ms = (C.c_double * 8)()
        _check(self._lib.dg_autotune(self._h, cfg, ms))
        return dict(zip(self.CONFIG_KEYS, list(cfg))), {k: (v if v >= 0 else None)
                                                        for k, v in zip(self.TUNE_KEYS, list(ms))}

    def set_config(self, lift_epb=0, vol_epb=0, vol_pairs=-1, side_block=0, stage_form=0, prefetch=1, persistent=0):
        cfg = (C.c_int * 7)(lift_epb, vol_epb, vol_pairs, side_block, stage_form, prefetch, persistent)
        _check(self._lib.dg_set_config(self._h, cfg))

    def selftest_wait_timeout(self, spin_polls=5000):
        """Runs one persistent step launch whose grid-wide barriers wait for a
        participant that does not exist (see dg_selftest_wait_timeout); returns
        the library's status code (DG_ERR_TIMEOUT when the waits ran out)."""
        return self._lib.dg_selftest_wait_timeout(self._h, int(spin_polls))

    def stage_form(self):
        """2: the two-kernel FP32-bulk stage; 4: the four-kernel stage."""
        r = self._lib.dg_stage_form(self._h)
        if r < 0:
            _check(r)
        return r

    def config(self):
        cfg = (C.c_int * 7)()
        _check(self._lib.dg_get_config(self._h, cfg))
        return dict(zip(self.CONFIG_KEYS, list(cfg)))

    #: kernel kinds reported by profile_step, in the library's order
    KERNELS = ("cfl", "surf_prims", "lift", "surf_flux", "volume")

    def profile_step(self, n_steps=1, dt=0.0):
        """Per-kernel summed device time (ms) and launch counts over n_steps
        eagerly launched steps (CUDA events on the solver's stream)."""
        ms = (C.c_double * 5)()
        cnt = (C.c_int64 * 5)()
        _check(self._lib.dg_profile_step(self._h, int(n_steps), float(dt), ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNELS)}

    def time_step(self):
        dt = C.c_double()
        _check(self._lib.dg_time_step(self._h, C.byref(dt)))
        return dt.value

    def kinetic(self):
        out = (C.c_double * 3)()
        _check(self._lib.dg_kinetic(self._h, out))
        return tuple(out)

    # -- verification -------------------------------------------------------------
    def debug(self, what):
        import torch
        E, n3, n2 = self.E, self.n ** 3, self.n ** 2
        dev = "cuda"
        if what == "metrics":
            Ja = torch.empty((E, n3, 3, 3), dtype=torch.float64, device=dev)
            J = torch.empty((E, n3), dtype=torch.float64, device=dev)
            _check(self._lib.dg_debug(self._h, DEBUG_METRICS, C.c_void_p(Ja.data_ptr()), C.c_void_p(J.data_ptr())))
            return Ja.cpu().numpy(), J.cpu().numpy()
        if what == "maps":
            nbr = torch.empty((E, 6, 3), dtype=torch.int32, device=dev)
            nodes = torch.empty((E, 6, n2), dtype=torch.int32, device=dev)
            _check(self._lib.dg_debug(self._h, DEBUG_MAPS, C.c_void_p(nbr.data_ptr()), C.c_void_p(nodes.data_ptr())))
            return nbr.cpu().numpy(), nodes.cpu().numpy()
        if what == "grad":
            g = torch.empty((E, n3, 4, 3), dtype=torch.float64, device=dev)
            _check(self._lib.dg_debug(self._h, DEBUG_GRAD, C.c_void_p(g.data_ptr()), None))
            return g.cpu().numpy()
        if what == "fstar":
            f = torch.empty((E, 6, n2, 5), dtype=torch.float64, device=dev)
            _check(self._lib.dg_debug(self._h, DEBUG_FSTAR, C.c_void_p(f.data_ptr()), None))
            return f.cpu().numpy()
        if what == "alpha":
            a = torch.empty((E,), dtype=torch.float64, device=dev)
            _check(self._lib.dg_debug(self._h, DEBUG_ALPHA, C.c_void_p(a.data_ptr()), None))
            return a.cpu().numpy()
        raise ValueError(what)


class Server:
    """Continuous-batching request loop (include/dg.h, "Serving").

    ``pool_elems`` maps a polynomial degree to its pool capacity in elements;
    cases of that degree are admitted while their pool has room.
    """

    STAT_KEYS = ("time_to_solution", "queue_wait", "service_time", "t_final", "steps", "elements", "N",
                 "nonfinite")

    def __init__(self, pool_elems=None, max_cases=64, precision=FP64, gamma=1.4, R=1.0, Pr=0.72, dfl=0.9,
                 max_resident_dof=0, priority_dof=0, persistent=0):
        lib = load()
        self._lib = lib
        cfg = ServerConfig()
        lib.dg_server_default_config(C.byref(cfg))
        cfg.gamma, cfg.R, cfg.Pr, cfg.dfl = gamma, R, Pr, dfl
        cfg.precision = precision
        cfg.max_cases = max_cases
        cfg.max_resident_dof = int(max_resident_dof)
        cfg.priority_dof = int(priority_dof)
        cfg.persistent = int(persistent)
        if pool_elems is not None:
            for N in range(8):
                cfg.pool_elems[N] = int(pool_elems.get(N, 0))
        self.cfg = cfg
        self.meta = {}
        h = C.c_void_p()
        _check(lib.dg_server_create(C.byref(h), C.byref(cfg)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, mesh, U0, t_end, mu=0.0, riemann=ROE, cfl=0.9):
        """Queue one case; returns its ticket.  Arrays are copied by the library."""
        if isinstance(riemann, str):
            riemann = {"roe": ROE, "lf": LF}[riemann]
        xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        cvid = np.ascontiguousarray(mesh["corner_vid"], dtype=np.int64)
        N, E = int(mesh["N"]), int(xyz.shape[0])
        _mesh_arrays(xyz, cvid, N)
        U0 = _host_buf(np.ascontiguousarray(U0, dtype=np.float64), E * (N + 1) ** 3 * 5, "U0")
        d = CaseDesc()
        fb, bc, nbc = _bc_arrays(mesh)
        d.mesh = MeshDesc(N, E, cvid.ctypes.data_as(C.POINTER(C.c_int64)), xyz.ctypes.data_as(C.POINTER(C.c_double)),
                          fb.ctypes.data_as(C.POINTER(C.c_int)) if fb is not None else None, nbc,
                          bc.ctypes.data_as(C.POINTER(C.c_double)) if bc is not None else None)
        d.U0 = U0.ctypes.data_as(C.POINTER(C.c_double))
        d.t_end, d.mu, d.riemann, d.cfl = float(t_end), float(mu), int(riemann), float(cfl)
        t = C.c_int64()
        _check(self._lib.dg_submit(self._h, C.byref(d), C.byref(t)))
        self.meta[t.value] = (N, E)
        return t.value

    def poll(self, ticket, with_state=True):
        """(done, U or None, stats dict or None)."""
        N, E = self.meta[ticket]
        U = np.empty((E, (N + 1) ** 3, 5)) if with_state else None
        st = (C.c_double * 8)()
        code = self._lib.dg_poll(self._h, int(ticket), C.c_void_p(U.ctypes.data) if U is not None else None, st)
        if code == DG_PENDING:
            return False, None, None
        _check(code)
        return True, U, dict(zip(self.STAT_KEYS, list(st)))

    def wait(self, ticket, timeout=600.0, with_state=True):
        import time
        t0 = time.time()
        while True:
            done, U, stats = self.poll(ticket, with_state)
            if done:
                return U, stats
            if time.time() - t0 > timeout:
                raise TimeoutError(f"case {ticket} not finished after {timeout} s")
            time.sleep(0.002)

    def stats(self):
        out = (C.c_double * 10)()
        _check(self._lib.dg_server_stats(self._h, out))
        return dict(zip(("steps", "finished", "resident", "waiting", "captures", "dof_stage_updates",
                         "step_device_s", "capture_host_s", "setup_host_s", "insert_host_s"), list(out)))
