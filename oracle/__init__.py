"""Python access to the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg import this package; the CUDA library and its binding never do.  Arrays use the oracle's
own layout: halo-padded [nvar][nz+4][ny+4][nx+4] float64 (see oracle.h).
"""
import ctypes
import numpy as np

from . import build as _build

HALO = 2


class Params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("viscous", ctypes.c_int),
        ("limiter", ctypes.c_int),
    ]


def params(gamma=1.4, mu=0.0, Pr=0.72, cfl=0.5, eps=0.1, viscous=False, limiter=0) -> Params:
    return Params(gamma, mu, Pr, cfl, eps, int(bool(viscous)), int(limiter))


PERIODIC, SLIP_WALL, FARFIELD = 0, 1, 2
FACES = {"-x": 0, "+x": 1, "-y": 2, "+y": 3, "-z": 4, "+z": 5}


class BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("inf", ctypes.c_double * 5)]


def bc(kinds=None, inf=(1.0, 0.0, 0.0, 0.0, 1.0 / 1.4)) -> BC:
    """kinds: {face name or index: kind} (faces not named stay periodic); inf: free-stream
    (rho, u, v, w, p) of FARFIELD faces"""
    k = [PERIODIC] * 6
    for f, v in (kinds or {}).items():
        k[FACES[f] if isinstance(f, str) else int(f)] = int(v)
    return BC((ctypes.c_int * 6)(*k), (ctypes.c_double * 5)(*inf))


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        i, sz = ctypes.c_int, ctypes.c_size_t
        L.oracle_cells.argtypes = [i, i, i]
        L.oracle_cells.restype = sz
        L.oracle_primitive.argtypes = [ctypes.c_double, _D, _D]
        L.oracle_primitive.restype = None
        L.oracle_muscl.argtypes = [i, _D, _D, _D, _D, _D, _D]
        L.oracle_muscl.restype = None
        L.oracle_roe_flux.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]
        L.oracle_roe_flux.restype = None
        L.oracle_metrics.argtypes = [i, i, i, _D, _D]
        L.oracle_fill_halo_periodic.argtypes = [i, i, i, i, _D]
        L.oracle_residual.argtypes = [P, i, i, i, _D, _D, _D]
        L.oracle_dt.argtypes = [P, i, i, i, _D, _D, _D]
        L.oracle_norms.argtypes = [sz, _D, _D]
        L.oracle_rk3_stage.argtypes = [i, sz, _D, _D, _D, ctypes.c_double, _D]
        L.oracle_step.argtypes = [P, i, i, i, _D, _D, i, _D, _D]
        L.oracle_step_fixed_dt.argtypes = [P, i, i, i, _D, _D, i, ctypes.c_double, _D]
        B = ctypes.POINTER(BC)
        L.oracle_metrics_bc.argtypes = [i, i, i, _D, B, _D]
        L.oracle_fill_halo_bc.argtypes = [ctypes.c_double, i, i, i, _D, B, _D]
        L.oracle_dt_local.argtypes = [P, i, i, i, _D, _D, _D]
        L.oracle_step_ex.argtypes = [P, i, i, i, _D, B, i, ctypes.c_double, _D, i, _D, _D]
        L.oracle_threads.argtypes = []
        L.oracle_set_threads.argtypes = [i]
        L.oracle_wcns_edge.argtypes = [i, _D]
        L.oracle_wcns_edge.restype = ctypes.c_double
        L.oracle_wcns_residual.argtypes = [P, i, i, i, _D, _D, _D]
        L.oracle_wcns_dt.argtypes = [P, i, i, i, _D, _D, _D]
        L.oracle_wcns_step.argtypes = [P, i, i, i, _D, _D, i, ctypes.c_double, _D, _D]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(n: int) -> int:
    """use n OpenMP threads from now on; returns the number in force"""
    return int(lib().oracle_set_threads(int(n)))


# ---- layout helpers -------------------------------------------------------------------------

def pad(q: np.ndarray) -> np.ndarray:
    """compact [nvar][nz][ny][nx] -> halo-padded copy (halo filled periodically)"""
    nvar, nz, ny, nx = q.shape
    out = np.zeros((nvar, nz + 2 * HALO, ny + 2 * HALO, nx + 2 * HALO))
    out[:, HALO:HALO + nz, HALO:HALO + ny, HALO:HALO + nx] = q
    _check(lib().oracle_fill_halo_periodic(nx, ny, nz, nvar, _ptr(out)), "fill_halo")
    return out


def interior(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a[:, HALO:-HALO, HALO:-HALO, HALO:-HALO])


# ---- point functions ------------------------------------------------------------------------

def primitive(U, gamma=1.4) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    W = np.zeros(5)
    lib().oracle_primitive(gamma, _ptr(U), _ptr(W))
    return W


def muscl(w0, w1, w2, w3, limiter=0):
    ws = [np.ascontiguousarray(w, dtype=np.float64) for w in (w0, w1, w2, w3)]
    wl, wr = np.zeros(5), np.zeros(5)
    lib().oracle_muscl(limiter, *[_ptr(w) for w in ws], _ptr(wl), _ptr(wr))
    return wl, wr


def roe_flux(wl, wr, S, gamma=1.4, eps=0.1) -> np.ndarray:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    F = np.zeros(5)
    lib().oracle_roe_flux(gamma, eps, _ptr(wl), _ptr(wr), _ptr(S), _ptr(F))
    return F


# ---- field functions ------------------------------------------------------------------------

def metrics(nodes: np.ndarray) -> np.ndarray:
    """nodes [3][nz+1][ny+1][nx+1] -> halo-padded metrics [10][nz+4][ny+4][nx+4]"""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    _, nz1, ny1, nx1 = nodes.shape
    nx, ny, nz = nx1 - 1, ny1 - 1, nz1 - 1
    M = np.zeros((10, nz + 2 * HALO, ny + 2 * HALO, nx + 2 * HALO))
    _check(lib().oracle_metrics(nx, ny, nz, _ptr(nodes), _ptr(M)), "metrics")
    return M


def _dims(Qp):
    _, nz4, ny4, nx4 = Qp.shape
    return nx4 - 2 * HALO, ny4 - 2 * HALO, nz4 - 2 * HALO


def residual(p: Params, Qp: np.ndarray, M: np.ndarray) -> np.ndarray:
    """R(Q) at interior cells, compact [5][nz][ny][nx]; Qp's halo must be filled"""
    nx, ny, nz = _dims(Qp)
    R = np.zeros((5, nz, ny, nx))
    _check(lib().oracle_residual(ctypes.byref(p), nx, ny, nz, _ptr(M), _ptr(Qp), _ptr(R)), "residual")
    return R


def dt(p: Params, Qp: np.ndarray, M: np.ndarray) -> float:
    nx, ny, nz = _dims(Qp)
    out = ctypes.c_double(0.0)
    _check(lib().oracle_dt(ctypes.byref(p), nx, ny, nz, _ptr(M), _ptr(Qp), ctypes.byref(out)), "dt")
    return out.value


def norms(R: np.ndarray) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.size // 5
    out = np.zeros(5)
    _check(lib().oracle_norms(n, _ptr(R), _ptr(out)), "norms")
    return out


def rk3_stage(stage: int, Qn, Qs, R, dt_: float) -> np.ndarray:
    Qn, Qs, R = (np.ascontiguousarray(a, dtype=np.float64) for a in (Qn, Qs, R))
    out = np.zeros_like(Qn)
    _check(lib().oracle_rk3_stage(stage, Qn.size, _ptr(Qn), _ptr(Qs), _ptr(R), dt_, _ptr(out)), "rk3_stage")
    return out


def step(p: Params, Qp: np.ndarray, M: np.ndarray, nsteps: int, dt_fixed=None):
    """nsteps SSP-RK3 steps on a periodic block; returns (Q padded, dts, stage-1 norms)"""
    Q = np.array(Qp, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = _dims(Q)
    norms_ = np.zeros((max(nsteps, 1), 5))
    if dt_fixed is None:
        dts = np.zeros(max(nsteps, 1))
        _check(lib().oracle_step(ctypes.byref(p), nx, ny, nz, _ptr(M), _ptr(Q), nsteps, _ptr(dts),
                                 _ptr(norms_)), "step")
    else:
        dts = np.full(max(nsteps, 1), float(dt_fixed))
        _check(lib().oracle_step_fixed_dt(ctypes.byref(p), nx, ny, nz, _ptr(M), _ptr(Q), nsteps,
                                          float(dt_fixed), _ptr(norms_)), "step_fixed_dt")
    return Q, dts[:nsteps], norms_[:nsteps]


# ---- boundary conditions and local time stepping ---------------------------------------------

def metrics_bc(nodes: np.ndarray, bcs: BC = None) -> np.ndarray:
    """metrics as metrics(); halo cells of non-periodic directions from reflected nodes"""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    _, nz1, ny1, nx1 = nodes.shape
    nx, ny, nz = nx1 - 1, ny1 - 1, nz1 - 1
    M = np.zeros((10, nz + 2 * HALO, ny + 2 * HALO, nx + 2 * HALO))
    _check(lib().oracle_metrics_bc(nx, ny, nz, _ptr(nodes), ctypes.byref(bcs) if bcs else None, _ptr(M)),
           "metrics_bc")
    return M


def fill_halo_bc(Qp: np.ndarray, M: np.ndarray, bcs: BC = None, gamma=1.4) -> np.ndarray:
    """copy of the halo-padded state with its halo filled (periodic, then boundary ghosts)"""
    Q = np.array(Qp, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = _dims(Q)
    _check(lib().oracle_fill_halo_bc(gamma, nx, ny, nz, _ptr(M), ctypes.byref(bcs) if bcs else None, _ptr(Q)),
           "fill_halo_bc")
    return Q


def dt_local(p: Params, Qp: np.ndarray, M: np.ndarray) -> np.ndarray:
    """per-cell CFL time step [nz][ny][nx]"""
    nx, ny, nz = _dims(Qp)
    out = np.zeros((nz, ny, nx))
    _check(lib().oracle_dt_local(ctypes.byref(p), nx, ny, nz, _ptr(M), _ptr(np.ascontiguousarray(Qp)), _ptr(out)),
           "dt_local")
    return out


def step_ex(p: Params, Qp: np.ndarray, M: np.ndarray, nsteps: int, bcs: BC = None, local_dt=False, dt_fixed=None):
    """nsteps SSP-RK3 steps with boundary conditions (None: periodic) and optionally local time
    steps or a fixed step; returns (Q padded, smallest dt per step, stage-1 norms)"""
    Q = np.array(Qp, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = _dims(Q)
    norms_ = np.zeros((max(nsteps, 1), 5))
    dts = np.zeros(max(nsteps, 1))
    _check(lib().oracle_step_ex(ctypes.byref(p), nx, ny, nz, _ptr(M), ctypes.byref(bcs) if bcs else None,
                                int(bool(local_dt)), float(dt_fixed or 0.0), _ptr(Q), nsteps, _ptr(dts),
                                _ptr(norms_)), "step_ex")
    return Q, dts[:nsteps], norms_[:nsteps]


# ---- the paper's own scheme: WCNS-E-5 (Eq. 2) on periodic uniform Cartesian blocks -----------
# compact arrays [5][nz][ny][nx]; p.limiter 0 = nonlinear interpolation weights, 1 = linear

def wcns_edge(u, linear=False) -> float:
    """value at i + 1/2 interpolated from the left, u = (u_{i-2} .. u_{i+2})"""
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size == 5
    return float(lib().oracle_wcns_edge(int(bool(linear)), _ptr(u)))


def wcns_residual(p: Params, Q: np.ndarray, h) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    _, nz, ny, nx = Q.shape
    hh = np.ascontiguousarray(h, dtype=np.float64)
    R = np.zeros_like(Q)
    _check(lib().oracle_wcns_residual(ctypes.byref(p), nx, ny, nz, _ptr(hh), _ptr(Q), _ptr(R)), "wcns_residual")
    return R


def wcns_dt(p: Params, Q: np.ndarray, h) -> float:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    _, nz, ny, nx = Q.shape
    hh = np.ascontiguousarray(h, dtype=np.float64)
    out = ctypes.c_double(0.0)
    _check(lib().oracle_wcns_dt(ctypes.byref(p), nx, ny, nz, _ptr(hh), _ptr(Q), ctypes.byref(out)), "wcns_dt")
    return out.value


def wcns_step(p: Params, Q: np.ndarray, h, nsteps: int, dt_fixed=None):
    """nsteps SSP-RK3 steps; returns (Q, dts, stage-1 norms)"""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    _, nz, ny, nx = Q.shape
    hh = np.ascontiguousarray(h, dtype=np.float64)
    dts = np.zeros(max(nsteps, 1))
    norms_ = np.zeros((max(nsteps, 1), 5))
    _check(lib().oracle_wcns_step(ctypes.byref(p), nx, ny, nz, _ptr(hh), _ptr(Q), nsteps, float(dt_fixed or 0.0),
                                  _ptr(dts), _ptr(norms_)), "wcns_step")
    return Q, dts[:nsteps], norms_[:nsteps]
