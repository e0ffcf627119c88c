"""Thin Python binding of the gbcfd C ABI (include/gbcfd.h).

Argument marshalling only: every step of the solver runs in the CUDA library.  PyTorch provides
the device memory (one uint8 tensor per block) and the stream.  Importing this module loads
libgbcfd.so (building it with nvcc if needed) and raises if that is impossible: there is no
CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

from . import build as _build

OK = 0
ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_STATE, ERR_MEMORY = -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
FACES = {"-x": 0, "+x": 1, "-y": 2, "+y": 3, "-z": 4, "+z": 5}
BC_NONE, BC_SLIP_WALL, BC_FARFIELD = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("entropy_eps", ctypes.c_double),
        ("viscous", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("local_dt", ctypes.c_int),
    ]


def params(gamma=1.4, mu=0.0, Pr=0.72, cfl=0.5, entropy_eps=0.1, viscous=False, limiter=0,
           precision=FP64, local_dt=False) -> Params:
    return Params(gamma, mu, Pr, cfl, entropy_eps, int(bool(viscous)), int(limiter), int(precision),
                  int(bool(local_dt)))


class GbcfdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gbcfd error {code}: {msg}")
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

# (name, argtypes) of every entry point declared in include/gbcfd.h
SIGNATURES = {
    "gbcfd_required_bytes": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                             ctypes.POINTER(ctypes.c_size_t)],
    "gbcfd_create_block": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), _VP,
                           ctypes.c_size_t, ctypes.POINTER(_VP)],
    "gbcfd_destroy_block": [_VP],
    "gbcfd_connect": [_VP, ctypes.c_int, _VP],
    "gbcfd_set_metrics": [_VP, _VP, _D, _VP],
    "gbcfd_set_state": [_VP, _VP, _VP],
    "gbcfd_get_state": [_VP, _VP, _VP],
    "gbcfd_exchange_halos": [ctypes.POINTER(_VP), ctypes.c_int, _VP],
    "gbcfd_compute_residual": [_VP, _VP, _VP],
    "gbcfd_stage": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP],
    "gbcfd_step": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP],
    "gbcfd_residual_norm": [_VP, _D, _VP],
    "gbcfd_get_dt": [_VP, _D, _VP],
    "gbcfd_time_step_noalloc": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), _D, _VP,
                                _VP],
    "gbcfd_set_boundary": [_VP, ctypes.c_int, ctypes.c_int, _D],
    "gbcfd_pipe_create": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)],
    "gbcfd_pipe_destroy": [_VP],
    "gbcfd_pipe_submit": [_VP, _VP, _VP, ctypes.c_int, _VP],
    "gbcfd_pipe_sync": [_VP],
    "gbcfd_wcns_pipe_create": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)],
    "gbcfd_group_pipe_create": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)],
    "gbcfd_group_required_bytes": [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
    "gbcfd_group_create": [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)],
    "gbcfd_group_destroy": [_VP],
    "gbcfd_group_step": [_VP, ctypes.c_int, _VP],
    "gbcfd_group_tune": [_VP, _VP, ctypes.POINTER(ctypes.c_int)],
    "gbcfd_group_tune_tile": [_VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "gbcfd_group_set_schedule": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP],
    "gbcfd_group_get_schedule": [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)],
    "gbcfd_group_set_timing": [_VP, ctypes.POINTER(_VP), ctypes.c_int],
    "gbcfd_accel_required_bytes": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
    "gbcfd_accel_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t,
                           ctypes.POINTER(_VP)],
    "gbcfd_accel_destroy": [_VP],
    "gbcfd_accel_set_params": [_VP, ctypes.POINTER(ctypes.c_float), _VP],
    "gbcfd_accel_get_params": [_VP, ctypes.POINTER(ctypes.c_float), _VP],
    "gbcfd_accel_forward": [_VP, _VP, _VP, _VP],
    "gbcfd_accel_train_step": [_VP, _VP, _VP, ctypes.c_float, ctypes.c_int, _D, _VP],
    "gbcfd_accel_get_train_state": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_float), _VP],
    "gbcfd_accel_features": [_VP, _VP, _VP, _VP],
    "gbcfd_accel_target": [_VP, _VP, _VP, _VP],
    "gbcfd_accel_try": [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_int), _D],
    "gbcfd_accel_try_smooth": [_VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_double, _VP,
                               ctypes.POINTER(ctypes.c_int), _D],
    "gbcfd_wcns_required_bytes": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                                  ctypes.POINTER(ctypes.c_size_t)],
    "gbcfd_wcns_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), _D, _VP, ctypes.c_size_t,
                          ctypes.POINTER(_VP)],
    "gbcfd_wcns_destroy": [_VP],
    "gbcfd_wcns_set_state": [_VP, _VP, _VP],
    "gbcfd_wcns_get_state": [_VP, _VP, _VP],
    "gbcfd_wcns_compute_residual": [_VP, _VP, _VP],
    "gbcfd_wcns_step": [_VP, ctypes.c_int, _VP],
    "gbcfd_wcns_connect": [_VP, ctypes.c_int, _VP],
    "gbcfd_wcns_step_many": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP],
    "gbcfd_wcns_residual_norm": [_VP, _D, _VP],
    "gbcfd_wcns_get_dt": [_VP, _D, _VP],
    "gbcfd_wcns_set_timing": [_VP, ctypes.POINTER(_VP), ctypes.c_int],
    "gbcfd_op_rate": [ctypes.c_int, _VP, _D, _VP],
    "gbcfd_last_error": [],
}


def lib():
    """Load libgbcfd.so (built in-tree on first use); raises if it cannot be built or loaded."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, argt in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = ctypes.c_char_p if name == "gbcfd_last_error" else ctypes.c_int
        _lib = L
    return _lib


def library_path() -> str:
    return os.path.abspath(_build.LIB)


def _check(rc):
    if rc != OK:
        raise GbcfdError(rc, lib().gbcfd_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


class Block:
    """One structured block: nx x ny x nz interior cells in a torch-owned device buffer."""

    def __init__(self, nx, ny, nz, prm: Params, device=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.params = prm
        nbytes = ctypes.c_size_t(0)
        _check(lib().gbcfd_required_bytes(self.nx, self.ny, self.nz, ctypes.byref(prm), ctypes.byref(nbytes)))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.memory = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.memory.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p(0)
        _check(lib().gbcfd_create_block(self.nx, self.ny, self.nz, ctypes.byref(prm),
                                        ctypes.c_void_p(base + off), nbytes.value, ctypes.byref(h)))
        self.handle = h

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gbcfd_destroy_block(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def connect(self, face, other: "Block"):
        f = FACES[face] if isinstance(face, str) else int(face)
        _check(lib().gbcfd_connect(self.handle, f, other.handle))

    def set_boundary(self, face, kind, inf=None):
        f = FACES[face] if isinstance(face, str) else int(face)
        arr = (ctypes.c_double * 5)(*inf) if inf is not None else None
        _check(lib().gbcfd_set_boundary(self.handle, f, int(kind), arr))

    def periodic(self):
        for d in range(3):
            self.connect(2 * d + 1, self)
        return self

    def set_metrics(self, spacing=None, nodes=None, stream=None):
        sp = (ctypes.c_double * 3)(*(spacing if spacing is not None else (1.0, 1.0, 1.0)))
        nptr = _ptr(nodes) if nodes is not None else None
        _check(lib().gbcfd_set_metrics(self.handle, nptr, sp, _stream(stream)))

    def set_state(self, q, stream=None):
        """q: compact [5][nz][ny][nx] float64, a CUDA tensor or a (pinned) host tensor/array"""
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        else:
            assert q.dtype == torch.float64 and q.is_contiguous()
        assert tuple(q.shape) == (5, self.nz, self.ny, self.nx)
        _check(lib().gbcfd_set_state(self.handle, _ptr(q), _stream(stream)))

    def get_state(self, out=None, stream=None):
        if out is None:
            out = torch.empty((5, self.nz, self.ny, self.nx), dtype=torch.float64, device=self.memory.device)
        _check(lib().gbcfd_get_state(self.handle, _ptr(out), _stream(stream)))
        return out

    def compute_residual(self, out=None, stream=None):
        if out is None:
            out = torch.empty((5, self.nz, self.ny, self.nx), dtype=torch.float64, device=self.memory.device)
        _check(lib().gbcfd_compute_residual(self.handle, _ptr(out), _stream(stream)))
        return out

    def residual_norm(self, stream=None) -> np.ndarray:
        out = np.zeros(5)
        _check(lib().gbcfd_residual_norm(self.handle, out.ctypes.data_as(_D), _stream(stream)))
        return out

    def get_dt(self, stream=None) -> float:
        out = ctypes.c_double(0.0)
        _check(lib().gbcfd_get_dt(self.handle, ctypes.byref(out), _stream(stream)))
        return out.value


def _handles(blocks):
    arr = (ctypes.c_void_p * len(blocks))(*[b.handle.value for b in blocks])
    return arr


def exchange_halos(blocks, stream=None):
    _check(lib().gbcfd_exchange_halos(_handles(blocks), len(blocks), _stream(stream)))


def stage(blocks, s, stream=None):
    _check(lib().gbcfd_stage(_handles(blocks), len(blocks), int(s), _stream(stream)))


def step(blocks, nsteps=1, stream=None):
    _check(lib().gbcfd_step(_handles(blocks), len(blocks), int(nsteps), _stream(stream)))


def create_block(nx, ny, nz, prm: Params, device=None) -> Block:
    return Block(nx, ny, nz, prm, device)


def block_for_case(case, precision=FP64, periodic=True, device=None, local_dt=None) -> Block:
    """Block configured from a cases.Case (physics, grid, initial state).  A case with boundary
    conditions (extra["bc"]: face -> kind, extra["inf"]: free stream) gets them on those faces,
    is periodic in the other directions and steps with local time steps unless told otherwise."""
    bcs = case.extra.get("bc") if case.extra else None
    if local_dt is None:
        local_dt = bool(bcs)
    prm = params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, case.limiter, precision, local_dt)
    b = Block(case.nx, case.ny, case.nz, prm, device)
    if bcs:
        for f, kind in bcs.items():
            b.set_boundary(f, kind, case.extra.get("inf"))
        for d, (lo, hi) in enumerate((("-x", "+x"), ("-y", "+y"), ("-z", "+z"))):
            if lo not in bcs and hi not in bcs:
                b.connect(2 * d + 1, b)
    elif periodic:
        b.periodic()
    if case.nodes is None:
        b.set_metrics(spacing=case.spacing)
    else:
        b.set_metrics(nodes=torch.from_numpy(np.ascontiguousarray(case.nodes)).to(b.memory.device))
    b.set_state(torch.from_numpy(np.ascontiguousarray(case.state)).to(b.memory.device))
    return b


def time_step_noalloc(q, prm: Params, spacing, out=None, stream=None):
    """CFL time step of a compact CUDA state q[5][nz][ny][nx] without any device allocation in the
    library; `out` is a caller-owned one-element float64 CUDA tensor (allocated here if None)."""
    assert q.is_cuda and q.dtype == torch.float64 and q.is_contiguous()
    _, nz, ny, nx = q.shape
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=q.device)
    sp = (ctypes.c_double * 3)(*spacing)
    _check(lib().gbcfd_time_step_noalloc(_ptr(q), nx, ny, nz, ctypes.byref(prm), sp, _ptr(out), _stream(stream)))
    return out


OP_DFMA, OP_FFMA, OP_DIV, OP_RCP_NEWTON, OP_RSQRT, OP_DADD, OP_DMUL, OP_DFMA_CONST = 0, 1, 2, 3, 4, 5, 6, 7


def op_rate(op, device=None, stream=None) -> float:
    """operations per second of one arithmetic operation on the GPU (gbcfd_op_rate): OP_DFMA,
    OP_FFMA, OP_DIV (FP64 1/x by IEEE division), OP_RCP_NEWTON (the FP64 path's reciprocal),
    OP_RSQRT (FP64)"""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.empty(8 * nsm, dtype=torch.float64, device=dev)
    out = ctypes.c_double(0.0)
    _check(lib().gbcfd_op_rate(int(op), _ptr(scratch), ctypes.byref(out), _stream(stream)))
    return out.value


class Pipe:
    """States in host memory advanced through identical blocks with the host-link copies
    overlapping the steps (gbcfd_pipe_*).  submit() enqueues one item; sync() waits for all.
    Buffers must be pinned (page-locked) float64 tensors of shape (5, nz, ny, nx); the pipeline
    holds references to them until sync()."""

    def __init__(self, blocks):
        """blocks: finite-volume Blocks, WcnsBlocks (the paper's scheme) or Groups built alike
        (an item is then the concatenation of the blocks' states, see item_numel)"""
        self.blocks = list(blocks)
        assert self.blocks and all(type(b) is type(self.blocks[0]) for b in self.blocks)
        h = ctypes.c_void_p(0)
        first = self.blocks[0]
        if isinstance(first, Group):
            create = lib().gbcfd_group_pipe_create
            self.item_numel = sum(5 * b.cells for b in first.blocks)
            self.norms_numel = 5 * len(first.blocks)
        else:
            create = lib().gbcfd_wcns_pipe_create if isinstance(first, WcnsBlock) else lib().gbcfd_pipe_create
            self.item_numel = 5 * first.cells
            self.norms_numel = 5
        _check(create(_handles(self.blocks), len(self.blocks), ctypes.byref(h)))
        self.handle = h
        self._inflight = []

    def submit(self, q_in, q_out, nsteps=1, norms=None):
        for t in (q_in, q_out):
            assert t.dtype == torch.float64 and t.is_contiguous() and t.numel() == self.item_numel
        if norms is not None:
            assert norms.dtype == torch.float64 and norms.is_contiguous() and norms.numel() == self.norms_numel
        self._inflight.append((q_in, q_out, norms))
        _check(lib().gbcfd_pipe_submit(self.handle, _ptr(q_in), _ptr(q_out), int(nsteps),
                                       _ptr(norms) if norms is not None else None))

    def sync(self):
        try:
            _check(lib().gbcfd_pipe_sync(self.handle))
        finally:
            self._inflight = []

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gbcfd_pipe_destroy(self.handle))
        self.handle = None
        self._inflight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many blocks advanced with one launch per stage and a CUDA graph per step (gbcfd_group_*)."""

    def __init__(self, blocks):
        self.blocks = list(blocks)
        nbytes = ctypes.c_size_t(0)
        _check(lib().gbcfd_group_required_bytes(len(self.blocks), ctypes.byref(nbytes)))
        dev = self.blocks[0].memory.device
        self.memory = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.memory.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p(0)
        _check(lib().gbcfd_group_create(_handles(self.blocks), len(self.blocks), ctypes.c_void_p(base + off),
                                        nbytes.value, ctypes.byref(h)))
        self.handle = h
        self.tile_rows = 8  # the default tile height until tune() or set_schedule()

    def step(self, nsteps=1, stream=None):
        _check(lib().gbcfd_group_step(self.handle, int(nsteps), _stream(stream)))

    def tune(self, stream=None) -> int:
        """choose the tile shape and grid split (gbcfd_group_tune_tile); returns the CTAs per SM,
        the tile height is kept in `tile_rows`"""
        c, t = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().gbcfd_group_tune_tile(self.handle, _stream(stream), ctypes.byref(c), ctypes.byref(t)))
        self.tile_rows = t.value
        return c.value

    def set_schedule(self, ctas_per_sm, tile_rows, halo_push=0, stream=None):
        """pin the tile height, grid split and halo fold (gbcfd_group_set_schedule)"""
        _check(lib().gbcfd_group_set_schedule(self.handle, int(ctas_per_sm), int(tile_rows), int(halo_push),
                                              _stream(stream)))
        self.tile_rows = int(tile_rows)

    def schedule(self):
        """(ctas_per_sm, tile_rows, halo_push) in force (gbcfd_group_get_schedule)"""
        c, t, p = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().gbcfd_group_get_schedule(self.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(p)))
        return c.value, t.value, p.value

    def set_timing(self, events):
        """events: 7 torch.cuda.Event(enable_timing=True) recorded inside every step (or None)"""
        self._events = events
        if events is None:
            _check(lib().gbcfd_group_set_timing(self.handle, None, 0))
            return
        for e in events:
            e.record()  # creates the underlying CUDA event
        torch.cuda.current_stream().synchronize()
        arr = (ctypes.c_void_p * 7)(*[e.cuda_event for e in events])
        _check(lib().gbcfd_group_set_timing(self.handle, arr, 7))

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gbcfd_group_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def blocks_for_lattice(lat, precision=MIXED, device=None):
    """The blocks of a cases.Lattice, connected face to face with periodic wrap and holding their
    part of the global state; returned in the lattice's block order (k slowest, then j, i)."""
    prm = params(lat.gamma, 0.0, 0.72, lat.cfl, lat.eps, False, 0, precision)
    nx, ny, nz = lat.shape
    sl = lat.block_slices()
    blk = {}
    for (i, j, k), (zs, ys, xs) in sl.items():
        b = Block(lat.sx[i], lat.sy[j], lat.sz[k], prm, device)
        b.set_metrics(spacing=lat.spacing)
        blk[(i, j, k)] = b
    for (i, j, k), b in blk.items():
        b.connect("+x", blk[((i + 1) % nx, j, k)])
        b.connect("+y", blk[(i, (j + 1) % ny, k)])
        b.connect("+z", blk[(i, j, (k + 1) % nz)])
    for key, b in blk.items():
        zs, ys, xs = sl[key]
        part = lat.state[:, zs, ys, xs]
        part = part.contiguous() if isinstance(part, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(part))
        b.set_state(part.to(b.memory.device))
    return [blk[key] for key in sl]


def gather_lattice(lat, blocks, out=None):
    """global state [5][Nz][Ny][Nx] float64 assembled from the lattice's blocks"""
    ox, oy, oz = lat.offsets()
    if out is None:
        out = torch.empty((5, oz[-1], oy[-1], ox[-1]), dtype=torch.float64, device=blocks[0].memory.device)
    for b, (zs, ys, xs) in zip(blocks, lat.block_slices().values()):
        out[:, zs, ys, xs] = b.get_state()
    return out


ACCEL_NPARAM = 40677


class Accel:
    """The learned convergence accelerator over `batch` volumes of nx x ny x nz cells
    (gbcfd_accel_*).  Features are bf16 [batch cells][16] tensors (torch.bfloat16), outputs and
    targets float32 [batch cells][8]."""

    def __init__(self, nx, ny, nz, batch=1, zperiodic=True, device=None):
        self.nx, self.ny, self.nz, self.batch = int(nx), int(ny), int(nz), int(batch)
        nbytes = ctypes.c_size_t(0)
        _check(lib().gbcfd_accel_required_bytes(self.nx, self.ny, self.nz, self.batch, ctypes.byref(nbytes)))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.memory = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.memory.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p(0)
        _check(lib().gbcfd_accel_create(self.nx, self.ny, self.nz, self.batch, int(bool(zperiodic)),
                                        ctypes.c_void_p(base + off), nbytes.value, ctypes.byref(h)))
        self.handle = h
        self.step_count = 0

    @property
    def cells(self):
        return self.nx * self.ny * self.nz * self.batch

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == ACCEL_NPARAM
        _check(lib().gbcfd_accel_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            _stream(stream)))
        self.step_count = 0

    def get_params(self, stream=None) -> np.ndarray:
        p = np.zeros(ACCEL_NPARAM, dtype=np.float32)
        _check(lib().gbcfd_accel_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            _stream(stream)))
        return p

    def forward(self, x, y=None, stream=None):
        if y is None:
            y = torch.empty((x.shape[0], 8), dtype=torch.float32, device=x.device)
        _check(lib().gbcfd_accel_forward(self.handle, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def train_step(self, x, t, lr, stream=None) -> float:
        self.step_count += 1
        loss = ctypes.c_double(0.0)
        _check(lib().gbcfd_accel_train_step(self.handle, _ptr(x), _ptr(t), float(lr), self.step_count,
                                            ctypes.byref(loss), _stream(stream)))
        return loss.value

    def train_state(self, stream=None):
        """(grad, m, v) after the last train_step: the gradient of its loss at the parameters it
        started from, and Adam's moments after its move (float32 arrays, parameter layout)"""
        out = [np.zeros(ACCEL_NPARAM, dtype=np.float32) for _ in range(3)]
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().gbcfd_accel_get_train_state(self.handle, *(a.ctypes.data_as(fp) for a in out), _stream(stream)))
        return tuple(out)

    def features(self, block, x=None, stream=None):
        _check(lib().gbcfd_accel_features(self.handle, block.handle, _ptr(x) if x is not None else None,
                                          _stream(stream)))
        return x

    def target(self, block, t, stream=None):
        _check(lib().gbcfd_accel_target(self.handle, block.handle, _ptr(t), _stream(stream)))
        return t

    def try_update(self, block, stream=None):
        """one accelerated update of the block; returns (accepted, rms R_rho before, after)"""
        acc = ctypes.c_int(0)
        norms = np.zeros(2)
        _check(lib().gbcfd_accel_try(self.handle, block.handle, _stream(stream), ctypes.byref(acc),
                                     norms.ctypes.data_as(_D)))
        return bool(acc.value), float(norms[0]), float(norms[1])

    def try_smooth(self, block, alpha, nsteps, ratio, stream=None):
        """prediction x alpha, nsteps plain steps, kept only below min(ratio, 1) x the residual before
        (gbcfd_accel_try_smooth); returns (accepted, rms R_rho before, after)"""
        acc = ctypes.c_int(0)
        norms = np.zeros(2)
        _check(lib().gbcfd_accel_try_smooth(self.handle, block.handle, float(alpha), int(nsteps), float(ratio),
                                            _stream(stream), ctypes.byref(acc), norms.ctypes.data_as(_D)))
        return bool(acc.value), float(norms[0]), float(norms[1])

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gbcfd_accel_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WcnsBlock:
    """A periodic uniform Cartesian block advanced with the paper's own WCNS-E-5 scheme (Eq. 2)
    and fourth-order central viscous terms (gbcfd_wcns_*); prm.limiter 0 = nonlinear weights,
    1 = linear."""

    def __init__(self, nx, ny, nz, prm: Params, spacing, device=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.params = prm
        nbytes = ctypes.c_size_t(0)
        _check(lib().gbcfd_wcns_required_bytes(self.nx, self.ny, self.nz, ctypes.byref(prm), ctypes.byref(nbytes)))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.memory = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.memory.data_ptr()
        off = (-base) % 256
        sp = (ctypes.c_double * 3)(*spacing)
        h = ctypes.c_void_p(0)
        _check(lib().gbcfd_wcns_create(self.nx, self.ny, self.nz, ctypes.byref(prm), sp, ctypes.c_void_p(base + off),
                                       nbytes.value, ctypes.byref(h)))
        self.handle = h

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def set_state(self, q, stream=None):
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        else:
            assert q.dtype == torch.float64 and q.is_contiguous()
        assert tuple(q.shape) == (5, self.nz, self.ny, self.nx)
        _check(lib().gbcfd_wcns_set_state(self.handle, _ptr(q), _stream(stream)))

    def get_state(self, out=None, stream=None):
        if out is None:
            out = torch.empty((5, self.nz, self.ny, self.nx), dtype=torch.float64, device=self.memory.device)
        _check(lib().gbcfd_wcns_get_state(self.handle, _ptr(out), _stream(stream)))
        return out

    def compute_residual(self, out=None, stream=None):
        if out is None:
            out = torch.empty((5, self.nz, self.ny, self.nx), dtype=torch.float64, device=self.memory.device)
        _check(lib().gbcfd_wcns_compute_residual(self.handle, _ptr(out), _stream(stream)))
        return out

    def step(self, nsteps=1, stream=None):
        _check(lib().gbcfd_wcns_step(self.handle, int(nsteps), _stream(stream)))

    def residual_norm(self, stream=None) -> np.ndarray:
        out = np.zeros(5)
        _check(lib().gbcfd_wcns_residual_norm(self.handle, out.ctypes.data_as(_D), _stream(stream)))
        return out

    def connect(self, face, other):
        """face 0..5 (-x, +x, -y, +y, -z, +z) of this block to the opposite face of `other`
        (gbcfd_wcns_connect); blocks connected to others advance with wcns_step_many"""
        _check(lib().gbcfd_wcns_connect(self.handle, int(face), other.handle))

    def get_dt(self, stream=None) -> float:
        out = ctypes.c_double(0.0)
        _check(lib().gbcfd_wcns_get_dt(self.handle, ctypes.byref(out), _stream(stream)))
        return out.value

    def set_timing(self, events, created=False):
        """events: 18 torch.cuda.Event(enable_timing=True), 6 per stage (or None).  created: the
        events have been recorded once already (so they exist), which skips a synchronisation."""
        self._events = events
        if events is None:
            _check(lib().gbcfd_wcns_set_timing(self.handle, None, 0))
            return
        if not created:
            for e in events:
                e.record()  # creates the underlying CUDA event
            torch.cuda.current_stream().synchronize()
        arr = (ctypes.c_void_p * 18)(*[e.cuda_event for e in events])
        _check(lib().gbcfd_wcns_set_timing(self.handle, arr, 18))

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().gbcfd_wcns_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wcns_step_many(blocks, nsteps=1, stream=None):
    """nsteps SSP-RK3 steps of connected WCNS blocks together (gbcfd_wcns_step_many)"""
    arr = (_VP * len(blocks))(*[b.handle for b in blocks])
    _check(lib().gbcfd_wcns_step_many(arr, len(blocks), int(nsteps), _stream(stream)))


def wcns_blocks_for_split(case, cuts, precision=FP64, linear=False, device=None):
    """A periodic uniform Cartesian case split into a lattice of WCNS blocks: cuts = the block
    sizes along x, y and z (each list sums to the case's size).  The blocks hold their part of
    the state and are connected face to face with periodic wrap; returned with k slowest, then j,
    then i (the order gather_wcns_split expects)."""
    assert case.nodes is None, "WCNS blocks are uniform Cartesian"
    sx, sy, sz = (list(map(int, c)) for c in cuts)
    assert (sum(sx), sum(sy), sum(sz)) == (case.nx, case.ny, case.nz)
    prm = params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, int(bool(linear)), precision)
    ox, oy, oz = np.cumsum([0] + sx), np.cumsum([0] + sy), np.cumsum([0] + sz)
    nxb, nyb, nzb = len(sx), len(sy), len(sz)
    blocks = []
    for k in range(nzb):
        for j in range(nyb):
            for i in range(nxb):
                b = WcnsBlock(sx[i], sy[j], sz[k], prm, case.spacing, device)
                part = case.state[:, oz[k]:oz[k + 1], oy[j]:oy[j + 1], ox[i]:ox[i + 1]]
                b.set_state(torch.from_numpy(np.ascontiguousarray(part)).to(b.memory.device))
                blocks.append(b)
    at = lambda i, j, k: blocks[((k % nzb) * nyb + (j % nyb)) * nxb + (i % nxb)]
    for k in range(nzb):
        for j in range(nyb):
            for i in range(nxb):
                at(i, j, k).connect(1, at(i + 1, j, k))
                at(i, j, k).connect(3, at(i, j + 1, k))
                at(i, j, k).connect(5, at(i, j, k + 1))
    return blocks


def gather_wcns_split(case, cuts, blocks):
    """the global state [5][nz][ny][nx] (float64, on the blocks' device) of a split lattice"""
    sx, sy, sz = (list(map(int, c)) for c in cuts)
    ox, oy, oz = np.cumsum([0] + sx), np.cumsum([0] + sy), np.cumsum([0] + sz)
    out = torch.empty((5, case.nz, case.ny, case.nx), dtype=torch.float64, device=blocks[0].memory.device)
    n = 0
    for k in range(len(sz)):
        for j in range(len(sy)):
            for i in range(len(sx)):
                out[:, oz[k]:oz[k + 1], oy[j]:oy[j + 1], ox[i]:ox[i + 1]] = blocks[n].get_state()
                n += 1
    return out


def wcns_block_for_case(case, precision=FP64, linear=False, device=None) -> WcnsBlock:
    """WCNS block configured from a periodic Cartesian cases.Case (physics, spacing, state)"""
    assert case.nodes is None, "WCNS blocks are uniform Cartesian"
    prm = params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, int(bool(linear)), precision)
    b = WcnsBlock(case.nx, case.ny, case.nz, prm, case.spacing, device)
    b.set_state(torch.from_numpy(np.ascontiguousarray(case.state)).to(b.memory.device))
    return b
