"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds only initial conditions and grids; none of the solver's arithmetic (no
reconstruction, flux, metric, residual or time stepping).  It imports neither the CUDA binding
nor the oracle, and both consume what it returns.

Arrays returned here:
  state  Q[5][nz][ny][nx] float64, conserved (rho, rho u, rho v, rho w, rho E) of Eq. 1
  nodes  X[3][nz+1][ny+1][nx+1] float64, the block's grid points (x, y, z)
The paper's meshes (NACA0012, DeltaWing, DLR-F6, CompCorner) are not available; these seeded
cases stand in for them with the sizes and flow regimes of the workloads the solver is built for.
"""
from dataclasses import dataclass, field
import math

import numpy as np

GAMMA = 1.4


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    state: np.ndarray
    nodes: np.ndarray = None          # None for a uniform Cartesian grid
    spacing: tuple = (1.0, 1.0, 1.0)  # cell size of the uniform Cartesian grid
    gamma: float = GAMMA
    mu: float = 0.0
    Pr: float = 0.72
    cfl: float = 0.5
    eps: float = 0.1
    viscous: bool = False
    limiter: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def grid_nodes(self) -> np.ndarray:
        """nodes of the block (uniform Cartesian ones when the case has none)"""
        if self.nodes is not None:
            return self.nodes
        return cartesian_nodes(self.nx, self.ny, self.nz, *self.spacing)


def conserved(rho, u, v, w, p, gamma=GAMMA) -> np.ndarray:
    """(rho, u, v, w, p) -> conserved state array (Eq. 1's Q)"""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    u, v, w, p = (np.broadcast_to(np.asarray(a, dtype=np.float64), shape) for a in (u, v, w, p))
    q = np.empty((5,) + shape)
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * v
    q[3] = rho * w
    q[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return q


def cartesian_nodes(nx, ny, nz, hx, hy, hz) -> np.ndarray:
    x = np.arange(nx + 1, dtype=np.float64) * hx
    y = np.arange(ny + 1, dtype=np.float64) * hy
    z = np.arange(nz + 1, dtype=np.float64) * hz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.ascontiguousarray(np.stack([X, Y, Z]))


def cell_centres(nx, ny, nz, hx, hy, hz):
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    z = (np.arange(nz) + 0.5) * hz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _periodic_delta(a, a0, period):
    d = a - a0
    return d - period * np.round(d / period)


# ---- 32^3 Gaussian pulse, Euler FP64 -------------------------------------------------------

def gaussian_pulse(n=32, seed=0, mach=0.5, amp=1e-2, width=0.1, gamma=GAMMA, nx=None, ny=None, nz=None) -> Case:
    """Unit periodic box, spacing 1/n, rho = 1, p = 1/gamma (so c = 1), u = Mach along x, plus
    amp * exp(-r^2 / width^2) added to rho and p/p_inf around a seeded centre (minimum-image r)."""
    nx, ny, nz = nx or n, ny or n, nz or n
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = rng.random(3)
    X, Y, Z = cell_centres(nx, ny, nz, *h)
    r2 = (_periodic_delta(X, x0[0], 1.0) ** 2 + _periodic_delta(Y, x0[1], 1.0) ** 2
          + _periodic_delta(Z, x0[2], 1.0) ** 2)
    g = np.exp(-r2 / width ** 2)
    rho = 1.0 + amp * g
    p = (1.0 / gamma) * (1.0 + amp * g)
    q = conserved(rho, mach, 0.0, 0.0, p, gamma)
    return Case("gaussian_pulse", nx, ny, nz, q, None, h, gamma=gamma, cfl=0.5, eps=0.1,
                extra={"centre": x0.tolist(), "seed": seed})


# ---- isentropic vortex (closed form), Navier-Stokes or Euler -------------------------------

def vortex_fields(X, Y, t, L, beta=5.0, mach=0.5, gamma=GAMMA, centre=None):
    """Closed-form isentropic vortex of strength beta convecting along x on a periodic box of
    side L (free stream rho = 1, p = 1, T = p / rho, c = sqrt(gamma)); exact for Euler."""
    uinf = mach * math.sqrt(gamma)
    xc0, yc0 = centre if centre is not None else (0.5 * L, 0.5 * L)
    dx = _periodic_delta(X, xc0 + uinf * t, L)
    dy = _periodic_delta(Y, yc0, L)
    r2 = dx * dx + dy * dy
    e = np.exp(0.5 * (1.0 - r2))
    u = uinf - beta / (2.0 * math.pi) * dy * e
    v = beta / (2.0 * math.pi) * dx * e
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return rho, u, v, p


def isentropic_vortex(n=256, L=10.0, nz=None, beta=5.0, mach=0.5, Re=1e4, Pr=0.72, viscous=True,
                      t=0.0, gamma=GAMMA, cfl=0.5, limiter=0, eps=0.1) -> Case:
    """z-invariant vortex on [0,L]^2 x [0, nz*h], h = L/n, periodic; mu = rho_inf |u_inf| / Re
    with reference length 1."""
    nz = nz or n
    h = L / n
    X, Y, _ = cell_centres(n, n, nz, h, h, h)
    rho, u, v, p = vortex_fields(X, Y, t, L, beta, mach, gamma)
    q = conserved(rho, u, v, 0.0, p, gamma)
    uinf = mach * math.sqrt(gamma)
    mu = uinf / Re if viscous else 0.0
    return Case("isentropic_vortex", n, n, nz, q, None, (h, h, h), gamma=gamma, mu=mu, Pr=Pr,
                cfl=cfl, eps=eps, viscous=viscous, limiter=limiter,
                extra={"L": L, "beta": beta, "mach": mach, "Re": Re})


# ---- warped curvilinear grid with broadband velocity perturbation -------------------------

def warped_nodes(nx, ny, nz, amp=0.05) -> np.ndarray:
    """[0,1]^3 mapped by x' = x + a sin(2 pi y) sin(2 pi z) and the cyclic permutations,
    applied simultaneously; periodic-compatible (the map shifts by whole periods)."""
    x = (np.arange(nx + 1, dtype=np.float64) / nx)[None, None, :]
    y = (np.arange(ny + 1, dtype=np.float64) / ny)[None, :, None]
    z = (np.arange(nz + 1, dtype=np.float64) / nz)[:, None, None]
    s = lambda a: np.sin(2.0 * math.pi * a)
    out = np.empty((3, nz + 1, ny + 1, nx + 1))
    out[0] = x + amp * s(y) * s(z)
    out[1] = y + amp * s(z) * s(x)
    out[2] = z + amp * s(x) * s(y)
    return out


def broadband_warped(nx=512, ny=512, nz=384, seed=0, mach=0.3, rms=0.05, kmax=16, Re=1e5,
                     Pr=0.72, amp=0.05, gamma=GAMMA, viscous=True, cfl=0.5, nmodes=48, device=None) -> Case:
    """Mean flow at Mach `mach` along x (rho = 1, p = 1/gamma, c = 1) on the warped unit box plus
    a seeded sum of Fourier modes with |k| <= kmax, each with its amplitude vector orthogonal to
    its wave vector (divergence-free in the logical coordinates), scaled to `rms` of |u_inf|.  The
    modes are evaluated at the logical cell centres as products of 1D complex exponentials
    (torch, on `device` when given) so that the 10^8-cell case generates in seconds."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    nodes = warped_nodes(nx, ny, nz, amp)
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = []
    while len(modes) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any() or np.dot(k, k) > kmax * kmax:
            continue
        a = rng.standard_normal(3)
        a -= np.dot(a, k) / np.dot(k, k) * k
        modes.append((k, a, rng.random() * 2.0 * math.pi))
    xi = [(torch.arange(n, dtype=torch.float64, device=dev) + 0.5) / n for n in (nx, ny, nz)]
    du = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=dev)
    for k, a, ph in modes:
        ex = torch.exp(1j * 2.0 * math.pi * k[0] * xi[0])
        ey = torch.exp(1j * 2.0 * math.pi * k[1] * xi[1])
        ez = torch.exp(1j * (2.0 * math.pi * k[2] * xi[2] + ph))
        field = (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag
        for c in range(3):
            du[c].add_(field, alpha=float(a[c]))
    uinf = mach
    du.mul_(rms * uinf / math.sqrt(float((du * du).sum(0).mean())))
    du = du.cpu().numpy()
    q = conserved(np.ones((nz, ny, nx)), uinf + du[0], du[1], du[2], 1.0 / gamma, gamma)
    mu = uinf / Re if viscous else 0.0
    return Case("broadband_warped", nx, ny, nz, q, nodes, (1.0 / nx, 1.0 / ny, 1.0 / nz), gamma=gamma,
                mu=mu, Pr=Pr, cfl=cfl, eps=0.1, viscous=viscous, extra={"seed": seed, "Re": Re})


# ---- random smooth states for parity sweeps -------------------------------------------------

def smooth_random(nx, ny, nz, seed=0, amp=0.05, mach=0.5, gamma=GAMMA, h=None, nodes=None,
                  viscous=False, mu=0.0, limiter=0, eps=0.1, cfl=0.5, nmodes=6) -> Case:
    """Free stream (rho = 1, p = 1/gamma, u = Mach along x) plus a few seeded periodic Fourier
    modes of relative amplitude `amp` in every primitive variable."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = h or (1.0 / nx, 1.0 / ny, 1.0 / nz)
    X, Y, Z = cell_centres(nx, ny, nz, *h)
    Lx, Ly, Lz = nx * h[0], ny * h[1], nz * h[2]
    prim = [np.ones_like(X), np.full_like(X, mach), np.zeros_like(X), np.zeros_like(X),
            np.full_like(X, 1.0 / gamma)]
    for m in range(5):
        scale = amp * (1.0 if m in (0, 4) else 1.0)
        ref = 1.0 if m in (0, 1, 2, 3) else 1.0 / gamma
        for _ in range(nmodes):
            k = rng.integers(-3, 4, size=3)
            ph = rng.random() * 2 * math.pi
            a = rng.standard_normal() / nmodes
            prim[m] = prim[m] + scale * ref * a * np.sin(
                2 * math.pi * (k[0] * X / Lx + k[1] * Y / Ly + k[2] * Z / Lz) + ph)
    q = conserved(*prim, gamma=gamma)
    return Case("smooth_random", nx, ny, nz, q, nodes, h, gamma=gamma, mu=mu, cfl=cfl, eps=eps,
                viscous=viscous, limiter=limiter, extra={"seed": seed})


def with_grid(case: Case, nodes: np.ndarray) -> Case:
    case.nodes = nodes
    return case


# ---- conforming lattice of uneven blocks, Euler at Mach 0.8 ---------------------------------

def lattice_sizes(seed, shape=(4, 4, 6), lo=16, hi=160):
    """per-slab cell counts of a shape[0] x shape[1] x shape[2] lattice of blocks, each drawn
    uniformly from lo..hi: block (i, j, k) has sx[i] x sy[j] x sz[k] cells, so every face is
    shared whole with exactly one neighbour (periodic wrap included)"""
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(rng.integers(lo, hi + 1, size=n).tolist() for n in shape)


def lattice_seed(shape=(4, 4, 6), lo=16, hi=160, total=(100_000_000, 140_000_000)):
    """the first seed 0, 1, 2, ... whose lattice holds between total[0] and total[1] cells"""
    s = 0
    while True:
        sx, sy, sz = lattice_sizes(s, shape, lo, hi)
        if total[0] <= sum(sx) * sum(sy) * sum(sz) <= total[1]:
            return s
        s += 1


@dataclass
class Lattice:
    sx: list
    sy: list
    sz: list
    state: object            # global state [5][Nz][Ny][Nx] float64 (torch tensor)
    spacing: tuple
    gamma: float = GAMMA
    mach: float = 0.8
    cfl: float = 0.5
    eps: float = 0.1
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return len(self.sx), len(self.sy), len(self.sz)

    @property
    def cells(self) -> int:
        return sum(self.sx) * sum(self.sy) * sum(self.sz)

    def offsets(self):
        c = lambda s: np.concatenate([[0], np.cumsum(s)]).astype(int).tolist()
        return c(self.sx), c(self.sy), c(self.sz)

    def block_slices(self):
        """(i, j, k) -> (z slice, y slice, x slice) of block (i, j, k) in the global arrays, in
        block order k (slowest), j, i"""
        ox, oy, oz = self.offsets()
        out = {}
        for k in range(len(self.sz)):
            for j in range(len(self.sy)):
                for i in range(len(self.sx)):
                    out[(i, j, k)] = (slice(oz[k], oz[k + 1]), slice(oy[j], oy[j + 1]), slice(ox[i], ox[i + 1]))
        return out


def lattice_case(sizes=None, seed=None, shape=(4, 4, 6), lo=16, hi=160, mach=0.8, amp=1e-2, gamma=GAMMA,
                 device=None) -> Lattice:
    """Periodic lattice of uneven Cartesian blocks, Euler: free stream rho = 1, p = 1/gamma (c = 1),
    u = Mach along x, with rho and p each perturbed by a sum of the 27 Fourier modes k in
    {1,2,3}^3 of the global box with seeded phases, scaled to a largest relative change of `amp`.
    Cells are cubes of side 1/Nx (Nx = sum of sx).  Without `sizes`, the lattice is the first seed
    whose total lies in 1.0e8..1.4e8 cells (`seed` picks the phases and defaults to that seed)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    if sizes is None:
        lseed = lattice_seed(shape, lo, hi)
        sizes = lattice_sizes(lseed, shape, lo, hi)
        seed = lseed if seed is None else seed
    seed = 0 if seed is None else seed
    sx, sy, sz = (list(map(int, s)) for s in sizes)
    Nx, Ny, Nz = sum(sx), sum(sy), sum(sz)
    h = 1.0 / Nx
    rng = np.random.Generator(np.random.PCG64(seed))
    xi = [(torch.arange(n, dtype=torch.float64, device=dev) + 0.5) / n for n in (Nx, Ny, Nz)]
    fields = []
    for _ in range(2):  # rho, then p
        ph = rng.random((3, 3, 3)) * 2.0 * math.pi
        d = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device=dev)
        for kz in range(1, 4):
            ez0 = torch.exp(1j * 2.0 * math.pi * kz * xi[2])
            for ky in range(1, 4):
                ey = torch.exp(1j * 2.0 * math.pi * ky * xi[1])
                for kx in range(1, 4):
                    ex = torch.exp(1j * 2.0 * math.pi * kx * xi[0])
                    ez = ez0 * complex(math.cos(ph[kz - 1, ky - 1, kx - 1]), math.sin(ph[kz - 1, ky - 1, kx - 1]))
                    d.add_((ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag)
        d.mul_(amp / float(d.abs().max()))
        fields.append(d)
    q = torch.empty((5, Nz, Ny, Nx), dtype=torch.float64, device=dev)
    rho = fields[0].add_(1.0)
    q[0] = rho
    q[1] = rho * mach
    q[2] = 0.0
    q[3] = 0.0
    q[4] = fields[1].add_(1.0).mul_(1.0 / (gamma * (gamma - 1.0))).add_(rho * (0.5 * mach * mach))
    return Lattice(sx, sy, sz, q, (h, h, h), gamma=gamma, mach=mach,
                   extra={"seed": seed, "shape": list(shape), "lo": lo, "hi": hi})


# ---- steady channel with a bump on the lower wall (inviscid) --------------------------------

def stretched_unit(n, ratio=1.1, cap=None) -> np.ndarray:
    """n + 1 points on [0, 1]: spacings h0 ratio^j from 0, each capped at `cap` (default 1.5 / n),
    with h0 found by bisection so that they sum to 1"""
    cap = 1.5 / n if cap is None else cap

    def total(h0):
        return sum(min(h0 * ratio ** j, cap) for j in range(n))

    lo, hi = 0.0, 1.0 / n
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < 1.0:
            lo = mid
        else:
            hi = mid
    h0 = 0.5 * (lo + hi)
    s = np.array([min(h0 * ratio ** j, cap) for j in range(n)])
    eta = np.concatenate([[0.0], np.cumsum(s)])
    eta /= eta[-1]
    return eta


def bump_wall(x, height):
    """lower wall y_w = height sin^2(pi x) on 0 <= x <= 1, flat elsewhere"""
    x = np.asarray(x, dtype=np.float64)
    return np.where((x >= 0.0) & (x <= 1.0), height * np.sin(math.pi * x) ** 2, 0.0)


def channel_nodes(nx=192, ny=96, nz=64, height=0.1, x0=-1.0, x1=2.0, lz=0.5, ratio=1.1) -> np.ndarray:
    """nodes of the channel x in [x0, x1], y from the bump wall to 1, z in [0, lz]: uniform in x
    and z, geometric from the lower wall in y (ratio `ratio`, capped at 1.5 / ny of the local
    height)"""
    x = x0 + (x1 - x0) * np.arange(nx + 1, dtype=np.float64) / nx
    z = lz * np.arange(nz + 1, dtype=np.float64) / nz
    eta = stretched_unit(ny, ratio)
    yw = bump_wall(x, height)
    out = np.empty((3, nz + 1, ny + 1, nx + 1))
    out[0] = x[None, None, :]
    out[1] = (yw[None, :] + (1.0 - yw[None, :]) * eta[:, None])[None, :, :]
    out[2] = z[:, None, None]
    return out


CHANNEL_BC = {"-x": 2, "+x": 2, "-y": 1, "+y": 1}   # far field in/out, slip walls, z periodic


def channel_case(nx=192, ny=96, nz=64, height=0.1, mach=0.6, gamma=GAMMA, cfl=0.9, ratio=1.1) -> Case:
    """Inviscid channel over a bump: the free stream (rho = 1, p = 1/gamma, c = 1, u = Mach along
    x) everywhere at the start; characteristic far field at x = -1 and x = 2, slip walls at the
    bump and at y = 1, periodic in z.  extra["bc"] names each face's condition (1 slip wall,
    2 far field) and extra["inf"] the free stream (rho, u, v, w, p)."""
    nodes = channel_nodes(nx, ny, nz, height, ratio=ratio)
    q = conserved(np.ones((nz, ny, nx)), mach, 0.0, 0.0, 1.0 / gamma, gamma)
    return Case("bump_channel", nx, ny, nz, q, nodes, (3.0 / nx, 1.0 / ny, 0.5 / nz), gamma=gamma, cfl=cfl,
                eps=0.1, extra={"bc": dict(CHANNEL_BC), "inf": (1.0, mach, 0.0, 0.0, 1.0 / gamma),
                                "height": height, "mach": mach})
