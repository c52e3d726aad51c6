"""Seeded case descriptions shaped like the paper's flow-over-orography tests.

The paper (Sec. 3.1) runs a stably stratified flow over a bell-shaped hill on
a terrain-following mesh that is refined, non-conformingly, near the ground.
The cases below reproduce those shapes synthetically:

* ``bubble2d`` -- 16x8 conforming quads over 20 km x 10 km, degree 2,
  isothermal 250 K atmosphere with a seeded warm cosine bubble.
* ``hill2d``   -- 64x32 base quads over 40 km x 20 km, degree 4, Gaussian
  hill of seeded height/width, two refinement levels near the ground giving
  2:1 hanging faces both horizontally and vertically, constant-N atmosphere
  (N = 0.01 1/s, Sec. 3.1) with a 10 m/s inflow.
* ``hill3d``   -- 32x32x16 base hexahedra over 40x40x20 km, degree 3, one
  refinement level below 1.5 km, Gaussian hill 400 m high.
* ``hill3d_big`` -- the same generator at 64x64x32 base cells (roofline sweep).

A case is pure data: integer cell coordinates per refinement level, and the
parameters of the terrain, the background atmosphere and the perturbation.
Cells are ordered base cell by base cell (x fastest, vertical slowest), and
depth-first (Morton) inside each base cell, so that neighbouring cells sit
close together in memory.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

# Physical constants of Sec. 2 (gravity, gas constant) and Sec. 3.1 (gamma).
GRAV = 9.81
R_GAS = 287.0
GAMMA = 1.4


@dataclasses.dataclass
class Case:
    """A seeded synthetic workload.

    Axis convention: axis 0 is x, axis 1 is y in 3D, and the last axis is the
    vertical (computational height zeta).  ``ijk[c, a]`` is the integer
    coordinate of cell ``c`` along axis ``a`` at its own refinement level
    ``levels[c]``; the cell covers ``[ijk*h, (ijk+1)*h]`` with
    ``h = extent[a] / base[a] / 2**level``.
    """

    name: str
    dim: int
    degree: int
    base: Tuple[int, ...]
    extent: Tuple[float, ...]
    periodic: Tuple[bool, ...]
    levels: np.ndarray  # uint8 [n_cells]
    ijk: np.ndarray  # int32 [n_cells, dim]
    hill: Dict[str, float]
    atmosphere: Dict[str, float]
    init: Dict[str, float]
    courant: float
    dt: float
    steps: int
    seed: int
    gravity: float = GRAV
    # Rayleigh damping layer below the top: {"depth": m, "rate": 1/s, "u0": m/s}, or None
    sponge: Optional[Dict[str, float]] = None

    @property
    def n_cells(self) -> int:
        return int(self.levels.shape[0])

    @property
    def n_vars(self) -> int:
        return self.dim + 2

    @property
    def nodes_per_cell(self) -> int:
        return (self.degree + 1) ** self.dim

    @property
    def n_nodes(self) -> int:
        return self.n_cells * self.nodes_per_cell

    @property
    def n_dof(self) -> int:
        return self.n_nodes * self.n_vars

    @property
    def max_level(self) -> int:
        return int(self.levels.max()) if self.n_cells else 0

    def cell_box(self, c: int) -> Tuple[np.ndarray, np.ndarray]:
        """Computational bounding box (lo, hi) of cell ``c``."""
        h = np.asarray(self.extent) / np.asarray(self.base) / (2 ** int(self.levels[c]))
        lo = self.ijk[c] * h
        return lo, lo + h

    def min_edge(self) -> float:
        """Smallest computational cell edge (the paper's H in the Courant number, Sec. 3)."""
        h = np.asarray(self.extent) / np.asarray(self.base)
        return float(h.min() / 2 ** self.max_level)


# ---------------------------------------------------------------------------
# refinement trees


def _cell_centre(level: int, ijk: Sequence[int], base, extent) -> np.ndarray:
    h = np.asarray(extent, dtype=np.float64) / np.asarray(base) / (2 ** level)
    return (np.asarray(ijk, dtype=np.float64) + 0.5) * h


def _neighbour(level, ijk, axis, side, base, periodic):
    """Same-level neighbour coordinate across a face, or None at a wall."""
    n = base[axis] * (2 ** level)
    c = list(ijk)
    c[axis] += 1 if side else -1
    if c[axis] < 0 or c[axis] >= n:
        if not periodic[axis]:
            return None
        c[axis] %= n
    return tuple(c)


def build_tree(dim, base, extent, periodic, rule: Optional[Callable], max_level: int):
    """Leaves of a 2:1 balanced quad/oct-tree forest over the base grid.

    ``rule(level, centre)`` says whether a leaf at ``level`` whose
    computational centre is ``centre`` should be split.
    """
    leaves = set()
    for idx in np.ndindex(*base):
        leaves.add((0, tuple(int(v) for v in idx)))
    for lvl in range(max_level):
        if rule is None:
            break
        new = set()
        for (l, c) in leaves:
            if l == lvl and rule(l, _cell_centre(l, c, base, extent)):
                for off in np.ndindex(*(2,) * dim):
                    new.add((l + 1, tuple(2 * c[a] + off[a] for a in range(dim))))
            else:
                new.add((l, c))
        leaves = new
    # 2:1 balance: a leaf must not touch, across a face, a leaf two levels finer.
    changed = True
    while changed:
        changed = False
        internal = set()
        for (l, c) in leaves:
            cc = c
            for ll in range(l - 1, -1, -1):
                cc = tuple(v // 2 for v in cc)
                internal.add((ll, cc))
        split = []
        for (l, c) in leaves:
            bad = False
            for a in range(dim):
                for side in (0, 1):
                    nb = _neighbour(l, c, a, side, base, periodic)
                    if nb is None or (l, nb) not in internal:
                        continue
                    # children of nb touching our face
                    for off in np.ndindex(*(2,) * dim):
                        if off[a] != (0 if side else 1):
                            continue
                        ch = (l + 1, tuple(2 * nb[b] + off[b] for b in range(dim)))
                        if ch in internal:
                            bad = True
            if bad:
                split.append((l, c))
        for (l, c) in split:
            leaves.discard((l, c))
            for off in np.ndindex(*(2,) * dim):
                leaves.add((l + 1, tuple(2 * c[a] + off[a] for a in range(dim))))
            changed = True
    return leaves


def _morton(v: Sequence[int], bits: int) -> int:
    key = 0
    d = len(v)
    for b in range(bits):
        for a in range(d):
            key |= ((int(v[a]) >> b) & 1) << (b * d + a)
    return key


def order_leaves(leaves, dim, base):
    """Order cells base cell by base cell, Morton order inside each."""
    lmax = max(l for (l, _) in leaves)
    strides = np.cumprod((1,) + tuple(base[:-1]))

    def key(item):
        l, c = item
        s = 2 ** l
        bc = [v // s for v in c]
        lin = int(sum(bc[a] * strides[a] for a in range(dim)))
        fine = [(v % s) * (2 ** (lmax - l)) for v in c]
        return (lin, _morton(fine, lmax), l)

    ordered = sorted(leaves, key=key)
    levels = np.array([l for (l, _) in ordered], dtype=np.uint8)
    ijk = np.array([c for (_, c) in ordered], dtype=np.int32).reshape(len(ordered), dim)
    return levels, ijk


# ---------------------------------------------------------------------------
# seeded random inputs shared by both sides


def noise(seed: int, n_vars: int, n_cells: int, nodes_per_cell: int) -> np.ndarray:
    """Standard-normal nodal noise, shape ``[n_vars, n_cells, nodes_per_cell]``."""
    return np.random.default_rng(seed).standard_normal((n_vars, n_cells, nodes_per_cell))


def smooth_modes(seed: int, case: Case, n_modes: int = 4) -> List[Dict]:
    """Parameters of a smooth random perturbation: sum of Fourier modes.

    Each mode is ``amp[v] * sin(k . x + phase)`` with integer wave numbers
    along periodic axes (so the field stays periodic) and half-integer ones
    along walled axes.  The caller evaluates it at its own node coordinates.
    """
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(n_modes):
        k = []
        for a in range(case.dim):
            m = int(rng.integers(1, 3))
            k.append(2.0 * math.pi * m / case.extent[a])
        modes.append(
            dict(k=np.array(k), phase=float(rng.uniform(0, 2 * math.pi)), amp=rng.standard_normal(case.n_vars))
        )
    return modes


# ---------------------------------------------------------------------------
# workloads


def _sound_speed_surface(atm: Dict[str, float]) -> float:
    if atm["kind"] == "none":
        return math.sqrt(GAMMA * R_GAS * 300.0)
    t = atm["T0"] if atm["kind"] == "isothermal" else atm["T_ref"]
    return math.sqrt(GAMMA * R_GAS * t)


def courant_dt(case_dim, degree, h_min, c, courant, sqrt_d=True) -> float:
    """Time step from the acoustic Courant number C = r c dt / (H sqrt(d)) (Sec. 3).

    ``sqrt_d=False`` drops the sqrt(d) factor, which is the reading under
    which the paper's worked example (r=4, dt=2 s, H=1 km -> C ~ 2.75) holds.
    """
    f = math.sqrt(case_dim) if sqrt_d else 1.0
    return courant * h_min * f / (degree * c)


def _finish(name, dim, degree, base, extent, periodic, leaves, hill, atm, init, courant, steps, seed):
    levels, ijk = order_leaves(leaves, dim, base)
    case = Case(
        name=name,
        dim=dim,
        degree=degree,
        base=tuple(base),
        extent=tuple(float(e) for e in extent),
        periodic=tuple(bool(p) for p in periodic),
        levels=levels,
        ijk=ijk,
        hill=hill,
        atmosphere=atm,
        init=init,
        courant=courant,
        dt=0.0,
        steps=steps,
        seed=seed,
    )
    case.dt = courant_dt(dim, degree, case.min_edge(), _sound_speed_surface(atm), courant)
    return case


def bubble2d(seed: int = 0, degree: int = 2, base=(16, 8)) -> Case:
    """16x8 conforming quads, isothermal 250 K, warm cosine bubble jittered by +-10%."""
    rng = np.random.default_rng(seed)
    j = rng.uniform(0.9, 1.1, size=4)
    extent = (20e3, 10e3)
    leaves = build_tree(2, base, extent, (True, False), None, 0)
    init = dict(kind="bubble", amp=2.0 * j[0], radius=2e3 * j[1], xc=10e3 * j[2], zc=2e3 * j[3])
    return _finish(
        "bubble2d", 2, degree, base, extent, (True, False), leaves,
        dict(kind="none"), dict(kind="isothermal", T0=250.0, p_ref=1e5), init, 1.0, 10, seed,
    )


def hill2d(seed: int = 0, degree: int = 4, base=(64, 32)) -> Case:
    """64x32 base quads over 40x20 km, Gaussian hill, two near-ground refinement levels.

    Level 1 where a base cell's centre is below 2 km; level 2 where a level-1
    cell's centre is below 1 km and within 5 km of the hill crest, so that the
    refined patch has hanging faces on its sides as well as on its top.
    """
    rng = np.random.default_rng(seed)
    extent = (40e3, 20e3)
    xc = 20e3
    hc = float(rng.uniform(200.0, 600.0))
    ah = float(rng.uniform(1e3, 3e3))
    sx = extent[0] / 40e3
    sz = extent[1] / 20e3

    def rule(level, centre):
        if level == 0:
            return centre[1] < 2e3 * sz
        if level == 1:
            return centre[1] < 1e3 * sz and abs(centre[0] - xc * sx) < 5e3 * sx
        return False

    leaves = build_tree(2, base, extent, (True, False), rule, 2)
    return _finish(
        "hill2d", 2, degree, base, extent, (True, False), leaves,
        dict(kind="gauss", hc=hc, half_width=ah, xc=xc * sx, yc=0.0),
        dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5),
        dict(kind="inflow", u0=10.0), 1.0, 200, seed,
    )


def hill3d(seed: int = 0, degree: int = 3, base=(32, 32, 16), name="hill3d") -> Case:
    """32x32x16 base hexahedra over 40x40x20 km, one refinement level below 1.5 km."""
    rng = np.random.default_rng(seed)
    extent = (40e3, 40e3, 20e3)
    jit = rng.uniform(-1e3, 1e3, size=2)
    band = 1.5e3

    def rule(level, centre):
        return level == 0 and centre[2] < band

    leaves = build_tree(3, base, extent, (True, True, False), rule, 1)
    return _finish(
        name, 3, degree, base, extent, (True, True, False), leaves,
        dict(kind="gauss", hc=400.0, half_width=2e3, xc=float(20e3 + jit[0]), yc=float(20e3 + jit[1])),
        dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5),
        dict(kind="inflow", u0=10.0), 1.0, 10, seed,
    )


def hill3d_big(seed: int = 0, degree: int = 3) -> Case:
    """Roofline-sweep size: the 3D generator at 64x64x32 base cells."""
    return hill3d(seed, degree, base=(64, 64, 32), name="hill3d_big")


def bell3d(seed: int = 0, degree: int = 4, refined: bool = True) -> Case:
    """Sec. 3.1's 3D medium-steep bell-shaped hill: 60 x 40 x 16 km, h = hc / (1 + r^2/a^2)^(3/2)
    with hc = 400 m, a = 1 km, crest at (30, 20) km; constant-N atmosphere (N = 0.01 1/s,
    T_ref = 293.15 K), 10 m/s inflow, degree 4, dt = 2 s.  The paper's non-reflecting top and
    lateral boundaries are read as absorbing layers (top 6 km; 10 km along the lateral boundaries,
    which are periodic).

    refined=False: the uniform 60 x 40 x 16 mesh of 1 km cells (250 m effective resolution at
    degree 4).  refined=True: 15 x 10 x 4 base cells of 4 km, refined to 2 km within 14 km of the
    crest below 8 km and to 1 km within 9 km of it below 4 km (2:1 balanced), 1972 cells whose
    finest resolution is the uniform mesh's (the paper's non-conforming mesh has 1958 cells)."""
    extent = (60e3, 40e3, 16e3)
    xc, yc = 30e3, 20e3
    if refined:
        base = (15, 10, 4)

        def rule(level, centre):
            r = math.hypot(centre[0] - xc, centre[1] - yc)
            if level == 0:
                return r < 14e3 and centre[2] < 8e3
            if level == 1:
                return r < 9e3 and centre[2] < 4e3
            return False

        leaves = build_tree(3, base, extent, (True, True, False), rule, 2)
    else:
        base = (60, 40, 16)
        leaves = build_tree(3, base, extent, (True, True, False), None, 0)
    case = _finish(
        "bell3d_nc" if refined else "bell3d_uniform", 3, degree, base, extent, (True, True, False), leaves,
        dict(kind="bell", hc=400.0, half_width=1e3, xc=xc, yc=yc),
        dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5),
        dict(kind="inflow", u0=10.0), 1.0, 1800, seed,
    )
    case.dt = 2.0  # Sec. 3.1
    case.sponge = dict(depth=6e3, rate=1.0 / 100.0, u0=10.0, lateral_width=10e3, lateral_rate=1.0 / 100.0)
    return case


def member2d(seed: int) -> Case:
    """One uneven ensemble member: base 16x8..128x64, 0-2 levels, degree 2-5."""
    rng = np.random.default_rng(seed)
    nx = int(rng.choice([16, 32, 64, 128]))
    base = (nx, nx // 2)
    levels = int(rng.integers(0, 3))
    degree = int(rng.integers(2, 6))
    extent = (40e3, 20e3)
    hc = float(rng.uniform(0.0, 1e3))
    xc = 20e3

    def rule(level, centre):
        return centre[1] < 2e3 / (2 ** level) and (level == 0 or abs(centre[0] - xc) < 5e3)

    leaves = build_tree(2, base, extent, (True, False), rule if levels else None, levels)
    if rng.uniform() < 0.5:
        init = dict(kind="bubble", amp=2.0, radius=2e3, xc=float(rng.uniform(5e3, 35e3)), zc=3e3)
    else:
        init = dict(kind="inflow", u0=10.0)
    return _finish(
        "member2d", 2, degree, base, extent, (True, False), leaves,
        dict(kind="gauss", hc=hc, half_width=2e3, xc=xc, yc=0.0),
        dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5), init, 1.0, 10, seed,
    )


def tiny_case(
    dim: int = 2,
    degree: int = 2,
    base=None,
    refine: Sequence[Tuple[int, ...]] = ((0, 0),),
    periodic=None,
    hill: Optional[Dict[str, float]] = None,
    atmosphere: Optional[Dict[str, float]] = None,
    extent=None,
    init: Optional[Dict[str, float]] = None,
    seed: int = 0,
    courant: float = 1.0,
) -> Case:
    """Small meshes for dense/brute-force checks: refine the listed base cells once."""
    if base is None:
        base = (3, 2) if dim == 2 else (2, 2, 2)
    if extent is None:
        extent = (3e3, 2e3) if dim == 2 else (2e3, 2e3, 2e3)
    if periodic is None:
        periodic = (True,) * (dim - 1) + (False,)
    if refine and len(refine[0]) != dim:
        refine = tuple(tuple(r) + (0,) * (dim - len(r)) for r in refine)
    targets = set(tuple(int(v) for v in r) for r in refine)

    def rule(level, centre):
        h = np.asarray(extent) / np.asarray(base)
        c = tuple(int(v) for v in np.floor(centre / h))
        return level == 0 and c in targets

    leaves = build_tree(dim, base, extent, periodic, rule if targets else None, 1 if targets else 0)
    return _finish(
        "tiny", dim, degree, base, extent, periodic, leaves,
        hill or dict(kind="none"),
        atmosphere or dict(kind="isothermal", T0=250.0, p_ref=1e5),
        init or dict(kind="rest"), courant, 1, seed,
    )


def request_case(seed: int, dof_lo: float = 1e4, dof_hi: float = 5e6) -> Case:
    """One serving request: 2D or 3D (50/50), degree 2-5, DoF log-uniform in [dof_lo, dof_hi].

    The base grid is sized to the drawn DoF (x by y by z/2 cells) with base
    cells of 1 km (finer when the domain would exceed 20 km in height, where the
    constant-N atmosphere's pressure runs out), so the domain grows with small
    requests and every request stays resolved (coarse cells of several km at
    low degree, run for hundreds of steps, go unstable in the collocated
    discretisation: the aliasing of the nonlinear fluxes is not damped).  A
    seeded hill of up
    to a fifth of the domain height (at most 1 km) and half-width a tenth of
    the domain length, a bubble (radius a fifth of the height) or an inflow,
    0 or 1 refinement level near the ground.
    """
    rng = np.random.default_rng(seed)
    dim = int(rng.choice([2, 3]))
    degree = int(rng.integers(2, 6))
    dof = float(np.exp(rng.uniform(np.log(dof_lo), np.log(dof_hi))))
    V = dim + 2
    cells = dof / (V * (degree + 1) ** dim)
    if dim == 2:
        nx = max(4, 2 * int(round(math.sqrt(2.0 * cells) / 2)))
        base, periodic = (nx, nx // 2), (True, False)
    else:
        nx = max(4, 2 * int(round((2.0 * cells) ** (1.0 / 3.0) / 2)))
        base, periodic = (nx, nx, nx // 2), (True, True, False)
    h = min(1e3, 20e3 / base[-1])
    extent = tuple(b * h for b in base)
    refine = bool(rng.uniform() < 0.5)
    dz = extent[-1] / base[-1]

    def rule(level, centre):
        return level == 0 and centre[-1] < 1.1 * dz

    leaves = build_tree(dim, base, extent, periodic, rule if refine else None, 1 if refine else 0)
    Lx, Lz = extent[0], extent[-1]
    hill = dict(kind="gauss", hc=float(rng.uniform(0.0, min(1e3, 0.2 * Lz))), half_width=0.1 * Lx,
                xc=0.5 * Lx, yc=0.5 * extent[1])
    if rng.uniform() < 0.5:
        init = dict(kind="bubble", amp=2.0, radius=0.2 * Lz, xc=float(rng.uniform(0.25, 0.75) * Lx), zc=0.35 * Lz,
                    yc=0.5 * extent[1])
    else:
        init = dict(kind="inflow", u0=10.0)
    return _finish(
        "request", dim, degree, base, extent, periodic, leaves, hill,
        dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5), init, 1.0, 10, seed,
    )


def serving_trace(seed: int, n: int, rate: float = 20.0, dof_lo: float = 1e4, dof_hi: float = 5e6,
                  steps_lo: int = 10, steps_hi: int = 500):
    """Poisson arrivals (mean `rate` per second) of n requests: (arrival s, case, steps, 'fp64'|'fp32')."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        case = request_case(seed * 100003 + i, dof_lo, dof_hi)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        prec = "fp64" if rng.uniform() < 0.5 else "fp32"
        out.append((t, case, steps, prec))
    return out


CONFIGS = {
    "bubble2d": bubble2d,
    "hill2d": hill2d,
    "hill3d": hill3d,
    "hill3d_big": hill3d_big,
    "bell3d_nc": lambda seed=0, **kw: bell3d(seed, refined=True, **kw),
    "bell3d_uniform": lambda seed=0, **kw: bell3d(seed, refined=False, **kw),
}


def make_case(name: str, seed: int = 0, **kw) -> Case:
    return CONFIGS[name](seed, **kw)
