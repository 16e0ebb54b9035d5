"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver.  It produces plain data only:
structured meshes, element partitions, Dirichlet and traction data, and the
per-cell coefficient fields k and f.  Every random number comes from the
counter-free splitmix64 generator (Steele, Lea, Flood 2014), so every workload
can be re-created bit for bit from its seed on any machine.

Workloads (node ids are lexicographic, x fastest; cell (i, j) has id j*n + i):

* ``diffusion_c1``  64x64 P1 cells, 4x4 regular boxes, overlap 1, homogeneous
  Dirichlet data on the whole boundary, k = f = 1 (nonlinear diffusion, Eq. 1).
* ``diffusion_c2``  1024x1024 P1 cells, 32 bands x 32 bricks, band heights and
  per-band brick widths drawn as nominal * (1 + 0.3 (U - 0.5)), overlap 2.
* ``neohooke_c3``   512x512 Q1 cells, 2 dofs per node, left edge clamped,
  vertical dead-load traction on the right edge (Eq. 2), 16x16 bricks, overlap 2.
* ``diffusion_c4``  512x512 P1 cells, log-normal k (Gaussian covariance,
  correlation length 1/16, sigma 1), f constant per instance drawn in [0.5, 2].
* ``neohooke_c5``   2048x2048 Q1 cells, 64x64 bricks, otherwise as c3.
* ``beam_problem``  the beam of Section 1: 5 x 1 Neo-Hooke rectangle clamped at both ends under
  a volume force f_x, laid out along y, m x 5m Q1 cells, px x py bricks.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MASK64 = (1 << 64) - 1

P1_TRI = 1
Q1_QUAD = 2
LAW_DIFFUSION = 1
LAW_NEOHOOKE = 2
LAMBDA_PRINTED = 0        # Eq. 2 with the Lame lambda as printed
LAMBDA_PLANE_STRESS = 1   # Eq. 2 with the plane-stress reduction of lambda


class SplitMix64:
    """The splitmix64 sequence: draw k (k = 1, 2, ...) mixes state0 + k * 0x9E3779B97F4A7C15."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.seed = seed & MASK64
        self.count = 0

    def next_u64(self, count: int) -> np.ndarray:
        k = np.arange(self.count + 1, self.count + count + 1, dtype=np.uint64)
        self.count += count
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + k * np.uint64(self.GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int) -> SplitMix64:
    return SplitMix64(seed)


def uniform01(gen: SplitMix64, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1): the top 53 bits of each splitmix64 draw times 2^-53."""
    return (gen.next_u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------------------------

def structured_mesh(n: int, elem_type: int, lx: float = 1.0, ly: float = 1.0):
    """Uniform n x n cell mesh of [0, lx] x [0, ly] (see structured_rect_mesh)."""
    return structured_rect_mesh(n, n, elem_type, lx, ly)


def structured_rect_mesh(nx: int, ny: int, elem_type: int, lx: float = 1.0, ly: float = 1.0):
    """Uniform nx x ny cell mesh of [0, lx] x [0, ly]; node (i, j) has id j (nx + 1) + i, cell (i, j)
    has id j nx + i.

    P1: every cell (i, j) is cut along its SW-NE diagonal into the triangles
    {(i,j),(i+1,j),(i+1,j+1)} (element 2c) and {(i,j),(i+1,j+1),(i,j+1)} (element 2c+1).
    Q1: the cell itself, nodes counter-clockwise from its SW corner.
    Returns (xy [n_nodes, 2] float64, conn [n_elems, nen] int32).
    """
    m = nx + 1
    jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(m), indexing="ij")
    xy = np.stack([ii.ravel() * (lx / nx), jj.ravel() * (ly / ny)], axis=1).astype(np.float64)
    cj, ci = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ci = ci.ravel()
    cj = cj.ravel()
    sw = cj * m + ci
    se = sw + 1
    ne = sw + m + 1
    nw = sw + m
    if elem_type == P1_TRI:
        conn = np.empty((2 * nx * ny, 3), dtype=np.int32)
        conn[0::2] = np.stack([sw, se, ne], axis=1)
        conn[1::2] = np.stack([sw, ne, nw], axis=1)
    elif elem_type == Q1_QUAD:
        conn = np.stack([sw, se, ne, nw], axis=1).astype(np.int32)
    else:
        raise ValueError("unknown element type")
    return xy, conn


def elems_per_cell(elem_type: int) -> int:
    return 2 if elem_type == P1_TRI else 1


def cell_to_elem_partition(cell_to_sub: np.ndarray, elem_type: int) -> np.ndarray:
    """Both triangles of a cell belong to the cell's subdomain."""
    return np.repeat(cell_to_sub.astype(np.int32), elems_per_cell(elem_type))


# ----------------------------------------------------------------------------------------------
# partitions (non-overlapping, by cells)
# ----------------------------------------------------------------------------------------------

def box_partition(n: int, nbx: int, nby: int) -> np.ndarray:
    """Regular nbx x nby boxes of cells; subdomain id = by * nbx + bx."""
    cx = np.minimum((np.arange(n) * nbx) // n, nbx - 1)
    cy = np.minimum((np.arange(n) * nby) // n, nby - 1)
    return (cy[:, None] * nbx + cx[None, :]).ravel().astype(np.int32)


def _cuts(n: int, sizes: np.ndarray) -> np.ndarray:
    """Integer cut positions floor(n * S_k / S_total + 0.5) of the prefix sums S_k."""
    s = np.concatenate([[0.0], np.cumsum(sizes)])
    c = np.floor(n * s / s[-1] + 0.5).astype(np.int64)
    c[0], c[-1] = 0, n
    if np.any(np.diff(c) <= 0):
        raise ValueError("partition produced an empty brick")
    return c


def brick_partition(n: int, n_bands: int, per_band: int, seed: int, spread: float = 0.3) -> np.ndarray:
    """Seeded uneven brick partition of an n x n cell grid (see rect_brick_partition)."""
    return rect_brick_partition(n, n, n_bands, per_band, seed, spread)


def rect_brick_partition(nx: int, ny: int, n_bands: int, per_band: int, seed: int,
                         spread: float = 0.3) -> np.ndarray:
    """Seeded uneven brick partition of an nx x ny cell grid: n_bands bands along y, per_band
    bricks along x in every band.

    Band heights h_j and, independently in every band, brick widths w_{j,k} are
    nominal * (1 + spread * (U - 0.5)) with U uniform in [0, 1) (each side varies by
    +-spread/2, each area by about +-spread).  Subdomain id = band * per_band + k.
    """
    gen = splitmix64(seed)
    heights = 1.0 + spread * (uniform01(gen, n_bands) - 0.5)
    ycut = _cuts(ny, heights)
    cell_to_sub = np.empty((ny, nx), dtype=np.int32)
    for j in range(n_bands):
        widths = 1.0 + spread * (uniform01(gen, per_band) - 0.5)
        xcut = _cuts(nx, widths)
        for k in range(per_band):
            cell_to_sub[ycut[j]:ycut[j + 1], xcut[k]:xcut[k + 1]] = j * per_band + k
    return cell_to_sub.ravel()


# ----------------------------------------------------------------------------------------------
# boundary data and coefficient fields
# ----------------------------------------------------------------------------------------------

def boundary_nodes(n: int) -> np.ndarray:
    m = n + 1
    j, i = np.divmod(np.arange(m * m), m)
    return np.nonzero((i == 0) | (i == n) | (j == 0) | (j == n))[0].astype(np.int64)


def left_edge_nodes(n: int) -> np.ndarray:
    return (np.arange(n + 1) * (n + 1)).astype(np.int64)


def right_edge_segments(n: int) -> np.ndarray:
    """The n boundary segments of the edge x = lx, as node pairs (bottom to top)."""
    m = n + 1
    nodes = np.arange(n + 1) * m + n
    return np.stack([nodes[:-1], nodes[1:]], axis=1).astype(np.int32)


def gaussian_random_field(n: int, seed: int, ell: float, sigma: float = 1.0) -> np.ndarray:
    """Stationary Gaussian field g on the n x n cell centres of the unit square.

    Spectral synthesis on a periodic 2n x 2n grid (period 2 in each direction, so the
    kept n x n corner sees no wrap-around correlation): complex white noise from
    splitmix64 + Box-Muller, filtered by the square root of the spectral density of the
    covariance exp(-r^2 / (2 ell^2)), real part taken, scaled to unit sample variance
    and then by sigma.  Returns g for cells in id order.
    """
    m = 2 * n
    gen = splitmix64(seed)
    u = uniform01(gen, 2 * m * m).reshape(2, m, m)
    u1 = np.maximum(u[0], 1e-300)
    rad = np.sqrt(-2.0 * np.log(u1))
    noise = rad * np.cos(2.0 * np.pi * u[1]) + 1j * rad * np.sin(2.0 * np.pi * u[1])
    h = 1.0 / n
    kx = np.fft.fftfreq(m, d=h) * 2.0 * np.pi
    kk = kx[:, None] ** 2 + kx[None, :] ** 2
    spec = np.exp(-0.5 * ell * ell * kk)  # spectral density of a Gaussian covariance (up to a constant)
    field = np.fft.ifft2(noise * np.sqrt(spec)).real[:n, :n]
    field = (field - field.mean()) / field.std()
    return (sigma * field).ravel()


# ----------------------------------------------------------------------------------------------
# complete problem descriptions
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Everything that defines one nonlinear problem F(u) = 0 plus its decomposition."""
    name: str
    n: int
    elem_type: int
    law: int
    xy: np.ndarray
    conn: np.ndarray
    dirichlet_nodes: np.ndarray          # every dof of these nodes is fixed to 0
    elem_to_sub: np.ndarray
    n_sub: int
    overlap: int
    k_elem: Optional[np.ndarray] = None  # diffusion coefficient per element (None = 1)
    f_elem: Optional[np.ndarray] = None  # source per element (None = 1)
    traction_edges: Optional[np.ndarray] = None   # [n_edges, 2] node pairs
    traction: Optional[np.ndarray] = None         # [n_edges, 2] force per unit length at load factor 1
    f_vol: Optional[np.ndarray] = None            # [n_elems, 2] Neo-Hooke volume force per unit area, load factor 1
    young: float = 210.0
    poisson: float = 0.3
    lambda_mode: int = LAMBDA_PRINTED
    load_steps: int = 1

    @property
    def ndof(self) -> int:
        return 2 if self.law == LAW_NEOHOOKE else 1

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    def dirichlet_dofs(self) -> np.ndarray:
        d = self.ndof
        return (self.dirichlet_nodes[:, None] * d + np.arange(d)[None, :]).ravel().astype(np.int64)


def diffusion_problem(n: int, cell_to_sub: np.ndarray, n_sub: int, overlap: int, name: str = "diffusion",
                      k_cell: Optional[np.ndarray] = None, f_cell: Optional[np.ndarray] = None) -> Problem:
    xy, conn = structured_mesh(n, P1_TRI)
    rep = elems_per_cell(P1_TRI)
    return Problem(name=name, n=n, elem_type=P1_TRI, law=LAW_DIFFUSION, xy=xy, conn=conn,
                   dirichlet_nodes=boundary_nodes(n), elem_to_sub=cell_to_elem_partition(cell_to_sub, P1_TRI),
                   n_sub=n_sub, overlap=overlap,
                   k_elem=None if k_cell is None else np.repeat(k_cell, rep),
                   f_elem=None if f_cell is None else np.repeat(f_cell, rep))


def neohooke_problem(n: int, cell_to_sub: np.ndarray, n_sub: int, overlap: int, traction_max: float,
                     load_steps: int = 5, name: str = "neohooke") -> Problem:
    xy, conn = structured_mesh(n, Q1_QUAD)
    edges = right_edge_segments(n)
    t = np.zeros((edges.shape[0], 2))
    t[:, 1] = -traction_max
    return Problem(name=name, n=n, elem_type=Q1_QUAD, law=LAW_NEOHOOKE, xy=xy, conn=conn,
                   dirichlet_nodes=left_edge_nodes(n), elem_to_sub=cell_to_elem_partition(cell_to_sub, Q1_QUAD),
                   n_sub=n_sub, overlap=overlap, traction_edges=edges, traction=t, load_steps=load_steps)


PARTITION_SEED = 2410
NEOHOOKE_TRACTION_MAX = 8.0


def diffusion_c1() -> Problem:
    return diffusion_problem(64, box_partition(64, 4, 4), 16, 1, name="diffusion_c1_64x64_P1_4x4_boxes_overlap1")


def diffusion_c2(n: int = 1024, per_side: int = 32, seed: int = PARTITION_SEED) -> Problem:
    return diffusion_problem(n, brick_partition(n, per_side, per_side, seed), per_side * per_side, 2,
                             name=f"diffusion_c2_{n}x{n}_P1_{per_side * per_side}_bricks_overlap2")


def neohooke_c3(n: int = 512, per_side: int = 16, seed: int = PARTITION_SEED,
                traction_max: float = NEOHOOKE_TRACTION_MAX, load_steps: int = 5) -> Problem:
    return neohooke_problem(n, brick_partition(n, per_side, per_side, seed), per_side * per_side, 2,
                            traction_max, load_steps, name=f"neohooke_c3_{n}x{n}_Q1_{per_side * per_side}_bricks")


def c4_cell_coefficients(field_seed: int, n: int = 512):
    """Per-cell k (log-normal field, correlation length 1/16, sigma 1) and f (one constant per
    instance, uniform in [0.5, 2]) of the learned-guess workload."""
    g = gaussian_random_field(n, field_seed, ell=1.0 / 16.0, sigma=1.0)
    f = 0.5 + 1.5 * uniform01(splitmix64(field_seed ^ 0x5DEECE66D), 1)[0]
    return np.exp(g), np.full(n * n, f)


def c4_elem_coefficients(field_seed: int, n: int = 512):
    """The same per element (both triangles of a cell share the cell's values)."""
    k, f = c4_cell_coefficients(field_seed, n)
    rep = elems_per_cell(P1_TRI)
    return np.repeat(k, rep), np.repeat(f, rep)


def diffusion_c4(field_seed: int, n: int = 512, per_side: int = 16, seed: int = PARTITION_SEED) -> Problem:
    k, f = c4_cell_coefficients(field_seed, n)
    return diffusion_problem(n, brick_partition(n, per_side, per_side, seed), per_side * per_side, 2,
                             name=f"diffusion_c4_{n}x{n}_P1_lognormal_k_seed{field_seed}",
                             k_cell=k, f_cell=f)


def neohooke_c5(n: int = 2048, per_side: int = 64, seed: int = PARTITION_SEED) -> Problem:
    return neohooke_c3(n=n, per_side=per_side, seed=seed)


BEAM_LENGTH = 5.0


def beam_problem(m: int, px: int, py: int, f_x: float, overlap: int = 2, seed: int = PARTITION_SEED,
                 load_steps: int = 1) -> Problem:
    """The beam of Section 1 (Eq. 2): a 5 x 1 rectangle of Neo-Hooke material (E = 210, nu = 0.3),
    clamped (u = 0) at both ends, g_N = 0 elsewhere, under a volume force of size f_x across the
    beam (the paper's f_vol = (0, -f_x) with E in GPa and f_x in GN / m^3).

    The beam is laid out along y -- the paper's beam turned by 90 degrees, the force pointing
    along -x -- so that the lexicographic node numbering runs across its short side and the
    local and coarse band widths stay those of the subdomains' widths: m x 5m Q1 cells, clamped
    edges y = 0 and y = 5, px x py uneven bricks (py bands along the length).
    """
    nx, ny = m, int(round(BEAM_LENGTH * m))
    xy, conn = structured_rect_mesh(nx, ny, Q1_QUAD, 1.0, BEAM_LENGTH)
    j = np.arange(xy.shape[0]) // (nx + 1)
    clamped = np.nonzero((j == 0) | (j == ny))[0].astype(np.int64)
    cell_to_sub = rect_brick_partition(nx, ny, py, px, seed)
    f_vol = np.zeros((conn.shape[0], 2))
    f_vol[:, 0] = -f_x
    return Problem(name=f"beam_{nx}x{ny}_Q1_{px * py}_bricks_f{f_x:g}", n=nx, elem_type=Q1_QUAD, law=LAW_NEOHOOKE,
                   xy=xy, conn=conn, dirichlet_nodes=clamped,
                   elem_to_sub=cell_to_elem_partition(cell_to_sub, Q1_QUAD), n_sub=px * py, overlap=overlap,
                   f_vol=f_vol, load_steps=load_steps)
