"""Seeded synthetic inputs for the partitioned bidomain step.

This module builds the *inputs* of a simulation and nothing else: node
coordinates, element connectivity, per-element fibre directions, stimulus node
sets, seeded perturbations of an initial state and the arrival stream of the
serving workload.  It holds none of the method's arithmetic (no assembly, no
ionic model, no time stepping), so that the FP64 oracle and the CUDA path can
both be fed from it without sharing any computation.

Workload shapes follow the paper's experiments (Sec. 4): structured P1 meshes
of the unit square / square sheets (Sec. 4.1-4.2; the paper uses Q1 quads of
the same node grid), a 3-D slab with transmural fibre rotation (Sec. 4.4) and
S1-S2 stimulation protocols (Sec. 4.3).  All randomness uses numpy's PCG64 with
an explicit seed.

Units throughout: cm, ms, mV, mS/cm, uA/cm^2, uF/cm^2, 1/cm.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------


def rect_grid(nx: int, ny: int, lx: float, ly: float) -> Tuple[np.ndarray, np.ndarray]:
    """Structured P1 triangle mesh of [0,lx]x[0,ly] with nx x ny nodes.

    Node (i, j) (i along x, j along y) has index j*nx + i.  Every grid cell is
    split along its (i,j)->(i+1,j+1) diagonal into two counter-clockwise
    triangles.  Returns (xyz[N,2] float64, tris[E,3] int32).
    """
    if nx < 2 or ny < 2:
        raise ValueError("rect_grid needs at least 2 nodes per direction")
    X, Y = np.meshgrid(np.linspace(0.0, lx, nx), np.linspace(0.0, ly, ny), indexing="xy")
    xyz = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    a = j * nx + i
    b = j * nx + i + 1
    c = (j + 1) * nx + i + 1
    d = (j + 1) * nx + i
    tris = np.empty((2 * len(a), 3), dtype=np.int32)
    tris[0::2] = np.stack([a, b, c], axis=1)
    tris[1::2] = np.stack([a, c, d], axis=1)
    return xyz, tris


def square_grid(n: int, length: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """n x n node P1 triangle mesh of [0,L]^2 (see rect_grid)."""
    return rect_grid(n, n, length, length)


def lattice_tets(xs: np.ndarray, ys: np.ndarray, zs: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Tensor-product lattice of the coordinate vectors xs, ys, zs split into
    P1 tetrahedra.  Node (i,j,k) has index (k*ny + j)*nx + i.  Every
    hexahedron is split into the six Kuhn tetrahedra that share its
    (0,0,0)->(1,1,1) diagonal, so the mesh is conforming."""
    nx, ny, nz = len(xs), len(ys), len(zs)
    if min(nx, ny, nz) < 2:
        raise ValueError("a lattice needs at least 2 nodes per direction")
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    k, j, i = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1),
                          indexing="ij")
    i = i.ravel().astype(np.int64)
    j = j.ravel().astype(np.int64)
    k = k.ravel().astype(np.int64)

    def node(di, dj, dk):
        return ((k + dk) * ny + (j + dj)) * nx + (i + di)

    v000 = node(0, 0, 0)
    v111 = node(1, 1, 1)
    # the six monotone lattice paths from (0,0,0) to (1,1,1)
    paths = [((1, 0, 0), (1, 1, 0)), ((1, 0, 0), (1, 0, 1)),
             ((0, 1, 0), (1, 1, 0)), ((0, 1, 0), (0, 1, 1)),
             ((0, 0, 1), (1, 0, 1)), ((0, 0, 1), (0, 1, 1))]
    tets = []
    for p1, p2 in paths:
        tets.append(np.stack([v000, node(*p1), node(*p2), v111], axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return xyz, tets


def slab_grid(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float
              ) -> Tuple[np.ndarray, np.ndarray]:
    """Structured P1 tetrahedral mesh of [0,lx]x[0,ly]x[0,lz] with
    nx x ny x nz nodes (see lattice_tets).  Returns (xyz[N,3], tets[E,4])."""
    return lattice_tets(np.linspace(0.0, lx, nx), np.linspace(0.0, ly, ny), np.linspace(0.0, lz, nz))


def graded_axis(lo: float, hi: float, h: float, margin: float, grade: float) -> np.ndarray:
    """Coordinates of [lo - margin, hi + margin]: spacing h on [lo, hi'] (hi'
    = lo + h*ceil((hi-lo)/h)), cells growing by the factor `grade` across each
    margin (rescaled to fill it exactly)."""
    n = int(np.ceil((hi - lo) / h - 1e-9))
    core = lo + h * np.arange(n + 1)
    cells = []
    d, tot = h, 0.0
    while tot < margin - 1e-12:
        d *= grade
        cells.append(d)
        tot += d
    cells = np.array(cells) * (margin / tot) if cells else np.zeros(0)
    left = core[0] - np.cumsum(cells)[::-1]
    right = core[-1] + np.cumsum(cells)
    return np.concatenate([left, core, right])


# ---------------------------------------------------------------------------
# fibres, stimulus sets, initial perturbations
# ---------------------------------------------------------------------------


def fibers_along_x(n_elems: int, dim: int) -> np.ndarray:
    """Unit fibre direction e_x for every element, shape [E, dim]."""
    f = np.zeros((n_elems, dim), dtype=np.float64)
    f[:, 0] = 1.0
    return f


def fibers_transmural(xyz: np.ndarray, elems: np.ndarray, z0: float, z1: float,
                      theta0_deg: float, theta1_deg: float) -> np.ndarray:
    """Fibre direction (cos t, sin t, 0) per tetrahedron, where the angle t
    varies linearly from theta0 at z=z0 to theta1 at z=z1, evaluated at the
    element centroid's z (slab workload of Sec. 4.4)."""
    zc = xyz[elems, 2].mean(axis=1)
    s = np.clip((zc - z0) / (z1 - z0), 0.0, 1.0)
    t = np.deg2rad(theta0_deg + (theta1_deg - theta0_deg) * s)
    f = np.zeros((len(elems), 3), dtype=np.float64)
    f[:, 0] = np.cos(t)
    f[:, 1] = np.sin(t)
    return f


def nodes_x_below(xyz: np.ndarray, x_max: float) -> np.ndarray:
    """uint8 node mask of the planar strip x < x_max (strict)."""
    return (xyz[:, 0] < x_max).astype(np.uint8)


def nodes_in_box(xyz: np.ndarray, lo: Sequence[float], hi: Sequence[float]) -> np.ndarray:
    """uint8 node mask of the closed box lo <= x <= hi (componentwise)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = len(lo)
    m = np.all((xyz[:, :d] >= lo) & (xyz[:, :d] <= hi), axis=1)
    return m.astype(np.uint8)


def perturb_rows(X: np.ndarray, rows: Sequence[int], frac: float, seed: int,
                 clip01: bool = True) -> np.ndarray:
    """Multiply the given state rows of a node-major SoA state X[ns, N] by
    (1 + U(-frac, frac)), drawn with numpy PCG64(seed) in row-then-node
    order, optionally clipping to [0, 1] (gating variables)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = np.array(X, dtype=np.float64, copy=True)
    for r in rows:
        Y[r] = Y[r] * (1.0 + rng.uniform(-frac, frac, size=Y.shape[1]))
        if clip01:
            np.clip(Y[r], 0.0, 1.0, out=Y[r])
    return Y


# ---------------------------------------------------------------------------
# workload descriptions
# ---------------------------------------------------------------------------

LR91 = 0            # Luo-Rudy 1991, original parameters
LR91_PAPER_MOD = 1  # LR91 with G_si=0.02, G_Na=4.0, G_K=0.423 (Sec. 4)
TP06_EPI = 2        # ten Tusscher-Panfilov 2006, epicardial parameters

N_STATES = {LR91: 8, LR91_PAPER_MOD: 8, TP06_EPI: 19}


@dataclasses.dataclass
class Stimulus:
    mask: np.ndarray        # uint8 per node
    t_on: float             # ms
    duration: float         # ms
    amplitude: float        # uA/cm^2 (membrane current density, depolarising)


def tissue_first(xyz: np.ndarray, elems: np.ndarray, elem_bath: np.ndarray):
    """Renumber the nodes so that the nodes of tissue elements come first
    (each group in its original order).  Returns (xyz, elems, new_of_old)."""
    tis = np.zeros(len(xyz), dtype=bool)
    tis[elems[np.asarray(elem_bath) == 0].ravel()] = True
    order = np.concatenate([np.nonzero(tis)[0], np.nonzero(~tis)[0]])
    new_of_old = np.empty(len(xyz), dtype=np.int64)
    new_of_old[order] = np.arange(len(xyz))
    return xyz[order].copy(), new_of_old[elems].astype(np.int32), new_of_old


@dataclasses.dataclass
class Workload:
    name: str
    xyz: np.ndarray
    elems: np.ndarray
    fibers: np.ndarray
    sigma: Tuple[float, float, float, float]   # (s_il, s_it, s_el, s_et) mS/cm
    chi: float
    cm: float
    model: int
    stimuli: List[Stimulus]
    dt: float
    n_steps: int
    n_sdc_nodes: int = 3
    n_sweeps: int = 2
    pin_node: int = 0
    cg_tol: float = 1e-10
    initial: Optional[np.ndarray] = None     # X[ns, N] or None => model rest
    elem_bath: Optional[np.ndarray] = None   # per element, 1 = bath (tissue nodes numbered first)
    sbath: float = 0.0                       # bath conductivity, mS/cm

    @property
    def n_tissue(self) -> int:
        if self.elem_bath is None:
            return self.n_nodes
        tis = np.zeros(self.n_nodes, dtype=bool)
        tis[self.elems[self.elem_bath == 0].ravel()] = True
        return int(tis.sum())

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def dim(self) -> int:
        return int(self.xyz.shape[1])


CONFIG0_SIGMA = (3.0, 0.31, 2.0, 1.35)
STIM_AMP = 80.0


def sheet(n: int, length: float, model: int, dt: float, n_steps: int,
          sigma=CONFIG0_SIGMA, strip: float = 0.1, s2: Optional[Tuple[float, float]] = None,
          name: str = "sheet", **kw) -> Workload:
    """2-D square sheet with fibres along x and a left-edge S1 strip at t=0
    (1 ms, 80 uA/cm^2).  s2=(t_on, side) adds an S2 on the corner square
    [0,side]^2."""
    xyz, tris = square_grid(n, length)
    stims = [Stimulus(nodes_x_below(xyz, strip), 0.0, 1.0, STIM_AMP)]
    if s2 is not None:
        stims.append(Stimulus(nodes_in_box(xyz, (0.0, 0.0), (s2[1], s2[1])), s2[0], 1.0, STIM_AMP))
    return Workload(name=name, xyz=xyz, elems=tris, fibers=fibers_along_x(len(tris), 2),
                    sigma=tuple(sigma), chi=2000.0, cm=1.0, model=model, stimuli=stims,
                    dt=dt, n_steps=n_steps, **kw)


BATH_SIGMA = 20.0      # mS/cm, bath conductivity of the bidomain-bath runs


def bath_sheet(n_cells: int, lo: float, hi: float, t_lo: float, t_hi: float, model: int,
               dt: float, n_steps: int, sigma=CONFIG0_SIGMA, sbath: float = BATH_SIGMA,
               strip: float = 0.1, s1_amp: float = 100.0, s1_dur: float = 2.0,
               s2: Optional[Tuple[float, float, float]] = None, name: str = "bath_sheet",
               **kw) -> Workload:
    """Bidomain-bath square (Sec. 4): the domain [lo, hi]^2 split into
    n_cells^2 squares (two triangles each); the elements whose centroid lies
    in the tissue square [t_lo, t_hi]^2 are tissue, the rest bath.  Tissue
    nodes are numbered first, fibres run along x.  Stimuli follow the reentry
    protocol of Sec. 4: S1 (s1_amp uA/cm^2, s1_dur ms, t = 0) on the tissue
    strip t_lo <= y < t_lo + strip along the bottom edge; s2 = (t_on, x_len,
    y_len) adds an S2 on [t_lo, t_lo + x_len] x [t_lo, t_lo + y_len].  u is
    pinned at the domain corner (lo, lo), a bath node."""
    L = hi - lo
    xyz, tris = square_grid(n_cells + 1, L)
    xyz = xyz + lo
    cen = xyz[tris].mean(axis=1)
    inside = np.all((cen > t_lo) & (cen < t_hi), axis=1)
    bath = (~inside).astype(np.uint8)
    corner = int(np.argmin(np.abs(xyz[:, 0] - lo) + np.abs(xyz[:, 1] - lo)))
    xyz, tris, new_of_old = tissue_first(xyz, tris, bath)
    nt = int(np.count_nonzero(np.bincount(tris[bath == 0].ravel(), minlength=len(xyz))))
    eps = 1e-9 * L
    tissue = np.zeros(len(xyz), dtype=bool)
    tissue[:nt] = True
    x, y = xyz[:, 0], xyz[:, 1]
    m1 = tissue & (y < t_lo + strip - eps)
    stims = [Stimulus(m1.astype(np.uint8), 0.0, s1_dur, s1_amp)]
    if s2 is not None:
        m2 = tissue & (x <= t_lo + s2[1] + eps) & (y <= t_lo + s2[2] + eps)
        stims.append(Stimulus(m2.astype(np.uint8), s2[0], s1_dur, s1_amp))
    return Workload(name=name, xyz=xyz, elems=tris, fibers=fibers_along_x(len(tris), 2),
                    sigma=tuple(sigma), chi=2000.0, cm=1.0, model=model, stimuli=stims,
                    dt=dt, n_steps=n_steps, pin_node=int(new_of_old[corner]), elem_bath=bath,
                    sbath=sbath, **kw)


def bath_paper_2d(n_steps: int = 12000, dt: float = 0.05) -> Workload:
    """The bidomain-bath run of Sec. 4: domain [-1, 7]^2 on 800 x 800 cells
    (801^2 = 641,601 nodes), tissue [0, 6]^2 (601^2 = 361,201 nodes), LR91,
    reentry protocol (S1 bottom edge at 0 ms, S2 on [0, 1] x [0, 3] at
    120 ms), 600 ms."""
    return bath_sheet(800, -1.0, 7.0, 0.0, 6.0, LR91, dt, n_steps, s2=(120.0, 1.0, 3.0),
                      name="lr91_bath_801x801")


# truncated prolate LV shell in a bath box (bidomain-bath, 3-D)
LV_ENDO = (2.5, 2.5, 5.0)     # endocardial semi-axes, cm
LV_WALL = 1.0                 # wall thickness, cm
LV_ZCUT = 2.5                 # base plane z = +2.5 cm


def _lv_radii(xyz: np.ndarray):
    a, b, c = LV_ENDO
    ri = np.sqrt((xyz[:, 0] / a) ** 2 + (xyz[:, 1] / b) ** 2 + (xyz[:, 2] / c) ** 2)
    t = LV_WALL
    ro = np.sqrt((xyz[:, 0] / (a + t)) ** 2 + (xyz[:, 1] / (b + t)) ** 2 + (xyz[:, 2] / (c + t)) ** 2)
    return ri, ro


def lv_shell_fibers(cen: np.ndarray, theta0: float = -60.0, theta1: float = 60.0) -> np.ndarray:
    """Helical fibres: in the tangent plane of the ellipsoidal level set
    through the centroid, f = cos(t) e_circ + sin(t) e_long with t rising
    linearly from theta0 (endocardium) to theta1 (epicardium) in the
    transmural coordinate e = (r_i - 1)/(r_i - r_o), r_i, r_o the scaled
    radii of the endo- and epicardial ellipsoids."""
    a, b, c = LV_ENDO
    ri, ro = _lv_radii(cen)
    e = np.clip((ri - 1.0) / np.maximum(ri - ro, 1e-12), 0.0, 1.0)
    t = np.deg2rad(theta0 + (theta1 - theta0) * e)
    n = np.stack([cen[:, 0] / a ** 2, cen[:, 1] / b ** 2, cen[:, 2] / c ** 2], axis=1)
    n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-300)
    circ = np.stack([-cen[:, 1], cen[:, 0], np.zeros(len(cen))], axis=1)
    cn = np.linalg.norm(circ, axis=1, keepdims=True)
    circ = np.where(cn > 1e-9, circ / np.maximum(cn, 1e-300), np.array([[1.0, 0.0, 0.0]]))
    lon = np.cross(n, circ)
    lon /= np.maximum(np.linalg.norm(lon, axis=1, keepdims=True), 1e-300)
    f = np.cos(t)[:, None] * circ + np.sin(t)[:, None] * lon
    return f / np.linalg.norm(f, axis=1, keepdims=True)


def lv_shell_bath(h: float = 0.04, margin: float = 1.0, grade: float = 1.3, jitter: float = 0.125,
                  seed: int = 3, model: int = TP06_EPI, dt: float = 0.025, n_steps: int = 4000,
                  sbath: float = BATH_SIGMA, s2_ms: float = 60.0, name: Optional[str] = None) -> Workload:
    """Bidomain-bath LV model: a truncated prolate-ellipsoid shell
    (endocardial semi-axes 2.5/2.5/5.0 cm, wall 1.0 cm, cut at z = +2.5 cm)
    with helical -60..+60 deg fibres, embedded in a box bath extending
    `margin` beyond it on every side.

    Mesh: a tensor lattice of spacing h over the shell's bounding box and
    geometrically growing cells across the margins (a coarser bath), every
    interior node moved by a seeded uniform jitter of at most jitter*h_local
    per axis (numpy PCG64(seed)), hexahedra split into Kuhn tetrahedra;
    elements whose centroid lies in the wall (r_i >= 1, r_o <= 1, z <= cut)
    are tissue, the rest bath (the cavity included).  Tissue nodes are
    numbered first.  Stimuli: apical pacing on the tissue nodes within
    0.3 cm of (0, 0, -(c + wall/2)) at t = 0 (2 ms, 100 uA/cm^2); an S2 on
    the quadrant x > 0, y > 0, z > -2 of the wall at s2_ms."""
    a, b, c = LV_ENDO
    t = LV_WALL
    xs = graded_axis(-(a + t), a + t, h, margin, grade)
    ys = graded_axis(-(b + t), b + t, h, margin, grade)
    zs = graded_axis(-(c + t), LV_ZCUT, h, margin, grade)
    xyz, tets = lattice_tets(xs, ys, zs)
    rng = np.random.Generator(np.random.PCG64(seed))
    for d, ax in enumerate((xs, ys, zs)):
        sp = np.minimum(np.diff(ax)[:-1], np.diff(ax)[1:]) if len(ax) > 2 else np.zeros(0)
        loc = np.concatenate([[0.0], sp, [0.0]])          # boundary nodes stay on the box faces
        shape = [1, 1, 1]
        shape[2 - d] = len(ax)
        amp = np.broadcast_to(loc.reshape(shape), (len(zs), len(ys), len(xs))).ravel()
        xyz[:, d] += jitter * amp * rng.uniform(-1.0, 1.0, size=len(xyz))
    cen = np.zeros((len(tets), 3))
    for q in range(4):                                   # centroids without a [E, 4, 3] temporary
        cen += xyz[tets[:, q]]
    cen *= 0.25
    ri, ro = _lv_radii(cen)
    tissue = (ri >= 1.0) & (ro <= 1.0) & (cen[:, 2] <= LV_ZCUT)
    bath = (~tissue).astype(np.uint8)
    fib = np.zeros((len(tets), 3))
    fib[:, 0] = 1.0                                      # bath elements: unused
    fib[tissue] = lv_shell_fibers(cen[tissue])
    del cen, ri, ro
    corner = 0                                           # (x_min, y_min, z_min), a bath node
    xyz, tets, new_of_old = tissue_first(xyz, tets, bath)
    nt = int(np.count_nonzero(np.bincount(tets[bath == 0].ravel(), minlength=len(xyz))))
    tis = np.zeros(len(xyz), dtype=bool)
    tis[:nt] = True
    apex = np.array([0.0, 0.0, -(c + 0.5 * t)])
    s1 = tis & (np.linalg.norm(xyz - apex, axis=1) <= 0.3)
    s2 = tis & (xyz[:, 0] > 0) & (xyz[:, 1] > 0) & (xyz[:, 2] > -2.0)
    stims = [Stimulus(s1.astype(np.uint8), 0.0, 2.0, 100.0),
             Stimulus(s2.astype(np.uint8), s2_ms, 2.0, 100.0)]
    return Workload(name=name or f"tp06_lv_shell_bath_h{h:g}", xyz=xyz, elems=tets, fibers=fib,
                    sigma=tuple(CONFIG0_SIGMA), chi=2000.0, cm=1.0, model=model, stimuli=stims, dt=dt,
                    n_steps=n_steps, pin_node=int(new_of_old[corner]), elem_bath=bath, sbath=sbath)


def config0() -> Workload:
    """LR91 on the unit square, 65x65 nodes, 10 ms at dt = 0.02 ms, FP64."""
    return sheet(65, 1.0, LR91, 0.02, 500, name="lr91_sheet_65x65", cg_tol=1e-10)


def config1() -> Workload:
    """TP06-epi on a 2.5 cm sheet, 257x257 nodes, S1 left edge, S2 corner
    quadrant at 310 ms; 600 ms at dt = 0.02 ms."""
    return sheet(257, 2.5, TP06_EPI, 0.02, 30000, s2=(310.0, 1.25),
                 name="tp06_sheet_257x257")


def config2(nx: int = 201, ny: int = 201, nz: int = 51, seed: int = 2,
            rest: Optional[np.ndarray] = None, gate_rows: Sequence[int] = ()) -> Workload:
    """TP06 in a 2x2x0.5 cm slab with -60..+60 deg transmural fibre rotation,
    seeded +-2% gate perturbation around rest, S1 plane x<0.1 at 0 ms and S2
    on the half-slab y<1 at 150 ms; 200 ms at dt = 0.025 ms."""
    xyz, tets = slab_grid(nx, ny, nz, 2.0, 2.0, 0.5)
    fib = fibers_transmural(xyz, tets, 0.0, 0.5, -60.0, 60.0)
    stims = [Stimulus(nodes_x_below(xyz, 0.1), 0.0, 1.0, STIM_AMP),
             Stimulus((xyz[:, 1] < 1.0).astype(np.uint8), 150.0, 1.0, STIM_AMP)]
    init = None
    if rest is not None:
        X = np.repeat(np.asarray(rest, dtype=np.float64)[:, None], len(xyz), axis=1)
        init = perturb_rows(X, gate_rows, 0.02, seed)
    return Workload(name=f"tp06_slab_{nx}x{ny}x{nz}", xyz=xyz, elems=tets, fibers=fib,
                    sigma=CONFIG0_SIGMA, chi=2000.0, cm=1.0, model=TP06_EPI,
                    stimuli=stims, dt=0.025, n_steps=8000, initial=init)


# ---------------------------------------------------------------------------
# serving workload: a seeded stream of independent sheet simulations
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    side: int
    model: int
    sigma: Tuple[float, float, float, float]
    strip_x: float
    s2_time: float
    t_end: float = 400.0
    dt: float = 0.02


def request_stream(n_requests: int = 512, rate_per_s: float = 40.0, seed: int = 4,
                   sides: Sequence[int] = (33, 65, 129, 257, 513),
                   t_end: float = 400.0) -> List[Request]:
    """Poisson arrivals of independent square-sheet requests: side uniform
    over `sides`, LR91/TP06 50/50, each conductivity jittered by U(-20%, 20%),
    S1 strip whose left edge x0/L is U(0, 0.5) (width 0.1 L), S2 time
    U(250, 350) ms on the quadrant opposite the strip."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        side = int(sides[rng.integers(0, len(sides))])
        model = LR91 if rng.uniform() < 0.5 else TP06_EPI
        sig = tuple(float(s * (1.0 + rng.uniform(-0.2, 0.2))) for s in CONFIG0_SIGMA)
        strip = float(rng.uniform(0.0, 0.5))
        s2 = float(rng.uniform(250.0, 350.0))
        out.append(Request(r, t, side, model, sig, strip, s2, t_end=t_end))
    return out


def request_workload(req: Request, length: float = 1.0, n_steps: Optional[int] = None) -> Workload:
    """Materialise one serving request as a Workload on [0,L]^2: S1 on the
    strip [x0, x0 + 0.1 L) at t=0, S2 on the upper-right quadrant at s2_time."""
    xyz, tris = square_grid(req.side, length)
    x0 = req.strip_x * length
    s1 = ((xyz[:, 0] >= x0) & (xyz[:, 0] < x0 + 0.1 * length)).astype(np.uint8)
    s2 = nodes_in_box(xyz, (0.5 * length, 0.5 * length), (length, length))
    steps = n_steps if n_steps is not None else int(round(req.t_end / req.dt))
    return Workload(name=f"req{req.rid}", xyz=xyz, elems=tris,
                    fibers=fibers_along_x(len(tris), 2), sigma=req.sigma, chi=2000.0,
                    cm=1.0, model=req.model,
                    stimuli=[Stimulus(s1, 0.0, 1.0, STIM_AMP),
                             Stimulus(s2, req.s2_time, 1.0, STIM_AMP)],
                    dt=req.dt, n_steps=steps)
