"""Seeded synthetic inputs for the corrector-step solves.

This module only draws and lays out inputs: vertices and triangles of a
jittered triangular lattice, the Dirichlet side list, nodal (or cellular)
porosity and inverse-permeability fields, and right-hand sides.  It holds none
of the method's arithmetic (no circumcentres, transmissibilities, matrices or
solves).  Both the CPU oracle and the CUDA path are fed from here, so the two
sides always see the same arrays.

Input recipe (the paper's own meshes come from an unpublished in-house
generator, Sec. 4; these lattices stand in for them):

* Lattice of n x n vertices, unit spacing, vertex (i, j) at
  (i + (j mod 2)/2, j*sqrt(3)/2), id j*n + i.  Each row strip j holds 2(n-1)
  counter-clockwise triangles interleaved "up, down, up, down ...", triangle
  id j*2(n-1) + 2i + {0: up, 1: down}.  Up and down triangles only touch each
  other, so the parity of the id is a red/black colouring of the cells.
* Interior vertices are moved uniformly inside a disk of radius 0.05 (5% of
  the edge); boundary vertices stay put.  Every angle stays below 90 degrees,
  so the mesh is Delaunay and all circumcentre distances are positive (Sec. 3.1).
* Sides whose two vertices lie on the right column (i = n-1) are Dirichlet;
  all other boundary sides are no-flux.
* Porosity eps and the inverse permeability tensor (K^-1, stored xx, xy, yy)
  follow the workloads: a centred porous square (1/4 of the area, Test 1 of
  Sec. 4.1) with a tanh transition (Eq. 3), or a porous block in a channel
  (Test 5 geometry) filled with a random-Fourier porosity field; K from the
  Kozeny-Carman law, optionally anisotropic as K = R diag(k/beta, k) R^T
  (Eq. "aniso").
* Right-hand side b_e = A_e * N(0, 1) with A_e the triangle area.

Random numbers come from numpy.random.default_rng(seed) only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants of the workloads: kinematic viscosity of water
# (Sec. 4.1, Test 1) and the Test 1 coarse time step.
NU = 1.5e-5
DT = 0.225
# Kozeny-Carman grain diameter of the workloads.
KC_D = 1e-3

PER_VERTEX = 0
PER_CELL = 1


@dataclass
class Mesh:
    n: int                       # vertices per lattice side
    xy: np.ndarray               # float64 [nv, 2]
    tri: np.ndarray              # int32 [nt, 3], counter-clockwise
    dirichlet: np.ndarray        # int32 [nb], entries tri*3 + local side
    # local side j of triangle (v0, v1, v2) joins v[(j+1)%3] and v[(j+2)%3]

    @property
    def nv(self) -> int:
        return self.xy.shape[0]

    @property
    def nt(self) -> int:
        return self.tri.shape[0]

    @property
    def width(self) -> float:
        return float(self.n - 1)

    @property
    def height(self) -> float:
        return (self.n - 1) * math.sqrt(3.0) / 2.0


@dataclass
class Problem:
    mesh: Mesh
    eps: np.ndarray              # float64 [nv] or [nt]
    kinv: np.ndarray             # float64 [nv or nt, 3] (xx, xy, yy)
    field_loc: int
    nu: float = NU
    dt: float = DT
    meta: dict = field(default_factory=dict)


def lattice_vertices(n: int) -> np.ndarray:
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = i + 0.5 * (j % 2)
    y = j * (math.sqrt(3.0) / 2.0)
    return np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float64)


def lattice_triangles(n: int) -> np.ndarray:
    if n < 2:
        raise ValueError("lattice needs n >= 2")
    tris = np.empty((n - 1, n - 1, 2, 3), dtype=np.int64)
    i = np.arange(n - 1)
    for j in range(n - 1):
        b = j * n + i
        t = (j + 1) * n + i
        if j % 2 == 0:
            tris[j, :, 0] = np.stack([b, b + 1, t], axis=1)          # up
            tris[j, :, 1] = np.stack([t, b + 1, t + 1], axis=1)      # down
        else:
            tris[j, :, 0] = np.stack([b, b + 1, t + 1], axis=1)      # up
            tris[j, :, 1] = np.stack([t, b, t + 1], axis=1)          # down
    return tris.reshape(-1, 3).astype(np.int32)


def _boundary_vertex_mask(n: int) -> np.ndarray:
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return ((i == 0) | (i == n - 1) | (j == 0) | (j == n - 1)).ravel()


def sides_on_vertex_set(tri: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """tri*3 + j for every local side j whose two vertices are both in mask."""
    a = mask[tri[:, [1, 2, 0]]]
    b = mask[tri[:, [2, 0, 1]]]
    e, j = np.nonzero(a & b)
    return (e * 3 + j).astype(np.int32)


def lattice(n: int, seed: int = 0, jitter: float = 0.05) -> Mesh:
    """Jittered n x n triangular lattice with Dirichlet sides on the right."""
    xy = lattice_vertices(n)
    tri = lattice_triangles(n)
    if jitter > 0.0 and n > 2:
        rng = np.random.default_rng(seed)
        interior = ~_boundary_vertex_mask(n)
        k = int(interior.sum())
        r = jitter * np.sqrt(rng.random(k))
        phi = 2.0 * math.pi * rng.random(k)
        xy[interior, 0] += r * np.cos(phi)
        xy[interior, 1] += r * np.sin(phi)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    right = (i == n - 1).ravel()
    dirichlet = sides_on_vertex_set(tri, right)
    return Mesh(n=n, xy=xy, tri=tri, dirichlet=dirichlet)


def defect_lattice(n: int, seed: int = 0, defects: int = 4) -> Mesh:
    """Jittered lattice with `defects` interior sides bisected at their
    midpoint: the two cells of such a side become four, and the two vertices
    opposite the side get odd degree, so the cell graph has odd cycles (it is
    not two-colourable).  Every circumcentre distance stays positive."""
    base = lattice(n, seed)
    xy = [row for row in base.xy]
    tri = [list(t) for t in base.tri]
    rng = np.random.default_rng(seed + 271828)
    nt0 = len(tri)
    used = set()
    side_of = {}
    for e, t in enumerate(tri):
        for j in range(3):
            a, b = t[(j + 1) % 3], t[(j + 2) % 3]
            side_of.setdefault((min(a, b), max(a, b)), []).append(e)
    cands = [k for k, v in side_of.items() if len(v) == 2]
    rng.shuffle(cands)
    made = 0
    for a, b in cands:
        if made == defects:
            break
        e1, e2 = side_of[(a, b)]
        if e1 in used or e2 in used or e1 >= nt0 or e2 >= nt0:
            continue
        # keep defects apart: no shared vertex with earlier ones
        verts = set(tri[e1]) | set(tri[e2])
        if any(v in used for v in verts):
            continue
        m = len(xy)
        xy.append(0.5 * (np.asarray(xy[a]) + np.asarray(xy[b])))
        for e in (e1, e2):
            t = tri[e]
            k = [i for i in range(3) if t[i] not in (a, b)][0]
            c, p, q = t[k], t[(k + 1) % 3], t[(k + 2) % 3]   # side p -> q opposite c
            tri[e] = [p, m, c]
            tri.append([m, q, c])
        used.update({e1, e2})
        used.update(verts)
        made += 1
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int32)
    right = np.zeros(len(xy), dtype=bool)
    right[: n * n] = (np.arange(n * n) % n) == n - 1
    return Mesh(n=n, xy=xy, tri=tri, dirichlet=sides_on_vertex_set(tri, right))


def defect_problem(n: int, seed: int = 0) -> Problem:
    """Random-Fourier porosity in [0.3, 1] with isotropic Kozeny-Carman K on
    a lattice with bisected sides (a mesh that needs more than two colours)."""
    mesh = defect_lattice(n, seed)
    rng = np.random.default_rng(seed + 3571)
    f = random_fourier_field(mesh.xy, rng, mesh.width, mesh.height)
    eps = np.clip(0.65 + 0.175 * f, 0.3, 1.0)
    return Problem(mesh, eps, iso_kinv(kozeny_carman_kinv(eps)), PER_VERTEX,
                   meta={"workload": f"defect-lattice n={n}", "seed": seed})


def _tri_lattice(h: float, W: float, H: float) -> np.ndarray:
    """Triangular-lattice points of spacing h covering [0, W] x [0, H]."""
    dy = h * math.sqrt(3.0) / 2.0
    rows = np.arange(0.0, H + dy, dy)
    pts = []
    for j, y in enumerate(rows):
        xs = np.arange(0.5 * h * (j % 2), W + h, h)
        pts.append(np.stack([xs, np.full_like(xs, y)], axis=1))
    return np.concatenate(pts)


def _morton(c: np.ndarray, bits: int = 16) -> np.ndarray:
    """Morton (Z-order) key of points c [n, 2] scaled to the unit square."""
    lo, hi = c.min(axis=0), c.max(axis=0)
    q = ((c - lo) / np.maximum(hi - lo, 1e-300) * ((1 << bits) - 1)).astype(np.uint64)
    key = np.zeros(c.shape[0], dtype=np.uint64)
    for b in range(bits):
        for d in range(2):
            key |= ((q[:, d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + d)
    return key


def graded_mesh(n: int, seed: int = 0, levels: int = 2, band: float = 6.0,
                jitter: float = 0.05, order: str = "morton") -> Mesh:
    """Unstructured Delaunay mesh graded toward the porous block's interface
    (the transition layer the paper refines, Sec. 4): a triangular lattice of
    spacing 1 on [0, n-1] x [0, (n-1) sqrt3/2], replaced within distance
    band / 2^(k-1) of the block boundary (x in [W/3, 2W/3], y < 0.8 H) by a
    lattice of spacing 2^-k, k = 1..levels; interior points jittered by
    jitter x spacing; the boundary points lie on a rectangle bulged outward by
    1e-3 (strictly convex, so the Delaunay triangulation keeps every boundary
    point).  Cells are numbered along a Morton curve of their centroids
    (order="morton") or as triangulated ("none").  Dirichlet sides on the
    right edge.  Needs scipy (the triangulation is an input-generation step).
    """
    from scipy.spatial import Delaunay
    W, H = float(n - 1), (n - 1) * math.sqrt(3.0) / 2.0
    rng = np.random.default_rng(seed)
    lo, hi = (W / 3, -H), (2 * W / 3, 0.8 * H)

    def dist(p):
        return np.abs(box_signed_distance(p, lo, hi))

    pts, spacing = [], []
    for k in range(levels + 1):
        h = 2.0 ** (-k)
        q = _tri_lattice(h, W, H)
        d = dist(q)
        keep = np.ones(q.shape[0], dtype=bool)
        if k > 0:
            keep &= d < band / 2.0 ** (k - 1)
        if k < levels:
            keep &= d >= band / 2.0 ** k
        q = q[keep]
        # interior only, off the boundary by a third of the spacing
        inner = ((q[:, 0] > h / 3) & (q[:, 0] < W - h / 3) & (q[:, 1] > h / 3) &
                 (q[:, 1] < H - h / 3))
        q = q[inner]
        pts.append(q)
        spacing.append(np.full(q.shape[0], h))
    pts = np.concatenate(pts)
    spacing = np.concatenate(spacing)
    r = jitter * spacing * np.sqrt(rng.random(pts.shape[0]))
    phi = 2.0 * math.pi * rng.random(pts.shape[0])
    pts = pts + np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)
    # boundary: the local interior spacing along each edge, then bulged outward
    def edge_points(a, b):
        # vertical edges at the lattice's row height, so that every boundary
        # point sits on a row and the cell opposite a boundary side is acute
        rowf = math.sqrt(3.0) / 2.0 if a[0] == b[0] else 1.0
        length = math.hypot(b[0] - a[0], b[1] - a[1])
        t = np.linspace(0.0, 1.0, 8 * int(math.ceil(length)) * 2 ** levels + 1)
        probe = np.asarray(a)[None, :] + t[:, None] * (np.asarray(b) - np.asarray(a))[None, :]
        dd = dist(probe)
        hloc = np.ones_like(dd)
        for k in range(1, levels + 1):
            hloc = np.where(dd < band / 2.0 ** (k - 1), 2.0 ** (-k), hloc)
        out, s_ = [np.asarray(a, dtype=float)], 0.0
        while True:
            i = min(int(s_ / length * (t.size - 1)), t.size - 1)
            s_ += rowf * hloc[i]
            if s_ >= length - 0.5 * rowf * hloc[i]:
                break
            out.append(np.asarray(a) + (s_ / length) * (np.asarray(b) - np.asarray(a)))
        return np.array(out)

    corners = [(0.0, 0.0), (W, 0.0), (W, H), (0.0, H)]
    bnd = np.concatenate([edge_points(corners[i], corners[(i + 1) % 4]) for i in range(4)])
    # bulge: push each boundary point outward by 1e-3 x (distance-to-corner profile)
    bx, by = bnd[:, 0], bnd[:, 1]
    eps_b = 1e-3
    on_bottom, on_top = by == 0.0, by == H
    on_left, on_right = (bx == 0.0) & ~on_bottom & ~on_top, (bx == W) & ~on_bottom & ~on_top
    u = bx / W
    v = by / H
    bnd = bnd.copy()
    bnd[on_bottom, 1] -= eps_b * 4 * u[on_bottom] * (1 - u[on_bottom])
    bnd[on_top, 1] += eps_b * 4 * u[on_top] * (1 - u[on_top])
    bnd[on_left, 0] -= eps_b * 4 * v[on_left] * (1 - v[on_left])
    bnd[on_right, 0] += eps_b * 4 * v[on_right] * (1 - v[on_right])
    right = np.zeros(bnd.shape[0] + pts.shape[0], dtype=bool)
    right[: bnd.shape[0]] = (bx == W)
    xy = np.concatenate([bnd, pts])
    tri = Delaunay(xy).simplices.astype(np.int64)
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = cross < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    if order == "morton":
        cen = xy[tri].mean(axis=1)
        tri = tri[np.argsort(_morton(cen), kind="stable")]
    tri = np.ascontiguousarray(tri.astype(np.int32))
    dirichlet = sides_on_vertex_set(tri, right)
    return Mesh(n=n, xy=xy, tri=tri, dirichlet=dirichlet)


def graded_problem(n: int, seed: int = 0, levels: int = 2, beta: float = 100.0,
                   alpha_deg: float = 30.0, order: str = "morton") -> Problem:
    """The channel-block fields (random-Fourier porosity in the block, clear
    fluid outside, anisotropic Kozeny-Carman) on the graded mesh."""
    mesh = graded_mesh(n, seed, levels=levels, order=order)
    W, H = mesh.width, mesh.height
    rng = np.random.default_rng(seed + 7919)
    f = random_fourier_field(mesh.xy, rng, W, H)
    eps_blk = np.clip(0.45 + 0.1 * f, 0.3, 0.6)
    sd = box_signed_distance(mesh.xy, (W / 3, -H), (2 * W / 3, 0.8 * H))
    w = transition_weight(sd, 2.0 / 1.5 * 2 ** levels)
    eps = 1.0 + (eps_blk - 1.0) * w
    kinv = aniso_kinv(kozeny_carman_kinv(eps), beta, math.radians(alpha_deg))
    return Problem(mesh, eps, kinv, PER_VERTEX,
                   meta={"workload": f"graded-delaunay n={n} levels={levels}", "seed": seed})


def triangle_areas(mesh: Mesh) -> np.ndarray:
    """Shoelace area of each triangle (used to scale the random RHS)."""
    p = mesh.xy[mesh.tri]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def cell_centroids(mesh: Mesh) -> np.ndarray:
    return mesh.xy[mesh.tri].mean(axis=1)


# ---------------------------------------------------------------- fields

def kozeny_carman_kinv(eps: np.ndarray, d: float = KC_D) -> np.ndarray:
    """1/K for the Kozeny-Carman law K = d^2 eps^3 / (180 (1 - eps)^2).

    Zero in clear fluid (eps = 1), finite everywhere else."""
    eps = np.asarray(eps, dtype=np.float64)
    return 180.0 * (1.0 - eps) ** 2 / (d * d * eps ** 3)


def box_signed_distance(p: np.ndarray, lo, hi) -> np.ndarray:
    """Signed distance to an axis-aligned box, positive outside it."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    q = np.abs(p - c) - h
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
    inside = np.minimum(np.maximum(q[:, 0], q[:, 1]), 0.0)
    return outside + inside


def transition_weight(sd: np.ndarray, theta: float) -> np.ndarray:
    """Porous weight in [0, 1] of the tanh transition layer (Eq. 3).

    With sd > 0 toward the free fluid, eps = 1 + (eps0 - 1) * w reproduces
    Eq. 3a: eps = (1 - eps0)/2 * tanh(sd*theta) + (1 + eps0)/2."""
    return 0.5 * (1.0 - np.tanh(sd * theta))


def random_fourier_field(p: np.ndarray, rng: np.random.Generator, lx: float,
                         ly: float, modes: int = 32, kmax: int = 8) -> np.ndarray:
    """Standardised sum of `modes` random cosines with integer wave vectors."""
    ks = []
    while len(ks) < modes:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k[0] != 0 or k[1] != 0:
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    a = rng.standard_normal(modes)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    arg = 2.0 * math.pi * (np.outer(p[:, 0] / lx, ks[:, 0])
                           + np.outer(p[:, 1] / ly, ks[:, 1])) + ph
    f = np.cos(arg) @ a
    s = f.std()
    return (f - f.mean()) / (s if s > 0 else 1.0)


def aniso_kinv(kinv_scalar: np.ndarray, beta: float, alpha: float) -> np.ndarray:
    """Components (xx, xy, yy) of K^-1 for K = R diag(k/beta, k) R^T (Eq. aniso).

    K^-1 = R diag(beta/k, 1/k) R^T, with 1/k given (zero in clear fluid)."""
    c, s = math.cos(alpha), math.sin(alpha)
    l1 = beta * kinv_scalar
    l2 = kinv_scalar
    xx = c * c * l1 + s * s * l2
    xy = c * s * (l1 - l2)
    yy = s * s * l1 + c * c * l2
    return np.stack([xx, xy, yy], axis=1)


def iso_kinv(kinv_scalar: np.ndarray) -> np.ndarray:
    z = np.zeros_like(kinv_scalar)
    return np.stack([kinv_scalar, z, kinv_scalar], axis=1)


def centred_block_problem(n: int, seed: int = 0, eps0: float = 0.4) -> Problem:
    """Porous square in the middle (1/4 of the domain), isotropic Kozeny-Carman
    K, tanh transition about 3 cells wide (theta = 2/(1.5 h), h = 1)."""
    mesh = lattice(n, seed)
    W, H = mesh.width, mesh.height
    sd = box_signed_distance(mesh.xy, (W / 4, H / 4), (3 * W / 4, 3 * H / 4))
    w = transition_weight(sd, 2.0 / 1.5)
    eps = 1.0 + (eps0 - 1.0) * w
    kinv = iso_kinv(kozeny_carman_kinv(eps))
    return Problem(mesh, eps, kinv, PER_VERTEX,
                   meta={"workload": f"centred-block n={n}", "seed": seed})


def channel_block_problem(n: int, seed: int = 0, beta: float = 100.0,
                          alpha_deg: float = 30.0) -> Problem:
    """Porous block in a channel (x in [W/3, 2W/3], y in [0, 0.8 H]) whose
    porosity is a 32-mode random Fourier field (mean 0.45, std 0.1, clipped to
    [0.3, 0.6]); clear fluid eps = 1 outside; anisotropic Kozeny-Carman K with
    principal ratio beta rotated by alpha."""
    mesh = lattice(n, seed)
    W, H = mesh.width, mesh.height
    rng = np.random.default_rng(seed + 7919)
    f = random_fourier_field(mesh.xy, rng, W, H)
    eps_blk = np.clip(0.45 + 0.1 * f, 0.3, 0.6)
    sd = box_signed_distance(mesh.xy, (W / 3, -H), (2 * W / 3, 0.8 * H))
    w = transition_weight(sd, 2.0 / 1.5)
    eps = 1.0 + (eps_blk - 1.0) * w
    kinv = aniso_kinv(kozeny_carman_kinv(eps), beta, math.radians(alpha_deg))
    return Problem(mesh, eps, kinv, PER_VERTEX,
                   meta={"workload": f"channel-block-aniso n={n}", "seed": seed})


def ensemble_member_problem(nt_target: int, seed: int) -> Problem:
    """One member of the uneven ensemble: square lattice with about nt_target
    cells, random-Fourier porosity in [0.3, 1], isotropic Kozeny-Carman K."""
    n = max(3, 1 + int(round(math.sqrt(nt_target / 2.0))))
    mesh = lattice(n, seed)
    rng = np.random.default_rng(seed + 104729)
    f = random_fourier_field(mesh.xy, rng, mesh.width, mesh.height)
    eps = np.clip(0.65 + 0.175 * f, 0.3, 1.0)
    kinv = iso_kinv(kozeny_carman_kinv(eps))
    return Problem(mesh, eps, kinv, PER_VERTEX,
                   meta={"workload": f"ensemble-member n={n}", "seed": seed})


def ensemble_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)


def log_permeability_problem(n: int, seed: int = 0, eps0: float = 0.4,
                             theta_std: float = 1.0):
    """Cell-wise isotropic K = exp(theta) with theta = ln K_KC(eps0) + field
    (std theta_std); uniform porosity eps0.  Returns (problem, theta)."""
    mesh = lattice(n, seed)
    rng = np.random.default_rng(seed + 15485863)
    c = cell_centroids(mesh)
    f = random_fourier_field(c, rng, mesh.width, mesh.height)
    theta = -math.log(float(kozeny_carman_kinv(np.array(eps0)))) + theta_std * f
    kinv = iso_kinv(np.exp(-theta))
    eps = np.full(mesh.nt, eps0)
    return Problem(mesh, eps, kinv, PER_CELL,
                   meta={"workload": f"log-permeability n={n}", "seed": seed}), theta


def cell_vector_field(mesh: Mesh, seed: int, mean=(0.0, 0.0), scale: float = 1.0) -> np.ndarray:
    """[2, nt]: two independent random-Fourier fields at the cell centroids
    (standardised, times scale) plus a uniform mean -- the stand-in for the
    first corrector's cell velocity u^{k+2/3} (not divergence free) and for the
    cell field eps grad(Psi^k) entering the second corrector."""
    rng = np.random.default_rng(seed + 104729)
    c = cell_centroids(mesh)
    f = np.stack([random_fourier_field(c, rng, mesh.width, mesh.height) for _ in range(2)])
    return np.asarray(mean, dtype=np.float64)[:, None] + scale * f


def rhs(mesh: Mesh, seed: int) -> np.ndarray:
    """b_e = A_e * N(0, 1)."""
    rng = np.random.default_rng(seed)
    return triangle_areas(mesh) * rng.standard_normal(mesh.nt)


def normal_noise(size: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(size)


def workload(name: str, seed: int = 0) -> Problem:
    """Named workloads: 'block64' (small centred block, n=64),
    'channel1024' (anisotropic channel block, n=1024), 'channel<n>' and
    'block<n>' for other sizes."""
    if name.startswith("block"):
        return centred_block_problem(int(name[5:]), seed)
    if name.startswith("channel"):
        return channel_block_problem(int(name[7:]), seed)
    raise ValueError(f"unknown workload {name!r}")
