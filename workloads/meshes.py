"""Seeded synthetic simplex meshes for the P1-P1 IPCS workloads.

This module only builds inputs: vertex coordinates, cell-to-vertex tables,
periodic vertex-to-dof maps, boundary dof lists and dof renumberings.  It
holds none of the scheme's arithmetic (no element integrals, no assembly, no
solves) and is shared by the CPU oracle, the tests and the benchmark.

Conventions (the paper only says "split into 2 triangles / 6 tets", Sec. 6):
  * 2D: every square cell (i, j) is cut along the diagonal (i, j)-(i+1, j+1).
  * 3D: the Kuhn/Freudenthal split of every cube into the 6 tetrahedra that
    share the (0,0,0)-(1,1,1) diagonal.  The split is translation invariant,
    so the mesh is conforming and stays conforming under periodic wrap.
  * Every cell is stored with positive orientation (det J > 0).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    dim: int
    coords: np.ndarray            # [n_vertices, dim] float64
    cells: np.ndarray             # [n_cells, dim+1] int32, vertex indices
    dof_of_vertex: np.ndarray     # [n_vertices] int32 (identity if not periodic)
    n_dofs: int
    boundary_dofs: dict = field(default_factory=dict)   # name -> sorted int32 dofs

    @property
    def n_vertices(self) -> int:
        return self.coords.shape[0]

    @property
    def n_cells(self) -> int:
        return self.cells.shape[0]

    def dof_coords(self) -> np.ndarray:
        """Coordinates of one representative vertex per dof [n_dofs, dim]."""
        out = np.empty((self.n_dofs, self.dim))
        # the last vertex written wins; periodic images share all non-periodic
        # coordinates, and the periodic coordinate is taken from the lowest image
        order = np.argsort(-np.arange(self.n_vertices))
        out[self.dof_of_vertex[order]] = self.coords[order]
        return out


def _signed_measure_sign(coords, cells):
    d = coords.shape[1]
    x0 = coords[cells[:, 0]]
    J = np.stack([coords[cells[:, k + 1]] - x0 for k in range(d)], axis=1)
    return np.linalg.det(J)


def _orient_positive(coords, cells):
    det = _signed_measure_sign(coords, cells)
    neg = det < 0
    cells = cells.copy()
    cells[neg, 0], cells[neg, 1] = cells[neg, 1].copy(), cells[neg, 0].copy()
    return cells


def box_mesh_2d(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0, periodic=False,
                diagonal="right") -> Mesh:
    """(nx x ny) square cells, each cut into 2 right triangles.

    ``diagonal="right"`` cuts along (i, j)-(i+1, j+1), ``"left"`` along
    (i+1, j)-(i, j+1).  ``periodic`` identifies both pairs of opposite sides.
    """
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = np.arange((nx + 1) * (ny + 1)).reshape(nx + 1, ny + 1)
    v00 = vid[:-1, :-1].ravel()
    v10 = vid[1:, :-1].ravel()
    v11 = vid[1:, 1:].ravel()
    v01 = vid[:-1, 1:].ravel()
    if diagonal == "right":
        t1 = np.stack([v00, v10, v11], axis=1)
        t2 = np.stack([v00, v11, v01], axis=1)
    elif diagonal == "left":
        t1 = np.stack([v00, v10, v01], axis=1)
        t2 = np.stack([v10, v11, v01], axis=1)
    else:
        raise ValueError(diagonal)
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    cells = _orient_positive(coords, cells)
    n = coords.shape[0]
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    if periodic:
        key = (ii % nx) * ny + (jj % ny)
        uniq, dof = np.unique(key.ravel(), return_inverse=True)
        m = Mesh(2, coords, cells, dof.astype(np.int32), uniq.size)
        m.boundary_dofs["all"] = np.zeros(0, dtype=np.int32)
        return m
    bnd = (ii == 0) | (ii == nx) | (jj == 0) | (jj == ny)
    m = Mesh(2, coords, cells, np.arange(n, dtype=np.int32), n)
    m.boundary_dofs["all"] = np.nonzero(bnd.ravel())[0].astype(np.int32)
    return m


# The 6 Kuhn tetrahedra of the unit cube: walk from (0,0,0) to (1,1,1) adding
# one unit vector at a time, in every possible axis order.
def _kuhn_offsets():
    tets = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros(3, dtype=int)
        verts = [p.copy()]
        for ax in perm:
            p[ax] += 1
            verts.append(p.copy())
        tets.append(verts)
    return np.array(tets)          # [6, 4, 3]


def box_mesh_3d(nx: int, ny: int, nz: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                y_coords: np.ndarray | None = None, periodic=(False, False, False)) -> Mesh:
    """(nx x ny x nz) cubes, each cut into the 6 Kuhn tetrahedra.

    ``y_coords`` (length ny+1) replaces the uniform y spacing (stretched
    meshes).  ``periodic[a]`` identifies the vertex planes 0 and n_a of axis a
    through ``dof_of_vertex``; the geometry keeps both planes.
    """
    n = (nx, ny, nz)
    axes = [np.linspace(lo[a], hi[a], n[a] + 1) for a in range(3)]
    if y_coords is not None:
        assert len(y_coords) == ny + 1
        axes[1] = np.asarray(y_coords, dtype=np.float64)
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = np.arange((nx + 1) * (ny + 1) * (nz + 1)).reshape(nx + 1, ny + 1, nz + 1)
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    offs = _kuhn_offsets()
    cells = np.empty((ci.size, 6, 4), dtype=np.int64)
    for t in range(6):
        for v in range(4):
            o = offs[t, v]
            cells[:, t, v] = vid[ci + o[0], cj + o[1], ck + o[2]]
    cells = cells.reshape(-1, 4).astype(np.int32)
    cells = _orient_positive(coords, cells)

    # periodic identification: index along a periodic axis wraps n_a -> 0
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    I2, J2, K2 = I.copy(), J.copy(), K.copy()
    if periodic[0]:
        I2[I2 == nx] = 0
    if periodic[1]:
        J2[J2 == ny] = 0
    if periodic[2]:
        K2[K2 == nz] = 0
    key = (I2 * (ny + 1) + J2) * (nz + 1) + K2
    uniq, dof = np.unique(key.ravel(), return_inverse=True)
    dof_of_vertex = dof.astype(np.int32)
    n_dofs = uniq.size

    on = np.zeros(I.shape, dtype=bool)
    for a, (idx, na) in enumerate(((I, nx), (J, ny), (K, nz))):
        if not periodic[a]:
            on |= (idx == 0) | (idx == na)
    m = Mesh(3, coords, cells, dof_of_vertex, n_dofs)
    m.boundary_dofs["all"] = np.unique(dof_of_vertex[on.ravel()]).astype(np.int32)
    walls = (J == 0) | (J == ny)
    m.boundary_dofs["walls_y"] = np.unique(dof_of_vertex[walls.ravel()]).astype(np.int32)
    return m


def jitter_interior(mesh: Mesh, frac: float, spacing: float, seed: int, max_rounds: int = 50) -> Mesh:
    """Move every interior vertex by U(-frac*h, frac*h) per coordinate.

    Any cell left with det J <= 0 gets its vertices redrawn from the same seeded
    stream (deterministic for a given seed) until all cells are positive.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    coords0 = mesh.coords
    interior = np.ones(mesh.n_vertices, dtype=bool)
    interior[np.isin(mesh.dof_of_vertex, mesh.boundary_dofs["all"])] = False
    idx = np.nonzero(interior)[0]
    coords = coords0.copy()
    coords[idx] += rng.uniform(-frac * spacing, frac * spacing, size=(idx.size, mesh.dim))
    for _ in range(max_rounds):
        det = _signed_measure_sign(coords, mesh.cells)
        bad = det <= 0
        if not bad.any():
            break
        verts = np.unique(mesh.cells[bad].ravel())
        verts = verts[interior[verts]]
        coords[verts] = coords0[verts] + rng.uniform(-frac * spacing, frac * spacing,
                                                     size=(verts.size, mesh.dim))
    else:
        raise RuntimeError("jitter could not produce a positive mesh")
    return Mesh(mesh.dim, coords, mesh.cells, mesh.dof_of_vertex, mesh.n_dofs,
                dict(mesh.boundary_dofs))


def vertex_graph(mesh: Mesh):
    """Symmetric dof adjacency (scipy CSR, ones) of the P1 pattern, without values."""
    import scipy.sparse as sp
    d1 = mesh.dim + 1
    c = mesh.dof_of_vertex[mesh.cells]
    r = np.repeat(c, d1, axis=1).ravel()
    s = np.tile(c, (1, d1)).ravel()
    g = sp.coo_matrix((np.ones(r.size, dtype=np.int8), (r, s)), shape=(mesh.n_dofs, mesh.n_dofs)).tocsr()
    g.data[:] = 1
    return g


def rcm_permutation(mesh: Mesh) -> np.ndarray:
    """new_of_old dof permutation from reverse Cuthill-McKee on the dof graph."""
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    order = reverse_cuthill_mckee(vertex_graph(mesh), symmetric_mode=True)   # old index at new position
    new_of_old = np.empty_like(order)
    new_of_old[order] = np.arange(order.size)
    return new_of_old.astype(np.int32)


def random_permutation(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.permutation(n).astype(np.int32)


def renumber_dofs(mesh: Mesh, new_of_old: np.ndarray) -> Mesh:
    """Relabel dofs: dof d becomes new_of_old[d].  Geometry is unchanged."""
    new_of_old = np.asarray(new_of_old, dtype=np.int32)
    dov = new_of_old[mesh.dof_of_vertex]
    bd = {k: np.sort(new_of_old[v]).astype(np.int32) for k, v in mesh.boundary_dofs.items()}
    return Mesh(mesh.dim, mesh.coords, mesh.cells, dov, mesh.n_dofs, bd)
