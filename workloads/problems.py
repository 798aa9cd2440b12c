"""Seeded problem definitions (mesh + data) for the five IPCS workloads.

A ``Problem`` carries everything the solver is given: the mesh, nu, dt, the
constant body force f, the velocity Dirichlet dof set (shared by all
components), the initial fields u^{n-1}, u^{n-2}, p* and a callable giving the
Dirichlet values at a time t.  Exact solutions (Taylor-Green) are problem data,
used to initialise and to measure errors; nothing here evaluates the scheme.

Readings of the paper where it is silent (Sec. 6 and the workload list):
  * initial staggering: u^{n-1} = u_e(t0), u^{n-2} = u_e(t0 - dt), p* = p_e(t0 - dt/2);
  * 3D Taylor-Green, channel and stress meshes: u^{n-2} = u^{n-1} = u_0 and
    Dirichlet values held at the initial field on the boundary;
  * channel: periodic in x and z, no-slip walls at y = +-1, f = (1, 0, 0),
    Poiseuille 90 (1 - y^2) plus 0.1*90*U(-1, 1) on every interior dof and
    component.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

import numpy as np

from . import meshes as M


@dataclass
class Scalars:
    """Passive scalars c_alpha (the scalar equation of Sec. 3): initial values,
    diffusivities D_alpha, constant sources f_alpha, one Dirichlet dof set shared
    by every scalar and a callable giving its values at a time t."""
    c0: np.ndarray                      # [ns, N] float64
    diffusivity: np.ndarray             # [ns]
    source: np.ndarray                  # [ns] constant f_alpha
    dirichlet: np.ndarray               # [n_sdir] int32 dofs
    g: Callable[[float], np.ndarray]    # t -> [ns, n_sdir]
    exact: Callable | None = None       # (x [N,d], t) -> [ns, N]


@dataclass
class Problem:
    name: str
    mesh: M.Mesh
    nu: float
    dt: float
    f: np.ndarray                       # [dim] constant body force
    dirichlet: np.ndarray               # [n_dir] int32 dofs (velocity, all components)
    u_nm1: np.ndarray                   # [dim, N] float64
    u_nm2: np.ndarray                   # [dim, N]
    p: np.ndarray                       # [N] p* for the first step
    t0: float
    g: Callable[[float], np.ndarray]    # t -> [dim, n_dir] Dirichlet values at time t
    n_steps: int
    rtol: float
    exact_u: Callable | None = None     # (x [N,d], t) -> [d, N]
    exact_p: Callable | None = None     # (x [N,d], t) -> [N]
    scalars: Scalars | None = None      # passive scalars transported by the flow
    perm: np.ndarray | None = None      # [N] dof renumbering handed to the solver library
                                        # (perm[d] = its internal index of dof d); the
                                        # problem's own arrays stay in mesh order


# ---------------------------------------------------------------- 2D Taylor-Green
def tg2d_u(x, t, nu):
    e = np.exp(-2.0 * np.pi ** 2 * nu * t)
    return np.stack([-np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * e,
                     np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * e])


def tg2d_p(x, t, nu):
    e = np.exp(-4.0 * np.pi ** 2 * nu * t)
    return -0.25 * (np.cos(2 * np.pi * x[:, 0]) + np.cos(2 * np.pi * x[:, 1])) * e


def taylor_green_2d(n: int = 32, nu: float = 0.01, dt: float = 1e-3, n_steps: int = 100,
                    rtol: float = 1e-12) -> Problem:
    """Unit square, n x n cells x 2 triangles, Dirichlet from the exact solution."""
    mesh = M.box_mesh_2d(n, n)
    x = mesh.dof_coords()
    bd = mesh.boundary_dofs["all"]
    xb = x[bd]
    return Problem(
        name=f"tg2d_{n}", mesh=mesh, nu=nu, dt=dt, f=np.zeros(2), dirichlet=bd,
        u_nm1=tg2d_u(x, 0.0, nu), u_nm2=tg2d_u(x, -dt, nu), p=tg2d_p(x, -0.5 * dt, nu),
        t0=0.0, g=lambda t: tg2d_u(xb, t, nu), n_steps=n_steps, rtol=rtol,
        exact_u=lambda xx, t: tg2d_u(xx, t, nu), exact_p=lambda xx, t: tg2d_p(xx, t, nu))


def taylor_green_2d_periodic(n: int = 10, nu: float = 0.01, dt: float = 1e-3, n_steps: int = 1000,
                             rtol: float = 1e-12, diagonal: str = "right",
                             start: str = "staggered") -> Problem:
    """Doubly periodic [0, 2]^2, n x n cells x 2 triangles (the setting of Table 1).

    ``start="staggered"``: u^{n-2} = u_e(-dt), p* = p_e(-dt/2);
    ``start="flat"``: u^{n-2} = u^{n-1} = u_e(0), p* = p_e(0).
    """
    mesh = M.box_mesh_2d(n, n, 0.0, 2.0, 0.0, 2.0, periodic=True, diagonal=diagonal)
    x = mesh.dof_coords()
    if start == "staggered":
        u2, p0 = tg2d_u(x, -dt, nu), tg2d_p(x, -0.5 * dt, nu)
    else:
        u2, p0 = tg2d_u(x, 0.0, nu), tg2d_p(x, 0.0, nu)
    empty = np.zeros(0, dtype=np.int32)
    return Problem(
        name=f"tg2d_periodic_{n}", mesh=mesh, nu=nu, dt=dt, f=np.zeros(2), dirichlet=empty,
        u_nm1=tg2d_u(x, 0.0, nu), u_nm2=u2, p=p0, t0=0.0, g=lambda t: np.zeros((2, 0)),
        n_steps=n_steps, rtol=rtol,
        exact_u=lambda xx, t: tg2d_u(xx, t, nu), exact_p=lambda xx, t: tg2d_p(xx, t, nu))


# ---------------------------------------------------------------- 3D Taylor-Green
def tg3d_u(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return np.stack([np.sin(x) * np.cos(y) * np.cos(z),
                     -np.cos(x) * np.sin(y) * np.cos(z),
                     np.zeros_like(x)])


def tg3d_p(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0


def _held_problem(name, mesh, nu, dt, f, u0, p0, n_steps, rtol, dirichlet):
    ub = u0[:, dirichlet].copy()
    return Problem(name=name, mesh=mesh, nu=nu, dt=dt, f=np.asarray(f, dtype=np.float64),
                   dirichlet=dirichlet, u_nm1=u0.copy(), u_nm2=u0.copy(), p=p0, t0=0.0,
                   g=lambda t: ub, n_steps=n_steps, rtol=rtol)


def taylor_green_3d(n: int = 64, nu: float = 1.0 / 1600, dt: float = 1e-3, n_steps: int = 200,
                    rtol: float = 1e-8) -> Problem:
    """[-pi, pi]^3, n^3 cubes x 6 Kuhn tets, Dirichlet = initial field on the boundary."""
    mesh = M.box_mesh_3d(n, n, n, lo=(-np.pi,) * 3, hi=(np.pi,) * 3)
    x = mesh.dof_coords()
    return _held_problem(f"tg3d_{n}", mesh, nu, dt, np.zeros(3), tg3d_u(x), tg3d_p(x),
                         n_steps, rtol, mesh.boundary_dofs["all"])


# ---------------------------------------------------------------- channel
def channel_y(ny_vertices: int, stretch: float = 2.0) -> np.ndarray:
    eta = np.linspace(-1.0, 1.0, ny_vertices)
    return np.tanh(stretch * eta) / np.tanh(stretch)


def channel(nx: int = 128, ny: int = 96, nz: int = 96, nu: float = 1.0 / 180, dt: float = 5e-3,
            n_steps: int = 200, rtol: float = 1e-8, seed: int = 3, perturb: float = 0.1,
            lx: float = 4 * np.pi, lz: float = 4 * np.pi / 3) -> Problem:
    """4pi x 2 x 4pi/3 box, nx x ny x nz dofs (periodic x, z; ny vertices in y)."""
    mesh = M.box_mesh_3d(nx, ny - 1, nz, lo=(0.0, -1.0, 0.0), hi=(lx, 1.0, lz),
                         y_coords=channel_y(ny), periodic=(True, False, True))
    x = mesh.dof_coords()
    walls = mesh.boundary_dofs["walls_y"]
    fx = 1.0
    uc = fx / (2.0 * nu)
    u0 = np.zeros((3, mesh.n_dofs))
    u0[0] = uc * (1.0 - x[:, 1] ** 2)
    rng = np.random.Generator(np.random.PCG64(seed))
    interior = np.ones(mesh.n_dofs, dtype=bool)
    interior[walls] = False
    u0[:, interior] += perturb * uc * rng.uniform(-1.0, 1.0, size=(3, int(interior.sum())))
    u0[:, walls] = 0.0
    return _held_problem(f"channel_{nx}x{ny}x{nz}", mesh, nu, dt, (fx, 0.0, 0.0), u0,
                         np.zeros(mesh.n_dofs), n_steps, rtol, walls)


# ---------------------------------------------------------------- stress mesh
def stress_cube(n: int = 128, nu: float = 1e-3, dt: float = 1e-3, n_steps: int = 100,
                rtol: float = 1e-8, jitter: float = 0.2, seed: int = 4,
                ordering: str = "natural", perm_seed: int = 44) -> Problem:
    """Unit cube n^3 x 6 tets, interior vertices jittered, optional dof reordering.

    ``ordering``: "natural", "random" (seeded permutation) or "rcm": the order the
    solver library stores and computes in, handed to it as ``perm``; the mesh and
    every array of the problem stay in the natural (lexicographic) vertex order.
    3D Taylor-Green data on X = 2 pi x - pi (same for y, z).
    """
    mesh = M.box_mesh_3d(n, n, n)
    if jitter > 0:
        mesh = M.jitter_interior(mesh, jitter, 1.0 / n, seed)
    if ordering == "random":
        perm = M.random_permutation(mesh.n_dofs, perm_seed)
    elif ordering == "rcm":
        perm = M.rcm_permutation(mesh)
    elif ordering == "natural":
        perm = None
    else:
        raise ValueError(ordering)
    X = 2 * np.pi * mesh.dof_coords() - np.pi
    pb = _held_problem(f"stress_{n}_{ordering}", mesh, nu, dt, np.zeros(3), tg3d_u(X),
                       tg3d_p(X), n_steps, rtol, mesh.boundary_dofs["all"])
    pb.perm = perm
    return pb


# ---------------------------------------------------------------- scalars
def with_scalars(pb: Problem, ns: int = 2, diffusivity=(1e-3, 2e-2), source=(0.0, 0.5),
                 seed: int = 7) -> Problem:
    """Attach ``ns`` seeded scalars to a problem: a smooth field (a product of
    cosines in the box's own coordinates) plus 5 % seeded noise; Dirichlet set:
    the walls of a channel (c = (1 + y) / 2 there), else the velocity's Dirichlet
    set with the initial values held."""
    x = pb.mesh.dof_coords()
    lo, hi = x.min(axis=0), x.max(axis=0)
    xi = (x - lo) / np.maximum(hi - lo, 1e-300)
    rng = np.random.Generator(np.random.PCG64(seed))
    c0 = np.empty((ns, pb.mesh.n_dofs))
    for a in range(ns):
        c0[a] = np.prod(np.cos(np.pi * (a + 1) * xi), axis=1) + 0.05 * rng.uniform(-1.0, 1.0, pb.mesh.n_dofs)
    walls = pb.mesh.boundary_dofs.get("walls_y") if pb.mesh.boundary_dofs else None
    if walls is not None and pb.name.startswith("channel"):
        sd = np.asarray(walls, dtype=np.int32)
        c0[:, sd] = 0.5 * (1.0 + x[sd, 1])[None, :]
    else:
        sd = np.asarray(pb.dirichlet, dtype=np.int32)
    held = c0[:, sd].copy()
    dif = np.resize(np.asarray(diffusivity, dtype=np.float64), ns)
    src = np.resize(np.asarray(source, dtype=np.float64), ns)
    pb.scalars = Scalars(c0=c0, diffusivity=dif, source=src, dirichlet=sd, g=lambda t: held)
    return pb


def uniform_advection_2d(n: int = 16, U=(1.0, 0.5), nu: float = 0.01, D: float = 0.01,
                         dt: float = 1e-2, n_steps: int = 50) -> Problem:
    """Doubly periodic unit square with the uniform flow u = U, p = 0 (an exact
    Navier-Stokes solution) carrying one scalar with the exact solution
    c = exp(-8 pi^2 D t) sin(2 pi (x - U_x t)) sin(2 pi (y - U_y t))."""
    mesh = M.box_mesh_2d(n, n, 0.0, 1.0, 0.0, 1.0, periodic=True)
    x = mesh.dof_coords()
    N = mesh.n_dofs
    u0 = np.tile(np.asarray(U, dtype=np.float64)[:, None], (1, N))
    empty = np.zeros(0, dtype=np.int32)

    def exact(xx, t):
        e = np.exp(-8.0 * np.pi ** 2 * D * t)
        return (e * np.sin(2 * np.pi * (xx[:, 0] - U[0] * t)) * np.sin(2 * np.pi * (xx[:, 1] - U[1] * t)))[None, :]

    pb = Problem(name=f"advection_2d_{n}", mesh=mesh, nu=nu, dt=dt, f=np.zeros(2), dirichlet=empty,
                 u_nm1=u0.copy(), u_nm2=u0.copy(), p=np.zeros(N), t0=0.0, g=lambda t: np.zeros((2, 0)),
                 n_steps=n_steps, rtol=1e-12)
    pb.scalars = Scalars(c0=exact(x, 0.0), diffusivity=np.array([D]), source=np.zeros(1),
                         dirichlet=empty, g=lambda t: np.zeros((1, 0)), exact=exact)
    return pb


def by_name(name: str, **kw) -> Problem:
    table = {"tg2d": taylor_green_2d, "tg3d": taylor_green_3d, "channel": channel,
             "stress": stress_cube}
    return table[name](**kw)
