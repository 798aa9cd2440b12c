"""One P1-P1 IPCS (ABCN) time step, naive route (CPU, float64).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline of the benchmark, never by the product path.

The step follows the naive formulation of Sec. 4 (every form assembled from
element integrals each step), not the in-place Algorithm 2 of Sec. 5; the two
are algebraically identical, which is what the GPU parity tests check.

Per step, with d velocity components (inner iterations: see below):
  ubar   = 1.5 u^{n-1} - 0.5 u^{n-2}                          (Eq. 22)
  A      = M/dt + C(ubar)/2 + nu K/2                          (Eq. 33, A_ij)
  b_k    = (M/dt - C/2 - nu K/2) u_k^{n-1} + int f_k phi - G^k p*   (Eqs. 33, 31)
  rows i in the Dirichlet set: A_i. = e_i, b_k,i = g_k(x_i, t^n)
  A u_k^I = b_k,  k = 1..d
  K p = K p* - (1/dt) sum_k G^k u_k^I                         (Eq. 38, pressure)
      with the right-hand side projected on sum_i b_i = 0 (no pressure BC),
      p normalised to zero arithmetic mean, phi = p - p*
  u_k^n = u_k^I - dt (G^k phi)_i / ML_i, Dirichlet rows reset to g  (Eq. 41, lumping)

Convection (Sec. 3): `convection="abcn"` (default, Eq. 22) is the form above;
`convection="abe"` is the explicit Adams-Bashforth form of Eq. 21,
B = 1.5 u^{n-1}.grad u^{n-1} - 0.5 u^{n-2}.grad u^{n-2}, which moves convection
to the right-hand side:
  A   = M/dt + nu K/2   (constant)
  b_k = (M/dt - nu K/2) u_k^{n-1} - 1.5 C(u^{n-1}) u_k^{n-1} + 0.5 C(u^{n-2}) u_k^{n-2}
        + int f_k phi - G^k p*
with C(w)_ij = int phi_i w . grad phi_j.

Velocity update (Sec. 5): `velocity_update="lumped"` (default) is the lumped
update above; `"consistent"` solves the update with the mass matrix,
  M u_k^n = M u_k^I - dt G^k phi,   rows in the Dirichlet set: u_k^n = g_k,
by a sparse LU solve.

Passive scalars (the scalar equation of Sec. 3, solved after the velocity
update in Algorithm 1), when the problem carries them: for each scalar alpha
with diffusivity D_a and constant source f_a, convected by the same
ubar = 1.5 u^{n-1} - 0.5 u^{n-2} (B_a = ubar . grad c~, c~ = (c^n + c^{n-1}) / 2),
  A_a = M/dt + C(ubar)/2 + D_a K/2
  b_a = (M/dt - C(ubar)/2 - D_a K/2) c_a^{n-1} + f_a ML
  rows i in the scalars' Dirichlet set: A_a,i. = e_i, b_a,i = g_a(x_i, t^n)
  (the values are re-imposed after the solve, as for the velocity)
whichever form the velocity's convection takes.

Inner iterations (Algorithm 1): the tentative and pressure solves are repeated
`inner_iters` times within a step, each time with p* = the newest pressure (the
matrix A, which holds only old velocities, is unchanged); phi is the increment
of the last repetition, and the lumped velocity update follows the loop with
the last u^I and that phi.  inner_iters = 1 is the default of the paper's runs.

Readings where the paper is silent or self-contradictory:
  * Eq. 18 and its weak form carry the opposite sign to Eq. 19; the algebraic
    pressure equation of Sec. 5 (K P = K P* - ...) is consistent with Eq. 19
    and is the one used.
  * Eq. 41 is written with p^{n-1/2}; Eq. 19 and the naive form use phi.  phi
    is used, since the tentative step already carries -grad p*.
  * "normalize" is read as subtracting the arithmetic mean of the dof values.

Linear systems are solved exactly (sparse LU, the paper's default direct
solver) unless ``iterative=True``, in which case Jacobi-preconditioned
BiCGStab (velocity, as in Sec. 6) and Jacobi-preconditioned CG (pressure) run
to relative residual ``rtol``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .p1 import Discretization


@dataclass
class State:
    u_nm1: np.ndarray      # [d, N]
    u_nm2: np.ndarray      # [d, N]
    p: np.ndarray          # [N]  (p* of the next step)
    t: float
    c: np.ndarray | None = None   # [ns, N] passive scalars, if the problem has any


def replace_rows(A: sp.csr_matrix, rows: np.ndarray) -> sp.csr_matrix:
    """Return A with every row in ``rows`` replaced by the unit row e_i."""
    A = A.tolil(copy=True)
    for i in rows:
        A.rows[i] = [int(i)]
        A.data[i] = [1.0]
    return A.tocsr()


def _jacobi(A):
    dinv = 1.0 / A.diagonal()
    return spla.LinearOperator(A.shape, matvec=lambda x: dinv * x)


class IPCS:
    def __init__(self, problem, iterative: bool = False, rtol: float = 1e-12,
                 maxiter: int = 100000, inner_iters: int = 1, convection: str = "abcn",
                 velocity_update: str = "lumped"):
        self.pb = problem
        self.inner_iters = max(1, int(inner_iters))
        if convection not in ("abcn", "abe"):
            raise ValueError(convection)
        self.convection = convection
        if velocity_update not in ("lumped", "consistent"):
            raise ValueError(velocity_update)
        self.velocity_update = velocity_update
        self._Mlu = None
        self.disc = Discretization(problem.mesh)
        self.iterative = iterative
        self.rtol = rtol
        self.maxiter = maxiter
        D = self.disc
        self.dirichlet = np.asarray(problem.dirichlet, dtype=np.int64)
        # int f_k phi_i dx for a constant force
        self.b0 = np.asarray(problem.f, dtype=np.float64)[:, None] * D.ML[None, :]
        self.iters = {"u": [], "p": []}
        # pressure operator with dof 0 pinned: the pinned row is e_0, b_0 = 0
        self._Kpin_lu = None

    # ------------------------------------------------------------------ pieces
    def tentative_system(self, u_nm1, u_nm2, p_star, t_new):
        D, pb = self.disc, self.pb
        if self.convection == "abe":
            C1 = D.convection(u_nm1)
            C2 = D.convection(u_nm2)
            A = D.M / pb.dt + 0.5 * pb.nu * D.K
            E = D.M / pb.dt - 0.5 * pb.nu * D.K
            b = np.stack([E @ u_nm1[k] - 1.5 * (C1 @ u_nm1[k]) + 0.5 * (C2 @ u_nm2[k]) + self.b0[k]
                          - D.G[k] @ p_star for k in range(D.d)])
        else:
            ubar = 1.5 * u_nm1 - 0.5 * u_nm2
            C = D.convection(ubar)
            A = D.M / pb.dt + 0.5 * C + 0.5 * pb.nu * D.K
            E = D.M / pb.dt - 0.5 * C - 0.5 * pb.nu * D.K
            b = np.stack([E @ u_nm1[k] + self.b0[k] - D.G[k] @ p_star for k in range(D.d)])
        A = replace_rows(A, self.dirichlet)
        b[:, self.dirichlet] = pb.g(t_new)
        return A, b

    def scalar_system(self, u_nm1, u_nm2, c_nm1, alpha, t_new):
        """A_a, b_a of scalar ``alpha`` (Sec. 3, the scalar equation)."""
        D, pb = self.disc, self.pb
        sc = pb.scalars
        C = D.convection(1.5 * u_nm1 - 0.5 * u_nm2)
        Da = float(sc.diffusivity[alpha])
        A = D.M / pb.dt + 0.5 * C + 0.5 * Da * D.K
        E = D.M / pb.dt - 0.5 * C - 0.5 * Da * D.K
        b = E @ c_nm1 + float(sc.source[alpha]) * D.ML
        rows = np.asarray(sc.dirichlet, dtype=np.int64)
        A = replace_rows(A, rows)
        if len(rows):
            b[rows] = sc.g(t_new)[alpha]
        return A, b

    def pressure_rhs(self, u_I, p_star):
        D = self.disc
        bp = D.K @ p_star - (1.0 / self.pb.dt) * sum(D.G[k] @ u_I[k] for k in range(D.d))
        return bp - bp.mean()

    def solve_tentative(self, A, b, x0):
        if not self.iterative:
            lu = spla.splu(A.tocsc())
            return np.stack([lu.solve(b[k]) for k in range(b.shape[0])])
        out = []
        for k in range(b.shape[0]):
            x, info = spla.bicgstab(A, b[k], x0=x0[k], rtol=self.rtol, atol=0.0,
                                    maxiter=self.maxiter, M=_jacobi(A))
            if info != 0:
                raise RuntimeError(f"oracle BiCGStab did not converge (info={info})")
            out.append(x)
        return np.stack(out)

    def solve_pressure(self, bp, p_star):
        K = self.disc.K
        if not self.iterative:
            if self._Kpin_lu is None:
                self._Kpin_lu = spla.splu(replace_rows(K, np.array([0])).tocsc())
            rhs = bp.copy()
            rhs[0] = 0.0
            p = self._Kpin_lu.solve(rhs)
        else:
            p, info = spla.cg(K, bp, x0=p_star, rtol=self.rtol, atol=0.0,
                              maxiter=self.maxiter, M=_jacobi(K))
            if info != 0:
                raise RuntimeError(f"oracle CG did not converge (info={info})")
        return p - p.mean()

    # ------------------------------------------------------------------ step
    def step(self, s: State):
        pb, D = self.pb, self.disc
        t_new = s.t + pb.dt
        p_star = s.p
        increments = []
        for _ in range(self.inner_iters):
            A, b = self.tentative_system(s.u_nm1, s.u_nm2, p_star, t_new)
            u_I = self.solve_tentative(A, b, s.u_nm1)
            bp = self.pressure_rhs(u_I, p_star)
            p = self.solve_pressure(bp, p_star)
            phi = p - p_star
            increments.append(phi)
            p_star = p
        if self.velocity_update == "consistent":
            Mr = replace_rows(D.M, self.dirichlet)
            g = pb.g(t_new)
            rhs = np.stack([D.M @ u_I[k] - pb.dt * (D.G[k] @ phi) for k in range(D.d)])
            if len(self.dirichlet):
                rhs[:, self.dirichlet] = g
            if not self.iterative:
                if self._Mlu is None:
                    self._Mlu = spla.splu(Mr.tocsc())
                u_n = np.stack([self._Mlu.solve(rhs[k]) for k in range(D.d)])
            else:
                # iterative mode (the timed baseline): the same system by the
                # tentative solver's Jacobi BiCGStab, from u^I
                u_n = self.solve_tentative(Mr, rhs, u_I)
        else:
            u_n = np.stack([u_I[k] - pb.dt * (D.G[k] @ phi) / D.ML for k in range(D.d)])
        u_n[:, self.dirichlet] = pb.g(t_new)
        c_n = None
        if s.c is not None:
            c_n = np.empty_like(s.c)
            for a in range(s.c.shape[0]):
                Aa, ba = self.scalar_system(s.u_nm1, s.u_nm2, s.c[a], a, t_new)
                c_n[a] = self.solve_tentative(Aa, ba[None, :], s.c[a][None, :])[0]
            rows = np.asarray(pb.scalars.dirichlet, dtype=np.int64)
            if len(rows):
                c_n[:, rows] = pb.scalars.g(t_new)
        out = State(u_n, s.u_nm1, p, t_new, c_n)
        out.u_I, out.phi, out.bp = u_I, phi, bp
        out.increments = increments
        return out

    def initial_state(self) -> State:
        pb = self.pb
        c = None if getattr(pb, "scalars", None) is None else pb.scalars.c0.copy()
        return State(pb.u_nm1.copy(), pb.u_nm2.copy(), pb.p.copy(), pb.t0, c)

    def run(self, n_steps: int, state: State | None = None) -> State:
        s = state if state is not None else self.initial_state()
        for _ in range(n_steps):
            s = self.step(s)
        return s


def mesh_size(coords: np.ndarray, cells: np.ndarray) -> float:
    """h = 2 x (largest) circumradius over the cells, the convention of Sec. 6.1."""
    d = coords.shape[1]
    x = coords[cells]                              # [T, d+1, d]
    # circumcentre c solves 2 (x_k - x_0) . c = |x_k|^2 - |x_0|^2
    Amat = 2.0 * (x[:, 1:, :] - x[:, :1, :])
    rhs = (x[:, 1:, :] ** 2).sum(-1) - (x[:, :1, :] ** 2).sum(-1)
    c = np.linalg.solve(Amat, rhs[..., None])[..., 0]
    R = np.linalg.norm(x[:, 0, :] - c, axis=1)
    del d
    return float(2.0 * R.max())


def convergence_order(E_prev, E, h_prev, h):
    """k = ln(E_i / E_{i-1}) / ln(h_i / h_{i-1}) (Sec. 6.1)."""
    return float(np.log(E / E_prev) / np.log(h / h_prev))
