"""Convenience wrapper around the C ABI: one mesh + one solver for a problem.

Argument marshalling only; the problem object needs the attributes ``mesh``
(dim, coords, cells, dof_of_vertex, n_dofs), ``nu``, ``dt``, ``f``,
``dirichlet``, ``u_nm1``, ``u_nm2``, ``p``, ``t0`` and ``g(t)``, and may carry
``perm`` (a dof renumbering for the library; fields stay in the problem's order).
"""
from __future__ import annotations

import numpy as np

from . import capi


class IPCSRun:
    def __init__(self, problem, precision=capi.OASIS_FP64, rtol_u=1e-12, rtol_p=1e-12, max_it_u=2000,
                 max_it_p=50000, inner_rtol=1e-4, batch_rhs=1, use_graph=0, guess=capi.OASIS_GUESS_ZERO,
                 spmv_variant=0, pressure_pc=0, inner_iters=1, convection=0, velocity_update=0,
                 scalars=True, stream=None, bicg_variant=0):
        pb = problem
        self.pb = pb
        self.stream = stream
        m = pb.mesh
        self.dim, self.n = m.dim, m.n_dofs
        self.mesh = capi.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs,
                                           perm=getattr(pb, "perm", None))
        capi.oasis_assemble_constant(self.mesh, stream)
        self.nnz = capi.oasis_mesh_info(self.mesh)[2]
        self.params = capi.make_params(pb.nu, pb.dt, tuple(pb.f), rtol_u, rtol_p, max_it_u, max_it_p,
                                       precision, inner_rtol, batch_rhs, use_graph, guess, spmv_variant,
                                       pressure_pc, inner_iters, convection, velocity_update, bicg_variant)
        self.solver = capi.oasis_solver_create(self.mesh, self.params, pb.dirichlet, stream)
        self.t = pb.t0
        capi.oasis_set_fields(self.solver, pb.u_nm1, pb.u_nm2, pb.p, pb.t0, False, stream)
        self.stats = []
        self.net = None
        self.ns = 0
        sc = getattr(pb, "scalars", None)
        if sc is not None and scalars:
            self.ns = sc.c0.shape[0]
            capi.oasis_solver_set_scalars(self.solver, sc.diffusivity, sc.source, sc.dirichlet)
            capi.oasis_set_scalar_fields(self.solver, sc.c0, False, stream)

    def set_dirichlet_for_next_step(self):
        if len(self.pb.dirichlet):
            capi.oasis_set_dirichlet(self.solver, self.pb.g(self.t + self.pb.dt), False, self.stream)
        if self.ns and len(self.pb.scalars.dirichlet):
            capi.oasis_set_scalar_dirichlet(self.solver, self.pb.scalars.g(self.t + self.pb.dt), False,
                                            self.stream)

    def scalar_fields(self):
        """c^n of every scalar, [ns, n] (host)."""
        return capi.oasis_get_scalar_fields(self.solver, self.ns, self.n, False, None, self.stream)

    def step(self, n_steps=1, want_stats=True, time_dependent_bc=True):
        st = None
        for _ in range(n_steps):
            if time_dependent_bc or self.t == self.pb.t0:
                self.set_dirichlet_for_next_step()
            st = capi.oasis_step(self.solver, self.stream, want_stats)
            self.t += self.pb.dt
            if st is not None:
                self.stats.append(st.as_dict())
        return st

    def attach_guess_net(self, net):
        """Use a GuessNet (or None) when the solver's guess is OASIS_GUESS_LEARNED."""
        capi.oasis_solver_set_guess_net(self.solver, None if net is None else net.handle)
        self.net = net

    def record_guess(self, on=True):
        capi.oasis_solver_record_guess(self.solver, on)

    def guess_sample(self):
        """(features [n][3], target [n]) of the last step, as new device tensors."""
        import torch
        feat = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
        target = torch.empty(self.n, dtype=torch.float32, device="cuda")
        capi.oasis_get_guess_sample(self.solver, feat, target, self.stream)
        return feat, target

    def fields(self):
        u, p, phi = capi.oasis_get_fields(self.solver, self.dim, self.n, False, stream=self.stream)
        return u, p, phi

    def tentative_system(self):
        return capi.oasis_get_tentative_system(self.solver, self.dim, self.n, self.nnz, self.stream)

    def close(self):
        if self.solver is not None:
            capi.oasis_solver_destroy(self.solver)
            self.solver = None
        if self.mesh is not None:
            capi.oasis_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
