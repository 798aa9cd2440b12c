"""P1 simplex element integrals and global assembly (CPU, float64).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously correct
restatement of the scheme; only the tests, the smoke check and the CPU
baseline of the benchmark may import it.  It shares no code with the CUDA path.

Every integral here is the textbook closed form for linear Lagrange elements
on a simplex T with barycentric coordinates lambda_0..lambda_d:

  int_T lambda_i lambda_j dx = |T| (1 + delta_ij) / ((d+1)(d+2))
  int_T lambda_i dx          = |T| / (d+1)
  grad lambda_k, k >= 1      = row k-1 of J^{-1},  grad lambda_0 = -sum_k grad lambda_k

with J = [x_1 - x_0, ..., x_d - x_0].  The matrices are those of Sec. 5:
  M_ij   = int phi_j phi_i                       (mass)
  K_ij   = int grad phi_j . grad phi_i           (stiffness)
  G^k_ij = int d_k phi_j phi_i                   (pressure-gradient matrices dP^k, Eq. 31)
  C_ij   = int (ubar . grad phi_j) phi_i         (convection, Sec. 5)
All are assembled by summing element matrices into a scipy COO matrix and
converting to CSR (duplicates summed): no blocking, colouring or reordering.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def geometry(coords: np.ndarray, cells: np.ndarray):
    """Per-cell volume |T| [T] and barycentric gradients [T, d+1, d]."""
    d = coords.shape[1]
    x0 = coords[cells[:, 0]]
    J = np.stack([coords[cells[:, k + 1]] - x0 for k in range(d)], axis=2)   # columns x_k - x_0
    det = np.linalg.det(J)
    if np.any(det == 0):
        raise ValueError("degenerate cell")
    vol = np.abs(det) / math.factorial(d)
    Jinv = np.linalg.inv(J)                     # [T, d, d]
    grads = np.empty((cells.shape[0], d + 1, d))
    grads[:, 1:, :] = Jinv                      # row k-1 of J^{-1} is grad lambda_k
    grads[:, 0, :] = -Jinv.sum(axis=1)
    return vol, grads


def element_mass(vol: np.ndarray, d: int) -> np.ndarray:
    """M^T_ij = |T| (1 + delta_ij) / ((d+1)(d+2))  -> [T, d+1, d+1]."""
    base = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    return vol[:, None, None] * base[None]


def element_stiffness(vol, grads):
    """K^T_ij = |T| grad lambda_i . grad lambda_j."""
    return vol[:, None, None] * np.einsum("tik,tjk->tij", grads, grads)


def element_gradient(vol, grads, k):
    """G^{k,T}_ij = int_T d_k lambda_j lambda_i = d_k lambda_j |T| / (d+1)."""
    d = grads.shape[2]
    col = grads[:, :, k] * (vol / (d + 1))[:, None]      # [T, j]
    return np.broadcast_to(col[:, None, :], (grads.shape[0], d + 1, d + 1)).copy()


def element_convection(vol, grads, ubar_cell):
    """C^T_ij = int_T (ubar . grad lambda_j) lambda_i with ubar = sum_m ubar_m lambda_m.

    ubar . grad lambda_j is sum_m (ubar_m . grad lambda_j) lambda_m, so
    C^T_ij = sum_m (ubar_m . grad lambda_j) int lambda_m lambda_i
           = sum_m M^T_im (ubar_m . grad lambda_j).
    ``ubar_cell`` is [T, d+1 (vertex m), d (component)].
    """
    d = grads.shape[2]
    Me = element_mass(vol, d)                              # [T, i, m]
    dots = np.einsum("tmk,tjk->tmj", ubar_cell, grads)     # ubar_m . grad lambda_j
    return np.einsum("tim,tmj->tij", Me, dots)


class Discretization:
    """Mesh-dependent constants of the P1-P1 scheme (Sec. 5 preassembly)."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.d = mesh.dim
        self.N = mesh.n_dofs
        self.cdofs = mesh.dof_of_vertex[mesh.cells].astype(np.int64)     # [T, d+1]
        self.vol, self.grads = geometry(mesh.coords, mesh.cells)
        d1 = self.d + 1
        self._rows = np.repeat(self.cdofs, d1, axis=1).ravel()
        self._cols = np.tile(self.cdofs, (1, d1)).ravel()
        self.M = self.assemble(element_mass(self.vol, self.d))
        self.K = self.assemble(element_stiffness(self.vol, self.grads))
        self.G = [self.assemble(element_gradient(self.vol, self.grads, k)) for k in range(self.d)]
        # int phi_i dx, the lumped mass (row sums of M, Sec. 5 velocity update)
        self.ML = np.bincount(self.cdofs.ravel(), weights=np.repeat(self.vol / d1, d1),
                              minlength=self.N)

    def assemble(self, elem: np.ndarray) -> sp.csr_matrix:
        """Sum element matrices [T, d+1, d+1] (row i, col j) into an N x N CSR."""
        A = sp.coo_matrix((elem.ravel(), (self._rows, self._cols)), shape=(self.N, self.N)).tocsr()
        A.sum_duplicates()
        A.sort_indices()
        return A

    def convection(self, ubar: np.ndarray) -> sp.csr_matrix:
        """C(ubar) for ubar given per dof as [d, N]."""
        ubar_cell = np.transpose(ubar[:, self.cdofs], (1, 2, 0))          # [T, d+1, d]
        return self.assemble(element_convection(self.vol, self.grads, ubar_cell))

    def pattern(self) -> sp.csr_matrix:
        """The shared sparsity pattern of all matrices (structural, incl. zeros)."""
        P = sp.coo_matrix((np.ones(self._rows.size), (self._rows, self._cols)),
                          shape=(self.N, self.N)).tocsr()
        P.sum_duplicates()
        P.sort_indices()
        return P
