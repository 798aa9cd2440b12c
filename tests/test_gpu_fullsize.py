"""The benchmark's own workload and launch configuration, checked at full size.

The oracle cannot run these steps (exact solves at 274,625 dofs), so the GPU
step is checked against properties that hold at any size, with the oracle's
float64 operators (oracle/p1.py, oracle/ipcs.py) built from the GPU's state:

  * the assembled A and initial residual b - A u^{n-1} of the next step equal
    the oracle's (float32 rounding);
  * the tentative velocity u^I (recovered from u^n and phi through the lumped
    update, Sec. 5) solves the oracle's tentative system A u^I = b (Algorithm 2);
  * phi solves the pressure-correction system K phi = -(1/dt) sum_k dP^k u^I
    projected on sum b = 0 (Sec. 5), and p is normalised to zero mean;
  * Dirichlet values hold.

Tolerances: the mixed path solves with float32 operators inside float64-quality
refinement to 1e-8; against the exact float64 operators the residuals are
bounded by the float32 rounding of A (~6e-8 relative) times the conditioning:
2e-6 of the initial residual for the velocity; the pressure right-hand side and
residual are formed with float-float operators, 1e-6 of b_phi.

The 2.1M-dof stress cube (both dof orderings, handed to the library as its
renumbering) and the 1.18M-dof channel are checked the same way, except that
the oracle assembles only the rows of a seeded sample of 4,000 dofs (the cells
incident to them form a sub-mesh on which those rows are complete and exact):
A, r0, K, dP^k and ML agree on the sampled rows, and the solve properties are
checked at full size with the library's float64 operators and its A.
"""
import dataclasses
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.ipcs import IPCS
from workloads import problems as WP

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03643_gb300 import build
    build.build()
    torch.cuda.init()


def capi():
    from paper_1602_03643_gb300 import capi as c
    return c


@pytest.fixture(scope="module")
def tg3d_64():
    pb = WP.taylor_green_3d(64, n_steps=200, rtol=1e-8)
    return pb, IPCS(pb)


@pytest.mark.parametrize("pc", ["amg", "jacobi"])
def test_tg3d_64_bench_configuration(tg3d_64, pc):
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb, o = tg3d_64
    D = o.disc
    run = IPCSRun(pb, precision=c.OASIS_MIXED, rtol_u=1e-8, rtol_p=1e-8, max_it_u=5000, max_it_p=200000,
                  inner_rtol=1e-4, use_graph=1, batch_rhs=1, guess=c.OASIS_GUESS_PREV_PHI,
                  pressure_pc=c.OASIS_PC_AMG if pc == "amg" else c.OASIS_PC_JACOBI)
    try:
        st1 = run.step(1)
        u1, p1, _ = run.fields()
        # the assembly of the next step alone (Algorithm 2 on the current state)
        run.set_dirichlet_for_next_step()
        A_gpu, r0_gpu = run.tentative_system()
        rp, col = c.oasis_mesh_get_pattern(run.mesh)
        st2 = run.step(1)
        u2, p2, phi2 = run.fields()
    finally:
        run.close()
    assert st1.status == c.OASIS_OK and st2.status == c.OASIS_OK
    t2 = 2 * pb.dt
    # the step-2 tentative system of the oracle, from the GPU's state after step 1
    A, b = o.tentative_system(u1, pb.u_nm1, p1, t2)
    Ag = sp.csr_matrix((A_gpu, col, rp), shape=A.shape)
    assert np.abs((Ag - A).data).max() <= 2e-7 * np.abs(A.data).max()
    r0 = np.stack([b[k] - A @ u1[k] for k in range(D.d)])
    assert np.abs(r0_gpu - r0).max() <= 1e-5 * np.abs(r0).max()
    # u^I from the lumped update u^n = u^I - dt dP^k phi / ML (interior rows)
    uI = np.stack([u2[k] + pb.dt * (D.G[k] @ phi2) / D.ML for k in range(D.d)])
    uI[:, pb.dirichlet] = u2[:, pb.dirichlet]
    for k in range(D.d):
        res = b[k] - A @ uI[k]
        assert np.linalg.norm(res) <= 2e-6 * np.linalg.norm(r0[k]), k
    np.testing.assert_allclose(u2[:, pb.dirichlet], pb.g(t2), rtol=0, atol=1e-12)
    # pressure correction
    bphi = -(1.0 / pb.dt) * sum(D.G[k] @ uI[k] for k in range(D.d))
    bphi -= bphi.mean()
    assert np.linalg.norm(D.K @ phi2 - bphi) <= 1e-6 * np.linalg.norm(bphi)
    assert abs(p2.mean()) <= 1e-9 * np.abs(p2).max()
    np.testing.assert_allclose(phi2, p2 - p1, rtol=0, atol=1e-12 * np.abs(p2).max())


# ------------------------------------------------------------------ sampled-row checks
def _sub_problem(pb, rows):
    """The problem restricted to the cells incident to `rows` (dof numbering and
    Dirichlet data unchanged): the oracle's rows for those dofs are complete."""
    from workloads.meshes import Mesh
    m = pb.mesh
    cd = m.dof_of_vertex[m.cells]
    mark = np.zeros(m.n_dofs, dtype=bool)
    mark[rows] = True
    keep = mark[cd].any(axis=1)
    sub = Mesh(m.dim, m.coords, np.ascontiguousarray(m.cells[keep]), m.dof_of_vertex, m.n_dofs,
               dict(m.boundary_dofs))
    return dataclasses.replace(pb, mesh=sub, perm=None)


def _rows_close(got, want, rows, scale, tol):
    d = (got[rows] - want[rows]).tocsr()
    return (np.abs(d.data).max() if d.nnz else 0.0) <= tol * scale


def check_full_size(pb, n_sample=4000, seed=21):
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    run = IPCSRun(pb, precision=c.OASIS_MIXED, rtol_u=1e-8, rtol_p=1e-8, max_it_u=20000, max_it_p=200000,
                  inner_rtol=1e-4, use_graph=1, batch_rhs=1, guess=c.OASIS_GUESS_PREV_PHI,
                  pressure_pc=c.OASIS_PC_AMG)
    try:
        st1 = run.step(1)
        u1, p1, _ = run.fields()
        run.set_dirichlet_for_next_step()
        A_gpu, r0_gpu = run.tentative_system()
        rp, col = c.oasis_mesh_get_pattern(run.mesh)
        K = sp.csr_matrix((c.oasis_mesh_get_matrix(run.mesh, c.OASIS_MAT_K), col, rp), shape=(run.n, run.n))
        G = [sp.csr_matrix((c.oasis_mesh_get_matrix(run.mesh, c.OASIS_MAT_G0 + k), col, rp), shape=(run.n, run.n))
             for k in range(run.dim)]
        ML = c.oasis_mesh_get_matrix(run.mesh, -1)
        st2 = run.step(1)
        u2, p2, phi2 = run.fields()
    finally:
        run.close()
    assert st1.status == c.OASIS_OK and st2.status == c.OASIS_OK, (st1.as_dict(), st2.as_dict())
    N, D, t2 = pb.mesh.n_dofs, pb.mesh.dim, pb.t0 + 2 * pb.dt
    Ag = sp.csr_matrix((A_gpu, col, rp), shape=(N, N))
    # sampled rows: the oracle's A, r0 and constant operators
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([rng.choice(N, n_sample, replace=False), [0, N - 1],
                                     rng.choice(pb.dirichlet, 50, replace=False)]))
    o = IPCS(_sub_problem(pb, rows))
    A_o, b_o = o.tentative_system(u1, pb.u_nm1, p1, t2)
    assert _rows_close(Ag, A_o, rows, np.abs(A_o[rows].data).max(), 2e-7)
    r0_o = np.stack([b_o[k] - A_o @ u1[k] for k in range(D)])
    # r0 = f ML - (C + nu K) u^{n-1} - dP^k p* is formed from float32 shares: its
    # error scales with the size of those terms, which cancel to a much smaller r0
    Do = o.disc
    interior = np.setdiff1d(rows, pb.dirichlet)
    CK = abs(2.0 * (A_o - Do.M / pb.dt))[interior]
    scale = max(float((CK @ np.abs(u1[k]) + abs(Do.G[k])[interior] @ np.abs(p1)).max()) for k in range(D))
    assert np.abs(r0_gpu[:, rows] - r0_o[:, rows]).max() <= 1e-5 * scale
    assert _rows_close(K, Do.K, rows, np.abs(Do.K[rows].data).max(), 1e-13)
    for k in range(D):
        assert _rows_close(G[k], Do.G[k], rows, np.abs(Do.G[k][rows].data).max(), 1e-13), k
    np.testing.assert_allclose(ML[rows], Do.ML[rows], rtol=1e-13)
    # full size: the tentative velocity solves A u^I = b (b - A u^I = r0 - A (u^I - u^{n-1}))
    uI = np.stack([u2[k] + pb.dt * (G[k] @ phi2) / ML for k in range(D)])
    uI[:, pb.dirichlet] = u2[:, pb.dirichlet]
    for k in range(D):
        res = r0_gpu[k] - Ag @ (uI[k] - u1[k])
        assert np.linalg.norm(res) <= 2e-6 * np.linalg.norm(r0_gpu[k]), k
    np.testing.assert_allclose(u2[:, pb.dirichlet], pb.g(t2), rtol=0, atol=1e-12)
    # the pressure correction solves K phi = b_phi (projected), p has zero mean
    bphi = -(1.0 / pb.dt) * sum(G[k] @ uI[k] for k in range(D))
    bphi -= bphi.mean()
    assert np.linalg.norm(K @ phi2 - bphi) <= 1e-6 * np.linalg.norm(bphi)
    assert abs(p2.mean()) <= 1e-9 * np.abs(p2).max()
    np.testing.assert_allclose(phi2, p2 - p1, rtol=0, atol=1e-12 * np.abs(p2).max())
    return st2


@pytest.fixture(scope="module")
def stress128():
    return WP.stress_cube(128, ordering="natural")


@pytest.mark.parametrize("ordering", ["rcm", "random"])
def test_stress128_bench_configuration(stress128, ordering):
    """The 128^3 jittered cube (2,146,689 dofs, 12.6M cells), the library storing
    it in RCM or in random dof order (the caller's arrays stay in mesh order)."""
    from workloads import meshes as WM
    perm = WM.rcm_permutation(stress128.mesh) if ordering == "rcm" else \
        WM.random_permutation(stress128.mesh.n_dofs, 44)
    check_full_size(dataclasses.replace(stress128, perm=perm))


def test_channel_bench_configuration():
    """The 128 x 96 x 96 channel (1,179,648 dofs, periodic in x and z, stretched
    walls), mixed precision, multigrid, graph: the first two steps."""
    check_full_size(WP.channel())
