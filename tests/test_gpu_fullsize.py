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
"""
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
