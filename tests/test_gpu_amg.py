"""Multigrid-preconditioned pressure CG on the GPU.

The preconditioner changes how fast the pressure CG converges, not what it
converges to: steps with OASIS_PC_AMG must match the float64 oracle as the
Jacobi steps do (1e-10 for float64 at rtol 1e-12, 1e-6 per field for the mixed
path at rtol 1e-8).  The V-cycle itself must be symmetric and positive on the
complement of the constants, as CG requires.
"""
import numpy as np
import pytest

from oracle.ipcs import IPCS
from workloads import meshes as WM
from workloads import problems as WP

pytestmark = pytest.mark.gpu


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


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _run(pb, precision, pc, graph=1, rtol=None, guess=None, bicg_variant=0):
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    rt = rtol if rtol is not None else (1e-12 if precision == c.OASIS_FP64 else 1e-8)
    return IPCSRun(pb, precision=precision, rtol_u=rt, rtol_p=rt, use_graph=graph, pressure_pc=pc,
                   guess=c.OASIS_GUESS_PREV_PHI if guess is None else guess, bicg_variant=bicg_variant)


PROBLEMS = {
    "tg3d_8": lambda: WP.taylor_green_3d(8, dt=1e-2),
    "channel_8x7x6": lambda: WP.channel(nx=8, ny=7, nz=6),
    "stress_10_random": lambda: WP.stress_cube(10, ordering="random"),
    "tg2d_24": lambda: WP.taylor_green_2d(24),
}


@pytest.mark.parametrize("name", ["stress_10_random", "channel_8x7x6"])
def test_vcycle_symmetric_positive(name):
    import torch
    c = capi()
    pb = PROBLEMS[name]()
    run = _run(pb, c.OASIS_FP64, c.OASIS_PC_AMG)
    try:
        info = c.oasis_get_amg_info(run.solver)
        assert info["levels"] >= 2 and info["rows"][0] == pb.mesh.n_dofs
        assert all(a > b for a, b in zip(info["rows"], info["rows"][1:]))
        rng = np.random.default_rng(5)
        x = rng.normal(size=pb.mesh.n_dofs)
        y = rng.normal(size=pb.mesh.n_dofs)
        x -= x.mean()
        y -= y.mean()
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        U, W = torch.empty_like(X), torch.empty_like(Y)
        c.oasis_amg_apply(run.solver, X, U)
        c.oasis_amg_apply(run.solver, Y, W)
        u, w = U.cpu().numpy(), W.cpu().numpy()
        assert abs(x @ w - y @ u) <= 1e-11 * np.sqrt((x @ u) * (y @ w))
        assert x @ u > 0 and y @ w > 0
    finally:
        run.close()


@pytest.mark.parametrize("name", ["stress_10_random", "channel_8x7x6"])
def test_float32_vcycle_symmetric_and_close_to_float64(name):
    """The float32 cycle (its finest-level smoother reading K rounded to
    bfloat16) is symmetric and positive to float32 rounding, and within the
    smoother's few digits of the float64 cycle."""
    import torch
    c = capi()
    pb = PROBLEMS[name]()
    rng = np.random.default_rng(6)
    x = rng.normal(size=pb.mesh.n_dofs)
    y = rng.normal(size=pb.mesh.n_dofs)
    x -= x.mean()
    y -= y.mean()
    out = {}
    for prec, dt in ((c.OASIS_FP64, torch.float64), (c.OASIS_MIXED, torch.float32)):
        run = _run(pb, prec, c.OASIS_PC_AMG)
        try:
            X, Y = torch.from_numpy(x).to(dt).cuda(), torch.from_numpy(y).to(dt).cuda()
            U, W = torch.empty_like(X), torch.empty_like(Y)
            c.oasis_amg_apply(run.solver, X, U)
            c.oasis_amg_apply(run.solver, Y, W)
            out[prec] = (U.double().cpu().numpy(), W.double().cpu().numpy())
        finally:
            run.close()
    u, w = out[c.OASIS_MIXED]
    assert abs(x @ w - y @ u) <= 2e-6 * np.sqrt((x @ u) * (y @ w))
    assert x @ u > 0 and y @ w > 0
    u64, w64 = out[c.OASIS_FP64]
    # bfloat16 keeps 8 significant bits (relative rounding 2^-9) of each entry
    assert 1e-9 < relerr(u, u64) <= 2e-2
    assert 1e-9 < relerr(w, w64) <= 2e-2


@pytest.mark.parametrize("n,ordering", [(90, "rcm"), (96, "random")])
def test_float32_vcycle_on_packed_operators(n, ordering):
    """Meshes large enough that the float32 cycle reads its level-1 matrix and
    the level-0 transfers in pair-packed SELL-32 form (16-bit column offsets in
    RCM order, whole 32-bit columns in random order, where columns spread over
    the whole level): the cycle stays symmetric and positive to float32 rounding
    and within bfloat16's few digits of the float64 cycle (CSR, never packed)."""
    import torch
    c = capi()
    pb = WP.stress_cube(n, ordering=ordering)
    rng = np.random.default_rng(7)
    x = rng.normal(size=pb.mesh.n_dofs)
    y = rng.normal(size=pb.mesh.n_dofs)
    x -= x.mean()
    y -= y.mean()
    out = {}
    for prec, dt in ((c.OASIS_FP64, torch.float64), (c.OASIS_MIXED, torch.float32)):
        run = _run(pb, prec, c.OASIS_PC_AMG)
        try:
            info = c.oasis_get_amg_info(run.solver)
            X, Y = torch.from_numpy(x).to(dt).cuda(), torch.from_numpy(y).to(dt).cuda()
            U, W = torch.empty_like(X), torch.empty_like(Y)
            c.oasis_amg_apply(run.solver, X, U)
            c.oasis_amg_apply(run.solver, Y, W)
            out[prec] = (U.double().cpu().numpy(), W.double().cpu().numpy())
        finally:
            run.close()
    packed = info["packed"]
    # level 0: restriction and prolongation packed; level 1: its matrix packed
    assert packed[0] & 6 == 6 and packed[1] & 1, packed
    if ordering == "random":
        assert packed[0] & 48 == 48 and packed[1] & 8, packed      # 32-bit columns
    else:
        assert packed[0] & 32 == 0 and packed[1] & 8 == 0, packed  # 16-bit offsets
    u, w = out[c.OASIS_MIXED]
    assert abs(x @ w - y @ u) <= 2e-6 * np.sqrt((x @ u) * (y @ w))
    assert x @ u > 0 and y @ w > 0
    u64, w64 = out[c.OASIS_FP64]
    assert 1e-9 < relerr(u, u64) <= 2e-2
    assert 1e-9 < relerr(w, w64) <= 2e-2


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_amg_steps_match_oracle_fp64(name):
    c = capi()
    pb = PROBLEMS[name]()
    run = _run(pb, c.OASIS_FP64, c.OASIS_PC_AMG)
    try:
        st = run.step(3)
        u, p, _ = run.fields()
    finally:
        run.close()
    assert st.status == c.OASIS_OK
    s = IPCS(pb).run(3)
    assert relerr(u, s.u_nm1) <= 1e-10
    assert relerr(p, s.p) <= 1e-9


def test_amg_mixed_per_field_error_and_fewer_iterations():
    c = capi()
    pb = WP.taylor_green_3d(12)
    out = {}
    for pc in (c.OASIS_PC_JACOBI, c.OASIS_PC_AMG):
        run = _run(pb, c.OASIS_MIXED, pc)
        try:
            its = [run.step(1).it_p for _ in range(20)]
            out[pc] = (its, run.fields())
        finally:
            run.close()
    s = IPCS(pb).run(20)
    u, p, _ = out[c.OASIS_PC_AMG][1]
    for k in range(3):
        if np.abs(s.u_nm1[k]).max() > 0:
            assert relerr(u[k], s.u_nm1[k]) <= 1e-6
    assert relerr(p, s.p) <= 1e-6
    print("\nCG iterations per step, Jacobi:", out[c.OASIS_PC_JACOBI][0], "\nmultigrid:", out[c.OASIS_PC_AMG][0])
    assert sum(out[c.OASIS_PC_AMG][0]) * 3 < sum(out[c.OASIS_PC_JACOBI][0])


def test_amg_graph_equals_eager_bitwise():
    """Same bits from the graph and the eager step (the BiCGStab product shape is
    fixed: the autotuner of each solver could pick another summation order)."""
    c = capi()
    pb = WP.stress_cube(8, ordering="rcm")
    out = []
    for g in (1, 0):
        run = _run(pb, c.OASIS_MIXED, c.OASIS_PC_AMG, graph=g, bicg_variant=2)
        try:
            run.step(3)
            out.append(run.fields())
        finally:
            run.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
