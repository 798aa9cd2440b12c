"""Passive scalars (the scalar equation of Sec. 3) on the GPU against the oracle.

Each scalar is convected by ubar = 1.5 u^{n-1} - 0.5 u^{n-2} with a
Crank-Nicolson c~, its own diffusivity, source and Dirichlet set.  Tolerances
as for the velocity: float64 path 1e-10 relative L2 after each of 3 steps
(solves at rtol 1e-13); mixed path 1e-6 per scalar at rtol 1e-8.
"""
import numpy as np
import pytest

from oracle.ipcs import IPCS
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


def _perturbed(pb, seed=5):
    rng = np.random.default_rng(seed)
    u2 = pb.u_nm2 + 0.05 * rng.normal(size=pb.u_nm2.shape)
    u2[:, pb.dirichlet] = pb.u_nm1[:, pb.dirichlet]
    pb.u_nm2 = u2
    return pb


PROBLEMS = {
    "tg2d_8": lambda: WP.taylor_green_2d(8),
    "tg3d_6": lambda: WP.taylor_green_3d(6),
    "channel_6x6x4": lambda: WP.channel(nx=6, ny=6, nz=4),
    "stress_5_random": lambda: WP.stress_cube(5, ordering="random"),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("use_graph", [0, 1])
def test_scalars_match_oracle_fp64(name, use_graph):
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.with_scalars(_perturbed(PROBLEMS[name]()), ns=2)
    sc = pb.scalars
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=use_graph, guess=1)
    o = IPCS(pb)
    s = o.initial_state()
    try:
        for it in range(3):
            st = run.step()
            assert st.status == 0
            assert st.it_c > 0 and st.res_c <= 1e-13
            s = o.step(s)
            c = run.scalar_fields()
            assert relerr(c, s.c) < 1e-10, it
            np.testing.assert_array_equal(c[:, sc.dirichlet], sc.g(s.t))
            u, p, _ = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
    finally:
        run.close()


@pytest.mark.parametrize("pc", [0, 1])
def test_scalars_with_every_option(pc):
    """Scalars beside explicit convection (ubar still from both velocities), two
    inner iterations and the consistent-mass update, graph mode."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c_ = capi()
    pb = WP.with_scalars(_perturbed(PROBLEMS["channel_6x6x4"]()), ns=3, diffusivity=(0.0, 1e-3, 0.2),
                         source=(0.3, 0.0, -1.0))
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=1, guess=1, pressure_pc=pc, inner_iters=2,
                  convection=1, velocity_update=c_.OASIS_UPDATE_CONSISTENT)
    o = IPCS(pb, inner_iters=2, convection="abe", velocity_update="consistent")
    s = o.initial_state()
    try:
        for it in range(3):
            assert run.step().status == 0
            s = o.step(s)
            assert relerr(run.scalar_fields(), s.c) < 1e-10, it
            assert relerr(run.fields()[0], s.u_nm1) < 1e-10, it
    finally:
        run.close()


def test_uniform_advection_matches_oracle_and_exact():
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.uniform_advection_2d(n=16, dt=0.02)
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=1)
    try:
        run.step(10)
        c = run.scalar_fields()
    finally:
        run.close()
    s = IPCS(pb).run(10)
    assert relerr(c, s.c) < 1e-10
    exact = pb.scalars.exact(pb.mesh.dof_coords(), s.t)
    assert relerr(c, exact) < 0.05


def test_scalars_mixed_per_field():
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.with_scalars(WP.taylor_green_3d(10), ns=2)
    run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=1, pressure_pc=1, guess=1)
    try:
        for _ in range(10):
            st = run.step()
            assert st.status == 0 and st.res_c <= 1e-8
        c = run.scalar_fields()
    finally:
        run.close()
    s = IPCS(pb).run(10)
    for a in range(2):
        assert relerr(c[a], s.c[a]) <= 1e-6, a


def test_scalars_graph_equals_eager_bitwise():
    from paper_1602_03643_gb300.driver import IPCSRun
    out = []
    for g in (0, 1):
        pb = WP.with_scalars(WP.taylor_green_3d(6), ns=2)
        run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=g, bicg_variant=4)
        try:
            run.step(4)
            out.append(run.scalar_fields())
        finally:
            run.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_scalar_arguments_and_removal():
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.with_scalars(WP.taylor_green_3d(4), ns=1)
    run = IPCSRun(pb, rtol_u=1e-10, rtol_p=1e-10, use_graph=1)
    try:
        bad = [(np.ones(c.OASIS_MAX_SCALARS + 1), np.zeros(c.OASIS_MAX_SCALARS + 1), []),
               ([-1.0], [0.0], []),
               ([0.1], [0.0], [3, 3]),
               ([0.1], [0.0], [run.n])]
        for dif, src, dirs in bad:
            with pytest.raises(c.OasisError) as e:
                c.oasis_solver_set_scalars(run.solver, dif, src, dirs)
            assert e.value.code == c.OASIS_EINVAL
        assert run.step().status == 0
        # removing the scalars: the step runs without them, their API refuses
        c.oasis_solver_set_scalars(run.solver, [], [], [])
        run.ns = 0
        st = run.step()
        assert st.status == 0 and st.it_c == 0
        with pytest.raises(c.OasisError):
            c.oasis_get_scalar_fields(run.solver, 1, run.n)
    finally:
        run.close()
