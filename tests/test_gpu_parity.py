"""GPU path (through the C ABI) against the CPU float64 oracle, element by element.

Tolerances: float64 path -- matrices to 1e-13 relative, one step to 1e-10,
100 steps to 1e-9 relative L2 (solves at rtol 1e-12 on both sides); the
mixed path -- 1e-6 relative L2 per field at rtol 1e-8.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import p1
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


def csr_from(mesh_h, values):
    c = capi()
    rp, col = c.oasis_mesh_get_pattern(mesh_h)
    n = rp.size - 1
    return sp.csr_matrix((values, col, rp), shape=(n, n))


MESHES = {
    "sq_7x5": lambda: WM.box_mesh_2d(7, 5, 0.0, 1.3, -0.5, 0.5),
    "cube_5x4x3": lambda: WM.box_mesh_3d(5, 4, 3, hi=(1.0, 0.7, 0.6)),
    "jitter_6": lambda: WM.jitter_interior(WM.box_mesh_3d(6, 6, 6), 0.2, 1 / 6, seed=4),
    "periodic_channel": lambda: WM.box_mesh_3d(6, 5, 4, lo=(0, -1, 0), hi=(2, 1, 1),
                                               y_coords=WP.channel_y(6), periodic=(True, False, True)),
    "random_perm": lambda: WM.renumber_dofs(WM.box_mesh_3d(5, 5, 5), WM.random_permutation(216, 44)),
}


@pytest.mark.parametrize("renumber", [False, True])
@pytest.mark.parametrize("name", list(MESHES))
def test_constant_matrices_match_oracle(name, renumber):
    """Every constant matrix against the oracle's, in the caller's order; with
    `renumber` the library stores the mesh under a seeded random dof permutation
    (the perm of oasis_mesh_create) and must still return the caller's order."""
    c = capi()
    m = MESHES[name]()
    D = p1.Discretization(m)
    perm = WM.random_permutation(m.n_dofs, 17) if renumber else None
    h = c.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs, perm=perm)
    try:
        c.oasis_assemble_constant(h)
        rp, col = c.oasis_mesh_get_pattern(h)
        P = D.pattern()
        np.testing.assert_array_equal(rp, P.indptr)
        np.testing.assert_array_equal(col, P.indices)
        for which, ref in [(c.OASIS_MAT_M, D.M), (c.OASIS_MAT_K, D.K)] + \
                          [(c.OASIS_MAT_G0 + k, D.G[k]) for k in range(m.dim)]:
            got = c.oasis_mesh_get_matrix(h, which)
            np.testing.assert_allclose(got, ref.data, rtol=0, atol=1e-13 * np.abs(ref.data).max())
        np.testing.assert_allclose(c.oasis_mesh_get_matrix(h, -1), D.ML, rtol=1e-13)
    finally:
        c.oasis_mesh_destroy(h)


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_spmv_f64_f32(lanes):
    import torch
    c = capi()
    m = WM.jitter_interior(WM.box_mesh_3d(9, 8, 7), 0.2, 1 / 9, seed=2)
    D = p1.Discretization(m)
    h = c.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs)
    try:
        c.oasis_assemble_constant(h)
        rng = np.random.default_rng(lanes)
        x = rng.normal(size=m.n_dofs)
        for which, ref in [(c.OASIS_MAT_K, D.K), (c.OASIS_MAT_G1, D.G[1])]:
            xd = torch.tensor(x, device="cuda")
            yd = torch.empty_like(xd)
            c.oasis_spmv_f64(h, which, xd, yd, lanes)
            torch.cuda.synchronize()
            want = ref @ x
            np.testing.assert_allclose(yd.cpu().numpy(), want, rtol=0, atol=1e-13 * np.abs(want).max())
            xf = xd.float()
            yf = torch.empty_like(xf)
            c.oasis_spmv_f32(h, which, xf, yf, lanes)
            torch.cuda.synchronize()
            assert relerr(yf.cpu().numpy(), want) < 2e-6
    finally:
        c.oasis_mesh_destroy(h)


@pytest.mark.parametrize("name", ["jitter_6", "random_perm", "sq_7x5"])
def test_spmv_dot_f64(name):
    import torch
    c = capi()
    m = MESHES[name]()
    D = p1.Discretization(m)
    h = c.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs)
    try:
        c.oasis_assemble_constant(h)
        x = np.random.default_rng(3).normal(size=m.n_dofs)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        xy = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            c.oasis_spmv_dot_f64(h, c.OASIS_MAT_K, xd, yd, xy)
            torch.cuda.synchronize()
            want = D.K @ x
            np.testing.assert_allclose(yd.cpu().numpy(), want, rtol=0, atol=1e-13 * np.abs(want).max())
            assert abs(xy.item() - x @ want) <= 1e-12 * abs(x) @ abs(want)
    finally:
        c.oasis_mesh_destroy(h)


def _perturbed_state(pb, seed=5):
    """Make u^{n-2} differ from u^{n-1} so that ubar exercises both."""
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
@pytest.mark.parametrize("precision", [0, 1])
def test_tentative_system_alg2_matches_naive(name, precision):
    """Algorithm 2 (fused on the GPU) gives the naive A and b - A u^{n-1}."""
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = _perturbed_state(PROBLEMS[name]())
    run = IPCSRun(pb, precision=precision)
    try:
        run.set_dirichlet_for_next_step()
        A_gpu, r0_gpu = run.tentative_system()
        o = IPCS(pb)
        A_ref, b_ref = o.tentative_system(pb.u_nm1, pb.u_nm2, pb.p, pb.t0 + pb.dt)
        A_ref = A_ref.tocsr()
        A_ref.sort_indices()
        Ag = csr_from(run.mesh, A_gpu)
        tol = 1e-13 if precision == 0 else 2e-6
        diff = (Ag - A_ref).tocsr()
        assert abs(diff).max() <= tol * abs(A_ref).max()
        r0_ref = b_ref - np.stack([A_ref @ pb.u_nm1[k] for k in range(pb.mesh.dim)])
        scale = np.abs(r0_ref).max()
        tol_r = 1e-11 if precision == 0 else 1e-5
        np.testing.assert_allclose(r0_gpu, r0_ref, rtol=0, atol=tol_r * scale)
    finally:
        run.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("use_graph", [0, 1])
def test_fp64_steps_match_oracle(name, use_graph):
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = _perturbed_state(PROBLEMS[name]())
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=use_graph)
    o = IPCS(pb)
    s = o.initial_state()
    try:
        for it in range(3):
            st = run.step()
            assert st.status == 0
            s = o.step(s)
            u, p, phi = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
            assert relerr(phi, s.phi) < 1e-9, it
    finally:
        run.close()


def test_fp64_100_steps_tg2d_32():
    """The float64 GPU path stays within 1e-9 (relative L2) of the oracle over 100 steps."""
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.taylor_green_2d(32)
    run = IPCSRun(pb, rtol_u=1e-12, rtol_p=1e-12, use_graph=1)
    try:
        run.step(100, want_stats=False)
        u, p, _ = run.fields()
    finally:
        run.close()
    s = IPCS(pb).run(100)
    assert relerr(u, s.u_nm1) <= 1e-9
    assert relerr(p, s.p) <= 1e-9


@pytest.mark.parametrize("bicg_variant", [1, 2, 7])
def test_graph_equals_eager_bitwise(bicg_variant):
    """Same bits from the graph and the eager step, for a row-tile and a
    row-split BiCGStab product (each solver would otherwise tune its own)."""
    from paper_1602_03643_gb300.driver import IPCSRun
    out = []
    for g in (0, 1):
        pb = WP.taylor_green_3d(8)
        run = IPCSRun(pb, rtol_u=1e-10, rtol_p=1e-10, use_graph=g, precision=1, bicg_variant=bicg_variant)
        run.step(4)
        out.append(run.fields())
        run.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("pb_name", ["tg3d_8", "stress_9_rcm", "channel_6x5x6"])
def test_bicg_product_16bit_columns_bitwise(pb_name):
    """The BiCGStab product shape reading its columns as 16-bit offsets from the
    row (modulo n: periodic neighbours wrap) gives the same bits as the same
    shape reading int32 columns: the decoded columns are the same and the
    products are added in the same order (small meshes: the same grid)."""
    from paper_1602_03643_gb300.driver import IPCSRun
    make = {"tg3d_8": lambda: WP.taylor_green_3d(8),
            "stress_9_rcm": lambda: WP.stress_cube(9, ordering="rcm"),
            "channel_6x5x6": lambda: WP.channel(nx=6, ny=5, nz=6)}[pb_name]
    out = []
    for v in (3, 7):                          # (4 lanes, 4 rows, 5 blocks/SM): int32, 16-bit columns
        run = IPCSRun(make(), rtol_u=1e-10, rtol_p=1e-10, use_graph=1, precision=1, bicg_variant=v)
        try:
            tun = capi().oasis_get_tuning(run.solver)
            cand = tun["bicg_candidates"][v - 1]
            assert (cand["lanes"], cand["rows"], cand["min_blocks"], cand["col16"]) == (4, 4, 5, int(v == 7))
            st = run.step(3)
            assert st.status == 0
            out.append(run.fields())
        finally:
            run.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", [0, 1])
def test_explicit_convection_tentative_system(name, precision):
    """Explicit Adams-Bashforth convection (Eq. 21): A = M/dt + nu K/2 and the
    initial tentative residual b - A u^{n-1} against the oracle's."""
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = _perturbed_state(PROBLEMS[name]())
    run = IPCSRun(pb, precision=precision, convection=1)
    try:
        run.set_dirichlet_for_next_step()
        A_gpu, r0_gpu = run.tentative_system()
        o = IPCS(pb, convection="abe")
        A_ref, b_ref = o.tentative_system(pb.u_nm1, pb.u_nm2, pb.p, pb.t0 + pb.dt)
        A_ref = A_ref.tocsr()
        A_ref.sort_indices()
        Ag = csr_from(run.mesh, A_gpu)
        tol = 1e-13 if precision == 0 else 2e-6
        assert abs((Ag - A_ref).tocsr()).max() <= tol * abs(A_ref).max()
        r0_ref = b_ref - np.stack([A_ref @ pb.u_nm1[k] for k in range(pb.mesh.dim)])
        tol_r = 1e-11 if precision == 0 else 1e-5
        np.testing.assert_allclose(r0_gpu, r0_ref, rtol=0, atol=tol_r * np.abs(r0_ref).max())
    finally:
        run.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("use_graph", [0, 1])
def test_explicit_convection_steps_match_oracle_fp64(name, use_graph):
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = _perturbed_state(PROBLEMS[name]())
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=use_graph, convection=1)
    o = IPCS(pb, convection="abe")
    s = o.initial_state()
    try:
        for it in range(3):
            st = run.step()
            assert st.status == 0
            s = o.step(s)
            u, p, phi = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
    finally:
        run.close()


def test_explicit_convection_mixed_per_field():
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.taylor_green_3d(10)
    run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=1, pressure_pc=1, convection=1)
    try:
        run.step(10)
        u, p, _ = run.fields()
    finally:
        run.close()
    s = IPCS(pb, convection="abe").run(10)
    for k in range(3):
        if np.abs(s.u_nm1[k]).max() > 0:
            assert relerr(u[k], s.u_nm1[k]) <= 1e-6, k
    assert relerr(p, s.p) <= 1e-6


@pytest.mark.parametrize("name", ["tg2d_8", "tg3d_6", "channel_6x6x4"])
@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("pc", [0, 1])
def test_inner_iterations_match_oracle_fp64(name, use_graph, pc):
    """Algorithm 1 with 3 inner iterations per step (p* advanced between the
    repetitions, the last increment in the update) against the oracle."""
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = _perturbed_state(PROBLEMS[name]())
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=use_graph, inner_iters=3, pressure_pc=pc,
                  guess=1)
    o = IPCS(pb, inner_iters=3)
    s = o.initial_state()
    try:
        for it in range(2):
            st = run.step()
            assert st.status == 0
            s = o.step(s)
            u, p, phi = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
            assert relerr(phi, s.phi) < 1e-8, it
    finally:
        run.close()


def test_inner_iterations_mixed_per_field():
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.taylor_green_3d(10)
    run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=1, inner_iters=2, pressure_pc=1)
    try:
        run.step(5)
        u, p, _ = run.fields()
    finally:
        run.close()
    s = IPCS(pb, inner_iters=2).run(5)
    for k in range(3):
        if np.abs(s.u_nm1[k]).max() > 0:
            assert relerr(u[k], s.u_nm1[k]) <= 1e-6, k
    assert relerr(p, s.p) <= 1e-6


@pytest.mark.parametrize("name", list(PROBLEMS) + ["tg2d_periodic_8"])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_consistent_update_matches_oracle_fp64(name, use_graph):
    """Consistent-mass velocity update (Sec. 5): M u^n = M u^I - dt dP^k phi with
    Dirichlet rows u^n = g, against the oracle's direct solve; the lumped oracle
    is farther away than the tolerance, so the comparison tells the two apart."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    # the periodic case has no Dirichlet rows: the mass CG runs on all of M
    make = PROBLEMS.get(name, lambda: WP.taylor_green_2d_periodic(8, dt=0.05))
    pb = _perturbed_state(make())
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=use_graph, guess=1,
                  velocity_update=c.OASIS_UPDATE_CONSISTENT)
    o = IPCS(pb, velocity_update="consistent")
    ol = IPCS(pb)
    s, sl = o.initial_state(), ol.initial_state()
    try:
        for it in range(3):
            st = run.step()
            assert st.status == 0
            assert st.it_m > 0
            assert max(st.res_m[:pb.mesh.dim]) <= 1e-13
            s, sl = o.step(s), ol.step(sl)
            u, p, phi = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
            assert relerr(sl.u_nm1, s.u_nm1) > 1e-8, it
    finally:
        run.close()


@pytest.mark.parametrize("pc", [0, 1])
def test_consistent_update_with_inner_iterations_and_explicit_convection(pc):
    """All three options at once: explicit convection (Eq. 21), 2 inner
    iterations (Algorithm 1), consistent-mass update, graph mode."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = _perturbed_state(PROBLEMS["channel_6x6x4"]())
    run = IPCSRun(pb, rtol_u=1e-13, rtol_p=1e-13, use_graph=1, guess=1, pressure_pc=pc, inner_iters=2,
                  convection=1, velocity_update=c.OASIS_UPDATE_CONSISTENT)
    o = IPCS(pb, inner_iters=2, convection="abe", velocity_update="consistent")
    s = o.initial_state()
    try:
        for it in range(3):
            assert run.step().status == 0
            s = o.step(s)
            u, p, _ = run.fields()
            assert relerr(u, s.u_nm1) < 1e-10, it
            assert relerr(p, s.p) < 1e-10, it
    finally:
        run.close()


def test_consistent_update_mixed_per_field():
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.taylor_green_3d(10)
    run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=1, pressure_pc=1, guess=1,
                  velocity_update=c.OASIS_UPDATE_CONSISTENT)
    try:
        for _ in range(10):
            st = run.step()
            assert st.status == 0 and st.it_m > 0
            assert max(st.res_m) <= 1e-6
        u, p, _ = run.fields()
    finally:
        run.close()
    s = IPCS(pb, velocity_update="consistent").run(10)
    for k in range(3):
        if np.abs(s.u_nm1[k]).max() > 0:
            assert relerr(u[k], s.u_nm1[k]) <= 1e-6, k
    assert relerr(p, s.p) <= 1e-6


def test_consistent_update_graph_equals_eager_bitwise():
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    out = []
    for g in (0, 1):
        pb = WP.taylor_green_3d(6)
        run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=g,
                      velocity_update=c.OASIS_UPDATE_CONSISTENT, bicg_variant=3)
        try:
            run.step(4)
            out.append(run.fields())
        finally:
            run.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("pc", [0, 1])
@pytest.mark.parametrize("precision,case", [(0, "stress"), (1, "stress"), (1, "channel")])
def test_cg_shapes_bitwise_equal_and_tuned(precision, case, pc):
    """Every candidate shape of the pressure-CG product kernel -- the fused
    Jacobi iteration (pc 0; including 16-bit column offsets taken modulo n,
    which the periodic channel needs) or the multigrid CG product (pc 1) --
    gives the same bits; the autotuner timed every candidate and kept the
    fastest."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.stress_cube(12, ordering="random") if case == "stress" else WP.channel(nx=12, ny=9, nz=10)
    run = IPCSRun(pb, precision=precision, rtol_u=1e-9, rtol_p=1e-9, use_graph=1, pressure_pc=pc)
    try:
        tun = c.oasis_get_tuning(run.solver)
    finally:
        run.close()
    cands = tun["candidates"]
    assert len(cands) >= 3
    assert all(x["us"] > 0 for x in cands)
    assert cands[tun["chosen"] - 1]["us"] == min(x["us"] for x in cands)
    out = []
    for v in range(1, len(cands) + 1):
        run = IPCSRun(pb, precision=precision, rtol_u=1e-9, rtol_p=1e-9, use_graph=1, spmv_variant=v,
                      pressure_pc=pc, bicg_variant=1)
        try:
            assert c.oasis_get_tuning(run.solver)["chosen"] == v
            st = run.step(3)
            out.append((run.fields(), st.it_p))
        finally:
            run.close()
    for f, it in out[1:]:
        assert it == out[0][1]
        for a, b in zip(f, out[0][0]):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_bicg_product_shapes_agree_with_oracle_and_tuned(precision):
    """Every candidate shape of the batched BiCGStab product (row tiles, or G
    lanes per row with several rows in flight) gives steps that match the
    oracle (the shapes differ in summation order only); the autotuner timed
    every candidate and kept the fastest; a forced shape is kept."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.stress_cube(10, ordering="random")
    rtol = 1e-12 if precision == 0 else 1e-9
    run = IPCSRun(pb, precision=precision, rtol_u=rtol, rtol_p=rtol, use_graph=1, pressure_pc=c.OASIS_PC_AMG)
    try:
        tun = c.oasis_get_tuning(run.solver)
    finally:
        run.close()
    cands = tun["bicg_candidates"]
    assert len(cands) >= 4 and cands[0]["lanes"] == 0
    assert all(x["us"] > 0 for x in cands)
    assert cands[tun["bicg_chosen"] - 1]["us"] == min(x["us"] for x in cands)
    ref = IPCS(pb).run(3)
    tol = 1e-10 if precision == 0 else 1e-6
    for v in range(1, len(cands) + 1):
        run = IPCSRun(pb, precision=precision, rtol_u=rtol, rtol_p=rtol, use_graph=1,
                      pressure_pc=c.OASIS_PC_AMG, bicg_variant=v)
        try:
            assert c.oasis_get_tuning(run.solver)["bicg_chosen"] == v
            st = run.step(3)
            u, p, _ = run.fields()
        finally:
            run.close()
        assert st.status == c.OASIS_OK
        assert relerr(u, ref.u_nm1) <= tol, (v, relerr(u, ref.u_nm1))
        assert relerr(p, ref.p) <= 10 * tol, (v, relerr(p, ref.p))


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_unbatched(precision):
    from paper_1602_03643_gb300.driver import IPCSRun
    out = []
    for batch in (1, 0):
        pb = WP.channel(nx=8, ny=7, nz=6)
        run = IPCSRun(pb, rtol_u=1e-12 if precision == 0 else 1e-9, rtol_p=1e-12 if precision == 0 else 1e-9,
                      batch_rhs=batch, precision=precision)
        run.step(3)
        out.append(run.fields())
        run.close()
    assert relerr(out[0][0], out[1][0]) < (1e-10 if precision == 0 else 1e-7)
    assert relerr(out[0][1], out[1][1]) < (1e-9 if precision == 0 else 1e-6)


def test_mixed_precision_per_field_error():
    """Mixed precision at rtol 1e-8 against the float64 oracle (exact solves): <= 1e-6 per field."""
    from paper_1602_03643_gb300.driver import IPCSRun
    pb = WP.taylor_green_3d(12)
    run = IPCSRun(pb, precision=1, rtol_u=1e-8, rtol_p=1e-8, use_graph=1)
    try:
        run.step(20)
        u, p, _ = run.fields()
    finally:
        run.close()
    s = IPCS(pb).run(20)
    for k in range(3):
        if np.abs(s.u_nm1[k]).max() > 0:
            assert relerr(u[k], s.u_nm1[k]) <= 1e-6, k
    assert relerr(p, s.p) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_permutation_invariance(precision):
    """A dof renumbering handed to oasis_mesh_create (random, RCM) changes the
    library's internal order only: the same caller-order arrays go in, and the
    fields, the pattern and the matrices come out in the caller's order, equal to
    the unrenumbered run to the solvers' tolerance (sums run in another order).
    No renumbering happens on the host."""
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    rtol = 1e-12 if precision == 0 else 1e-8
    out = {}
    for ordering in ("natural", "random", "rcm"):
        pb = WP.stress_cube(6, ordering=ordering)
        assert (pb.perm is None) == (ordering == "natural")
        run = IPCSRun(pb, precision=precision, rtol_u=rtol, rtol_p=rtol, use_graph=1,
                      pressure_pc=c.OASIS_PC_AMG if precision else c.OASIS_PC_JACOBI,
                      guess=c.OASIS_GUESS_PREV_PHI)
        try:
            A, r0 = run.tentative_system()
            run.step(3)
            rp, col = c.oasis_mesh_get_pattern(run.mesh)
            K = c.oasis_mesh_get_matrix(run.mesh, c.OASIS_MAT_K)
            ML = c.oasis_mesh_get_matrix(run.mesh, -1)
            out[ordering] = (run.fields(), rp, col, K, ML, A, r0)
        finally:
            run.close()
    (u1, p1, f1), rp1, col1, K1, ML1, A1, r01 = out["natural"]
    tol_u = 1e-10 if precision == 0 else 1e-6
    for ordering in ("random", "rcm"):
        (u2, p2, f2), rp2, col2, K2, ML2, A2, r02 = out[ordering]
        np.testing.assert_array_equal(rp2, rp1)
        np.testing.assert_array_equal(col2, col1)
        np.testing.assert_allclose(K2, K1, rtol=0, atol=1e-14 * np.abs(K1).max())
        np.testing.assert_allclose(ML2, ML1, rtol=1e-14)
        np.testing.assert_allclose(A2, A1, rtol=0, atol=(1e-13 if precision == 0 else 1e-6) * np.abs(A1).max())
        np.testing.assert_allclose(r02, r01, rtol=0, atol=(1e-12 if precision == 0 else 1e-6) * np.abs(r01).max())
        assert relerr(u2, u1) <= tol_u, (ordering, relerr(u2, u1))
        assert relerr(p2, p1) <= 10 * tol_u, (ordering, relerr(p2, p1))


def _table1_rows():
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_p1p1.txt")
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, h, eu, ku, ep, kp = line.split()
                rows.append((int(n), float(eu), float(ep)))
    return rows


@pytest.mark.parametrize("row", range(5))
@pytest.mark.parametrize("precision", [0, 1])
def test_table1_p1p1_rows_on_gpu(row, precision):
    """The GPU path reproduces the printed P1P1 errors of Table 1 (periodic
    Taylor-Green on [0, 2]^2, 10..50 cells per side, 1000 steps to t = 1), in
    float64 and in the mixed path (rtol 1e-8), to the oracle's tolerances."""
    from paper_1602_03643_gb300.driver import IPCSRun
    n, eu_paper, ep_paper = _table1_rows()[row]
    pb = WP.taylor_green_2d_periodic(n)
    rtol = 1e-12 if precision == 0 else 1e-8
    run = IPCSRun(pb, precision=precision, rtol_u=rtol, rtol_p=rtol, use_graph=1, guess=1,
                  pressure_pc=1 if precision else 0)
    try:
        run.step(1000, want_stats=False)
        st = capi().oasis_last_stats(run.solver)
        assert st.status == 0
        u, p, _ = run.fields()
    finally:
        run.close()
    x = pb.mesh.dof_coords()
    t = 1.0
    eu = np.sqrt(np.mean((u - pb.exact_u(x, t)) ** 2))
    pe = pb.exact_p(x, t - 0.5 * pb.dt)
    ep = np.sqrt(np.mean(((p - p.mean()) - (pe - pe.mean())) ** 2))
    assert abs(eu - eu_paper) < 0.006 * eu_paper, (eu, eu_paper)
    assert abs(ep - ep_paper) < 0.01 * ep_paper, (ep, ep_paper)


def test_notconv_status():
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.taylor_green_3d(8)
    run = IPCSRun(pb, max_it_p=2, rtol_p=1e-12)
    try:
        with pytest.raises(c.OasisError) as ei:
            run.step()
        assert ei.value.code == c.OASIS_ENOTCONV
    finally:
        run.close()


def test_nan_input_status():
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    pb = WP.taylor_green_3d(6)
    pb.u_nm1 = pb.u_nm1.copy()
    pb.u_nm1[0, 100] = np.nan
    run = IPCSRun(pb)
    try:
        with pytest.raises(c.OasisError) as ei:
            run.step()
        assert ei.value.code in (c.OASIS_ENAN, c.OASIS_ENOTCONV)
    finally:
        run.close()


def test_degenerate_cell_rejected():
    c = capi()
    m = WM.box_mesh_2d(3, 3)
    coords = m.coords.copy()
    cells = m.cells.copy()
    cells[0] = [0, 1, 2]            # three collinear vertices on the bottom edge
    h = c.oasis_mesh_create(2, coords, cells)
    try:
        with pytest.raises(c.OasisError) as ei:
            c.oasis_assemble_constant(h)
        assert ei.value.code == c.OASIS_EMESH
    finally:
        c.oasis_mesh_destroy(h)
