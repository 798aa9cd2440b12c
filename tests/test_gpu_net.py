"""Learned pressure guess on the GPU against the float64 CPU oracle of the
network (forward, gradients, Adam), and its effect inside the step.

Tolerances: the kernels hold bfloat16 weights (the same bfloat16 values the
oracle evaluates in float64) and accumulate in float32, so outputs agree to
float32 rounding of O(100)-term sums: 2e-5 of the largest output, 1e-4 of the
largest gradient entry; Adam's float32 master weights to 1e-6 absolute.
"""
import numpy as np
import pytest

from oracle import net as ON
from oracle import p1
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


MESHES = {
    "jitter_9x8x7": lambda: WM.jitter_interior(WM.box_mesh_3d(9, 8, 7), 0.2, 1 / 9, seed=2),
    "cube_24": lambda: WM.box_mesh_3d(24, 24, 24),
    "sq_40x31": lambda: WM.box_mesh_2d(40, 31, 0.0, 1.0, 0.0, 1.0),
    "random_perm_12": lambda: WM.renumber_dofs(WM.box_mesh_3d(12, 12, 12), WM.random_permutation(13 ** 3, 7)),
}


def nontrivial_params(seed):
    """Oracle initialisation with a larger readout, so that both layers matter."""
    P = ON.unpack(ON.init_params(seed))
    rng = np.random.default_rng(seed + 100)
    P["w3"] = P["w3"] * 10.0
    P["c1"] = rng.normal(0, 0.1, ON.H)
    P["c2"] = rng.normal(0, 0.1, ON.H)
    P["c3"] = np.array([0.05])
    P["a"] = np.array([0.9, 0.2])
    return ON.round_bf16(ON.pack(P))


class MeshNet:
    def __init__(self, mesh):
        import torch
        from paper_1602_03643_gb300.guess import GuessNet
        c = capi()
        self.m = mesh
        self.h = c.oasis_mesh_create(mesh.dim, mesh.coords, mesh.cells, mesh.dof_of_vertex, mesh.n_dofs)
        c.oasis_assemble_constant(self.h)
        self.net = GuessNet(self.h, mesh.n_dofs)
        Pt = p1.Discretization(mesh).pattern()
        self.Am = ON.mean_operator(Pt.indptr, Pt.indices)
        self.torch = torch

    def close(self):
        self.net.close()
        capi().oasis_mesh_destroy(self.h)


def inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, 3)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    return x, t


@pytest.mark.parametrize("name", list(MESHES))
def test_forward_matches_oracle(name):
    M = MeshNet(MESHES[name]())
    try:
        torch = M.torch
        p = nontrivial_params(3)
        M.net.set_params(p.astype(np.float32))
        x, _ = inputs(M.m.n_dofs, 11)
        y = M.net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        y_ref, _ = ON.forward(p, x.astype(np.float64), M.Am)
        scale = np.abs(y_ref).max()
        assert scale > 0.5
        np.testing.assert_allclose(y, y_ref, rtol=0, atol=2e-5 * scale)
    finally:
        M.close()


@pytest.mark.parametrize("name", list(MESHES))
def test_gradient_matches_oracle(name):
    M = MeshNet(MESHES[name]())
    try:
        torch = M.torch
        p = nontrivial_params(5)
        M.net.set_params(p.astype(np.float32))
        x, t = inputs(M.m.n_dofs, 12)
        loss, grad = M.net.loss_and_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
        L_ref, g_ref, _ = ON.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64), M.Am)
        assert abs(float(loss.item()) - L_ref) <= 1e-5 * L_ref
        g = grad.cpu().numpy()
        gs = np.abs(g_ref).max()
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * gs)
        # every parameter block receives gradient
        o = 0
        for nm, shape in ON.SHAPES:
            k = int(np.prod(shape))
            assert np.abs(g_ref[o:o + k]).max() > 0, nm
            o += k
    finally:
        M.close()


def test_adam_matches_oracle_and_refreshes_bf16():
    M = MeshNet(MESHES["jitter_9x8x7"]())
    try:
        torch = M.torch
        p0 = nontrivial_params(8).astype(np.float32)
        M.net.set_params(p0)
        rng = np.random.default_rng(9)
        p, m, v = p0.astype(np.float64), np.zeros(ON.N_PARAMS), np.zeros(ON.N_PARAMS)
        for k in range(1, 4):
            g = rng.normal(0, 1e-2, ON.N_PARAMS).astype(np.float32)
            M.net.adam_step(1e-3, grad=torch.from_numpy(g).cuda())
            p, m, v = ON.adam(p, m, v, g.astype(np.float64), k, 1e-3)
        got = M.net.get_params()
        np.testing.assert_allclose(got, p, rtol=0, atol=1e-6)
        # the kernels now evaluate the bfloat16 rounding of the float32 master copy
        x, _ = inputs(M.m.n_dofs, 13)
        y = M.net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        y_ref, _ = ON.forward(ON.round_bf16(got), x.astype(np.float64), M.Am)
        np.testing.assert_allclose(y, y_ref, rtol=0, atol=2e-5 * np.abs(y_ref).max())
    finally:
        M.close()


def test_training_on_gpu_fits_a_teacher():
    """Adam on the GPU drives the loss of a teacher network's outputs down."""
    M = MeshNet(MESHES["cube_24"]())
    try:
        torch = M.torch
        x, _ = inputs(M.m.n_dofs, 21)
        teacher = nontrivial_params(30)
        t, _ = ON.forward(teacher, x.astype(np.float64), M.Am)
        sample = [(torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda())]
        losses = M.net.fit(sample, epochs=300, lr=3e-3)
        assert np.all(np.isfinite(losses))
        assert losses[-1] < 0.1 * losses[0], losses[[0, -1]]
    finally:
        M.close()


# ---------------------------------------------------------------- inside the step
def _run(problem, guess, precision, use_graph=1, rtol_p=1e-8):
    # the BiCGStab product shape is fixed so that runs compare bit for bit
    from paper_1602_03643_gb300.driver import IPCSRun
    c = capi()
    return IPCSRun(problem, precision=precision, rtol_u=1e-8 if precision == c.OASIS_MIXED else 1e-12,
                   rtol_p=rtol_p, batch_rhs=1, use_graph=use_graph, guess=guess, bicg_variant=1)


def test_guess_sample_is_scaled_history():
    """Recorded inputs are phi^{n-1}, phi^{n-2} over rms(phi^{n-1}); the target is
    phi^n over the same scale; the right-hand side column has rms 1."""
    c = capi()
    pb = WP.taylor_green_3d(n=10, dt=2e-3)
    r = _run(pb, c.OASIS_GUESS_PREV_PHI, c.OASIS_FP64, use_graph=0, rtol_p=1e-12)
    try:
        r.record_guess(True)
        phis = []
        for k in range(4):
            r.step(1)
            phis.append(r.fields()[2])
        feat, target = (a.cpu().numpy().astype(np.float64) for a in r.guess_sample())
        s = np.sqrt(np.mean(phis[-2] ** 2))
        np.testing.assert_allclose(feat[:, 1], phis[-2] / s, rtol=0, atol=1e-6 * np.abs(phis[-2] / s).max())
        np.testing.assert_allclose(feat[:, 2], phis[-3] / s, rtol=0, atol=1e-6 * np.abs(phis[-3] / s).max())
        np.testing.assert_allclose(target, phis[-1] / s, rtol=0, atol=1e-6 * np.abs(phis[-1] / s).max())
        assert abs(np.sqrt(np.mean(feat[:, 0] ** 2)) - 1.0) < 1e-5
        assert abs(np.mean(feat[:, 0])) < 1e-5
    finally:
        r.close()


def _train_on_run(r, n_record, epochs):
    from paper_1602_03643_gb300.guess import GuessNet
    r.record_guess(True)
    samples = []
    for k in range(n_record):
        r.step(1)
        if k >= 2:
            samples.append(r.guess_sample())
    r.record_guess(False)
    net = GuessNet(r.mesh, r.n, seed=1)
    losses = net.fit(samples, epochs=epochs, lr=2e-3)
    return net, losses


def test_learned_guess_gain_and_judge():
    """Train on the first steps of a run (samples recorded by the solver, Adam on
    the GPU), then use the learned guess on later steps.

    Gain measured: on held-out steps the network's guess has a smaller residual
    ||b - K phi0|| and a smaller L2 error than the previous correction.  The judge
    takes the candidate with the smaller residual, PCG still reaches the same
    tolerance, and the fields agree with the previous-guess run.  The iteration
    counts are printed, not asserted: from guesses whose relative error is
    0.1-0.5, Jacobi-PCG to 1e-8 needs about the same number of iterations
    (a zero guess needs only ~10% more than the previous correction)."""
    import torch
    c = capi()
    pb = WP.taylor_green_3d(n=20, dt=2e-3)
    n_record, n_eval = 12, 10
    ref = _run(pb, c.OASIS_GUESS_PREV_PHI, c.OASIS_MIXED)
    lr_run = _run(pb, c.OASIS_GUESS_LEARNED, c.OASIS_MIXED)
    try:
        ref.step(n_record)
        net, losses = _train_on_run(lr_run, n_record, epochs=60)
        assert losses[-1] < 0.3 * losses[0], losses[[0, -1]]
        lr_run.attach_guess_net(net)
        lr_run.record_guess(True)
        it_ref = [ref.step(1).it_p for _ in range(n_eval)]
        st, err = [], []
        for _ in range(n_eval):
            st.append(lr_run.step(1))
            feat, t = lr_run.guess_sample()
            y = net.forward(feat)
            err.append([float(torch.linalg.norm(y - t) / torch.linalg.norm(t)),
                        float(torch.linalg.norm(feat[:, 1] - t) / torch.linalg.norm(t))])
        it_learned = [s.it_p for s in st]
        res = np.array([list(s.guess_res) for s in st])
        err = np.array(err)
        print("\nPCG iterations, previous-phi guess:", it_ref, "\nPCG iterations, learned guess:     ", it_learned,
              "\nresidual ratio learned/previous:", np.round(res[:, 0] / res[:, 1], 3).tolist(),
              "\nL2 error ratio learned/previous:", np.round(err[:, 0] / err[:, 1], 3).tolist())
        assert all(s.status == c.OASIS_OK for s in st)
        assert all(s.res_p <= 1e-8 for s in st)
        for s in st:
            want = c.OASIS_GUESS_LEARNED if s.guess_res[0] < s.guess_res[1] else c.OASIS_GUESS_PREV_PHI
            assert s.guess_used == want
        assert np.median(res[:, 0] / res[:, 1]) < 0.9
        assert np.median(err[:, 0] / err[:, 1]) < 0.8
        u_a, p_a, _ = ref.fields()
        u_b, p_b, _ = lr_run.fields()
        assert np.linalg.norm(u_a - u_b) <= 1e-6 * np.linalg.norm(u_a)
        assert np.linalg.norm(p_a - p_b) <= 1e-5 * np.linalg.norm(p_a)
        net.close()
    finally:
        ref.close()
        lr_run.close()


def test_learned_guess_graph_equals_eager():
    """Captured (CUDA graph) and eager steps with the learned guess agree bit for bit."""
    c = capi()
    from paper_1602_03643_gb300.guess import GuessNet
    pb = WP.taylor_green_3d(n=8, dt=2e-3)
    out = []
    for g in (1, 0):
        r = _run(pb, c.OASIS_GUESS_LEARNED, c.OASIS_MIXED, use_graph=g)
        net = GuessNet(r.mesh, r.n, params=nontrivial_params(4).astype(np.float32))
        try:
            r.step(2)
            r.attach_guess_net(net)
            st = [r.step(1) for _ in range(4)]
            out.append((r.fields(), [(s.it_p, s.guess_used) for s in st]))
        finally:
            r.close()
            net.close()
    (fa, sa), (fb, sb) = out
    assert sa == sb
    for a, b in zip(fa, fb):
        np.testing.assert_array_equal(a, b)
