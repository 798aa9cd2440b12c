"""Pins of the learned-guess oracle: closed forms of the forward pass on a path
graph (each term and each weight's orientation isolated by a choice of
weights, neighbour means taken from the graph itself), permutation
equivariance, finite differences of the loss, the mean aggregation,
bfloat16 rounding, and a training sanity check."""
import numpy as np
import pytest

from oracle import net as N
from oracle.p1 import Discretization
from workloads import meshes as WM


def _graph(m):
    P = Discretization(m).pattern()
    return P.indptr, P.indices


def test_param_count():
    assert N.N_PARAMS == 2339
    p = N.init_params(0)
    np.testing.assert_array_equal(N.pack(N.unpack(p)), p)


def test_bf16_rounding_examples():
    # 1 + 2^-8 is halfway between bf16 1.0 and 1.0078125: ties to even -> 1.0
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-3], dtype=np.float32)
    r = N.round_bf16(x)
    np.testing.assert_array_equal(r[:5], [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 0.0])
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3            # half an ulp of bf16 (8 significant bits)


def test_gradient_matches_central_differences():
    m = WM.jitter_interior(WM.box_mesh_3d(4, 3, 3), 0.2, 0.25, seed=1)
    rp, col = _graph(m)
    Am = N.mean_operator(rp, col)
    rng = np.random.default_rng(0)
    x = rng.normal(size=(m.n_dofs, 3))
    t = rng.normal(size=m.n_dofs)
    p = N.init_params(3) + 0.05 * rng.normal(size=N.N_PARAMS)   # off the bf16 grid: any point works
    p[N.N_PARAMS - 2:] = [0.7, -0.2]
    L, g, _ = N.loss_and_grad(p, x, t, Am)
    idx = rng.choice(N.N_PARAMS, size=80, replace=False)
    idx = np.unique(np.concatenate([idx, [0, 100, 200, 300, 1300, 2280, 2310, 2336, 2337, 2338]]))
    h = 1e-6
    for k in idx:
        e = np.zeros(N.N_PARAMS)
        e[k] = h
        fd = (N.loss_and_grad(p + e, x, t, Am)[0] - N.loss_and_grad(p - e, x, t, Am)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_mean_operator_rows_and_symmetry_of_pattern():
    m = WM.box_mesh_2d(5, 4)
    rp, col = _graph(m)
    Am = N.mean_operator(rp, col)
    np.testing.assert_allclose(np.asarray(Am.sum(axis=1)).ravel(), 1.0)
    assert Am.diagonal().max() == 0.0
    # the pattern is symmetric, so the transpose aggregation uses the same neighbours
    A = (Am != 0).astype(int)
    assert (A != A.T).nnz == 0


def test_adam_training_reduces_loss():
    m = WM.box_mesh_3d(4, 4, 4)
    rp, col = _graph(m)
    Am = N.mean_operator(rp, col)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(m.n_dofs, 3))
    t = 0.5 * x[:, 1] + 0.3 * (Am @ x[:, 0])                  # representable by the network
    p = N.init_params(5)
    mom, var = np.zeros_like(p), np.zeros_like(p)
    L0 = N.loss_and_grad(p, x, t, Am)[0]
    for k in range(1, 301):
        L, g, _ = N.loss_and_grad(p, x, t, Am)
        p, mom, var = N.adam(p, mom, var, g, k, 3e-3)
    assert L < 0.05 * L0, (L0, L)


# ---------------------------------------------------------------- Adam pins
# Kingma & Ba (2015), Algorithm 1: m_t = b1 m + (1 - b1) g, v_t = b2 v + (1 - b2) g^2,
# step lr * mhat / (sqrt(vhat) + eps) with mhat = m_t / (1 - b1^t), vhat = v_t / (1 - b2^t).
# The pins below use consequences of that definition, evaluated by hand, so that a
# dropped bias correction, swapped moments or a wrong sign each fail one of them.

def test_adam_first_step_moves_by_lr_times_sign():
    """t = 1: mhat = g and vhat = g^2 exactly, so every parameter moves by
    -lr g / (|g| + eps), i.e. lr against the sign of its gradient."""
    g = np.array([0.5, -3.0, 1e-3, 250.0])
    p0 = np.array([1.0, 2.0, -1.0, 0.0])
    p, m, v = N.adam(p0, np.zeros(4), np.zeros(4), g, 1, 0.01, eps=1e-8)
    np.testing.assert_allclose(p - p0, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=0)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)          # (1 - b1) g
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-13)    # (1 - b2) g^2


def test_adam_constant_gradient_keeps_step_size():
    """With a constant gradient m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so
    after bias correction every step has the size of the first one."""
    g = np.array([0.5, -2.0])
    p = np.array([0.0, 0.0])
    m, v = np.zeros(2), np.zeros(2)
    for t in range(1, 41):
        p_prev = p
        p, m, v = N.adam(p, m, v, g, t, 0.05, eps=0.0)
        np.testing.assert_allclose(p - p_prev, [-0.05, 0.05], rtol=1e-12, atol=0)
    np.testing.assert_allclose(p, [-2.0, 2.0], rtol=1e-12)


def test_adam_three_steps_by_hand():
    """Two scalars, b1 = 0.9, b2 = 0.999, lr = 0.01, eps = 0, moments by hand.

    Scalar A, gradients 1, -1, 1 (|g| = 1, so v_t = 1 - b2^t and vhat = 1):
      t=1  m = 0.1                      mhat = 0.1 / 0.1 = 1
      t=2  m = 0.09 - 0.1 = -0.01        mhat = -0.01 / 0.19 = -1/19
      t=3  m = -0.009 + 0.1 = 0.091      mhat = 0.091 / 0.271 = 91/271
    Scalar B, gradients 2, 0, -4:
      t=1  m = 0.2,    v = 0.004           mhat = 2,            vhat = 4
      t=2  m = 0.18,   v = 0.003996        mhat = 18/19,        vhat = 3996/1999
      t=3  m = -0.238, v = 0.019992004     mhat = -0.238/0.271, vhat = 0.019992004/0.002997001
    """
    lr = 0.01
    want_steps = [
        [1.0, 2.0 / 2.0],
        [-1.0 / 19.0, (18.0 / 19.0) / np.sqrt(3996.0 / 1999.0)],
        [91.0 / 271.0, (-0.238 / 0.271) / np.sqrt(0.019992004 / 0.002997001)],
    ]
    grads = [[1.0, 2.0], [-1.0, 0.0], [1.0, -4.0]]
    p = np.array([0.3, -0.7])
    m, v = np.zeros(2), np.zeros(2)
    for t, (g, want) in enumerate(zip(grads, want_steps), start=1):
        p_prev = p
        p, m, v = N.adam(p, m, v, np.array(g), t, lr, b1=0.9, b2=0.999, eps=0.0)
        np.testing.assert_allclose(p_prev - p, lr * np.array(want), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, [0.091, -0.238], rtol=1e-12)
    np.testing.assert_allclose(v, [0.002997001, 0.019992004], rtol=1e-12)


def test_adam_eps_bounds_the_step_of_a_tiny_gradient():
    """t = 1 with |g| << eps: the step is lr g / (|g| + eps) ~ lr g / eps, not lr."""
    g = np.array([1e-12])
    p, _, _ = N.adam(np.zeros(1), np.zeros(1), np.zeros(1), g, 1, 1.0, eps=1e-8)
    np.testing.assert_allclose(-p, 1e-12 / (1e-12 + 1e-8), rtol=1e-12)


def test_features_scale_invariance():
    rng = np.random.default_rng(2)
    b, f1, f2 = rng.normal(size=(3, 50))
    x1, s1 = N.features(b, f1, f2)
    x2, s2 = N.features(7 * b, 3 * f1, 3 * f2)
    np.testing.assert_allclose(x1, x2, rtol=1e-12)
    assert abs(s2 / s1 - 3) < 1e-12


# ---------------------------------------------------------------- forward pins
def _path_graph(n):
    """CSR pattern of a path 0-1-...-(n-1) with its diagonal (like a P1 pattern)."""
    rp, col = [0], []
    for i in range(n):
        col += [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rp.append(len(col))
    return np.array(rp), np.array(col)


def _neighbour_mean_path(v):
    """Mean over the path neighbours, written from the graph, not the operator."""
    n = v.shape[0]
    out = np.empty_like(v)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        out[i] = sum(v[j] for j in nb) / len(nb)
    return out


def _zero():
    return {name: np.zeros(shape) for name, shape in N.SHAPES}


def test_forward_readout_skip_terms_closed_form():
    rp, col = _path_graph(7)
    x = np.random.default_rng(1).normal(size=(7, 3))
    P = _zero()
    P["c3"][0], P["a"][:] = 0.25, [0.5, -2.0]
    y, _ = N.forward(N.pack(P), x, N.mean_operator(rp, col))
    np.testing.assert_allclose(y, 0.25 + 0.5 * x[:, 1] - 2.0 * x[:, 2], rtol=0, atol=1e-15)


def test_forward_neighbour_mean_and_weight_orientation():
    """Layer 1 through W1b only, layer 2 through a shift in W2a: y = relu(mean x_0)."""
    rp, col = _path_graph(9)
    x = np.random.default_rng(2).normal(size=(9, 3))
    P = _zero()
    for c in range(3):
        P["W1b"][c, c] = 1.0              # h1_c = relu(mean_N x_c)
    for k in range(1, N.H):
        P["W2a"][k, k - 1] = 1.0          # h2_k = relu(h1_{k-1}): row k = output channel
    P["w3"][1] = 1.0
    y, _ = N.forward(N.pack(P), x, N.mean_operator(rp, col))
    np.testing.assert_allclose(y, np.maximum(_neighbour_mean_path(x)[:, 0], 0.0), rtol=0, atol=1e-14)


def test_forward_second_aggregation_and_biases():
    """Layer 1 through W1a, layer 2 through W2b: y = mean_N relu(x_1) + biases."""
    rp, col = _path_graph(8)
    x = np.random.default_rng(3).normal(size=(8, 3))
    P = _zero()
    for c in range(3):
        P["W1a"][c, c] = 1.0              # h1_c = relu(x_c)
    P["W2b"][4, 1] = 1.0                  # h2_4 = relu(mean_N h1_1 + c2_4)
    P["c2"][4] = 0.5
    P["w3"][4] = 2.0
    P["c3"][0] = -1.0
    y, _ = N.forward(N.pack(P), x, N.mean_operator(rp, col))
    want = 2.0 * np.maximum(_neighbour_mean_path(np.maximum(x, 0.0))[:, 1] + 0.5, 0.0) - 1.0
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-14)
    # the layer-1 bias reaches the output through W2a
    P = _zero()
    P["c1"][:] = 1.0
    P["W2a"][0, :] = 1.0 / N.H
    P["c2"][0] = -0.25
    P["w3"][0] = 3.0
    y, _ = N.forward(N.pack(P), x, N.mean_operator(rp, col))
    np.testing.assert_allclose(y, 3.0 * 0.75, rtol=0, atol=1e-14)


def test_forward_permutation_equivariance():
    m = WM.jitter_interior(WM.box_mesh_3d(3, 3, 2), 0.2, 1 / 3, seed=5)
    rp, col = _graph(m)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(m.n_dofs, 3))
    p = N.init_params(7)
    y, _ = N.forward(p, x, N.mean_operator(rp, col))
    perm = rng.permutation(m.n_dofs)
    mp = WM.renumber_dofs(m, perm)
    rp2, col2 = _graph(mp)
    xp = np.empty_like(x)
    xp[perm] = x                          # dof d of the old numbering is perm[d] in the new one
    y2, _ = N.forward(p, xp, N.mean_operator(rp2, col2))
    np.testing.assert_allclose(y2[perm], y, rtol=0, atol=1e-12)
