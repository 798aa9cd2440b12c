"""Pins of the learned-guess oracle: finite differences of the loss, the
gradient of the mean aggregation, bfloat16 rounding, and a training sanity
check (the loss of a solvable toy problem falls)."""
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


def test_features_scale_invariance():
    rng = np.random.default_rng(2)
    b, f1, f2 = rng.normal(size=(3, 50))
    x1, s1 = N.features(b, f1, f2)
    x2, s2 = N.features(7 * b, 3 * f1, 3 * f2)
    np.testing.assert_allclose(x1, x2, rtol=1e-12)
    assert abs(s2 / s1 - 3) < 1e-12
