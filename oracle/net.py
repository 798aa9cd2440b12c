"""Learned initial guess for the pressure-correction solve: CPU float64 oracle.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).  Shares no
code with the CUDA path.

The paper has no learned component; this project adds one.  The network is
defined here and implemented independently on the GPU:

  per dof i, inputs x_i = (b_i / s_b, phi1_i / s_phi, phi2_i / s_phi), where b is
  the projected right-hand side of the pressure-correction system, phi1, phi2
  the last two corrections, s_b = rms(b), s_phi = rms(phi1) (1 if zero);
  neighbour mean  m(v)_i = (1 / deg_i) sum_{j in N(i), j != i} v_j over the P1
  sparsity pattern;
  layer 1:  h1 = relu(x W1a^T + m(x) W1b^T + c1)          (3 -> 32)
  layer 2:  h2 = relu(h1 W2a^T + m(h1) W2b^T + c2)         (32 -> 32)
  readout:  y = h2 w3 + c3 + a0 x_2 + a1 x_3
  guess:    phi0 = s_phi * y;  training target t = phi / s_phi,
  loss:     L = (1/N) sum_i (y_i - t_i)^2.

Flat parameter order (2339 values): W1a[32][3], W1b[32][3], c1[32], W2a[32][32],
W2b[32][32], c2[32], w3[32], c3, a[2].  The GPU stores the weights in bfloat16
(round to nearest even of the float32 value) and accumulates in float32; the
oracle evaluates the same bfloat16-representable weights in float64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 32
SHAPES = [("W1a", (H, 3)), ("W1b", (H, 3)), ("c1", (H,)), ("W2a", (H, H)), ("W2b", (H, H)),
          ("c2", (H,)), ("w3", (H,)), ("c3", (1,)), ("a", (2,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64.

    A bfloat16 keeps the upper 16 bits of the float32 pattern; rounding adds
    0x7FFF plus the lowest kept bit before truncation."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    r = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """Seeded He-style initialisation (bfloat16-representable)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {"W1a": rng.normal(0, np.sqrt(2 / 6), (H, 3)), "W1b": rng.normal(0, np.sqrt(2 / 6), (H, 3)),
         "c1": np.zeros(H), "W2a": rng.normal(0, np.sqrt(2 / 64), (H, H)),
         "W2b": rng.normal(0, np.sqrt(2 / 64), (H, H)), "c2": np.zeros(H),
         "w3": rng.normal(0, np.sqrt(1 / 32), H) * 0.1, "c3": np.zeros(1), "a": np.array([1.0, 0.0])}
    return round_bf16(pack(d))


def mean_operator(row_ptr: np.ndarray, col: np.ndarray) -> sp.csr_matrix:
    """Row-normalised adjacency of the pattern without its diagonal."""
    n = row_ptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    keep = col != rows
    A = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], col[keep])), shape=(n, n))
    deg = np.asarray(A.sum(axis=1)).ravel()
    return sp.diags(1.0 / np.maximum(deg, 1)) @ A


def features(b, phi1, phi2):
    """Network inputs and the scale of the guess (see module docstring)."""
    s_b = np.sqrt(np.mean(b ** 2))
    s_b = s_b if s_b > 0 else 1.0
    s_phi = np.sqrt(np.mean(phi1 ** 2))
    s_phi = s_phi if s_phi > 0 else 1.0
    return np.stack([b / s_b, phi1 / s_phi, phi2 / s_phi], axis=1), s_phi


def forward(p: np.ndarray, x: np.ndarray, Am: sp.csr_matrix):
    P = unpack(p)
    m1 = Am @ x
    z1 = x @ P["W1a"].T + m1 @ P["W1b"].T + P["c1"]
    h1 = np.maximum(z1, 0.0)
    m2 = Am @ h1
    z2 = h1 @ P["W2a"].T + m2 @ P["W2b"].T + P["c2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["c3"][0] + P["a"][0] * x[:, 1] + P["a"][1] * x[:, 2]
    return y, dict(x=x, m1=m1, z1=z1, h1=h1, m2=m2, z2=z2, h2=h2)


def loss_and_grad(p: np.ndarray, x: np.ndarray, t: np.ndarray, Am: sp.csr_matrix):
    """L = mean((y - t)^2) and dL/dp by the chain rule (no autograd)."""
    P = unpack(p)
    y, c = forward(p, x, Am)
    n = x.shape[0]
    r = y - t
    L = float(np.mean(r ** 2))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = c["h2"].T @ dy
    g["c3"] = np.array([dy.sum()])
    g["a"] = np.array([dy @ x[:, 1], dy @ x[:, 2]])
    dz2 = np.outer(dy, P["w3"]) * (c["z2"] > 0)
    g["W2a"] = dz2.T @ c["h1"]
    g["W2b"] = dz2.T @ c["m2"]
    g["c2"] = dz2.sum(axis=0)
    # m2 = Am h1, so the gradient reaching h1 through the mean is Am^T (dz2 W2b)
    dh1 = dz2 @ P["W2a"] + Am.T @ (dz2 @ P["W2b"])
    dz1 = dh1 * (c["z1"] > 0)
    g["W1a"] = dz1.T @ x
    g["W1b"] = dz1.T @ c["m1"]
    g["c1"] = dz1.sum(axis=0)
    return L, pack(g), y


def adam(p, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the float64 master parameters."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad ** 2
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
