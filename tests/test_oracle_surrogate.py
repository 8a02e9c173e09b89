"""Pins of the surrogate oracle (oracle/surrogate.c): the MLP forward and
backward against torch's float64 autograd (a library routine) and central
finite differences, bfloat16 rounding against torch's conversion, and the
pose features against their definition (counts, charge sums, unit sin/cos
pairs, scipy's rotation matrix, brute-force shell assignment)."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import oracle as o
from paper_2509_12232_gb300 import synth

NP = 164865


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(NP)
    W1, b1, W2, b2, W3, b3, W4, b4 = o.mlp_unpack(p)
    for W, fan in ((W1, 128), (W2, 256), (W3, 256)):
        W[...] = rng.normal(0, scale * math.sqrt(2.0 / fan), W.shape)
    W4[...] = rng.normal(0, math.sqrt(1.0 / 256), W4.shape)
    for b in (b1, b2, b3, b4):
        b[...] = rng.normal(0, 0.1, b.shape)
    return p


def torch_forward(p, X):
    W1, b1, W2, b2, W3, b3, W4, b4 = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
                                      for a in o.mlp_unpack(p)]
    x = torch.tensor(X, dtype=torch.float64)
    h = torch.nn.functional.gelu(x @ W1 + b1, approximate="none")
    h = torch.nn.functional.gelu(h @ W2 + b2, approximate="none")
    h = torch.nn.functional.gelu(h @ W3 + b3, approximate="none")
    y = h @ W4 + b4
    return y, (W1, b1, W2, b2, W3, b3, W4, b4)


def test_mlp_forward_matches_torch():
    p = random_params(0)
    X = np.random.default_rng(1).normal(size=(37, 128))
    y, _ = torch_forward(p, X)
    np.testing.assert_allclose(o.mlp_forward(p, X), y.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_mlp_backward_matches_torch_autograd():
    p = random_params(2)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(19, 128))
    T = rng.normal(size=19)
    loss, g = o.mlp_backward(p, X, T)
    y, params = torch_forward(p, X)
    tl = ((y - torch.tensor(T)) ** 2).mean()
    tl.backward()
    assert loss == pytest.approx(float(tl), rel=1e-12)
    ref = np.concatenate([t.grad.numpy().ravel() for t in params])
    np.testing.assert_allclose(g, ref, rtol=1e-9, atol=1e-12)


def test_mlp_backward_matches_finite_differences():
    p = random_params(4)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(5, 128))
    T = rng.normal(size=5)
    _, g = o.mlp_backward(p, X, T)
    h = 1e-3

    def loss_at(idx, d):
        q = p.copy()
        q[idx] += d
        return o.mlp_backward(q, X, T)[0]

    for idx in rng.choice(NP, 40, replace=False).tolist() + [NP - 1, 0, 128 * 256]:
        # fourth-order central difference (truncation error O(h^4))
        fd = (-loss_at(idx, 2 * h) + 8 * loss_at(idx, h) - 8 * loss_at(idx, -h)
              + loss_at(idx, -2 * h)) / (12 * h)
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-9)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.0e38]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(o.to_bf16(x), ref)


@pytest.fixture(scope="module")
def posed():
    rng = np.random.Generator(np.random.Philox(8))
    ls = synth.make_ligands(rng, [30], [9])
    lig = o.Ligand(**ls.ligand(0))
    g = np.array([1.5, -2.0, 0.7, 0.3, -0.4, 0.5, 0.7] + list(rng.uniform(-3, 3, 9)), np.float32)
    center = np.array([0.5, 0.25, -1.0])
    xyz = o.pose(lig, g, center)
    return lig, g, center, xyz


def test_features_definition(posed):
    lig, g, center, xyz = posed
    R = 12.0
    f = o.features(lig, xyz, center, g, R)
    assert f.shape == (128,)
    d = np.linalg.norm(xyz - center, axis=1)
    shell = np.minimum(np.floor(d / (R / 8)), 7).astype(int)
    counts = np.zeros((7, 8))
    for t, s in zip(lig.a["type"], shell):
        counts[t, s] += 1
    np.testing.assert_allclose(f[:56].reshape(7, 8), counts / 8, atol=1e-15)
    q = lig.a["q"].astype(np.float64)
    np.testing.assert_allclose(f[56:64], np.bincount(shell, weights=q, minlength=8), atol=1e-12)
    np.testing.assert_allclose(f[64:72], np.bincount(shell, weights=np.abs(q), minlength=8), atol=1e-12)
    sc = f[72:104].reshape(16, 2)
    np.testing.assert_allclose((sc[:lig.k] ** 2).sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.arctan2(sc[:lig.k, 0], sc[:lig.k, 1]),
                               np.angle(np.exp(1j * g[7:].astype(np.float64))), atol=1e-12)
    assert np.all(sc[lig.k:] == 0)
    qq = g[3:7].astype(np.float64)
    np.testing.assert_allclose(f[104:113].reshape(3, 3),
                               Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix(), atol=1e-14)
    np.testing.assert_allclose(f[113:116], g[:3] / R, atol=1e-15)
    assert f[116] == pytest.approx(lig.n / 100) and f[117] == pytest.approx(lig.k / 16)
    assert np.all(f[118:] == 0)
    assert f[:56].sum() == pytest.approx(lig.n / 8)


# ---------------------------------------------------------------------------
# Training: Adam and the order of the training rows
# ---------------------------------------------------------------------------
def test_adam_step_equals_torch_adam_float64():
    """Five steps of the oracle's Adam equal torch.optim.Adam's (float64,
    lr 1e-3, betas (0.9, 0.999), eps 1e-8, bias-corrected) on the same
    gradients, including tiny and zero gradients where eps matters."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    n = 4000
    p = rng.normal(size=n)
    m = np.zeros(n)
    v = np.zeros(n)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.normal(size=n) * np.exp(rng.uniform(-20, 2, size=n))
        g[:7] = 0.0
        o.adam_step(p, m, v, g, t)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-16)
    # the first step moves every parameter with |g| >> eps by lr, against g
    p2, m2, v2 = np.zeros(3), np.zeros(3), np.zeros(3)
    o.adam_step(p2, m2, v2, np.array([5.0, -2e-3, 0.0]), 1)
    np.testing.assert_allclose(p2, [-1e-3 * 5 / (5 + 1e-8), 1e-3 * 2e-3 / (2e-3 + 1e-8), 0.0],
                               rtol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 100, 128, 1000, 1024, 4097, 65536])
def test_train_order_is_a_permutation(n):
    """A permutation of [0, n) for sizes with and without cycle walking
    (n = 1024 = 4^5 and 65536 = 4^8 use the Feistel network alone, so it
    must be a bijection itself)."""
    p = o.train_order(11, n)
    np.testing.assert_array_equal(np.sort(p), np.arange(n))


def test_train_order_depends_on_seed_and_looks_shuffled():
    from scipy.stats import chisquare, spearmanr
    n = 1000
    a, b = o.train_order(1, n), o.train_order(2, n)
    assert (a != b).mean() > 0.9
    assert abs(spearmanr(np.arange(n), a)[0]) < 0.1
    # where row 0 lands, over many seeds, is uniform over ten bins
    pos = np.array([int(np.nonzero(o.train_order(s, n) == 0)[0][0]) for s in range(400)])
    assert chisquare(np.bincount(pos * 10 // n, minlength=10)).pvalue > 1e-3
