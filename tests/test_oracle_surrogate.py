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
