"""The surrogate's training loop on the GPU against the oracle's training
steps: target standardisation, the order of the rows and Adam.

Each run here has one batch per epoch (the batch covers the training set, in
the order the seed fixes), so epoch k is Adam step k. Three runs of one, two
and three epochs from the same initial network give the FP32 masters after
steps 1, 2 and 3. The gradient of step k is taken again through
dock_surrogate_gradients at the masters before it, on the rows in the
oracle's order with the targets standardised as training does; the oracle's
FP64 Adam steps from the initial masters with those gradients must then give
the GPU's masters after every step, to FP32 rounding.
"""
import numpy as np
import pytest

from oracle import oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import to_dev  # noqa: E402

N_ROWS, CLIP, LR = 512, 20.0, 1e-3


@pytest.fixture(scope="module")
def dock():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock as d
    return d


def _bf16_bits(x):
    return (o.to_bf16(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(21)
    X = rng.normal(0, 0.6, size=(N_ROWS, 128))
    X[:, 118:] = 0.0
    scores = rng.normal(-6.0, 3.0, size=N_ROWS).astype(np.float32)
    scores[rng.choice(N_ROWS, N_ROWS // 10, replace=False)] = 1.0e4   # clashes, clipped
    return _bf16_bits(X), scores


def test_adam_steps_and_row_order_match_oracle(dock, data):
    Xb, scores = data
    seed_w, seed_order = 3, 99
    dX = to_dev(torch, Xb.view(np.int16))
    ds = to_dev(torch, scores)
    W0 = dock.dock_surrogate_get_params(dock.dock_surrogate_create(seed=seed_w))[0]
    W, stats = {}, {}
    for ep in (1, 2, 3):
        S = dock.dock_surrogate_create(seed=seed_w)
        dock.dock_surrogate_train(S, dX, ds, epochs=ep, batch=N_ROWS, lr=LR, score_clip=CLIP,
                                  seed=seed_order)
        W[ep], tm, ts, tc = dock.dock_surrogate_get_params(S)
        stats[ep] = (tm, ts, tc)
        S.close()
    assert stats[1] == stats[2] == stats[3]
    tm, ts, tc = stats[1]
    mean, std = o.standardize_targets(scores, CLIP)
    assert tm == pytest.approx(mean, rel=1e-6) and ts == pytest.approx(std, rel=1e-6)
    assert tc == np.float32(CLIP)
    # the rows of the batch in the training order, targets standardised as the
    # training loop does in FP32
    order = o.train_order(seed_order, N_ROWS)
    inv = np.float32(1.0) / np.float32(ts)
    tgt = ((np.minimum(scores[order], np.float32(CLIP)) - np.float32(tm)) * inv).astype(np.float32)
    dXo, dt = to_dev(torch, Xb[order].view(np.int16)), to_dev(torch, tgt)
    G = dock.dock_surrogate_create(seed=seed_w)
    grad = torch.zeros(dock.DOCK_MLP_N_PARAMS, dtype=torch.float32, device="cuda")
    p = W0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    prev = W0
    for step in (1, 2, 3):
        dock.dock_surrogate_set_params(G, prev, tm, ts, CLIP)
        dock.dock_surrogate_gradients(G, dXo, dt, grad)
        torch.cuda.synchronize()
        o.adam_step(p, m, v, grad.cpu().numpy().astype(np.float64), step, lr=LR)
        got = W[step].astype(np.float64)
        err = np.abs(got - p)
        # FP32 masters and moments; 1 - 0.999^t in FP32 loses ~1e-5 of the
        # bias correction at t = 2, 3: 5e-8 absolute on an lr-sized update
        tol = 5e-8 + 3e-7 * np.abs(p)
        assert np.all(err <= tol), (step, int(np.argmax(err / tol)), float((err / tol).max()))
        # the step moved the masters (the test is not vacuous)
        assert np.median(np.abs(got - prev)) > 0.3 * LR
        prev = W[step]


def test_two_batch_epoch_uses_the_order_in_batches(dock, data):
    """With two batches per epoch, step 1 is taken on the first half of the
    order and step 2 on the second half."""
    Xb, scores = data
    seed_w, seed_order, B = 4, 7, N_ROWS // 2
    dX, ds = to_dev(torch, Xb.view(np.int16)), to_dev(torch, scores)
    S = dock.dock_surrogate_create(seed=seed_w)
    W0 = dock.dock_surrogate_get_params(S)[0]
    dock.dock_surrogate_train(S, dX, ds, epochs=1, batch=B, lr=LR, score_clip=CLIP, seed=seed_order)
    W2, tm, ts, _ = dock.dock_surrogate_get_params(S)
    order = o.train_order(seed_order, N_ROWS)
    inv = np.float32(1.0) / np.float32(ts)
    G = dock.dock_surrogate_create(seed=seed_w)
    grad = torch.zeros(dock.DOCK_MLP_N_PARAMS, dtype=torch.float32, device="cuda")
    p, m, v = W0.astype(np.float64), np.zeros(W0.size), np.zeros(W0.size)
    at = W0
    for step, rows in ((1, order[:B]), (2, order[B:])):
        tgt = ((np.minimum(scores[rows], np.float32(CLIP)) - np.float32(tm)) * inv).astype(np.float32)
        dock.dock_surrogate_set_params(G, at, tm, ts, CLIP)
        dock.dock_surrogate_gradients(G, to_dev(torch, Xb[rows].view(np.int16)), to_dev(torch, tgt),
                                      grad)
        torch.cuda.synchronize()
        o.adam_step(p, m, v, grad.cpu().numpy().astype(np.float64), step, lr=LR)
        at = p.astype(np.float32)
    err = np.abs(W2.astype(np.float64) - p)
    # Step 2's BF16 weight copies are rounded from FP32 masters that differ by
    # an FP32 ulp between the two runs (FP32 Adam in training, FP64 Adam here),
    # so a copy near a BF16 rounding boundary can round the other way and move
    # that step's gradients by a BF16 step: a few masters then differ by a
    # small fraction of the learning rate. Taking the batches in another order
    # moves them by about the learning rate (1e-3).
    tight = err <= 1e-7 + 1e-6 * np.abs(p)
    assert tight.mean() >= 0.999, (float(tight.mean()), float(err.max()))
    assert np.all(err <= 2e-6 + 1e-5 * np.abs(p)), float(err.max())


@pytest.mark.parametrize("rows", [16384, 65536])
def test_large_batch_step_matches_oracle(dock, rows):
    """One Adam step on a batch of 16,384 or 65,536 rows (the sizes the
    training benchmark times; the training products then span hundreds of
    tiles and the reductions many blocks): the FP32 masters after the step
    equal the oracle's FP64 Adam step from the initial masters with the
    gradient at them, to FP32 rounding."""
    rng = np.random.default_rng(rows)
    X = rng.normal(0, 0.6, size=(rows, 128))
    X[:, 118:] = 0.0
    Xb = _bf16_bits(X)
    scores = rng.normal(-6.0, 3.0, size=rows).astype(np.float32)
    seed_w, seed_order = 5, 11
    S = dock.dock_surrogate_create(seed=seed_w)
    W0 = dock.dock_surrogate_get_params(S)[0]
    dock.dock_surrogate_train(S, to_dev(torch, Xb.view(np.int16)), to_dev(torch, scores), epochs=1,
                              batch=rows, lr=LR, score_clip=CLIP, seed=seed_order)
    W1, tm, ts, _ = dock.dock_surrogate_get_params(S)
    order = o.train_order(seed_order, rows)
    inv = np.float32(1.0) / np.float32(ts)
    tgt = ((np.minimum(scores[order], np.float32(CLIP)) - np.float32(tm)) * inv).astype(np.float32)
    G = dock.dock_surrogate_create(seed=seed_w)
    dock.dock_surrogate_set_params(G, W0, tm, ts, CLIP)
    grad = torch.zeros(dock.DOCK_MLP_N_PARAMS, dtype=torch.float32, device="cuda")
    dock.dock_surrogate_gradients(G, to_dev(torch, Xb[order].view(np.int16)), to_dev(torch, tgt), grad)
    torch.cuda.synchronize()
    p = W0.astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    o.adam_step(p, m, v, grad.cpu().numpy().astype(np.float64), 1, lr=LR)
    err = np.abs(W1.astype(np.float64) - p)
    assert np.all(err <= 5e-8 + 3e-7 * np.abs(p)), float(err.max())
    assert np.median(np.abs(W1 - W0)) > 0.3 * LR
    S.close()
    G.close()
