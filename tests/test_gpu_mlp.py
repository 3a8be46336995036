"""Surrogate network kernels (through include/mlp.h) against the FP64 oracle.

The kernels round every GEMM operand to bfloat16 and accumulate in FP32.  The
oracle's bf16 mode performs the same roundings with exact FP64 sums, so the
two differ only by FP32 summation order and by the rare bfloat16 rounding
decision that the different sums tip the other way (one bf16 unit, 2^-8
relative, on that element): bounds of 2e-3 of the output scale and 2e-2 of
the gradient norm.  Against the plain FP64 network the difference is the
bfloat16 rounding itself (8 significant bits): bounded by 5e-2.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net_mod():
    from paper_0807_0602_gb300.build import build
    build()
    from paper_0807_0602_gb300 import surrogate
    return surrogate


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 6)).astype(np.float32)
    T = np.stack([np.tanh(X[:, 0] - X[:, 1]), X[:, 2] * X[:, 3] * 0.5, np.cos(X[:, 4]) + 0.1 * X[:, 5]], 1)
    return X, T.astype(np.float32)


@pytest.mark.parametrize("n", [1, 16, 37, 300])
def test_forward_matches_oracle(net_mod, n):
    th = net_mod.init_params(3)
    X, _ = _data(n, 1)
    net = net_mod.Network(max_batch=512, params=th)
    y = net.forward(X).cpu().numpy()
    yb, _ = M.forward(th.astype(np.float64), X.astype(np.float64), bf16=True)
    y64, _ = M.forward(th.astype(np.float64), X.astype(np.float64), bf16=False)
    scale = np.abs(y64).max()
    assert np.max(np.abs(y - yb)) <= 2e-3 * scale
    assert np.max(np.abs(y - y64)) <= 5e-2 * scale
    net.close()


def test_gradients_match_oracle_and_are_deterministic(net_mod):
    th = net_mod.init_params(4)
    X, T = _data(200, 2)
    net = net_mod.Network(max_batch=512, params=th)
    g, loss = net.gradients(X, T)
    g2, loss2 = net.gradients(X, T)
    g, g2 = g.cpu().numpy(), g2.cpu().numpy()
    assert np.array_equal(g, g2) and float(loss) == float(loss2)
    lb, gb = M.backward(th.astype(np.float64), X.astype(np.float64), T.astype(np.float64), bf16=True)
    assert abs(float(loss) - lb) <= 1e-3 * lb
    assert np.linalg.norm(g - gb) <= 2e-2 * np.linalg.norm(gb)
    # element by element, per parameter block (each layer's weights and
    # biases): the largest difference within 2e-2 of the block's largest
    # gradient (a flipped bf16 rounding moves an element by one bf16 unit of
    # an operand), and the median element within 1e-3 relative; a wrong or
    # transposed block fails both
    off = 0
    for a, b in ((6, 128), (128, 128), (128, 128), (128, 3)):
        for size in (a * b, b):
            gk, bk = g[off:off + size], gb[off:off + size]
            off += size
            assert np.max(np.abs(gk - bk)) <= 2e-2 * np.max(np.abs(bk)), (a, b, size)
            big = np.abs(bk) > 1e-3 * np.max(np.abs(bk))
            assert np.median(np.abs(gk - bk)[big] / np.abs(bk)[big]) <= 1e-3, (a, b, size)
    assert off == g.size
    # the output layer's biases are plain FP32 sums of FP32 residuals
    assert np.allclose(g[-3:], gb[-3:], rtol=1e-3, atol=1e-7)
    net.close()


def test_adam_step_matches_oracle(net_mod):
    th = net_mod.init_params(5)
    X, T = _data(64, 3)
    net = net_mod.Network(max_batch=128, params=th)
    g, _ = net.gradients(X, T)
    g = g.cpu().numpy().astype(np.float64)
    net.train_step(X, T, 1e-3)
    got = net.params
    want, _, _ = M.adam(th.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g, 1, 1e-3)
    assert np.max(np.abs(got - want)) <= 2e-6
    assert net.steps == 1
    net.close()


def test_training_reduces_loss(net_mod):
    import torch
    X, T = _data(1024, 4)
    net = net_mod.Network(max_batch=1024, params=net_mod.init_params(6))
    first = None
    for s in range(300):
        loss = net.train_step(X, T, 3e-3)
        if first is None:
            first = float(loss)
    torch.cuda.synchronize()
    assert float(loss) < 0.2 * first
    net.close()
