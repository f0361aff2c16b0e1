"""The warm-start network on the GPU (tcgen05 BF16 GEMMs, FP32 accumulation,
FP32 Adam) against the FP64 reference in oracle/mlp.py.  The reference sees
the same BF16-rounded inputs, weights and hidden activations the GPU uses, so
the remaining differences are FP32 accumulation order and the BF16 rounding
of the backward operands: outputs within 1e-2 relative, gradients with cosine
>= 0.999 and relative error <= 3e-2 (the first layer's gradient passes
through three BF16-rounded operands of 2^-9 relative error each)."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _net(P, dims, batch, seed=0):
    rng = np.random.default_rng(seed)
    params = ref.glorot_uniform(rng, dims)
    params = [(W, 0.1 * rng.standard_normal(b.shape)) for W, b in params]
    net = P.Mlp(dims[0], dims[-1], hidden=dims[1], n_hidden=len(dims) - 2, max_batch=batch)
    for l, (W, b) in enumerate(params):
        net.set_layer(l, W, b)
    # the GPU multiplies BF16 weights; the reference uses the same values
    return net, [(bf16(W), np.float32(b).astype(np.float64)) for W, b in params], rng


def _ref_forward_bf16(params, X):
    """FP64 forward with the GPU's BF16 roundings of the GEMM operands."""
    H = bf16(X)
    for l, (W, b) in enumerate(params):
        Z = H @ W.T + b
        H = bf16(np.maximum(Z, 0.0)) if l + 1 < len(params) else Z
    return H


DIMS = [300, 136, 136, 200]  # ragged sizes: partial 128-tiles and 64-wide K blocks
# long K with few output tiles: the first layer's forward product and the
# backward product through the last layer take the split-K path
DIMS_SPLIT = [2000, 136, 136, 4000]


@pytest.mark.parametrize("dims,batch", [(DIMS, 40), (DIMS_SPLIT, 40), (DIMS, 200)])
def test_forward_matches_the_reference(dims, batch):
    """batch 200: two 128-row tiles of the activations (a TMA box past the
    last row, zero-filled)."""
    P = _P()
    net, params, rng = _net(P, dims, batch)
    X = rng.standard_normal((batch, dims[0]))
    with net:
        Y = net.predict(X)
    R = _ref_forward_bf16(params, X)
    assert np.max(np.abs(Y - R)) <= 1e-2 * (1.0 + np.max(np.abs(R)))


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("dims", [DIMS, DIMS_SPLIT])
def test_gradients_match_the_reference(dims):
    P = _P()
    net, params, rng = _net(P, dims, 40, seed=1)
    X = rng.standard_normal((40, dims[0]))
    T = rng.standard_normal((40, dims[-1]))
    # reference gradients at the BF16-rounded point, with BF16 hidden activations
    Xb = bf16(X)
    _, grads = ref.gradients(params, Xb, T)
    with net:
        for l in range(len(params)):
            loss, dW, db = net.gradients(X, T, l)
            gW, gb = grads[l]
            assert _cos(dW, gW) >= 0.999, (l, _cos(dW, gW))
            assert np.linalg.norm(dW - gW) <= 3e-2 * np.linalg.norm(gW), l
            assert np.linalg.norm(db - gb) <= 3e-2 * np.linalg.norm(gb), l
        assert abs(loss - ref.loss(params, Xb, T)) <= 1e-2 * ref.loss(params, Xb, T)


def test_adam_step_matches_the_reference_on_the_gpu_gradients():
    P = _P()
    net, params, rng = _net(P, DIMS, 40, seed=2)
    X = rng.standard_normal((40, DIMS[0]))
    T = rng.standard_normal((40, DIMS[-1]))
    with net:
        master = [net.get_layer(l) for l in range(len(params))]
        g = [net.gradients(X, T, l)[1:] for l in range(len(params))]
        net.train_step(X, T)
        after = [net.get_layer(l) for l in range(len(params))]
    opt = ref.Adam([(W.astype(np.float64), b.astype(np.float64)) for W, b in master])
    want = opt.step([(W.astype(np.float64), b.astype(np.float64)) for W, b in master],
                    [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in g])
    for (W, b), (Ww, bw) in zip(after, want):
        assert np.max(np.abs(W - Ww)) <= 1e-6
        assert np.max(np.abs(b - bw)) <= 1e-6


def test_training_reduces_the_loss():
    P = _P()
    rng = np.random.default_rng(5)
    A = rng.standard_normal((64, 48)) / 8.0
    X = rng.standard_normal((256, 64))
    T = np.maximum(X @ A, 0.0)
    with P.Mlp(64, 48, hidden=128, n_hidden=2, max_batch=64, lr=3e-3, seed=3) as net:
        first = None
        for it in range(300):
            sl = slice((it % 4) * 64, (it % 4 + 1) * 64)
            loss = net.train_step(X[sl], T[sl])
            first = loss if first is None else first
        final = np.mean((net.predict(X[:64]) - T[:64]) ** 2)
    assert final < 0.1 * first, (first, final)


def test_full_size_shapes_run():
    """20001 inputs, three hidden layers of 512, 40204 outputs."""
    P = _P()
    rng = np.random.default_rng(7)
    X = rng.standard_normal((64, 20001)).astype(np.float32)
    T = (0.1 * rng.standard_normal((64, 40204))).astype(np.float32)
    with P.Mlp(20001, 40204, max_batch=64) as net:
        l0 = net.train_step(X, T)
        l1 = net.train_step(X, T)
        Y = net.predict(X[:8])
    assert np.isfinite(Y).all() and np.isfinite(l0) and l1 < l0
