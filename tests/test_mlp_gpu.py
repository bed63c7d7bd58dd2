"""The ordering network's GPU kernels against the CPU reference.

Forward logits and the loss gradient of every parameter, computed by the
hand-written tensor-core kernels (bf16 operands, fp32 accumulation), must
match oracle/mlp_ref.py evaluated with the same bf16 roundings, within a
relative tolerance of 2e-2 per tensor (accumulation order differs); training
on the GPU must drive the loss of a learnable task down.
"""
import numpy as np
import pytest

from oracle import mlp_ref

pytestmark = pytest.mark.gpu
REL_TOL = 2e-2


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _data(mlp, rows, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, mlp.D0), np.float32)
    X[:, :min(mlp.D0, 3 * 10)] = rng.normal(0.5, 0.4, (rows, min(mlp.D0, 30)))
    T = (rng.random((rows, mlp.O)) < 0.3).astype(np.float32)
    M = (rng.random((rows, mlp.O)) < 0.5).astype(np.float32)
    M[:, 1 + mlp.P:] = 0
    return X, T, M


@pytest.mark.parametrize("m,rows", [(5, 37), (10, 203), (20, 64)])
def test_forward_and_gradients_match_reference(pf, m, rows):
    mlp = pf.pfsp_mlp_create(m, seed=7)
    flat = pf.pfsp_mlp_get_params(mlp)
    rng = np.random.default_rng(m)
    flat = flat + rng.normal(0, 0.02, flat.size).astype(np.float32)  # non-zero biases too
    pf.pfsp_mlp_set_params(mlp, flat)
    params = mlp.split(flat)
    X, T, M = _data(mlp, rows, 11 + m)
    Y = pf.pfsp_mlp_forward(mlp, X)
    Yr, _ = mlp_ref.forward(params, X)
    assert np.linalg.norm(Y - Yr) <= REL_TOL * np.linalg.norm(Yr)
    loss, grad = pf.pfsp_mlp_loss_grad(mlp, X, T, M)
    lr, gr = mlp_ref.loss_and_grads(params, X, T, M)
    assert abs(loss - lr) <= REL_TOL * abs(lr)
    for g_gpu, g_ref in zip(mlp.split(grad), gr):
        assert np.linalg.norm(g_gpu - g_ref) <= REL_TOL * np.linalg.norm(g_ref) + 1e-7


def test_training_reduces_loss(pf):
    # targets are a fixed function of the inputs: pair k of the output is on
    # when feature k exceeds feature k + 1
    mlp = pf.pfsp_mlp_create(5, seed=3)
    rows = 8192
    rng = np.random.default_rng(5)
    X = np.zeros((rows, mlp.D0), np.float32)
    X[:, :15] = rng.random((rows, 15))
    T = np.zeros((rows, mlp.O), np.float32)
    M = np.zeros((rows, mlp.O), np.float32)
    for k in range(10):
        T[:, 1 + k] = X[:, k] > X[:, k + 1]
        M[:, 1 + k] = 1
    losses = pf.pfsp_mlp_train(mlp, X, T, M, epochs=8, batch=1024, lr=3e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0], losses
    Y = pf.pfsp_mlp_forward(mlp, X)
    acc = ((Y[:, 1:11] > 0) == (T[:, 1:11] > 0.5)).mean()
    assert acc > 0.9, acc


@pytest.mark.parametrize("m", [5, 10, 20])
def test_batched_forward_many_tiles(pf, m):
    # the batched forward (tcgen05 kernel, 128-row tiles, TMEM accumulators)
    # on more rows than one pass of the grid covers, with a ragged last tile:
    # every row against the reference with the same bf16 roundings
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mlp = pf.pfsp_mlp_create(m, seed=21)
    flat = pf.pfsp_mlp_get_params(mlp)
    rng = np.random.default_rng(100 + m)
    flat = flat + rng.normal(0, 0.02, flat.size).astype(np.float32)
    pf.pfsp_mlp_set_params(mlp, flat)
    params = mlp.split(flat)
    rows = 128 * nsm * 2 + 77
    X, _, _ = _data(mlp, rows, 7 + m)
    Y = pf.pfsp_mlp_forward(mlp, X)
    Yr, _ = mlp_ref.forward(params, X)
    assert Y.shape == Yr.shape
    assert np.isfinite(Y).all()
    assert np.linalg.norm(Y - Yr) <= REL_TOL * np.linalg.norm(Yr)
    # row by row too: no tile or row is misplaced
    err = np.linalg.norm(Y - Yr, axis=1)
    ref = np.linalg.norm(Yr, axis=1)
    assert (err <= 5e-2 * ref + 1e-3).all(), (int(np.argmax(err - 5e-2 * ref)), float(err.max()))
