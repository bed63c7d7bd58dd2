"""Pins of the CPU reference of the ordering network (oracle/mlp_ref.py).

The reference's gradients (unquantised) must match central finite differences
of its own loss, and a one-unit network worked by hand must give the printed
values; the bf16 rounding helper must match the IEEE round-to-nearest-even
definition on chosen bit patterns.  CPU only.
"""
import numpy as np

from oracle import mlp_ref


def _params(rng, D0, H, O, scale=0.5):
    return [rng.normal(0, scale, (D0, H)).astype(np.float32), rng.normal(0, 0.1, H).astype(np.float32),
            rng.normal(0, scale / 3, (H, H)).astype(np.float32), rng.normal(0, 0.1, H).astype(np.float32),
            rng.normal(0, scale / 3, (H, O)).astype(np.float32), rng.normal(0, 0.1, O).astype(np.float32)]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    D0, H, O, rows = 6, 8, 5, 7
    P = [p.astype(np.float64) for p in _params(rng, D0, H, O)]
    X = rng.normal(0, 1, (rows, D0))
    T = (rng.random((rows, O)) < 0.4).astype(np.float64)
    M = (rng.random((rows, O)) < 0.7).astype(np.float64)
    _, grads = mlp_ref.loss_and_grads([p.copy() for p in P], X, T, M, quantised=False)
    eps = 1e-5
    for pi, g in enumerate(grads):
        flat = P[pi].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp_ref.loss_and_grads(P, X, T, M, quantised=False)
            flat[idx] = old - eps
            lm, _ = mlp_ref.loss_and_grads(P, X, T, M, quantised=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g.reshape(-1)[idx]) < 1e-3 * max(1.0, abs(fd)), (pi, idx, fd, g.reshape(-1)[idx])


def test_one_unit_network_by_hand():
    # X = [[2]], W1 = [[1]], b1 = [-1] -> H1 = 1; W2 = [[3]], b2 = [0] -> H2 = 3;
    # W3 = [[0.5]], b3 = [0.25] -> y = 1.75; target 1, mask 1:
    # loss = log(1 + exp(-1.75)) = log(1.1737739) = 0.1602242, dy = sigmoid(1.75) - 1 = -0.1480472
    P = [np.array([[1.0]]), np.array([-1.0]), np.array([[3.0]]), np.array([0.0]), np.array([[0.5]]), np.array([0.25])]
    P = [p.astype(np.float32) for p in P]
    loss, g = mlp_ref.loss_and_grads(P, np.array([[2.0]], np.float32), np.array([[1.0]], np.float32),
                                     np.array([[1.0]], np.float32), quantised=False)
    assert abs(loss - 0.1602242) < 1e-6
    dy = 1 / (1 + np.exp(-1.75)) - 1
    assert abs(g[5][0] - dy) < 1e-6            # db3
    assert abs(g[4][0, 0] - 3 * dy) < 1e-6     # dW3 = H2 * dy
    assert abs(g[2][0, 0] - 1 * 0.5 * dy) < 1e-6  # dW2 = H1 * (W3 * dy)
    assert abs(g[0][0, 0] - 2 * 3 * 0.5 * dy) < 1e-6  # dW1 = X * W2 * W3 * dy


def test_bf16_rounding_is_round_to_nearest_even():
    def f32(bits):
        return np.array([bits], dtype=np.uint32).view(np.float32)

    # exactly halfway, even low part -> down; odd -> up; above half -> up
    assert mlp_ref.bf16(f32(0x3F808000)).view(np.uint32)[0] == 0x3F800000
    assert mlp_ref.bf16(f32(0x3F818000)).view(np.uint32)[0] == 0x3F820000
    assert mlp_ref.bf16(f32(0x3F808001)).view(np.uint32)[0] == 0x3F810000
    assert mlp_ref.bf16(np.array([1.0, -2.5], np.float32)).tolist() == [1.0, -2.5]
