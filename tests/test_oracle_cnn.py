"""Pins of the network oracle: central finite differences in FP64."""
import numpy as np

from oracle import cnn


def _net(rng, chans):
    return [(rng.standard_normal((9, a, b)) * 0.3, rng.standard_normal(b) * 0.1) for a, b in zip(chans[:-1], chans[1:])]


def test_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((1, 5, 6, 3))
    W = rng.standard_normal((9, 3, 4))
    b = rng.standard_normal(4)
    dY = rng.standard_normal((1, 5, 6, 4))
    dX, dW, db = cnn.conv_bwd(X, W, dY)
    f = lambda X_, W_, b_: float((cnn.conv_fwd(X_, W_, b_) * dY).sum())
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (0, 2, 3, 1), (0, 4, 5, 2)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += eps
        Xm[idx] -= eps
        assert abs((f(Xp, W, b) - f(Xm, W, b)) / (2 * eps) - dX[idx]) < 1e-7
    for idx in [(0, 0, 0), (4, 2, 3), (8, 1, 2)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        assert abs((f(X, Wp, b) - f(X, Wm, b)) / (2 * eps) - dW[idx]) < 1e-7
    for i in range(4):
        bp, bm = b.copy(), b.copy()
        bp[i] += eps
        bm[i] -= eps
        assert abs((f(X, W, bp) - f(X, W, bm)) / (2 * eps) - db[i]) < 1e-7


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    layers = _net(rng, [3, 4, 4, 2])
    X = rng.standard_normal((1, 6, 5, 3))
    T = rng.standard_normal((1, 6, 5, 2))
    loss, grads = cnn.net_loss_grads(X, T, layers, used=2)
    eps = 1e-6
    for li in range(3):
        W, b = layers[li]
        for idx in [(0, 0, 0), (4, 1, 1), (7, 2, 0)]:
            if idx[1] >= W.shape[1] or idx[2] >= W.shape[2]:
                continue
            Wp = [(w.copy(), bb) for w, bb in layers]
            Wm = [(w.copy(), bb) for w, bb in layers]
            Wp[li][0][idx] += eps
            Wm[li][0][idx] -= eps
            num = (cnn.net_loss_grads(X, T, Wp, 2)[0] - cnn.net_loss_grads(X, T, Wm, 2)[0]) / (2 * eps)
            assert abs(num - grads[li][0][idx]) < 1e-6 * max(1.0, abs(num))


def test_identity_kernel_is_a_copy():
    """A kernel that is 1 at the centre tap on the diagonal reproduces its input."""
    X = np.random.default_rng(2).standard_normal((2, 4, 7, 3))
    W = np.zeros((9, 3, 3))
    W[4] = np.eye(3)
    assert np.array_equal(cnn.conv_fwd(X, W, np.zeros(3)), X)
