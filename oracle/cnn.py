"""Oracle for the learned-guess network: plain FP64 numpy 3x3 convolutions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Same-padding 3x3
convolution in NHWC, weights W[tap][cin][cout] with tap = 3(dy+1) + (dx+1),
ReLU between layers, mean squared error on the first `used` output
channels.  The backward pass follows the definitions (chain rule written out
per layer); it is pinned by central finite differences
(tests/test_oracle_cnn.py).
"""
import numpy as np

TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def _shift(X, dy, dx):
    """S[b, y, x] = X[b, y + dy, x + dx] (zero outside the image)."""
    B, H, W, C = X.shape
    out = np.zeros_like(X)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[:, ys:ye, xs:xe] = X[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv_fwd(X, W, b):
    """Y[p] = sum_tap X[p + d(tap)] @ W[tap] + b."""
    Y = np.zeros(X.shape[:3] + (W.shape[2],))
    for t, (dy, dx) in enumerate(TAPS):
        Y += _shift(X, dy, dx) @ W[t]
    return Y + b


def conv_bwd(X, W, dY):
    """Gradients of sum(dY * conv_fwd(X, W, b)) w.r.t. X, W, b."""
    dW = np.zeros_like(W)
    dX = np.zeros_like(X)
    for t, (dy, dx) in enumerate(TAPS):
        Xs = _shift(X, dy, dx)
        dW[t] = np.einsum("bhwi,bhwo->io", Xs, dY)
        dX += _shift(dY @ W[t].T, -dy, -dx)
    db = dY.sum(axis=(0, 1, 2))
    return dX, dW, db


def net_forward(X, layers, round_act=None):
    """layers: list of (W, b); ReLU after every layer but the last.
    round_act(A) optionally models the storage rounding of hidden activations."""
    acts = [X]
    A = X
    for i, (W, b) in enumerate(layers):
        Z = conv_fwd(A, W, b)
        if i < len(layers) - 1:
            A = np.maximum(Z, 0.0)
            if round_act is not None:
                A = round_act(A)
        else:
            A = Z
        acts.append(A)
    return acts


def net_loss_grads(X, T, layers, used, round_act=None, round_grad=None):
    """loss = mean over pixels and the first `used` channels of (net(X) - T)^2;
    returns loss and [(dW, db)] per layer."""
    acts = net_forward(X, layers, round_act)
    out = acts[-1]
    P = out.shape[0] * out.shape[1] * out.shape[2]
    diff = np.zeros_like(out)
    diff[..., :used] = out[..., :used] - T[..., :used]
    loss = float((diff ** 2).sum() / (P * used))
    g = 2.0 * diff / (P * used)
    if round_grad is not None:
        g = round_grad(g)
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        if i < len(layers) - 1:
            g = g * (acts[i + 1] > 0)
        dX, dW, db = conv_bwd(acts[i], W, g)
        grads[i] = (dW, db)
        g = dX
        if round_grad is not None:
            g = round_grad(g)
    return loss, grads
