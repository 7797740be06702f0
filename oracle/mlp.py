"""FP64 forward/backward of the preconditioner-correction network.

Test infrastructure only (see ``oracle/__init__``).  Not part of the paper: a small
per-macro-face MLP that corrects the block-Jacobi preconditioner inside FGMRES
(FGMRES allows a variable preconditioner, Sec. 4.2).

Network: x [n_in] -> h1 = relu(W1 x + b1) [hid] -> h2 = relu(W2 h1 + b2) [hid]
-> y = W3 h2 + b3 [n_out].  Loss: mean over samples and outputs of (y - t)^2.
Parameters are packed [W1 (hid x n_in), b1, W2 (hid x hid), b2, W3 (n_out x hid), b3]
in row-major order, the layout of the library's mehdg_mlp_params.
Pinned by central finite differences in tests/test_oracle_pins.py.
"""
import numpy as np


def unpack(p, nin, hid, nout):
    o = 0
    out = []
    for shape in [(hid, nin), (hid,), (hid, hid), (hid,), (nout, hid), (nout,)]:
        n = int(np.prod(shape))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    return out


def n_params(nin, hid, nout):
    return hid * nin + hid + hid * hid + hid + nout * hid + nout


def forward(p, X, nin, hid, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, hid, nout)
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    return H1, H2, H2 @ W3.T + b3


def loss_and_grad(p, X, T, nin, hid, nout):
    """Mean-squared loss and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, hid, nout)
    H1, H2, Y = forward(p, X, nin, hid, nout)
    n = X.shape[0]
    loss = np.mean((Y - T) ** 2)
    dY = 2.0 * (Y - T) / (n * nout)
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dH2 = (dY @ W3) * (H2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(0)
    dH1 = (dH2 @ W2) * (H1 > 0)
    gW1 = dH1.T @ X
    gb1 = dH1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def bf16_round(x):
    """Round FP32 values to BF16 (round to nearest even) and back, as the library stores weights."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((a >> 16) & 1) + 0x7FFF
    b = ((a + rounding) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)
