"""CPU float64 reference of the surrogate network and its gradients. Test infrastructure only.

Definition (the network of the learned energy grid): layers l = 0..L-1 with y_l = a_{l-1} W_l + b_l,
a_l = GELU(y_l) for the hidden layers and the last layer linear; GELU(z) = 0.5 z (1 + tanh(c (z +
0.044715 z^3))), c = sqrt(2/pi); loss = mean over batch and outputs of (y - t)^2. Gradients by the
chain rule written out layer by layer; a central finite-difference check of these gradients is a
separate pin in the tests.
"""
import numpy as np

C = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C * (1.0 + 3 * 0.044715 * z * z)


def unpack(params, n_in, width, hidden, n_out):
    """Split the flat parameter vector into [(W_l, b_l)] (W_l: d_in x d_out)."""
    dims = [n_in] + [width] * hidden + [n_out]
    out, o = [], 0
    for l in range(hidden + 1):
        di, do = dims[l], dims[l + 1]
        W = params[o:o + di * do].reshape(di, do)
        o += di * do
        b = params[o:o + do]
        o += do
        out.append((W, b))
    assert o == len(params)
    return out


def forward(params, x, n_in, width, hidden, n_out):
    layers = unpack(np.asarray(params, dtype=np.float64), n_in, width, hidden, n_out)
    a = np.asarray(x, dtype=np.float64)
    for l, (W, b) in enumerate(layers):
        z = a @ W + b
        a = z if l == len(layers) - 1 else gelu(z)
    return a


def loss_and_grad(params, x, t, n_in, width, hidden, n_out):
    params = np.asarray(params, dtype=np.float64)
    layers = unpack(params, n_in, width, hidden, n_out)
    a = [np.asarray(x, dtype=np.float64)]
    zs = []
    for l, (W, b) in enumerate(layers):
        z = a[-1] @ W + b
        zs.append(z)
        a.append(z if l == len(layers) - 1 else gelu(z))
    y = a[-1]
    d = y - t
    loss = np.mean(d * d)
    dz = 2.0 * d / d.size
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = a[l].T @ dz
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            dz = (dz @ W.T) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in reversed(grads)])
    return loss, flat
