"""FP64 reference of the selector's MLP — TEST INFRASTRUCTURE ONLY.

The network (no counterpart in the paper): x -> relu(x W1 + b1) -> relu(h1 W2 + b2)
-> z = h2 W3 + b3, loss = mean over the batch of -sum_o q_o log softmax(z)_o,
trained with Adam (Kingma & Ba, Algorithm 1).  Parameters are one flat
array, row-major: W1[in][h], b1[h], W2[h][h], b2[h], W3[h][out], b3[out].
The gradient is the chain rule written out layer by layer; the tests pin it
against central finite differences of `loss` and the loss against closed
forms.
"""
import numpy as np


def split(params, dims):
    i, h, o = dims
    p = np.asarray(params, dtype=np.float64)
    k = 0

    def take(sz, shape):
        nonlocal k
        a = p[k:k + sz].reshape(shape)
        k += sz
        return a
    W1 = take(i * h, (i, h))
    b1 = take(h, (h,))
    W2 = take(h * h, (h, h))
    b2 = take(h, (h,))
    W3 = take(h * o, (h, o))
    b3 = take(o, (o,))
    assert k == p.size
    return W1, b1, W2, b2, W3, b3


def param_count(dims):
    i, h, o = dims
    return i * h + h + h * h + h + h * o + o


def forward(params, X, dims):
    W1, b1, W2, b2, W3, b3 = split(params, dims)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return h1, h2, z


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def loss(params, X, Q, dims):
    _, _, z = forward(params, X, dims)
    return float(-(np.asarray(Q, np.float64) * log_softmax(z)).sum() / z.shape[0])


def grad(params, X, Q, dims):
    W1, b1, W2, b2, W3, b3 = split(params, dims)
    X = np.asarray(X, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    B = X.shape[0]
    h1, h2, z = forward(params, X, dims)
    P = np.exp(log_softmax(z))
    dz = (P - Q) / B                       # d loss / d z for softmax cross-entropy
    gW3 = h2.T @ dz
    gb3 = dz.sum(axis=0)
    dh2 = (dz @ W3.T) * (h2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    gW1 = X.T @ dh1
    gb1 = dh1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(params, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments), step number t >= 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def predict(params, X, dims):
    _, _, z = forward(params, X, dims)
    return np.argmax(z, axis=1)
