"""A9 learned post-equaliser: 1-D CNN forward, backward and Adam, FP64.

TEST INFRASTRUCTURE (see the package docstring).

The paper has no learned equaliser. Reading taken: the network maps the
carrier-recovered symbols z of both polarisations (4 real channels: I_x,
Q_x, I_y, Q_y) to corrected symbols, out = z + f(z), with
f = conv(C->4) . relu . conv(C->C) . relu . conv(C->C) . relu . conv(4->C),
every conv one-dimensional over the symbol index with kernel K and "same"
zero padding (K // 2 on each side):
  y[o, t] = b[o] + sum_i sum_{k<K} W[o, i, k] x[i, t + k - K//2]   (x = 0 outside).
Loss: mean squared error against the transmitted symbols,
L = mean over (channel, t) of (out - target)^2. Optimiser: Adam
(Kingma & Ba 2015) with bias correction:
  m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
  w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""

from __future__ import annotations

import numpy as np

LAYERS = 4


def shapes(C: int = 64, K: int = 9):
    """Parameter shapes per layer: (W [out, in, K], b [out])."""
    dims = [(4, C), (C, C), (C, C), (C, 4)]
    return [((o, i, K), (o,)) for i, o in dims]


def init_params(C: int = 64, K: int = 9, seed: int = 0, out_scale: float = 0.1):
    """He-normal weights, zero biases; the last layer scaled down so f starts near 0."""
    rng = np.random.default_rng(seed)
    params = []
    for li, (ws, bs) in enumerate(shapes(C, K)):
        fan_in = ws[1] * ws[2]
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=ws)
        if li == LAYERS - 1:
            W *= out_scale
        params.append([W, np.zeros(bs)])
    return params


def conv1d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[o, t] = b[o] + sum_i sum_k W[o, i, k] x[i, t + k - K//2], x zero outside [0, T)."""
    Cin, T = x.shape
    K = W.shape[2]
    pad = K // 2
    xp = np.zeros((Cin, T + 2 * pad))
    xp[:, pad:pad + T] = x
    y = np.tile(b[:, None], (1, T)).astype(np.float64)
    for k in range(K):
        y += W[:, :, k] @ xp[:, k:k + T]
    return y


def conv1d_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of conv1d: (dx, dW, db)."""
    Cin, T = x.shape
    K = W.shape[2]
    pad = K // 2
    xp = np.zeros((Cin, T + 2 * pad))
    xp[:, pad:pad + T] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for k in range(K):
        dW[:, :, k] = dy @ xp[:, k:k + T].T
        dxp[:, k:k + T] += W[:, :, k].T @ dy
    return dxp[:, pad:pad + T], dW, dy.sum(axis=1)


def forward(params, z: np.ndarray):
    """z [4, T] -> (out [4, T], cache)."""
    acts = [z]
    h = z
    for li, (W, b) in enumerate(params):
        pre = conv1d(h, W, b)
        h = np.maximum(pre, 0.0) if li < LAYERS - 1 else pre
        acts.append(h)
    return z + h, acts


def mse(out: np.ndarray, target: np.ndarray) -> float:
    return float(np.mean((out - target) ** 2))


def backward(params, acts, out: np.ndarray, target: np.ndarray):
    """Gradients of the MSE loss w.r.t. every parameter: [[dW, db], ...]."""
    d = 2.0 * (out - target) / out.size
    grads = [None] * LAYERS
    for li in range(LAYERS - 1, -1, -1):
        W, _ = params[li]
        if li < LAYERS - 1:
            d = d * (acts[li + 1] > 0)                  # through the ReLU of this layer
        dx, dW, db = conv1d_backward(acts[li], W, d)
        grads[li] = [dW, db]
        d = dx
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = [[np.zeros_like(p) for p in layer] for layer in params]
        self.v = [[np.zeros_like(p) for p in layer] for layer in params]

    def step(self, params, grads):
        self.t += 1
        for li in range(LAYERS):
            for j in range(2):
                g = grads[li][j]
                self.m[li][j] = self.b1 * self.m[li][j] + (1 - self.b1) * g
                self.v[li][j] = self.b2 * self.v[li][j] + (1 - self.b2) * g * g
                mh = self.m[li][j] / (1 - self.b1 ** self.t)
                vh = self.v[li][j] / (1 - self.b2 ** self.t)
                params[li][j] = params[li][j] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return params


def flatten(params) -> np.ndarray:
    return np.concatenate([p.ravel() for layer in params for p in layer])


def unflatten(vec: np.ndarray, C: int = 64, K: int = 9):
    out, o = [], 0
    for ws, bs in shapes(C, K):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append([vec[o:o + nw].reshape(ws), vec[o + nw:o + nw + nb].reshape(bs)])
        o += nw + nb
    return out


# ----------------------------------------------------------------------------
# Training labels of the learned post-equaliser (reading taken, no paper
# counterpart): the transmitted symbols put in the frame of the chain's
# outputs by the alignment A6 found, then each block of `block` symbols
# turned by the quarter turn that best matches the outputs, so that a
# carrier slip of the chain is followed by the labels, not learned.
# ----------------------------------------------------------------------------

def aligned_targets(pol_map, rotation, delay, symbols: np.ndarray, n_sym: int) -> np.ndarray:
    """Output q at index n carries s_{p_q}[n + d_q] turned by j^{r_q} (A6), so its label is
    s_{p_q}[n + d_q] (-j)^{r_q}; indices without a transmitted symbol get 0."""
    n_ref = symbols.shape[1]
    out = np.zeros((2, n_sym), dtype=np.complex128)
    for q in range(2):
        p, r, d = pol_map[q], rotation[q], delay[q]
        for n in range(n_sym):
            if 0 <= n + d < n_ref:
                out[q, n] = symbols[p, n + d] * (-1j) ** r
    return out


def quarter_turn_errors(z: np.ndarray, target: np.ndarray, block: int) -> np.ndarray:
    """err[u, q, j] = sum over block j of |z_q - target_q j^u|^2, u = 0..3 (whole blocks only)."""
    nb = z.shape[1] // block
    err = np.zeros((4, 2, nb))
    for u in range(4):
        diff = z[:, :nb * block] - target[:, :nb * block] * (1j ** u)
        err[u] = (np.abs(diff) ** 2).reshape(2, nb, block).sum(axis=-1)
    return err


def repair_quarter_turns(z: np.ndarray, target: np.ndarray, block: int = 1024) -> np.ndarray:
    """Labels of each whole block turned by its best quarter turn (first minimum); a tail shorter
    than a block keeps its labels."""
    err = quarter_turn_errors(z, target, block)
    best = np.argmin(err, axis=0)                       # [2, nb], ties to the smallest turn
    out = np.array(target, dtype=np.complex128)
    for q in range(2):
        for j in range(best.shape[1]):
            out[q, j * block:(j + 1) * block] *= 1j ** best[q, j]
    return out
