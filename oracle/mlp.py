"""Fully connected corrective-forcing network (Sec. 2.2, Fig. 2) in FP64.

Architecture (reading of Sec. 2.2: "first and last layers linear, relu for the
hidden layers"): the input layer is the identity on the scaled features, then
n_hidden Dense layers of width H with ReLU, then one linear Dense output layer.
The same network serves every element (Sec. 2.2).

Scaling (Sec. 2.2: values are rescaled): per-feature z-scores
    x_s = (x - mean_in) / std_in,   s = y * std_out + mean_out,
and the loss is the MSE between y and the scaled target (t - mean_out)/std_out.

Weights W_l have shape (out, in); a layer computes h W^T + b.

``bf16=True`` rounds (round-to-nearest-even, via float32) at the points where the
GPU path stores bfloat16 operands: scaled inputs, weights, hidden activations,
and in the backward pass the output gradient and every pre-activation gradient
used as a GEMM operand.  Accumulation stays FP64 here.

Test infrastructure only (see the package docstring).
"""
import numpy as np


def round_bf16(a):
    """float64 -> float32 (RNE) -> bfloat16 (RNE), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(a, on):
    return round_bf16(a) if on else a


def layer_dims(n_in, n_out, width, n_hidden):
    return [n_in] + [width] * n_hidden + [n_out]


def he_uniform_init(dims, draws):
    """W_l = u * sqrt(6 / fan_in) with u ~ U(-1, 1) given in ``draws[l]`` (shape
    (out, in)); biases zero.  Returns a list of (W, b)."""
    params = []
    for l in range(len(dims) - 1):
        fan_in = dims[l]
        W = np.asarray(draws[l], dtype=np.float64).reshape(dims[l + 1], dims[l]) * np.sqrt(6.0 / fan_in)
        params.append((W, np.zeros(dims[l + 1])))
    return params


def forward(params, x_scaled, bf16=False):
    """Returns (y, cache).  cache['h'][l] is the input of layer l (as used by
    the GEMM, i.e. rounded when bf16)."""
    L = len(params)
    h = _r(x_scaled, bf16)
    hs = [h]
    for l, (W, b) in enumerate(params):
        a = h @ _r(W, bf16).T + b
        if l < L - 1:
            h = _r(np.maximum(a, 0.0), bf16)
            hs.append(h)
        else:
            y = a
    return y, {'h': hs}


def infer(params, scalers, x, bf16=False):
    """Forcing s for raw element features x: scale, forward, unscale."""
    mean_in, std_in, mean_out, std_out = scalers
    y, _ = forward(params, (x - mean_in) / std_in, bf16)
    return y * std_out + mean_out


def mse_loss(y, t_scaled):
    """L = mean over batch and outputs of (y - t)^2; returns (L, dL/dy)."""
    diff = y - t_scaled
    return float((diff ** 2).mean()), 2.0 * diff / diff.size


def backward(params, cache, dy, bf16=False):
    """Gradients [(dW_l, db_l)] of the loss given dL/dy (plain reverse mode)."""
    L = len(params)
    grads = [None] * L
    g = dy
    for l in range(L - 1, -1, -1):
        W, _ = params[l]
        h_in = cache['h'][l]
        g_op = _r(g, bf16)                     # GEMM operand
        dW = g_op.T @ h_in
        db = g.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            dh = g_op @ _r(W, bf16)
            g = dh * (cache['h'][l] > 0.0)      # ReLU mask of the layer that produced h_in
    return grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7):
    """Adam (Kingma & Ba, Algorithm 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr * m_hat / (sqrt(v_hat) + eps), m_hat = m/(1-b1^t),
    v_hat = v/(1-b2^t).  ``state`` = {'t': int, 'm': [...], 'v': [...]} (updated)."""
    if not state:
        state['t'] = 0
        state['m'] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state['v'] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    state['t'] += 1
    t = state['t']
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        upd = []
        for idx, (p, g) in enumerate(((W, gW), (b, gb))):
            m = beta1 * state['m'][l][idx] + (1.0 - beta1) * g
            v = beta2 * state['v'][l][idx] + (1.0 - beta2) * g * g
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            upd.append((p - lr * mh / (np.sqrt(vh) + eps), m, v))
        new.append((upd[0][0], upd[1][0]))
        state['m'][l] = (upd[0][1], upd[1][1])
        state['v'][l] = (upd[0][2], upd[1][2])
    return new


def train_step(params, state, scalers, X, T, bf16=False, **adam):
    """One optimisation step on the batch (X raw features, T raw targets).
    Returns (new_params, loss, grads)."""
    mean_in, std_in, mean_out, std_out = scalers
    y, cache = forward(params, (X - mean_in) / std_in, bf16)
    loss, dy = mse_loss(y, (T - mean_out) / std_out)
    grads = backward(params, cache, dy, bf16)
    return adam_step(params, grads, state, **adam), loss, grads
