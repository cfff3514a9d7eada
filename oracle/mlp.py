"""Learned troubled-cell indicator: a plain FP64 multilayer perceptron.

The paper has no learned component.  This module is the FP64 reference for
the indicator that replaces the TVB detection test: a fully connected network
40 -> 64 -> 64 -> 64 -> 1 with ReLU hidden layers and one logit, trained with
class-weighted binary cross entropy and Adam.  Parity is pinned by central
finite differences of the loss (gradient check) and by closed forms of the
loss; the feature recipe is pinned by its invariances.  Test infrastructure.

Feature recipe (per cell, per variable q of the four conserved variables):
  d  = (ubar_E - ubar_K, ubar_W - ubar_K, ubar_N - ubar_K, ubar_S - ubar_K,
        u_(1,0), u_(0,1), u_(2,0), u_(1,1), u_(0,2))
  s_q = max(max |d|, 1e-30)
  features: d / s_q (9 numbers) and clip(log10(s_q / (M h^2)), -8, 8)
giving 4 * 10 = 40 inputs ordered [q0: 9 normalised, q1: ..., q3: ..., then
the 4 scale features].  h = max(dx, dy).
"""
import numpy as np


def init_params(rng, sizes=(40, 64, 64, 64, 1)):
    """He-normal weights, zero biases.  W[l] has shape (out, in)."""
    Ws, bs = [], []
    for a, b in zip(sizes[:-1], sizes[1:]):
        Ws.append(rng.normal(0.0, np.sqrt(2.0 / a), size=(b, a)))
        bs.append(np.zeros(b))
    return {"W": Ws, "b": bs}


def forward(params, X):
    """X (n, 40) -> logits (n,), plus the activations needed by backward."""
    acts = [X]
    zs = []
    h = X
    L = len(params["W"])
    for l in range(L):
        z = h @ params["W"][l].T + params["b"][l]
        zs.append(z)
        h = np.maximum(z, 0.0) if l < L - 1 else z
        acts.append(h)
    return h[:, 0], (acts, zs)


def bce_with_logits(logits, y, pos_weight=1.0):
    """Mean of  -[pw y log s(z) + (1 - y) log(1 - s(z))]  and its derivative
    with respect to the logits."""
    z = logits
    log_sig = -np.logaddexp(0.0, -z)
    log_1msig = -np.logaddexp(0.0, z)
    loss = -(pos_weight * y * log_sig + (1 - y) * log_1msig)
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (pos_weight * y * (sig - 1.0) + (1 - y) * sig) / len(z)
    return loss.mean(), dz


def backward(params, cache, dlogits):
    """Gradients of sum(dlogits * logits) with respect to W and b."""
    acts, zs = cache
    L = len(params["W"])
    gW = [None] * L
    gb = [None] * L
    g = dlogits[:, None]
    for l in range(L - 1, -1, -1):
        gW[l] = g.T @ acts[l]
        gb[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ params["W"][l]) * (zs[l - 1] > 0)
    return {"W": gW, "b": gb}


def adam_update(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba) on every tensor; state holds m, v, t."""
    if not state:
        state.update(t=0, m={k: [np.zeros_like(a) for a in params[k]] for k in ("W", "b")},
                     v={k: [np.zeros_like(a) for a in params[k]] for k in ("W", "b")})
    state["t"] += 1
    t = state["t"]
    for key in ("W", "b"):
        for l in range(len(params[key])):
            g = grads[key][l]
            m = state["m"][key][l] = b1 * state["m"][key][l] + (1 - b1) * g
            v = state["v"][key][l] = b2 * state["v"][key][l] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            params[key][l] = params[key][l] - lr * mh / (np.sqrt(vh) + eps)
    return params


def features(u, nb, M, h):
    """Feature matrix (ny*nx, 40) from a P^2 (or richer) 2D Euler state
    u[y, x, v, m] and neighbour averages nb[side][y, x, v]."""
    avg = u[..., 0]
    d = np.stack([nb["E"] - avg, nb["W"] - avg, nb["N"] - avg, nb["S"] - avg,
                  u[..., 1], u[..., 2], u[..., 3], u[..., 4], u[..., 5]], axis=-1)  # (y,x,v,9)
    s = np.maximum(np.max(np.abs(d), axis=-1), 1e-30)                                 # (y,x,v)
    norm = d / s[..., None]
    scale = np.clip(np.log10(s / (M * h * h)), -8.0, 8.0)
    n = u.shape[0] * u.shape[1]
    return np.concatenate([norm.reshape(n, -1), scale.reshape(n, -1)], axis=1)
