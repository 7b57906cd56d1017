"""Reference for the learned GMRES initial guess: per-bubble spherical-harmonic features and a
small multilayer perceptron with its backward pass and Adam update, in FP64.

TEST INFRASTRUCTURE: part of the CPU oracle (see oracle/__init__.py).

The paper starts each GMRES solve from the previous step's q (Sections 3.5, 3.8). The learned
variant keeps that as the fallback and predicts a better start from per-bubble data:
  features  f_m = [c(phi_m), c(q_prev,m), c(q_prev,m) - c(q_prev2,m)], with c(x) = G+ x the
            least-squares coefficients of x in real spherical harmonics of degree l <= L_sh on
            the bubble's initial directions (the same projector as the shape filter of
            Eqs. (3.22)-(3.23), at bandwidth L_sh+1) and q_prev2 the start of the solve before;
  network   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3), y = W4 h3 + b4;
  guess     q0_m = q_prev,m + G (y), i.e. the network predicts the change of q's coefficients;
  loss      mean over bubbles of |y - (c(q_m) - c(q_prev,m))|^2 / 2.
Row vectors: a batch F [B x d_in] maps to Y [B x d_out] with Y = relu(...) @ W^T + b.

The learned part fixes its arithmetic as BF16 weights with FP32 accumulation: every matrix
product takes BF16 operands. `forward_bf16` and `loss_and_grads_bf16` are the same network
with each product's operands rounded to BF16 (round to nearest, ties to even) and the sums,
biases, losses and bias gradients kept in full precision: the weights, the features, the
hidden activations after the relu, and the back-propagated errors where they enter a product.
They are the reference for a BF16 implementation; `forward` and `loss_and_grads` (no rounding)
measure what the BF16 rounding itself costs.
"""
from __future__ import annotations

import numpy as np


def init_params(sizes, seed):
    """He-initialised weights W_i [d_out x d_in] and zero biases, for layer sizes
    (d_in, h, h, h, d_out)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        params.append([rng.standard_normal((b, a)) * np.sqrt(2.0 / a), np.zeros(b)])
    return params


def forward(params, F):
    """Returns (Y, cache). Hidden layers use relu, the output layer is linear."""
    acts = [F]
    pre = []
    h = F
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if i + 1 < len(params) else z
        acts.append(h)
    return h, (acts, pre)


def bf16(x):
    """Nearest bfloat16 value (sign, 8 exponent bits, 8 significant bits), ties to even, of
    the float32 value of x: the float32 word rounded to its upper 16 bits. Returns float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, F, rnd=bf16):
    """forward() with BF16 operands in every product (see the module docstring): layer i
    computes z = rnd(h) @ rnd(W_i)^T + b_i and passes rnd(relu(z)) on. Returns (Y, cache)
    with cache = (the rounded layer inputs, the pre-activations)."""
    acts = [rnd(F)]
    pre = []
    for i, (W, b) in enumerate(params):
        z = acts[-1] @ rnd(W).T + b
        pre.append(z)
        if i + 1 < len(params):
            acts.append(rnd(np.maximum(z, 0.0)))
    return pre[-1], (acts, pre)


def loss_and_grads_bf16(params, F, T, rnd=bf16):
    """loss_and_grads() with BF16 operands in every product: the error g of a layer's output
    enters dW_i = rnd(g)^T a_i and the back-propagated error rnd(g) rnd(W_i) rounded; the bias
    gradient sums the unrounded g."""
    Y, (acts, pre) = forward_bf16(params, F, rnd)
    B = F.shape[0]
    L = 0.5 * float(np.sum((Y - T) ** 2)) / B
    g = (Y - T) / B
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        gr = rnd(g)
        grads[i] = [gr.T @ acts[i], g.sum(axis=0)]
        if i > 0:
            g = (gr @ rnd(W)) * (pre[i - 1] > 0.0)
    return L, grads


def loss_and_grads(params, F, T):
    """Mean squared error L = sum((Y - T)^2) / (2 B) and its gradients (dW_i, db_i)."""
    Y, (acts, pre) = forward(params, F)
    B = F.shape[0]
    dY = (Y - T) / B
    L = 0.5 * float(np.sum((Y - T) ** 2)) / B
    grads = [None] * len(params)
    g = dY
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        grads[i] = [g.T @ acts[i], g.sum(axis=0)]
        if i > 0:
            g = (g @ W) * (pre[i - 1] > 0.0)
    return L, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) with bias correction; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state.update({"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
                      "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]})
    state["t"] += 1
    t = state["t"]
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][i][j] = beta1 * state["m"][i][j] + (1 - beta1) * g
            v = state["v"][i][j] = beta2 * state["v"][i][j] + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            p -= lr * mh / (np.sqrt(vh) + eps)
    return params


def sh_coefficients(Gp, x, vert_off, shape_of):
    """Per-bubble least-squares coefficients c_m = G+_m x_m  ->  [M x P]."""
    M = len(vert_off) - 1
    out = np.zeros((M, Gp[0].shape[0]))
    for m in range(M):
        a, b = vert_off[m], vert_off[m + 1]
        out[m] = Gp[shape_of[m]] @ x[a:b]
    return out


def sh_synthesis(G, C, vert_off, shape_of):
    """x_m = G_m c_m per bubble -> [N]."""
    N = vert_off[-1]
    x = np.zeros(N)
    for m in range(len(vert_off) - 1):
        a, b = vert_off[m], vert_off[m + 1]
        x[a:b] = G[shape_of[m]] @ C[m]
    return x
