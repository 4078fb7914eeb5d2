"""CPU oracle of the learned part: MLP surrogate of log|M|^2 and the exact
two-stage unweighting it drives (test infrastructure only).

The paper has no learned component; this is the benchmark configuration's
surrogate pattern ("4-layer MLP (width 256, SiLU) on pairwise invariants
s_ij/s predicting log|M|^2 ... two-stage unweighting ... exact FP64 ME on the
accepted ones"), following the published rejection-sampling scheme with
network weight estimates (Danziger, Janssen, Schumann, Siegert, SciPost
Phys. 12 (2022) 164):

  features    x_k = log(s_ij / s) for all particle pairs i < j (physical
              momenta, s_ij = (p_i + p_j)^2 > 0, s = s_12), padded with zeros
              to nin; the logarithm of the pair invariants is the network's
              fixed input transform (|M|^2 varies as powers of the s_ij near
              its poles, so log|M|^2 is close to linear in log s_ij)
  network     z_1 = W_1 x + b_1, a_l = silu(z_l), z_{l+1} = W_{l+1} a_l + b_{l+1},
              f = z_L (no activation on the output), silu(z) = z / (1 + e^-z)
  target      y = (log|M|^2 - mu) / sigma, mu and sigma over the training set
  loss        mean over the batch of (f - y)^2
  optimiser   Adam (Kingma, Ba 2015), bias-corrected, eps added to sqrt(v_hat)
  unweighting w = |M|^2 Phi, w_hat = exp(sigma f + mu) Phi;
              stage 1 keeps u1 < w_hat / w_hat_max, stage 2 keeps
              u2 < (w / w_hat) / r_max; accepted events carry the weight
              max(1, w_hat / w_hat_max) * max(1, (w / w_hat) / r_max).
All arithmetic is FP64 numpy.
"""
from __future__ import annotations

import numpy as np


def features(mom: np.ndarray, nin: int = 32) -> np.ndarray:
    """log(s_ij / s) for i < j over the particles of mom [n][npar][4], zero padded."""
    n, npar, _ = mom.shape
    P = mom[:, 0] + mom[:, 1]
    s = P[:, 0] ** 2 - (P[:, 1:] ** 2).sum(1)
    out = np.zeros((n, nin))
    k = 0
    for i in range(npar):
        for j in range(i + 1, npar):
            q = mom[:, i] + mom[:, j]
            out[:, k] = np.log((q[:, 0] ** 2 - (q[:, 1:] ** 2).sum(1)) / s)
            k += 1
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def init_params(sizes, seed=0):
    """Weights W_l [out][in] uniform in +-sqrt(6/(in+out)) (Glorot), biases 0."""
    rng = np.random.default_rng(seed)
    ps = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / (a + b))
        ps.append([rng.uniform(-lim, lim, (b, a)), np.zeros(b)])
    return ps


def round_bf16(a):
    """Round to bfloat16 (8 significant bits), round-to-nearest-even, via the
    float32 bit pattern: keep the high 16 bits after adding 0x7FFF plus the
    lowest kept bit.  Returns float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, emulate_bf16=False):
    """Returns (f, cache) with cache = [(a_prev, z)] per layer.  With
    emulate_bf16 the hidden activations are rounded to bfloat16 where the
    BF16 training stores them (the arithmetic stays FP64)."""
    a = x
    cache = []
    for l, (W, b) in enumerate(params):
        z = a @ W.T + b
        cache.append((a, z))
        if l + 1 < len(params):
            a = silu(z)
            if emulate_bf16:
                a = round_bf16(a)
        else:
            a = z
    return a[:, 0], cache


def loss_and_grads(params, x, y, emulate_bf16=False):
    """Mean-squared error and its gradients (hand-derived chain rule).

    emulate_bf16: the backward operands of the BF16 training are rounded to
    bfloat16 where it rounds them (the output gradient dz of each layer before
    it multiplies weights or activations); bias gradients sum the unrounded dz."""
    f, cache = forward(params, x, emulate_bf16)
    n = len(y)
    loss = float(np.mean((f - y) ** 2))
    dz = (2.0 / n) * (f - y)[:, None]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        a_prev, z = cache[l]
        if l + 1 < len(params):
            dz = dz * dsilu(z)
        W, _ = params[l]
        dzq = round_bf16(dz) if emulate_bf16 else dz
        grads[l] = [dzq.T @ a_prev, dz.sum(0)]
        dz = dzq @ W
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state.update(t=0, m=[[np.zeros_like(p) for p in l] for l in params],
                     v=[[np.zeros_like(p) for p in l] for l in params])
    state["t"] += 1
    t = state["t"]
    for l in range(len(params)):
        for k in range(2):
            g = grads[l][k]
            m = state["m"][l][k] = b1 * state["m"][l][k] + (1 - b1) * g
            v = state["v"][l][k] = b2 * state["v"][l][k] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            params[l][k] = params[l][k] - lr * mh / (np.sqrt(vh) + eps)


def unweight_two_stage(w, w_hat, u1, u2, w_hat_max, r_max):
    """Accept mask after both stages, weights of the accepted events, and the
    stage-1 mask (the events whose exact matrix element is needed)."""
    s1 = u1 < w_hat / w_hat_max
    r = w / w_hat
    acc = s1 & (u2 < r / r_max)
    wt = np.maximum(1.0, w_hat / w_hat_max) * np.maximum(1.0, r / r_max)
    return acc, np.where(acc, wt, 0.0), s1
