"""FP64 reference of the warm-start MLP (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU leg use this module.
It is written from the chain rule, independently of the CUDA kernels in
``paper_1501_05810_gb300/csrc/mlp.cu``; the two share only the parameter
layout below (an interface, not code).

Network: 12 inputs -> 64 -> 64 -> 64 -> 3, SiLU after each hidden layer,
linear output layer, plus a skip connection that adds inputs 3..5 (the
previous-step impulse in the output frame) to the output, so the layers
learn the correction to the previous impulse.  Parameters, flat, in this
order: for each layer, the weight matrix W (out x in, row-major) then the
bias b (out).  9,347 values.  Loss of a batch of N rows:
L = sum((Y - T)^2) / (2 N).
"""
from __future__ import annotations

import numpy as np

SIZES = (12, 64, 64, 64, 3)
N_PARAMS = sum(o * i + o for i, o in zip(SIZES[:-1], SIZES[1:]))   # 9347


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, k = [], 0
    for i, o in zip(SIZES[:-1], SIZES[1:]):
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X):
    """Returns the output (N x 3) and the pre-activations of each layer."""
    a = np.asarray(X, dtype=np.float64)
    zs, acts = [], [a]
    layers = unflatten(theta)
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = silu(z) if li < len(layers) - 1 else z + acts[0][:, 3:6]   # skip: previous impulse
        acts.append(a)
    return a, zs, acts


def loss(theta, X, T):
    Y, _, _ = forward(theta, X)
    return float(np.sum((Y - np.asarray(T, dtype=np.float64)) ** 2) / (2.0 * len(Y)))


def loss_and_grad(theta, X, T):
    """Loss and its gradient by back-propagation (chain rule, layer by layer)."""
    Y, zs, acts = forward(theta, X)
    n = len(Y)
    layers = unflatten(theta)
    dz = (Y - np.asarray(T, dtype=np.float64)) / n          # dL/dY = dL/dz4 (linear layer + skip)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (dz.T @ acts[li], dz.sum(0))             # dL/dW = dZ^T A_prev, dL/db = sum dZ
        if li > 0:
            dz = (dz @ W) * silu_grad(zs[li - 1])
    L = float(np.sum((Y - T) ** 2) / (2.0 * n))
    return L, flatten(grads)


def loss_and_grad_rounded(theta, X, T, rnd=None):
    """Loss and gradient as loss_and_grad computes them, except that every
    operand of a matrix product is first passed through `rnd`: the inputs,
    the weights, the hidden activations and the back-propagated deltas
    (bfloat16 operands of tensor-core products, sums exact).  The biases, the
    skip connection, the loss and the bias gradients use the unrounded
    values, and the activations that feed the next layer are the rounded
    ones.  rnd = None rounds to bfloat16; the identity gives
    loss_and_grad."""
    rnd = bf16_round if rnd is None else rnd
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    layers = unflatten(theta)
    ops, zs = [rnd(X)], []
    for li, (W, b) in enumerate(layers):
        z = ops[-1] @ rnd(W).T + b
        zs.append(z)
        if li < len(layers) - 1:
            ops.append(rnd(silu(z)))
    Y = zs[-1] + X[:, 3:6]
    n = len(Y)
    dz = (Y - T) / n
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        dr = rnd(dz)
        grads[li] = (dr.T @ ops[li], dz.sum(0))
        if li > 0:
            dz = (dr @ rnd(W)) * silu_grad(zs[li - 1])
    L = float(np.sum((Y - T) ** 2) / (2.0 * n))
    return L, flatten(grads)


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; returns new
    (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init(seed=0):
    """He-style uniform initialisation (only used to give tests and training
    a starting point)."""
    rng = np.random.default_rng(seed)
    layers = []
    for i, o in zip(SIZES[:-1], SIZES[1:]):
        lim = np.sqrt(6.0 / (i + o))
        layers.append((rng.uniform(-lim, lim, (o, i)), np.zeros(o)))
    return flatten(layers)


def bf16_round(x):
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def contact_frame_np(n):
    """Duff et al. (JCGT 2017) tangent basis, vectorised (same construction as
    the C oracle's oracle_contact_frame)."""
    sign = np.copysign(1.0, n[:, 2])
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t = np.stack([1.0 + sign * n[:, 0] * n[:, 0] * a, sign * b, -sign * n[:, 0]], -1)
    o = np.stack([b, sign + n[:, 1] * n[:, 1] * a, -n[:, 1]], -1)
    return t, o


def contact_features(c, bodies, radius, invm, invI, params, v_ref, prev=None):
    """The 12 network inputs of every contact (plus cos, sin of e2 in (t, o),
    w_n and v_ref), in FP64, from the state at the start of a step.

    c: contacts (j1, j2, normal, xi) in canonical order; bodies: pos, vel,
    angvel at the start of the step; prev: previous step's contacts (j1, j2,
    normal, impulse) whose world impulses are matched by key, or None."""
    n_b = len(radius)
    j1, j2 = c["j1"].astype(np.int64), c["j2"].astype(np.int64)
    nrm, xi = c["normal"], c["xi"]
    dyn = j2 < n_b
    jb = np.where(dyn, j2, 0)
    dt, g = params["dt"], np.asarray(params["gravity"], dtype=np.float64)
    r_a = radius[j1]
    r_b = np.where(dyn, radius[jb], 0.0)
    la = xi + r_a                       # l_a = -la n, for spheres and walls
    lb = np.where(dyn, r_b, 0.0)        # l_b = lb n
    kick = lambda idx, ok: bodies["vel"][idx] + np.where((invm[idx] > 0) & ok, 1.0, 0.0)[:, None] * dt * g
    va = kick(j1, np.ones_like(dyn))
    vb = np.where(dyn[:, None], kick(jb, dyn), 0.0)
    wa = bodies["angvel"][j1]
    wb = np.where(dyn[:, None], bodies["angvel"][jb], 0.0)
    u = va + np.cross(wa, -la[:, None] * nrm) - vb - np.cross(wb, lb[:, None] * nrm)
    t, o = contact_frame_np(nrm)
    un = np.sum(u * nrm, 1)
    ut, uo = np.sum(u * t, 1), np.sum(u * o, 1)
    utl = np.hypot(ut, uo)
    big = utl > 1e-12 * v_ref
    cth = np.where(big, -ut / np.where(big, utl, 1.0), 1.0)
    sth = np.where(big, -uo / np.where(big, utl, 1.0), 0.0)
    e2 = cth[:, None] * t + sth[:, None] * o
    e3 = -sth[:, None] * t + cth[:, None] * o
    finite = (invm > 0) | (invI > 0)
    wn = invm[j1] + np.where(dyn, invm[jb], 0.0)
    wt = wn + invI[j1] * la * la + np.where(dyn, invI[jb], 0.0) * lb * lb
    P = np.zeros((len(j1), 3))
    if prev is not None and len(prev["j1"]):
        pk = (prev["j1"].astype(np.int64) << 32) | prev["j2"].astype(np.int64)
        pt_, po_ = contact_frame_np(prev["normal"])
        Pw = (prev["impulse"][:, :1] * prev["normal"] + prev["impulse"][:, 1:2] * pt_
              + prev["impulse"][:, 2:3] * po_)
        key = (j1 << 32) | j2
        pos = np.searchsorted(pk, key)
        pos = np.minimum(pos, len(pk) - 1)
        hit = pk[pos] == key
        P[hit] = Pw[pos[hit]]
        # previous impulse re-projected onto the new contact's cone (the warm start)
        pn = np.maximum(np.sum(P * nrm, 1), 0.0)
        ptt, poo = np.sum(P * t, 1), np.sum(P * o, 1)
        lim = params["mu"] * pn
        ln = np.hypot(ptt, poo)
        f = np.where(ln > lim, np.where(ln > 0, lim / np.where(ln > 0, ln, 1.0), 0.0), 1.0)
        P = pn[:, None] * nrm + (f * ptt)[:, None] * t + (f * poo)[:, None] * o
    deg = np.zeros(n_b)
    np.add.at(deg, j1[finite[j1]], 1)
    np.add.at(deg, jb[dyn & finite[jb]], 1)
    da = np.where(finite[j1], deg[j1], 0)
    db = np.where(dyn & finite[jb], deg[jb], 0)
    sc = wn / v_ref
    F = np.stack([un / v_ref, utl / v_ref, (xi / dt) / v_ref,
                  np.sum(P * nrm, 1) * sc, np.sum(P * e2, 1) * sc, np.sum(P * e3, 1) * sc,
                  np.log(wn), wt / wn, r_a, r_b, np.full(len(j1), params["mu"]), (da + db) / 12.0,
                  cth, sth, wn, np.full(len(j1), v_ref)], -1)
    return F
