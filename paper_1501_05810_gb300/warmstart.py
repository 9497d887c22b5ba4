"""Learned warm start: training data from the solver, training on the GPU,
evaluation.

Data: (features, converged impulse) pairs.  Scenes are stepped with the
previous-step warm start; at every step the features are read after the
colouring and the impulses after a tight solve (tol_data), expressed in the
network's frame (n, e2, e3) and scale (w_n / v_ref).  Training: mini-batch
Adam on the mean squared error, every forward/backward/update in the CUDA
kernels of libnbgs (nbgs_mlp_grad, nbgs_mlp_adam); torch only holds the
device buffers.  Evaluation: sweeps to a tolerance with cold, previous-step
and network warm starts on the same scenes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import nbgs

N_PARAMS = 9347
SIZES = (12, 64, 64, 64, 3)


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform initialisation with limits sqrt(6 / (fan_in + fan_out)), zero
    biases, in the flat layout of the library (W out x in, then b)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in zip(SIZES[:-1], SIZES[1:]):
        lim = np.sqrt(6.0 / (i + o))
        parts += [rng.uniform(-lim, lim, o * i), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def targets_in_frame(impulse: np.ndarray, feat16: np.ndarray) -> np.ndarray:
    """Contact-frame impulses (p_n, p_t, p_o) -> the network's output frame
    and scale: (p_n, p.e2, p.e3) * w_n / v_ref, e2 = cos t + sin o."""
    c, s = feat16[:, 12].astype(np.float64), feat16[:, 13].astype(np.float64)
    k = feat16[:, 14].astype(np.float64) / feat16[:, 15].astype(np.float64)
    pn, pt, po = impulse[:, 0], impulse[:, 1], impulse[:, 2]
    return np.stack([pn, pt * c + po * s, -pt * s + po * c], -1) * k[:, None]


def collect(scene_dicts, steps: int, tol_data: float = 1e-9, max_sweeps: int = 5000, skip_steps: int = 0,
            new_only: bool = False, device="cuda:0"):
    """Run each scene for skip_steps + steps steps (previous-step warm start,
    FP64 sweeps to tol_data) and return features X (N x 12) and targets
    T (N x 3) of the last `steps` steps (the first ones are the start-up
    transient, where no previous impulse exists yet); new_only keeps the
    contacts that had no previous-step impulse, the ones the network warm
    start predicts."""
    X, T = [], []
    for sc in scene_dicts:
        sc = dict(sc)
        sc["params"] = dict(sc["params"], warm_start="prev", precision="fp64")
        g = nbgs.Scene(sc, device=device)
        for _ in range(skip_steps):
            g.step(max_sweeps, tol_data, stats=False)
        for _ in range(steps):
            g.detect_contacts()
            g.colour_contacts()
            f = g.mlp_features()
            g.solve_nbgs(max_sweeps, tol_data)
            c = g.get_contacts()
            g.integrate()
            if len(f) == 0:
                continue
            keep = np.all(f[:, 3:6] == 0.0, axis=1) if new_only else np.ones(len(f), bool)
            X.append(f[keep, :12])
            T.append(targets_in_frame(c["impulse"][keep], f[keep]).astype(np.float32))
        g.close()
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, epochs: int = 20, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          theta0=None, device="cuda:0", log=None):
    """Adam on sum((Y - T)^2) / (2 n); returns (theta, list of epoch losses)."""
    import torch
    dev = torch.device(device)
    lib = nbgs.library()
    th = torch.as_tensor(init_params(seed) if theta0 is None else np.asarray(theta0, np.float32), device=dev).clone()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    g = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    Xd = torch.as_tensor(X, device=dev)
    Td = torch.as_tensor(T, device=dev)
    n = len(Xd)
    rng = np.random.default_rng(seed + 1)
    stream = torch.cuda.current_stream(dev).cuda_stream
    losses, step = [], 0
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(n), device=dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = order[b0:b0 + batch]
            xb, tb = Xd[idx].contiguous(), Td[idx].contiguous()
            rc = lib.nbgs_mlp_grad(th.data_ptr(), xb.data_ptr(), tb.data_ptr(), len(idx), g.data_ptr(),
                                   loss.data_ptr(), stream)
            assert rc == nbgs.NBGS_OK
            step += 1
            rc = lib.nbgs_mlp_adam(th.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), N_PARAMS, lr, 0.9, 0.999,
                                   1e-8, step, stream)
            assert rc == nbgs.NBGS_OK
            tot += float(loss.item()) * len(idx)
            cnt += len(idx)
        losses.append(tot / cnt)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.6g}")
    return th.cpu().numpy(), losses


def infer(theta, X, device="cuda:0"):
    """The tensor-core forward of the library on rows X."""
    import torch
    dev = torch.device(device)
    th = torch.as_tensor(np.asarray(theta, np.float32), device=dev)
    Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=dev)
    Y = torch.empty((len(Xd), 3), dtype=torch.float32, device=dev)
    rc = nbgs.library().nbgs_mlp_infer(th.data_ptr(), Xd.data_ptr(), Y.data_ptr(), len(Xd),
                                       torch.cuda.current_stream(dev).cuda_stream)
    assert rc == nbgs.NBGS_OK
    return Y.cpu().numpy()


def sweeps_to_tolerance(scene_dict, mode: str, theta=None, steps: int = 5, tol: float = 1e-6,
                        max_sweeps: int = 2000, warm_steps: int = 3, device="cuda:0"):
    """Sweeps each of `steps` consecutive steps needs to reach tol with the
    given warm start ('none', 'prev', 'mlp'), after `warm_steps` steps run
    with the previous-step warm start to reach a state with contact history."""
    sc = dict(scene_dict)
    sc["params"] = dict(sc["params"], warm_start="prev")
    g = nbgs.Scene(sc, device=device)
    if theta is not None:
        g.mlp_load(theta)
    for _ in range(warm_steps):
        g.step(max_sweeps, tol)
    out = []
    mode_code = {"none": nbgs.NBGS_WARM_NONE, "prev": nbgs.NBGS_WARM_PREV, "mlp": nbgs.NBGS_WARM_MLP}[mode]
    for _ in range(steps):
        _set_warm(g, mode_code)
        st = g.step(max_sweeps, tol)
        out.append(st["sweeps_done"])
    g.close()
    return np.array(out)


def _set_warm(g, code):
    # the warm-start mode is read from the scene's parameters at every solve
    rc = nbgs.library().nbgs_set_warm_start(g.h, int(code))
    if rc != nbgs.NBGS_OK:
        raise nbgs.NBGSError(rc, "nbgs_set_warm_start", nbgs.library().nbgs_last_error(g.h).decode())
