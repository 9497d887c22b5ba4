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
                        max_sweeps: int = 2000, warm_steps: int = 3, device="cuda:0", times: bool = False):
    """Sweeps each of `steps` consecutive steps needs to reach tol with the
    given warm start ('none', 'prev', 'mlp'), after `warm_steps` steps run
    with the previous-step warm start to reach a state with contact history.
    times: also the device time of each solve (CUDA events around
    nbgs_solve_nbgs: the network's prologue, fused into the sweep kernel, and
    the sweeps), in ms."""
    import torch
    sc = dict(scene_dict)
    sc["params"] = dict(sc["params"], warm_start="prev")
    g = nbgs.Scene(sc, device=device)
    if theta is not None:
        g.mlp_load(theta)
    for _ in range(warm_steps):
        g.step(max_sweeps, tol)
    out, ms = [], []
    mode_code = {"none": nbgs.NBGS_WARM_NONE, "prev": nbgs.NBGS_WARM_PREV, "mlp": nbgs.NBGS_WARM_MLP}[mode]
    for _ in range(steps):
        _set_warm(g, mode_code)
        g.detect_contacts()
        g.colour_contacts()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        k, _ = g.solve_nbgs(max_sweeps, tol)
        e1.record(g.stream)
        g.integrate()
        torch.cuda.synchronize()
        out.append(k)
        ms.append(e0.elapsed_time(e1))
    g.close()
    return (np.array(out), np.array(ms)) if times else np.array(out)


def _set_warm(g, code):
    # the warm-start mode is read from the scene's parameters at every solve
    rc = nbgs.library().nbgs_set_warm_start(g.h, int(code))
    if rc != nbgs.NBGS_OK:
        raise nbgs.NBGSError(rc, "nbgs_set_warm_start", nbgs.library().nbgs_last_error(g.h).decode())


def settling_training_data(target: int = 5_000_000, steps: int = 250, tol_data: float = 1e-7, first_seed: int = 100,
                           max_runs: int = 200, device="cuda:0", log=None):
    """(features, converged impulse) pairs of the contacts that appear while
    1,000-sphere lattice boxes (the FP64 workload's setup, dt = 2e-3) settle
    under gravity: every contact without a previous-step impulse, at every
    step; runs with seeds first_seed, first_seed + 1, ... until `target`
    pairs are collected (the last run's are kept whole)."""
    from . import scenes
    X, T, got = [], [], 0
    for s in range(first_seed, first_seed + max_runs):
        sc = scenes.lattice_box(seed=int(s), per_side=10, dt=2e-3, mu=0.5, tau=0.005, vel_sigma=0.1 + 0.05 * (s % 4))
        x, t = collect([sc], steps=steps, tol_data=tol_data, max_sweeps=5000, new_only=True, device=device)
        X.append(x)
        T.append(t)
        got += len(x)
        if log:
            log(f"settling run {s}: {len(x)} new-contact samples ({got} in all)")
        if got >= target:
            break
    return np.concatenate(X), np.concatenate(T)


def hopper_evaluation(n: int = 2_000_000, settle_steps: int = 600, settle_sweeps: int = 30, eval_steps: int = 4,
                      tol: float = 1e-6, max_sweeps: int = 4000, theta=None, train_epochs: int = 30, seed: int = 0,
                      samples: int = 5_000_000, checkpoint: str = "/tmp/nbgs_hopper_eval.ckpt", device="cuda:0",
                      log=None) -> dict:
    """Hopper discharge (conical hopper, 30 degree half-angle, orifice 8 r,
    mu = 0.5): sweeps and device time per step to residual tol with cold,
    previous-step and network warm starts, from the same state.

    The hopper runs settle_steps FP32 steps (previous-step warm start,
    settle_sweeps sweeps) until it discharges through the orifice; its state
    moves into an FP64 scene, which steps once with the previous-step warm
    start (the contact history every mode starts from) and is checkpointed.
    Each mode then restores the checkpoint and runs eval_steps steps with FP64
    sweeps to tol (FP32 sweeps stall above 1e-6 on dense packings).  The
    network is trained first on settling runs unless theta is given."""
    import time
    import torch
    from . import scenes
    say = log or (lambda *_: None)
    out = {"n": n, "tol": tol, "eval_steps": eval_steps, "settle_steps": settle_steps}
    if theta is None:
        t0 = time.perf_counter()
        X, T = settling_training_data(target=samples, device=device, log=say)
        theta, losses = train(X, T, epochs=train_epochs, batch=4096, lr=1e-3, seed=seed, device=device)
        out["training"] = {"samples": int(len(X)), "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                           "seconds": time.perf_counter() - t0}
        say(f"trained on {len(X)} samples: loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    sc = scenes.hopper(n, seed=seed)
    sc32 = dict(sc, params=dict(sc["params"], precision="fp32", warm_start="prev"))
    g = nbgs.Scene(sc32, device=device)
    t0 = time.perf_counter()
    for _ in range(settle_steps):
        st = g.step(settle_sweeps, 0.0, stats=False)
    torch.cuda.synchronize()
    b = g.get_bodies()
    nc = g.step(settle_sweeps, 0.0)["n_contacts"]
    g.close()
    cn = sc["cones"][0]
    z_o = cn["r_orifice"] / np.tan(cn["half_angle"])   # orifice height above the apex (apex at the origin)
    out["settle"] = {"seconds": time.perf_counter() - t0, "contacts": int(nc),
                     "below_orifice": int(np.count_nonzero(b["pos"][:, 2] < z_o))}
    say(f"settled: {nc} contacts, {out['settle']['below_orifice']} spheres discharged")
    sc64 = dict(sc, params=dict(sc["params"], precision="fp64", warm_start="prev"))
    h = nbgs.Scene(sc64, device=device)
    h.set_bodies(b["pos"], b["quat"], b["vel"], b["angvel"])
    h.mlp_load(theta)
    h.step(max_sweeps, tol)
    h.save_state(checkpoint)
    h.close()
    modes = {}
    for mode in ("none", "prev", "mlp"):
        s = nbgs.Scene(sc64, device=device)
        s.load_state(checkpoint)
        _set_warm(s, {"none": nbgs.NBGS_WARM_NONE, "prev": nbgs.NBGS_WARM_PREV, "mlp": nbgs.NBGS_WARM_MLP}[mode])
        sweeps, ms, res, ncon, nnew = [], [], [], [], []
        for _ in range(eval_steps):
            s.detect_contacts()
            s.colour_contacts()
            f = s.mlp_features()   # columns 3..5: previous impulse (0: new, or no push last step)
            nnew.append(int(np.count_nonzero(np.all(f[:, 3:6] == 0.0, axis=1))) if len(f) else 0)
            ncon.append(int(len(f)))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)   # the solve: the network's prologue (fused into the sweep kernel) and the sweeps
            k, r = s.solve_nbgs(max_sweeps, tol)
            e1.record(s.stream)
            s.integrate()
            torch.cuda.synchronize()
            sweeps.append(int(k))
            res.append(float(r))
            ms.append(e0.elapsed_time(e1))
        modes[mode] = {"sweeps": sweeps, "solve_ms": ms, "residual": res, "contacts": ncon, "zero_prev_impulse": nnew,
                       "total_solve_ms": float(sum(ms))}
        say(f"{mode}: sweeps {sweeps}, solve ms {[round(x, 1) for x in ms]}, R {['%.2g' % x for x in res]}, "
            f"zero previous impulse {nnew} of {ncon}")
        s.close()
    out["modes"] = modes
    return out


if __name__ == "__main__":  # pragma: no cover
    import argparse
    import json
    ap = argparse.ArgumentParser(description="warm-start evaluation on the hopper discharge")
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--settle-steps", type=int, default=600)
    ap.add_argument("--eval-steps", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--max-sweeps", type=int, default=4000)
    ap.add_argument("--samples", type=int, default=5_000_000, help="training pairs from settling runs")
    a = ap.parse_args()
    r = hopper_evaluation(n=a.n, settle_steps=a.settle_steps, eval_steps=a.eval_steps, train_epochs=a.epochs,
                          max_sweeps=a.max_sweeps, samples=a.samples, log=lambda m: print(m, flush=True))
    print(json.dumps(r))
