"""Learned warm start on the GPU against the FP64 references in oracle/:
tensor-core inference and training (tcgen05, BF16 operands, FP32 accumulation in
TMEM), Adam, the per-contact feature map, and the network inside the sweep
kernel's prologue."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs, warmstart
    return torch, nbgs, warmstart


def _forward_bf16(theta, X):
    """The FP64 reference with the GPU's roundings: BF16 weights, inputs and
    hidden activations, exact sums."""
    layers = omlp.unflatten(theta)
    a = omlp.bf16_round(X)
    for li, (W, b) in enumerate(layers):
        z = a @ omlp.bf16_round(W).T + np.asarray(b, dtype=np.float32)
        a = omlp.bf16_round(omlp.silu(z)) if li < 3 else z + X[:, 3:6]   # skip added in FP32
    return a


def test_tensor_core_inference_matches_reference(env):
    torch, nb, ws = env
    rng = np.random.default_rng(0)
    theta = ws.init_params(3) + rng.normal(0, 0.02, ws.N_PARAMS).astype(np.float32)
    for n in (1, 16, 17, 127, 128, 129, 1000, 4099):   # partial and full 128-row tiles
        X = rng.normal(0, 1.0, (n, 12)).astype(np.float32)
        Y = ws.infer(theta, X)
        ref = _forward_bf16(theta.astype(np.float64), X.astype(np.float64))
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(Y - ref).max() <= 2e-2 * scale, (n, np.abs(Y - ref).max())
        full = omlp.forward(theta.astype(np.float64), X.astype(np.float64))[0]
        assert np.abs(Y - full).max() <= 6e-2 * scale     # BF16 versus exact


@pytest.mark.parametrize("n", [1000, 40000])
def test_training_gradient_matches_reference(env, n):
    """Forward and backward on the tensor cores (BF16 operands, FP32
    accumulation in TMEM) against the FP64 reference with the same operand
    roundings (oracle.mlp.loss_and_grad_rounded): the loss to 1e-5, the
    gradient to 5e-4 of its largest entry, direction to 1e-8.  n = 1000: one
    ragged 128-sample tile per CTA; n = 40,000: two or three tiles per CTA,
    so the weight gradients accumulate in TMEM across tiles.  And within
    BF16 precision of the exact gradient."""
    torch, nb, ws = env
    rng = np.random.default_rng(1)
    theta = ws.init_params(4) + rng.normal(0, 0.02, ws.N_PARAMS).astype(np.float32)
    X = rng.normal(size=(n, 12)).astype(np.float32)
    T = rng.normal(size=(n, 3)).astype(np.float32)
    dev = torch.device("cuda:0")
    th, Xd, Td = (torch.as_tensor(a, device=dev) for a in (theta, X, T))
    g = torch.zeros(ws.N_PARAMS, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    assert nb.library().nbgs_mlp_grad(th.data_ptr(), Xd.data_ptr(), Td.data_ptr(), n, g.data_ptr(), loss.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream) == nb.NBGS_OK
    torch.cuda.synchronize()
    th64, X64, T64 = theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    L, G = omlp.loss_and_grad_rounded(th64, X64, T64)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - L) <= 1e-5 * L, (loss.item(), L)
    err = np.abs(gg - G).max() / np.abs(G).max()
    cos = np.dot(gg, G) / (np.linalg.norm(gg) * np.linalg.norm(G))
    print(f"n={n}: gradient vs rounded reference: max err {err:.2e} of the largest, 1 - cos {1 - cos:.2e}")
    assert err <= 5e-4 and cos > 1 - 1e-8   # measured on a GB300: 4.7e-5 / 1.3e-10 (n = 1000)
    Le, Ge = omlp.loss_and_grad(th64, X64, T64)
    assert np.dot(gg, Ge) / (np.linalg.norm(gg) * np.linalg.norm(Ge)) > 1 - 1e-3


def test_adam_step_matches_reference(env):
    torch, nb, ws = env
    rng = np.random.default_rng(2)
    th0 = rng.normal(size=ws.N_PARAMS).astype(np.float32)
    m0 = rng.normal(0, 0.1, ws.N_PARAMS).astype(np.float32)
    v0 = np.abs(rng.normal(0, 0.1, ws.N_PARAMS)).astype(np.float32)
    gr = rng.normal(size=ws.N_PARAMS).astype(np.float32)
    dev = torch.device("cuda:0")
    th, m, v, g = (torch.as_tensor(a, device=dev).clone() for a in (th0, m0, v0, gr))
    assert nb.library().nbgs_mlp_adam(th.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), ws.N_PARAMS, 1e-3,
                                      0.9, 0.999, 1e-8, 7, torch.cuda.current_stream().cuda_stream) == nb.NBGS_OK
    rt, rm, rv = omlp.adam(th0.astype(np.float64), gr.astype(np.float64), m0.astype(np.float64),
                           v0.astype(np.float64), 7, lr=1e-3)
    assert np.allclose(th.cpu().numpy(), rt, atol=1e-6) and np.allclose(m.cpu().numpy(), rm, atol=1e-6)


def test_features_match_reference(env, oracle_mod):
    torch, nb, ws = env
    sc = scenes.lattice_box(seed=5, per_side=5, spacing=1.02, vel_sigma=1.0, dt=2e-2, tau=0.01, warm_start="prev")
    sc["angvel"] = np.random.default_rng(6).normal(0, 1.0, sc["vel"].shape)
    g = nb.Scene(sc)
    o = oracle_mod.OracleScene(sc)
    g.step(30)
    o.step(30)
    prev = o.get_contacts()
    start = o.get_bodies()
    o.detect_contacts()
    co = o.get_contacts()
    g.set_bodies(start["pos"], start["quat"], start["vel"], start["angvel"])   # same start, FP rounding aside
    # set_bodies drops the previous-step impulses of the GPU scene: rerun the
    # previous step there from the oracle's previous start instead
    g2 = nb.Scene(sc)
    g2.step(30)
    g2.detect_contacts()
    g2.colour_contacts()
    F = g2.mlp_features()
    r, rho = sc["radius"], sc["density"]
    mass = rho * 4.0 / 3.0 * math.pi * r ** 3
    vref = max(np.linalg.norm(start["vel"], axis=1).max(), 9.81 * sc["params"]["dt"], 1e-12)
    ref = omlp.contact_features(co, start, r, 1.0 / mass, 1.0 / (0.4 * mass * r * r), sc["params"], vref, prev)
    assert len(F) == len(ref) > 100
    scale = np.maximum(1.0, np.abs(ref).max(0))
    assert np.all(np.abs(F - ref).max(0) <= 1e-5 * scale), np.abs(F - ref).max(0) / scale


def test_fused_prologue_equals_prologue_kernel(env):
    """The network's warm start inside the persistent sweep kernel (256
    threads per block, its dynamic shared memory as operand space) gives the
    same impulses, bit for bit, as the separate prologue kernel the per-colour
    solver launches (128 threads per block): every row of a 128-row tile is
    computed alone.  Zero sweeps: the impulses are the warm start itself."""
    torch, nb, ws = env
    rng = np.random.default_rng(9)
    theta = (ws.init_params(5) + rng.normal(0, 0.05, ws.N_PARAMS)).astype(np.float32)
    theta[ws.N_PARAMS - 3] = 2.0   # output bias of the normal impulse: positive predictions
    sc = scenes.periodic_cloud(seed=12, per_side=9, dt=2e-2, vel_sigma=1.0, mu=0.4)
    sc["params"]["warm_start"] = "mlp"
    out = []
    for solver in ("persistent", "per_colour"):
        g = nb.Scene(sc, solver=solver)
        g.mlp_load(theta)
        g.detect_contacts()
        g.colour_contacts()
        g.solve_nbgs(0, 0.0)
        out.append(g.get_contacts())
        g.close()
    assert len(out[0]["j1"]) > 300
    assert np.array_equal(out[0]["j1"], out[1]["j1"]) and np.array_equal(out[0]["j2"], out[1]["j2"])
    assert np.array_equal(out[0]["impulse"], out[1]["impulse"])
    assert np.abs(out[0]["impulse"]).max() > 0.0   # the network acted (every contact is new)
