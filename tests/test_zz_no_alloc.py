"""nbgs_final_residuals_noalloc: the residual evaluation for callers that
cannot allocate device memory (its scratch is a static device array inside
the library).  Called twice in a row through the C ABI, each time checked
against nbgs_final_residuals() of a scene holding the same contacts and
bodies, on a contact list that spans many blocks of the reduction; then once
at exactly the largest accepted size.  Kept in its own file, collected last."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu

KEYS = ("non_penetration", "cone", "complementarity", "dissipation")
TILE = 2048            # contacts per block of the reduction
MAX_CONTACTS = 2_097_152


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _call(torch, nbgs, lib, n_bodies, j1, j2, c, vel, ang, r, invm, invI, prm, v_ref, out, stream):
    args = [_dev(torch, j1.astype(np.int32), torch.int32), _dev(torch, j2.astype(np.int32), torch.int32),
            _dev(torch, c["normal"], torch.float64), _dev(torch, c["xi"], torch.float64),
            _dev(torch, c["impulse"], torch.float64), _dev(torch, vel, torch.float64),
            _dev(torch, ang, torch.float64), _dev(torch, r, torch.float64),
            _dev(torch, invm, torch.float64), _dev(torch, invI, torch.float64)]
    rc = lib.nbgs_final_residuals_noalloc(n_bodies, len(j1), *[a.data_ptr() for a in args], prm["dt"], prm["beta"],
                                          prm["mu"], v_ref, out.data_ptr(), C.c_void_p(stream.cuda_stream))
    assert rc == nbgs.NBGS_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_residuals_match_scene_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs

    sc = scenes.loose_pour(seed=2, n=9001)
    sc["vel"] = np.random.default_rng(7).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    prm = sc["params"]
    r, rho = sc["radius"], sc["density"]
    n = len(r)
    mass = rho * (4.0 / 3.0) * math.pi * r * r * r
    invm, invI = 1.0 / mass, 1.0 / (0.4 * mass * r * r)
    g = nbgs.Scene(sc, device="cuda:0")
    lib = nbgs.library()
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream()
    for call in range(2):
        st = g.step(8)            # few sweeps: residuals well above zero
        ref = g.final_residuals()
        c, b = g.get_contacts(), g.get_bodies()
        assert len(c["j1"]) > 3 * TILE   # several blocks of the reduction
        got = _call(torch, nbgs, lib, n, c["j1"], c["j2"], c, b["vel"], b["angvel"], r, invm, invI, prm,
                    st["v_ref"], out, stream)
        want = np.array([ref[k] for k in KEYS])
        assert np.all(want[[0, 2, 3]] > 1e-6)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-13), (call, got, want)
    # exactly the largest accepted size: the scene's contacts and bodies
    # repeated (each copy with its own bodies, walls past all of them) and cut
    # at 2,097,152 contacts; every copy is the same, so the maxima are the
    # scene's
    m = len(c["j1"])
    k = -(-MAX_CONTACTS // m)
    rep = np.repeat(np.arange(k, dtype=np.int64), m)[:MAX_CONTACTS]
    j1 = (np.tile(c["j1"].astype(np.int64), k)[:MAX_CONTACTS] + rep * n)
    j2s = np.tile(c["j2"].astype(np.int64), k)[:MAX_CONTACTS]
    j2 = np.where(j2s < n, j2s + rep * n, k * n)
    big = {f: np.tile(c[f], (k,) + (1,) * (c[f].ndim - 1))[:MAX_CONTACTS] for f in ("normal", "xi", "impulse")}
    got = _call(torch, nbgs, lib, k * n, j1, j2, big, np.tile(b["vel"], (k, 1)), np.tile(b["angvel"], (k, 1)),
                np.tile(r, k), np.tile(invm, k), np.tile(invI, k), prm, st["v_ref"], out, stream)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-13), (got, want)
    # sizes beyond the static scratch are refused
    assert lib.nbgs_final_residuals_noalloc(1, MAX_CONTACTS + 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1e-3, 1.0, 0.5, 1.0,
                                            out.data_ptr(), None) == nbgs.NBGS_ECAPACITY
    g.close()
