"""nbgs_final_residuals_noalloc: the residual evaluation for callers that
cannot allocate device memory (its scratch is a static device array inside
the library).  Called twice in a row through the C ABI, each time checked
against nbgs_final_residuals() of a scene holding the same contacts and
bodies.  Kept in its own file, collected last."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def test_noalloc_residuals_match_scene_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs

    sc = scenes.config1(2)
    sc["vel"][:, 2] -= 3.0
    sc["params"]["dt"] = 2e-2
    prm = sc["params"]
    r, rho = sc["radius"], sc["density"]
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
        assert len(c["j1"]) > 1000
        args = [_dev(torch, c["j1"].astype(np.int32), torch.int32), _dev(torch, c["j2"].astype(np.int32), torch.int32),
                _dev(torch, c["normal"], torch.float64), _dev(torch, c["xi"], torch.float64),
                _dev(torch, c["impulse"], torch.float64), _dev(torch, b["vel"], torch.float64),
                _dev(torch, b["angvel"], torch.float64), _dev(torch, r, torch.float64),
                _dev(torch, invm, torch.float64), _dev(torch, invI, torch.float64)]
        rc = lib.nbgs_final_residuals_noalloc(len(r), len(c["j1"]), *[a.data_ptr() for a in args],
                                              prm["dt"], prm["beta"], prm["mu"], st["v_ref"], out.data_ptr(),
                                              C.c_void_p(stream.cuda_stream))
        assert rc == nbgs.NBGS_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = np.array([ref[k] for k in ("non_penetration", "cone", "complementarity", "dissipation")])
        assert np.all(want[[0, 2]] > 1e-6)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-13), (call, got, want)
    # sizes beyond the static scratch are refused
    assert lib.nbgs_final_residuals_noalloc(1, 2_097_153, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1e-3, 1.0, 0.5, 1.0,
                                            out.data_ptr(), None) == nbgs.NBGS_ECAPACITY
    g.close()
