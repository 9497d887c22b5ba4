"""Checkpoint and resume through the C ABI (nbgs_save_state / nbgs_load_state).

A scene steps N times and saves; it steps M more times.  A second scene,
created from the same inputs, loads the checkpoint and steps M times.  The
two must end bit-identical: bodies, contacts, colours, impulses.  With the
previous-step warm start on, this also checks that the saved contacts and
world impulses feed the next step's warm start exactly as in the original
run.  Mismatched scenes and damaged files are refused."""
import os

import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def _state(g):
    b, c = g.get_bodies(), g.get_contacts()
    return b, c


def _assert_identical(s1, s2):
    (b1, c1), (b2, c2) = s1, s2
    for k in ("pos", "quat", "vel", "angvel"):
        assert np.array_equal(b1[k], b2[k]), k
    for k in ("j1", "j2", "colour", "normal", "xi", "impulse"):
        assert np.array_equal(c1[k], c2[k]), k


@pytest.mark.parametrize("case", ["config1_fp64", "hcp_fp32"])
def test_resume_is_bit_identical(nb, tmp_path, case):
    if case == "config1_fp64":
        sc = scenes.config1(0)
        sweeps, tol = 30, 0.0
    else:
        sc = scenes.hcp_packing(12, 12, 8, dt=1e-3, tau=0.005, mu=0.6, tilt_deg=10.0, v0=0.05, precision="fp32")
        sweeps, tol = 40, 1e-6
    sc["params"]["warm_start"] = "prev"
    a = nb.Scene(sc)
    for _ in range(3):
        a.step(sweeps, tol)
    path = str(tmp_path / f"{case}.nbgs")
    a.save_state(path)
    assert os.path.getsize(path) > 0
    for _ in range(2):
        a.step(sweeps, tol)
    ref = _state(a)

    b = nb.Scene(sc)
    b.step(sweeps, tol)   # its own history must not leak into the resumed run
    b.load_state(path)
    for _ in range(2):
        b.step(sweeps, tol)
    _assert_identical(ref, _state(b))


def test_resume_before_any_step_and_twice(nb, tmp_path):
    sc = scenes.column(6, dt=1e-3, warm_start="prev")
    sc["params"]["tau"] = 0.01
    a = nb.Scene(sc)
    a.step(5)
    p1 = str(tmp_path / "c1.nbgs")
    a.save_state(p1)
    b = nb.Scene(sc)
    b.load_state(p1)
    p2 = str(tmp_path / "c2.nbgs")
    b.save_state(p2)   # a restored, not yet stepped scene saves the same warm-start data
    c = nb.Scene(sc)
    c.load_state(p2)
    for g in (a, b, c):
        g.step(5)
        g.step(5)
    _assert_identical(_state(a), _state(b))
    _assert_identical(_state(a), _state(c))


def test_mismatched_scene_and_damaged_file_are_refused(nb, tmp_path):
    a = nb.Scene(scenes.column(4, dt=1e-3, warm_start="prev"))
    a.step(3)
    path = str(tmp_path / "col4.nbgs")
    a.save_state(path)
    other = nb.Scene(scenes.column(5, dt=1e-3, warm_start="prev"))
    with pytest.raises(nb.NBGSError, match="body count"):
        other.load_state(path)
    bad = str(tmp_path / "bad.nbgs")
    with open(path, "rb") as f:
        data = f.read()
    with open(bad, "wb") as f:
        f.write(data[:-16])   # the header survives; the impulses are cut short
    fresh = nb.Scene(scenes.column(4, dt=1e-3, warm_start="prev"))
    with pytest.raises(nb.NBGSError, match="truncated"):
        fresh.load_state(bad)
    fresh2 = nb.Scene(scenes.column(4, dt=1e-3, warm_start="prev"))
    with pytest.raises(nb.NBGSError, match="cannot open"):
        fresh2.load_state(str(tmp_path / "missing.nbgs"))


def test_corrupt_header_and_rows_are_refused(nb, tmp_path):
    """A damaged checkpoint is refused before anything reaches the device:
    cone and plane counts beyond the arrays, parameters a scene could not be
    created with, a precision other than the scene's, a non-finite largest
    radius, warm-start rows that leave [0, prev_count], a radius beyond the
    largest one.  The header layout (host byte order, natural alignment) is
    checked against known values first."""
    import struct
    sc = scenes.column(4, dt=1e-3, warm_start="prev")
    a = nb.Scene(sc)
    a.step(3)
    path = str(tmp_path / "ok.nbgs")
    a.save_state(path)
    data = bytearray(open(path, "rb").read())
    hb, n = struct.unpack_from("<I", data, 12)[0], struct.unpack_from("<q", data, 16)[0]
    prev_count = struct.unpack_from("<q", data, 32)[0]
    assert n == 4 and prev_count > 0 and struct.unpack_from("<i", data, 28)[0] == 1
    R_MAX, PRM, PLANES = 48, 56, 224
    assert struct.unpack_from("<d", data, R_MAX)[0] == 0.5
    assert struct.unpack_from("<d", data, PRM)[0] == 1e-3                       # prm.dt
    assert struct.unpack_from("<i", data, PRM + 124)[0] == nb.NBGS_FP64          # prm.precision
    assert struct.unpack_from("<i", data, PLANES)[0] == 1                       # planes.count
    NCONES = PLANES + 8 + 16 * 24 + 16 * 8
    assert struct.unpack_from("<i", data, NCONES)[0] == 0
    vbytes = 32                                                                   # FP64 velocity records
    OFF = hb + n * 32 + n * 32 + n * 2 * vbytes + n
    assert struct.unpack_from("<I", data, OFF)[0] == 0
    assert struct.unpack_from("<I", data, OFF + 4 * n)[0] == prev_count

    def damaged(fmt, at, value):
        d = bytearray(data)
        struct.pack_into(fmt, d, at, value)
        return d

    cases = [("corrupt header", damaged("<i", NCONES, 1000)),
             ("corrupt header", damaged("<i", PLANES, 17)),
             ("corrupt header", damaged("<d", PRM, -1.0)),
             ("corrupt header", damaged("<i", PRM + 124, nb.NBGS_FP32)),
             ("corrupt header", damaged("<d", R_MAX, float("nan"))),
             ("inconsistent", damaged("<I", OFF + 4, prev_count + 5)),
             ("inconsistent", damaged("<d", hb + 32 * 2 + 24, 0.75))]   # radius of body 2 above r_max
    for k, (msg, d) in enumerate(cases):
        bad = str(tmp_path / f"bad{k}.nbgs")
        open(bad, "wb").write(bytes(d))
        fresh = nb.Scene(sc)
        with pytest.raises(nb.NBGSError, match=msg) as e:
            fresh.load_state(bad)
        assert e.value.status == nb.NBGS_EINVAL
    # the undamaged file still loads and steps
    b = nb.Scene(sc)
    b.load_state(path)
    b.step(3)
