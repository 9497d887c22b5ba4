"""FP64 sequential CPU oracle of the NBGS time step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``nbgs_oracle.c`` (plain C,
double precision, brute-force detection) through ctypes and shares nothing
with the CUDA library in ``paper_1501_05810_gb300``: not a header, not a
helper, not a constant.

The C code follows Preclik & Ruede, arXiv:1501.05810: Sect. 2 (Newton-Euler,
eq. wrench, eq. contactpos), Sect. 3 (eq. integrationscheme,
eq. nonpenetration, eq. coulomb), Sect. 4 (eq. expansionradius), Sect. 5
(Alg. 1) and Sect. 6 (Alg. 2, velocity accumulators).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbgs_oracle.c")
_HDR = os.path.join(_HERE, "nbgs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

WARM_NONE = 0
WARM_PREV = 1
SUB_NONE, SUB_GRID, SUB_JACOBI = 0, 1, 2


class OracleParams(C.Structure):
    _fields_ = [
        ("dt", C.c_double),
        ("gravity", C.c_double * 3),
        ("mu", C.c_double),
        ("omega", C.c_double),
        ("tau", C.c_double),
        ("beta", C.c_double),
        ("box_lo", C.c_double * 3),
        ("box_hi", C.c_double * 3),
        ("periodic", C.c_int32 * 3),
        ("warm_start", C.c_int32),
        ("colour_seed", C.c_uint64),
        ("subdomain_mode", C.c_int32),
        ("subdomains", C.c_int32 * 3),
    ]


class OracleStepStats(C.Structure):
    _fields_ = [
        ("n_contacts", C.c_int64),
        ("n_colours", C.c_int32),
        ("sweeps_done", C.c_int32),
        ("residual", C.c_double),
        ("v_ref", C.c_double),
    ]


class OracleResiduals(C.Structure):
    _fields_ = [
        ("non_penetration", C.c_double),
        ("cone", C.c_double),
        ("complementarity", C.c_double),
        ("dissipation", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no contraction, so the hull predicate
    rounds exactly as written).  Returns the library path."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O3", "-ffp-contract=off", "-fno-fast-math", "-D_GNU_SOURCE",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        dp = P(C.c_double)
        L.oracle_create_scene.argtypes = [P(OracleParams), C.c_int64, dp, dp, dp, dp, dp, P(C.c_void_p)]
        L.oracle_destroy_scene.argtypes = [C.c_void_p]
        L.oracle_destroy_scene.restype = None
        L.oracle_add_plane.argtypes = [C.c_void_p, dp, C.c_double]
        L.oracle_add_cone.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_double, C.c_double]
        L.oracle_cone_distance.argtypes = [C.c_void_p, C.c_int32, dp, dp, dp]
        L.oracle_set_mass_properties.argtypes = [C.c_void_p, dp, dp]
        L.oracle_set_bodies.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.oracle_get_bodies.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.oracle_detect_contacts.argtypes = [C.c_void_p, P(C.c_int64)]
        L.oracle_colour_contacts.argtypes = [C.c_void_p, P(C.c_int32)]
        L.oracle_solve_nbgs.argtypes = [C.c_void_p, C.c_int32, C.c_double, P(C.c_int32), dp]
        L.oracle_integrate.argtypes = [C.c_void_p]
        L.oracle_step.argtypes = [C.c_void_p, C.c_int32, C.c_double, P(OracleStepStats)]
        L.oracle_get_contacts.argtypes = [C.c_void_p, C.c_int64, P(C.c_uint32), P(C.c_uint32),
                                          P(C.c_int32), dp, dp, dp, P(C.c_int64)]
        L.oracle_set_impulses.argtypes = [C.c_void_p, dp]
        L.oracle_contact_subdomains.argtypes = [C.c_void_p, P(C.c_int64)]
        L.oracle_create_composite_scene.argtypes = [P(OracleParams), C.c_int64, dp, dp, dp, dp, C.c_int64,
                                                    P(C.c_int32), dp, dp, P(C.c_void_p)]
        L.oracle_member_positions.argtypes = [C.c_void_p, dp]
        L.oracle_body_mass_properties.argtypes = [C.c_void_p, dp, dp]
        L.oracle_residual_history.argtypes = [C.c_void_p, dp, C.c_int32, P(C.c_int32)]
        L.oracle_final_residuals.argtypes = [C.c_void_p, P(OracleResiduals)]
        L.oracle_contact_frame.argtypes = [dp, dp, dp]
        L.oracle_contact_frame.restype = None
        L.oracle_one_contact.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
        L.oracle_one_contact.restype = None
        L.oracle_one_contact_general.argtypes = [dp, C.c_double, dp, dp]
        L.oracle_one_contact_general.restype = C.c_int
        L.oracle_splitmix64.argtypes = [C.c_uint64]
        L.oracle_splitmix64.restype = C.c_uint64
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle: {what} failed with code {rc}")


def make_params(p: dict) -> OracleParams:
    """Map a scene parameter dict (see paper_1501_05810_gb300.scenes) onto
    the oracle's own parameter struct."""
    o = OracleParams()
    o.dt = p["dt"]
    o.gravity[:] = list(p.get("gravity", (0.0, 0.0, 0.0)))
    o.mu = p.get("mu", 0.5)
    o.omega = p.get("omega", 1.0)
    o.tau = p.get("tau", 0.0)
    o.beta = p.get("beta", 1.0)
    o.box_lo[:] = list(p.get("box_lo", (0.0, 0.0, 0.0)))
    o.box_hi[:] = list(p.get("box_hi", (1.0, 1.0, 1.0)))
    o.periodic[:] = [int(b) for b in p.get("periodic", (0, 0, 0))]
    o.warm_start = WARM_PREV if p.get("warm_start", "none") == "prev" else WARM_NONE
    o.colour_seed = int(p.get("colour_seed", 0)) & 0xFFFFFFFFFFFFFFFF
    sub = p.get("subdomains")
    if sub is None:
        o.subdomain_mode = SUB_NONE
    elif isinstance(sub, str) and sub == "jacobi":
        o.subdomain_mode = SUB_JACOBI
    else:
        o.subdomain_mode = SUB_GRID
        o.subdomains[:] = [int(g) for g in sub]
    return o


class OracleScene:
    """One scene held by the C oracle; mirrors the C-ABI of the CUDA path."""

    def __init__(self, scene: dict):
        L = lib()
        self.params = make_params(scene["params"])
        self.composite = "members" in scene
        self.n = int(len(scene["pos"]))
        pos = _f64(scene["pos"], (self.n, 3))
        vel = _f64(scene["vel"], (self.n, 3))
        ang = _f64(scene["angvel"], (self.n, 3))
        den = _f64(scene["density"])
        h = C.c_void_p()
        if self.composite:
            mem = scene["members"]
            mb = np.ascontiguousarray(mem["body"], dtype=np.int32)
            self.nm = int(len(mb))
            mo = _f64(mem["offset"], (self.nm, 3))
            mr = _f64(mem["radius"])
            _check(L.oracle_create_composite_scene(C.byref(self.params), self.n, _dp(pos), _dp(vel), _dp(ang),
                                                   _dp(den), self.nm, mb.ctypes.data_as(C.POINTER(C.c_int32)),
                                                   _dp(mo), _dp(mr), C.byref(h)), "create_composite_scene")
        else:
            rad = _f64(scene["radius"])
            _check(L.oracle_create_scene(C.byref(self.params), self.n, _dp(pos), _dp(vel), _dp(ang),
                                         _dp(rad), _dp(den), C.byref(h)), "create_scene")
        self._h = h
        self.n_planes = 0
        for n_, c_ in scene.get("planes", []):
            nn = _f64(n_)
            _check(L.oracle_add_plane(self._h, _dp(nn), float(c_)), "add_plane")
            self.n_planes += 1
        self.n_cones = 0
        for cn in scene.get("cones", []):
            _check(L.oracle_add_cone(self._h, _dp(_f64(cn["apex"])), _dp(_f64(cn["axis"])), float(cn["half_angle"]),
                                     float(cn["r_orifice"]), float(cn["r_top"])), "add_cone")
            self.n_cones += 1

    def cone_distance(self, k: int, x):
        """(case, signed distance, unit normal) of point x against cone k:
        case 0 above the frustum, 1 face, 2 orifice rim."""
        x = _f64(x)
        sd, nrm = C.c_double(), np.empty(3)
        case = lib().oracle_cone_distance(self._h, int(k), _dp(x), C.byref(sd), _dp(nrm))
        return int(case), float(sd.value), nrm

    def close(self):
        if getattr(self, "_h", None):
            lib().oracle_destroy_scene(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mass_properties(self, invm=None, invI=None):
        a = _f64(invm) if invm is not None else None
        b = _f64(invI) if invI is not None else None
        _check(lib().oracle_set_mass_properties(self._h, _dp(a), _dp(b)), "set_mass_properties")

    def set_bodies(self, pos=None, quat=None, vel=None, angvel=None):
        arrs = [None if a is None else _f64(a) for a in (pos, quat, vel, angvel)]
        _check(lib().oracle_set_bodies(self._h, *[_dp(a) for a in arrs]), "set_bodies")

    def get_bodies(self):
        n = self.n
        pos, quat = np.empty((n, 3)), np.empty((n, 4))
        vel, ang = np.empty((n, 3)), np.empty((n, 3))
        _check(lib().oracle_get_bodies(self._h, _dp(pos), _dp(quat), _dp(vel), _dp(ang)), "get_bodies")
        return {"pos": pos, "quat": quat, "vel": vel, "angvel": ang}

    def detect_contacts(self) -> int:
        n = C.c_int64()
        _check(lib().oracle_detect_contacts(self._h, C.byref(n)), "detect_contacts")
        return n.value

    def colour_contacts(self) -> int:
        n = C.c_int32()
        _check(lib().oracle_colour_contacts(self._h, C.byref(n)), "colour_contacts")
        return n.value

    def solve_nbgs(self, max_sweeps: int, tol: float = 0.0):
        k = C.c_int32()
        r = C.c_double()
        _check(lib().oracle_solve_nbgs(self._h, int(max_sweeps), float(tol), C.byref(k), C.byref(r)),
               "solve_nbgs")
        return k.value, r.value

    def integrate(self):
        _check(lib().oracle_integrate(self._h), "integrate")

    def step(self, max_sweeps: int, tol: float = 0.0) -> dict:
        st = OracleStepStats()
        _check(lib().oracle_step(self._h, int(max_sweeps), float(tol), C.byref(st)), "step")
        return {f: getattr(st, f) for f, _ in OracleStepStats._fields_}

    def get_contacts(self) -> dict:
        L = lib()
        n = C.c_int64()
        _check(L.oracle_get_contacts(self._h, 0, None, None, None, None, None, None, C.byref(n)),
               "get_contacts")
        m = n.value
        j1 = np.empty(m, np.uint32)
        j2 = np.empty(m, np.uint32)
        col = np.empty(m, np.int32)
        nrm = np.empty((m, 3))
        xi = np.empty(m)
        imp = np.empty((m, 3))
        _check(L.oracle_get_contacts(self._h, m, j1.ctypes.data_as(C.POINTER(C.c_uint32)),
                                     j2.ctypes.data_as(C.POINTER(C.c_uint32)),
                                     col.ctypes.data_as(C.POINTER(C.c_int32)), _dp(nrm), _dp(xi),
                                     _dp(imp), C.byref(n)), "get_contacts")
        return {"j1": j1, "j2": j2, "colour": col, "normal": nrm, "xi": xi, "impulse": imp}

    def body_mass_properties(self):
        """(1/m per body, body-frame inertia n x 3 x 3) of a composite scene."""
        invm = np.empty(self.n)
        I0 = np.empty((self.n, 3, 3))
        _check(lib().oracle_body_mass_properties(self._h, _dp(invm), _dp(I0)), "body_mass_properties")
        return invm, I0

    def member_positions(self) -> np.ndarray:
        """World positions of the member spheres of a composite scene."""
        out = np.empty((self.nm, 3))
        _check(lib().oracle_member_positions(self._h, _dp(out)), "member_positions")
        return out

    def contact_subdomains(self) -> np.ndarray:
        """Subdomain s_c(j) of every contact (canonical order)."""
        m = len(self.get_contacts()["j1"])
        out = np.zeros(m, np.int64)
        _check(lib().oracle_contact_subdomains(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))),
               "contact_subdomains")
        return out

    def set_impulses(self, imp):
        a = _f64(imp)
        _check(lib().oracle_set_impulses(self._h, _dp(a)), "set_impulses")

    def residual_history(self) -> np.ndarray:
        n = C.c_int32()
        _check(lib().oracle_residual_history(self._h, None, 0, C.byref(n)), "residual_history")
        out = np.empty(n.value)
        _check(lib().oracle_residual_history(self._h, _dp(out), n.value, C.byref(n)), "residual_history")
        return out

    def final_residuals(self) -> dict:
        r = OracleResiduals()
        _check(lib().oracle_final_residuals(self._h, C.byref(r)), "final_residuals")
        return {f: getattr(r, f) for f, _ in OracleResiduals._fields_}


def contact_frame(n):
    n = _f64(n)
    t, o = np.empty(3), np.empty(3)
    lib().oracle_contact_frame(_dp(n), _dp(t), _dp(o))
    return t, o


def one_contact(w_n, w_t, mu, b):
    b = _f64(b)
    p = np.empty(3)
    lib().oracle_one_contact(float(w_n), float(w_t), float(mu), _dp(b), _dp(p))
    return p


def one_contact_general(W6, mu, b):
    """(p, status) of the one-contact problem with a full symmetric Delassus
    block W6 = (Wnn, Wtt, Woo, Wnt, Wno, Wto); status -1: diagonal fallback."""
    w = _f64(W6)
    bb = _f64(b)
    out = np.empty(3)
    st = lib().oracle_one_contact_general(_dp(w), float(mu), _dp(bb), _dp(out))
    return out, st


def splitmix64(x: int) -> int:
    return int(lib().oracle_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
