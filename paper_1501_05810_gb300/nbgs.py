"""Thin ctypes binding of libnbgs.so (include/nbgs.h).

Argument marshalling only: every step of the time step runs in the CUDA
library.  PyTorch supplies device memory (its caching allocator, handed to
the library as an ``nbgs_allocator``) and the CUDA stream.  If the library
has not been built this module raises on import; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnbgs.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "nbgs.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = C.CDLL(LIB_PATH)

NBGS_OK, NBGS_EINVAL, NBGS_ENOMEM, NBGS_ECUDA, NBGS_ECAPACITY, NBGS_ENOTCONV, NBGS_ENAN, NBGS_ETIMEOUT = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ECAPACITY", "ENOTCONV", "ENAN", "ETIMEOUT"]
NBGS_FP64, NBGS_FP32 = 0, 1
NBGS_WARM_NONE, NBGS_WARM_PREV, NBGS_WARM_MLP = 0, 1, 2
NBGS_SOLVER_PERSISTENT, NBGS_SOLVER_PER_COLOUR = 0, 1
NBGS_SWEEP_GLOBAL_SYNC, NBGS_SWEEP_TMA_STAGE, NBGS_SWEEP_WARP_SYNC, NBGS_SWEEP_GATHER2 = 1, 2, 4, 8
NBGS_SUB_NONE, NBGS_SUB_GRID, NBGS_SUB_JACOBI = 0, 1, 2


class nbgs_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p),
                ("alloc", C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p))]


class nbgs_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("mu", C.c_double), ("omega", C.c_double),
                ("tau", C.c_double), ("beta", C.c_double), ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int32 * 3), ("precision", C.c_int32), ("warm_start", C.c_int32),
                ("solver", C.c_int32), ("colour_seed", C.c_uint64), ("contacts_per_body", C.c_int32),
                ("sweep_flags", C.c_int32), ("subdomain_mode", C.c_int32), ("subdomains", C.c_int32 * 3)]


class nbgs_batch_desc(C.Structure):
    _fields_ = [("n_scenes", C.c_int64), ("body_offset", C.POINTER(C.c_int64)), ("box_lo", C.POINTER(C.c_double)),
                ("box_hi", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double))]


class nbgs_step_stats(C.Structure):
    _fields_ = [("n_contacts", C.c_int64), ("n_colours", C.c_int32), ("sweeps_done", C.c_int32),
                ("residual", C.c_double), ("v_ref", C.c_double)]


class nbgs_residuals(C.Structure):
    _fields_ = [("non_penetration", C.c_double), ("cone", C.c_double), ("complementarity", C.c_double),
                ("dissipation", C.c_double)]


_P = C.POINTER
_vp, _dp, _i64p, _i32p, _u32p = C.c_void_p, _P(C.c_double), _P(C.c_int64), _P(C.c_int32), _P(C.c_uint32)
_SIG = {
    "nbgs_create_scene": [_P(nbgs_params), C.c_int64, _vp, _vp, _vp, _vp, _vp, _P(nbgs_allocator), _vp, _P(_vp)],
    "nbgs_destroy_scene": [_vp],
    "nbgs_last_error": [_vp],
    "nbgs_add_plane": [_vp, _dp, C.c_double],
    "nbgs_add_cone": [_vp, _dp, _dp, C.c_double, C.c_double, C.c_double],
    "nbgs_set_mass_properties": [_vp, _vp, _vp],
    "nbgs_set_bodies": [_vp, _vp, _vp, _vp, _vp],
    "nbgs_update_bodies": [_vp, _vp, _vp, _vp, _vp],
    "nbgs_get_bodies": [_vp, _vp, _vp, _vp, _vp],
    "nbgs_detect_contacts": [_vp, _i64p],
    "nbgs_colour_contacts": [_vp, _i32p],
    "nbgs_solve_nbgs": [_vp, C.c_int32, C.c_double, _i32p, _dp],
    "nbgs_integrate": [_vp],
    "nbgs_step": [_vp, C.c_int32, C.c_double, _P(nbgs_step_stats)],
    "nbgs_get_contacts": [_vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _i64p],
    "nbgs_residual_history": [_vp, _dp, C.c_int32, _i32p],
    "nbgs_save_state": [_vp, C.c_char_p],
    "nbgs_load_state": [_vp, C.c_char_p],
    "nbgs_final_residuals": [_vp, _P(nbgs_residuals)],
    "nbgs_set_impulses": [_vp, _vp],
    "nbgs_sync": [_vp],
    "nbgs_enable_timing": [_vp, C.c_int32],
    "nbgs_get_timings": [_vp, _dp, _i64p],
    "nbgs_create_batch": [_P(nbgs_params), _P(nbgs_batch_desc), C.c_int64, _vp, _vp, _vp, _vp, _vp,
                          _P(nbgs_allocator), _vp, _P(_vp)],
    "nbgs_batch_step": [_vp, C.c_int32, C.c_double, _i32p, _dp],
    "nbgs_get_scene_stats": [_vp, _i32p, _dp],
    "nbgs_graph_step": [_vp, C.c_int32, C.c_double, C.c_int32],
    "nbgs_get_updates": [_vp, _i64p],
    "nbgs_one_contact": [C.c_int64, _vp, _vp, _vp, _vp, _vp],
    "nbgs_pair_normals": [C.c_int64, _vp, _vp, _vp],
    "nbgs_autotune": [_vp, C.c_int32, C.c_double, _i32p, _i32p],
    "nbgs_mlp_load": [_vp, _vp, C.c_int64],
    "nbgs_set_warm_start": [_vp, C.c_int32],
    "nbgs_set_subdomains": [_vp, C.c_int32, _i32p],
    "nbgs_create_composite_scene": [_P(nbgs_params), C.c_int64, _vp, _vp, _vp, _vp, C.c_int64, _vp, _vp, _vp,
                                    _P(nbgs_allocator), _vp, _P(_vp)],
    "nbgs_get_subdomains": [_vp, C.c_int64, _u32p, _i64p],
    "nbgs_mlp_features": [_vp, _vp, C.c_int64, _i64p],
    "nbgs_mlp_infer": [_vp, _vp, _vp, C.c_int64, _vp],
    "nbgs_mlp_grad": [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp],
    "nbgs_mlp_adam": [_vp, _vp, _vp, _vp, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32, _vp],
    "nbgs_final_residuals_noalloc": [C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                     C.c_double, C.c_double, C.c_double, C.c_double, _vp, _vp],
}
for _name, _args in _SIG.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.nbgs_destroy_scene.restype = None
_lib.nbgs_last_error.restype = C.c_char_p


def header_symbols() -> list:
    """Entry points declared in include/nbgs.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:nbgs_status|void|const char\*)\s+(nbgs_\w+)\s*\(", txt, re.M)))


def library() -> C.CDLL:
    return _lib


class NBGSError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: NBGS_{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


# ---------------------------------------------------------------------------
# thin wrappers with the C names (raw pointers as ints)
# ---------------------------------------------------------------------------
def nbgs_create_scene(params, n, pos, vel, angvel, radius, density, allocator, stream):
    h = C.c_void_p()
    st = _lib.nbgs_create_scene(C.byref(params), n, pos, vel, angvel, radius, density,
                                C.byref(allocator) if allocator is not None else None, stream, C.byref(h))
    return st, h


def _call(scene, name, *args):
    st = getattr(_lib, name)(scene, *args)
    if st != NBGS_OK:
        raise NBGSError(st, name, _lib.nbgs_last_error(scene).decode(errors="replace"))
    return st


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------------------
# torch-backed scene
# ---------------------------------------------------------------------------
_PREC = {"fp64": NBGS_FP64, "fp32": NBGS_FP32}
_SOLVER = {"persistent": NBGS_SOLVER_PERSISTENT, "per_colour": NBGS_SOLVER_PER_COLOUR}


def make_params(p: dict, solver: str = "persistent") -> nbgs_params:
    o = nbgs_params()
    o.dt = p["dt"]
    o.gravity[:] = list(p.get("gravity", (0.0, 0.0, 0.0)))
    o.mu = p.get("mu", 0.5)
    o.omega = p.get("omega", 1.0)
    o.tau = p.get("tau", 0.005)
    o.beta = p.get("beta", 1.0)
    o.box_lo[:] = list(p.get("box_lo", (0.0, 0.0, 0.0)))
    o.box_hi[:] = list(p.get("box_hi", (1.0, 1.0, 1.0)))
    o.periodic[:] = [int(b) for b in p.get("periodic", (0, 0, 0))]
    o.precision = _PREC[p.get("precision", "fp64")]
    o.warm_start = {"none": NBGS_WARM_NONE, "prev": NBGS_WARM_PREV, "mlp": NBGS_WARM_MLP}[p.get("warm_start", "none")]
    o.solver = _SOLVER[p.get("solver", solver)]
    o.colour_seed = int(p.get("colour_seed", 0)) & 0xFFFFFFFFFFFFFFFF
    o.contacts_per_body = int(p.get("contacts_per_body", 0))
    o.sweep_flags = int(p.get("sweep_flags", 0))
    o.subdomain_mode, grid = _subdomains(p.get("subdomains"))
    o.subdomains[:] = grid
    return o


def _subdomains(sub):
    """(mode, grid) of a scene's "subdomains" entry: None (classic NBGS),
    "jacobi" (one subdomain per contact) or a grid (g0, g1, g2)."""
    if sub is None:
        return NBGS_SUB_NONE, [1, 1, 1]
    if isinstance(sub, str):
        if sub != "jacobi":
            raise ValueError(f"unknown subdomains {sub!r}")
        return NBGS_SUB_JACOBI, [1, 1, 1]
    return NBGS_SUB_GRID, [int(g) for g in sub]


class TorchAllocator:
    """nbgs_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = torch.device(device).index or 0
        proto_a = nbgs_allocator._fields_[1][1]
        proto_f = nbgs_allocator._fields_[2][1]

        def _alloc(ctx, nbytes, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:
                return None

        def _free(ctx, ptr, stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._a = proto_a(_alloc)
        self._f = proto_f(_free)
        self.struct = nbgs_allocator(None, self._a, self._f)


class Scene:
    """A scene on the GPU: owns an ``nbgs_scene*`` created from a scene dict
    (see :mod:`paper_1501_05810_gb300.scenes`)."""

    def __init__(self, scene: dict, device="cuda:0", stream=None, solver: str = "persistent",
                 use_torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.composite = "members" in scene
        self.n = int(len(scene["pos"]))   # bodies (spheres, or composites)
        self.params = make_params(scene["params"], solver)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.allocator = TorchAllocator(self.device) if use_torch_allocator else None
        alloc = self.allocator.struct if self.allocator else None
        if self.composite:
            mem = scene["members"]
            arrs = [np.ascontiguousarray(scene[k], dtype=np.float64) for k in ("pos", "vel", "angvel", "density")]
            mb = np.ascontiguousarray(mem["body"], dtype=np.int32)
            mo = np.ascontiguousarray(mem["offset"], dtype=np.float64)
            mr = np.ascontiguousarray(mem["radius"], dtype=np.float64)
            self.n_members = len(mb)
            h = C.c_void_p()
            with torch.cuda.device(self.device):
                st = _lib.nbgs_create_composite_scene(C.byref(self.params), self.n, *[_ptr(a) for a in arrs],
                                                      self.n_members, _ptr(mb), _ptr(mo), _ptr(mr),
                                                      C.byref(alloc) if alloc is not None else None,
                                                      self.stream.cuda_stream, C.byref(h))
        else:
            arrs = [np.ascontiguousarray(scene[k], dtype=np.float64)
                    for k in ("pos", "vel", "angvel", "radius", "density")]
            with torch.cuda.device(self.device):
                st, h = nbgs_create_scene(self.params, self.n, *[_ptr(a) for a in arrs], alloc,
                                          self.stream.cuda_stream)
        if st != NBGS_OK:
            raise NBGSError(st, "nbgs_create_scene", "scene creation failed")
        self.h = h
        for n_, c_ in scene.get("planes", []):
            nn = (C.c_double * 3)(*n_)
            _call(self.h, "nbgs_add_plane", nn, float(c_))
        for cn in scene.get("cones", []):
            _call(self.h, "nbgs_add_cone", (C.c_double * 3)(*cn["apex"]), (C.c_double * 3)(*cn["axis"]),
                  float(cn["half_angle"]), float(cn["r_orifice"]), float(cn["r_top"]))

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            _lib.nbgs_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def set_mass_properties(self, invm=None, invI=None):
        a = None if invm is None else np.ascontiguousarray(invm, dtype=np.float64)
        b = None if invI is None else np.ascontiguousarray(invI, dtype=np.float64)
        _call(self.h, "nbgs_set_mass_properties", _ptr(a), _ptr(b))
        self.sync()

    def set_bodies(self, pos=None, quat=None, vel=None, angvel=None):
        arrs = [None if a is None else (a if not isinstance(a, (np.ndarray, list, tuple))
                                        else np.ascontiguousarray(a, dtype=np.float64))
                for a in (pos, quat, vel, angvel)]
        _call(self.h, "nbgs_set_bodies", *[_ptr(a) for a in arrs])
        self.sync()

    def update_bodies(self, pos=None, quat=None, vel=None, angvel=None):
        """Overwrite the body state and keep the warm-start history
        (nbgs_update_bodies)."""
        arrs = [None if a is None else (a if not isinstance(a, (np.ndarray, list, tuple))
                                        else np.ascontiguousarray(a, dtype=np.float64))
                for a in (pos, quat, vel, angvel)]
        _call(self.h, "nbgs_update_bodies", *[_ptr(a) for a in arrs])
        self.sync()

    def get_bodies(self) -> dict:
        n = self.n
        out = {"pos": np.empty((n, 3)), "quat": np.empty((n, 4)), "vel": np.empty((n, 3)),
               "angvel": np.empty((n, 3))}
        _call(self.h, "nbgs_get_bodies", *[_ptr(out[k]) for k in ("pos", "quat", "vel", "angvel")])
        return out

    # -- the time step
    def detect_contacts(self) -> int:
        n = C.c_int64()
        _call(self.h, "nbgs_detect_contacts", C.byref(n))
        return n.value

    def colour_contacts(self) -> int:
        k = C.c_int32()
        _call(self.h, "nbgs_colour_contacts", C.byref(k))
        return k.value

    def solve_nbgs(self, max_sweeps: int, tol: float = 0.0, sync: bool = True):
        if not sync:
            _call(self.h, "nbgs_solve_nbgs", int(max_sweeps), float(tol), None, None)
            return None
        k, r = C.c_int32(), C.c_double()
        _call(self.h, "nbgs_solve_nbgs", int(max_sweeps), float(tol), C.byref(k), C.byref(r))
        return k.value, r.value

    def integrate(self):
        _call(self.h, "nbgs_integrate")

    def step(self, max_sweeps: int, tol: float = 0.0, stats: bool = True):
        if not stats:
            _call(self.h, "nbgs_step", int(max_sweeps), float(tol), None)
            return None
        st = nbgs_step_stats()
        _call(self.h, "nbgs_step", int(max_sweeps), float(tol), C.byref(st))
        return {f: getattr(st, f) for f, _ in nbgs_step_stats._fields_}

    def graph_step(self, max_sweeps: int, tol: float = 0.0, n_steps: int = 1) -> None:
        """n_steps time steps replayed from captured CUDA graphs, without host
        synchronisation (asynchronous; read results with the usual calls)."""
        _call(self.h, "nbgs_graph_step", int(max_sweeps), float(tol), int(n_steps))

    def get_updates(self) -> int:
        """Contact updates since the last call (read and reset)."""
        u = C.c_int64()
        _call(self.h, "nbgs_get_updates", C.byref(u))
        return u.value

    def sync(self):
        _call(self.h, "nbgs_sync")

    # -- read-out
    def get_contacts(self) -> dict:
        n = C.c_int64()
        _call(self.h, "nbgs_get_contacts", 0, None, None, None, None, None, None, C.byref(n))
        m = n.value
        out = {"j1": np.empty(m, np.uint32), "j2": np.empty(m, np.uint32), "colour": np.empty(m, np.int32),
               "normal": np.empty((m, 3)), "xi": np.empty(m), "impulse": np.empty((m, 3))}
        _call(self.h, "nbgs_get_contacts", m, *[_ptr(out[k]) for k in ("j1", "j2", "colour", "normal", "xi",
                                                                        "impulse")], C.byref(n))
        return out

    def set_subdomains(self, sub) -> None:
        """Subdomains of later solves: None, "jacobi" or a grid (g0, g1, g2)."""
        mode, grid = _subdomains(sub)
        g = (C.c_int32 * 3)(*grid)
        _call(self.h, "nbgs_set_subdomains", mode, g)

    def get_subdomains(self) -> np.ndarray:
        """s_c(j) of every contact of the last colouring (canonical order)."""
        n = C.c_int64()
        _call(self.h, "nbgs_get_subdomains", 0, None, C.byref(n))
        out = np.zeros(n.value, np.uint32)
        _call(self.h, "nbgs_get_subdomains", n.value, out.ctypes.data_as(_u32p), C.byref(n))
        return out

    def save_state(self, path: str) -> None:
        """Checkpoint of everything the next step reads (nbgs_save_state)."""
        _call(self.h, "nbgs_save_state", os.fsencode(path))

    def load_state(self, path: str) -> None:
        """Restore a checkpoint written by save_state (nbgs_load_state)."""
        _call(self.h, "nbgs_load_state", os.fsencode(path))

    def residual_history(self) -> np.ndarray:
        n = C.c_int32()
        _call(self.h, "nbgs_residual_history", None, 0, C.byref(n))
        out = np.empty(n.value)
        _call(self.h, "nbgs_residual_history", out.ctypes.data_as(_dp), n.value, C.byref(n))
        return out

    def set_impulses(self, imp) -> None:
        """Impulses of the current contacts (n_contacts x 3, canonical order,
        contact frame)."""
        a = np.ascontiguousarray(imp, dtype=np.float64).reshape(-1, 3)
        _call(self.h, "nbgs_set_impulses", _ptr(a))

    def final_residuals(self) -> dict:
        r = nbgs_residuals()
        _call(self.h, "nbgs_final_residuals", C.byref(r))
        return {f: getattr(r, f) for f, _ in nbgs_residuals._fields_}

    def mlp_load(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _call(self.h, "nbgs_mlp_load", _ptr(a), a.size)
        self.sync()

    def mlp_features(self) -> np.ndarray:
        n = C.c_int64()
        _call(self.h, "nbgs_mlp_features", None, 0, C.byref(n))
        out = np.empty((n.value, 16), np.float32)
        _call(self.h, "nbgs_mlp_features", _ptr(out), n.value, C.byref(n))
        return out

    def enable_timing(self, on: bool = True):
        _call(self.h, "nbgs_enable_timing", 1 if on else 0)

    def get_timings(self):
        ms = (C.c_double * 5)()
        la = (C.c_int64 * 5)()
        _call(self.h, "nbgs_get_timings", ms, la)
        names = ("detect", "colour", "solve", "integrate", "sweep_kernel")
        return {k: ms[i] for i, k in enumerate(names)}, {k: la[i] for i, k in enumerate(names)}


class BatchScene(Scene):
    """Many independent walled-box scenes on the GPU in one nbgs_scene
    (nbgs_create_batch).  ``scenes`` is a list of scene dicts whose boxes do
    not overlap (see :func:`paper_1501_05810_gb300.scenes.layout_batch`);
    each keeps its own mu; dt, gravity, tau, beta, omega, precision,
    warm start and colour seed come from the first scene."""

    def __init__(self, scenes: list, device="cuda:0", stream=None, use_torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.n_scenes = len(scenes)
        sizes = [len(sc["radius"]) for sc in scenes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        lo = np.array([sc["params"]["box_lo"] for sc in scenes], dtype=np.float64)
        hi = np.array([sc["params"]["box_hi"] for sc in scenes], dtype=np.float64)
        mu = np.array([sc["params"]["mu"] for sc in scenes], dtype=np.float64)
        p = dict(scenes[0]["params"])
        p["box_lo"] = tuple(lo.min(0) - 1.0)
        p["box_hi"] = tuple(hi.max(0) + 1.0)
        p["periodic"] = (0, 0, 0)
        p["solver"] = "persistent"
        self.params = make_params(p)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.allocator = TorchAllocator(self.device) if use_torch_allocator else None
        cat = {k: np.ascontiguousarray(np.concatenate([sc[k] for sc in scenes]), dtype=np.float64)
               for k in ("pos", "vel", "angvel", "radius", "density")}
        self._keep = (self.offsets, np.ascontiguousarray(lo), np.ascontiguousarray(hi), np.ascontiguousarray(mu))
        desc = nbgs_batch_desc(self.n_scenes, self.offsets.ctypes.data_as(C.POINTER(C.c_int64)),
                               self._keep[1].ctypes.data_as(_dp), self._keep[2].ctypes.data_as(_dp),
                               self._keep[3].ctypes.data_as(_dp))
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = _lib.nbgs_create_batch(C.byref(self.params), C.byref(desc), self.n,
                                        *[_ptr(cat[k]) for k in ("pos", "vel", "angvel", "radius", "density")],
                                        C.byref(self.allocator.struct) if self.allocator else None,
                                        self.stream.cuda_stream, C.byref(h))
        if st != NBGS_OK:
            raise NBGSError(st, "nbgs_create_batch", "batch creation failed")
        self.h = h

    def step_scenes(self, max_sweeps: int, tol: float):
        k = np.empty(self.n_scenes, np.int32)
        r = np.empty(self.n_scenes)
        _call(self.h, "nbgs_batch_step", int(max_sweeps), float(tol), k.ctypes.data_as(_i32p), r.ctypes.data_as(_dp))
        return k, r

    def scene_stats(self):
        k = np.empty(self.n_scenes, np.int32)
        r = np.empty(self.n_scenes)
        _call(self.h, "nbgs_get_scene_stats", k.ctypes.data_as(_i32p), r.ctypes.data_as(_dp))
        return k, r


def autotune(scene: Scene, max_sweeps: int, tol: float):
    """Pick the fastest sweep schedule and blocks per SM for the scene's
    current contacts (nbgs_autotune); returns (sweep_flags, blocks_per_sm)."""
    f, b = C.c_int32(), C.c_int32()
    _call(scene.h, "nbgs_autotune", int(max_sweeps), float(tol), C.byref(f), C.byref(b))
    return f.value, b.value
