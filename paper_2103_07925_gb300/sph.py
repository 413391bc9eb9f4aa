"""ctypes binding of libsph (include/sph.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of ``libsph.so``; this module only
converts numpy arrays and scene dictionaries into the C structures, and raises
``SphError`` for any non-zero status.  There is no fallback: if the library is
missing or no CUDA device is present the calls fail.

The environment variable ``SPH_LIBRARY`` names another build of the same library to load
instead of the in-tree ``libsph.so`` (a build with different compile-time limits).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SPH_LIBRARY") or os.path.join(HERE, "libsph.so")

FLUID, RIGID, WALL = 0, 1, 2
FIELDS = dict(pos=0, vel=1, acc=2, rho=3, pres=4, temp=5, dtemp=6, mat=7, body=8, force=9,
              vext=10, cell=11, enth=12, bacc=13, conc=14, dconc=15)
_VEC = {"pos", "vel", "acc", "force", "vext", "bacc"}
_INT = {"mat", "body", "cell"}
STATUS = {0: "SPH_OK", -1: "SPH_ERR_INVALID", -2: "SPH_ERR_OOM", -3: "SPH_ERR_CUDA",
          -4: "SPH_ERR_NONFINITE", -5: "SPH_ERR_TIMEOUT", -6: "SPH_ERR_CAPACITY"}
EXPORTS = ["sph_create_scene", "sph_step", "sph_step_async", "sph_read_fields", "sph_write_fields",
           "sph_read_bodies", "sph_diagnostics", "sph_neighbors", "sph_info", "sph_destroy_scene",
           "sph_last_error", "sph_batch_create", "sph_job_footprint", "sph_batch_admit",
           "sph_batch_step", "sph_batch_poll", "sph_batch_read_fields", "sph_batch_job_diagnostics",
           "sph_batch_release", "sph_batch_info", "sph_batch_destroy", "sph_profile",
           "sph_profile_stage_name", "sph_density_static", "sph_set_launch", "sph_time_steps",
           "sph_batch_set_launch", "sph_batch_time_steps", "sph_batch_job_state", "sph_interpolate",
           "sph_fp32_peak"]
PROFILE_STAGES = 21


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rho0", C.c_double), ("c", C.c_double), ("eta", C.c_double),
                ("cp", C.c_double), ("kappa", C.c_double), ("T_transition", C.c_double),
                ("transitions_to", C.c_int32), ("latent_heat", C.c_double), ("mushy_width", C.c_double),
                ("diffusivity", C.c_double), ("C_transition", C.c_double), ("C_fixed", C.c_double),
                ("transition_by", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("dx", C.c_double), ("h", C.c_double), ("kernel_support", C.c_double),
                ("box_min", C.c_double * 3), ("box_max", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("gravity", C.c_double * 3), ("dt_mode", C.c_int32), ("dt_fixed", C.c_double),
                ("k_contact", C.c_double), ("d_contact", C.c_double), ("precision", C.c_int32),
                ("skin", C.c_double), ("rebin_interval", C.c_int32), ("key_order", C.c_int32), ("cells_per_group", C.c_int32),
                ("body_capacity", C.c_int32), ("n_materials", C.c_int32),
                ("materials", C.POINTER(Material)), ("src_power", C.c_double), ("src_radius", C.c_double),
                ("src_speed", C.c_double * 3), ("src_origin", C.c_double * 3), ("src_depth", C.c_double),
                ("src_ztop", C.c_double), ("p_background", C.c_double)]


class ParticlesIn(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p), ("mass", C.c_void_p),
                ("density", C.c_void_p), ("temperature", C.c_void_p), ("material", C.c_void_p),
                ("body", C.c_void_p), ("wall_velocity", C.c_void_p), ("wall_temperature", C.c_void_p),
                ("concentration", C.c_void_p)]


class BodiesIn(C.Structure):
    _fields_ = [("k", C.c_int32), ("quat", C.c_void_p), ("vel", C.c_void_p), ("omega", C.c_void_p)]


class BodiesOut(C.Structure):
    _fields_ = [("com", C.c_void_p), ("quat", C.c_void_p), ("vel", C.c_void_p), ("omega", C.c_void_p),
                ("mass", C.c_void_p), ("inertia", C.c_void_p), ("force", C.c_void_p), ("torque", C.c_void_p),
                ("alive", C.c_void_p)]


class JobDesc(C.Structure):
    _fields_ = [("params", C.POINTER(Params)), ("particles", C.POINTER(ParticlesIn)),
                ("bodies", C.POINTER(BodiesIn)), ("nsteps_total", C.c_int32)]


_lib = None


def lib():
    """Load libsph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SphError(-3, "%s is not built (run __graft_entry__.build())" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "sph_create_scene": [C.POINTER(Params), C.POINTER(ParticlesIn), C.POINTER(BodiesIn), vp, C.POINTER(vp)],
            "sph_step": [vp, i32], "sph_step_async": [vp, i32],
            "sph_read_fields": [vp, C.c_uint32, C.POINTER(vp), i32],
            "sph_write_fields": [vp, C.c_uint32, C.POINTER(vp)],
            "sph_read_bodies": [vp, C.POINTER(BodiesOut), C.POINTER(i32)],
            "sph_diagnostics": [vp, C.POINTER(C.c_double)],
            "sph_neighbors": [vp, vp, vp, i64, C.POINTER(i64)],
            "sph_info": [vp, C.POINTER(i64)],
            "sph_profile": [vp, i32, C.POINTER(C.c_double)],
            "sph_batch_create": [i32, C.c_size_t, i32, vp, C.POINTER(vp)],
            "sph_job_footprint": [C.POINTER(JobDesc), C.POINTER(C.c_size_t)],
            "sph_batch_admit": [vp, C.POINTER(JobDesc), C.POINTER(i64)],
            "sph_batch_step": [vp, i32],
            "sph_batch_poll": [vp, vp, i32, C.POINTER(i32)],
            "sph_batch_read_fields": [vp, i64, C.c_uint32, C.POINTER(vp)],
            "sph_batch_job_diagnostics": [vp, i64, C.POINTER(C.c_double)],
            "sph_batch_release": [vp, i64],
            "sph_batch_info": [vp, C.POINTER(i64)],
            "sph_set_launch": [vp, C.POINTER(i32), i32],
            "sph_time_steps": [vp, i32, C.POINTER(C.c_double)],
            "sph_batch_set_launch": [vp, i32, C.POINTER(i32), i32],
            "sph_batch_time_steps": [vp, i32, C.POINTER(C.c_double)],
            "sph_batch_job_state": [vp, i64, C.POINTER(i32)],
            "sph_interpolate": [vp, i64, vp, i32, C.c_uint32, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sph_destroy_scene.argtypes = [vp]
        L.sph_destroy_scene.restype = None
        L.sph_batch_destroy.argtypes = [vp]
        L.sph_batch_destroy.restype = None
        L.sph_density_static.argtypes = [i32, i64, vp, vp, C.c_double, C.c_double, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), vp, vp]
        L.sph_density_static.restype = C.c_int
        L.sph_fp32_peak.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(C.c_double)]
        L.sph_fp32_peak.restype = C.c_int
        L.sph_profile_stage_name.restype = C.c_char_p
        L.sph_profile_stage_name.argtypes = [i32]
        L.sph_last_error.restype = C.c_char_p
        L.sph_last_error.argtypes = []
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise SphError(st, lib().sph_last_error().decode(errors="replace"))


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _rows(name, a, n, dtype, cols=None):
    """``a`` as a C-contiguous array of ``dtype`` with n rows (and ``cols`` columns; a 2D
    vector field of n x 2 is padded with a zero third column), the layout the C ABI reads:
    raises ValueError for any other shape, so that the library never reads past a buffer."""
    a = np.asarray(a)
    if cols is not None and a.ndim == 2 and a.shape == (n, 2) and cols == 3:
        a = np.concatenate([a, np.zeros((n, 1), dtype=a.dtype)], axis=1)
    want = (n,) if cols is None else (n, cols)
    if a.shape != want:
        raise ValueError("%s: shape %s, expected %s" % (name, a.shape, want))
    return _arr(a, dtype)


def _out_field(name, a, n):
    """Checks a caller-supplied output array of field ``name`` for n particles: the dtype,
    shape and contiguity the library writes (it writes whole rows, unchecked)."""
    dtype = np.int32 if name in _INT else np.float64
    want = (n, 3) if name in _VEC else (n,)
    if not isinstance(a, np.ndarray) or a.dtype != dtype or a.shape != want or not a.flags["C_CONTIGUOUS"] \
            or not a.flags["WRITEABLE"]:
        raise ValueError("out[%r]: need a writeable C-contiguous %s array of shape %s" % (name, np.dtype(dtype).name,
                                                                                      want))
    return a


class _Inputs:
    """C structures built from a scene dictionary; keeps the arrays alive."""

    def __init__(self, scene, precision=None, overrides=None):
        p = dict(scene["params"])
        if precision is not None:
            p["precision"] = precision
        if overrides:
            p.update(overrides)
        mats = scene["materials"]
        self.mats = (Material * len(mats))()
        for q, m in enumerate(mats):
            for k in ("kind", "rho0", "c", "eta", "cp", "kappa", "T_transition", "transitions_to",
                      "latent_heat", "mushy_width"):
                setattr(self.mats[q], k, m[k])
            self.mats[q].diffusivity = m.get("diffusivity", 0.0)
            self.mats[q].C_transition = m.get("C_transition", float("nan"))
            self.mats[q].C_fixed = m.get("C_fixed", float("nan"))
            self.mats[q].transition_by = m.get("transition_by", 0)
        P = Params()
        for k in ("dim", "dx", "h", "kernel_support", "dt_mode", "dt_fixed", "k_contact", "d_contact",
                  "precision", "skin", "rebin_interval", "key_order", "cells_per_group", "body_capacity",
                  "src_power", "src_radius", "src_depth", "src_ztop"):
            setattr(P, k, p[k])
        P.p_background = p.get("p_background", 0.0)
        for d in range(3):
            P.box_min[d] = p["box_min"][d]
            P.box_max[d] = p["box_max"][d]
            P.periodic[d] = int(p["periodic"][d])
            P.gravity[d] = p["gravity"][d]
            P.src_speed[d] = p["src_speed"][d]
            P.src_origin[d] = p["src_origin"][d]
        P.n_materials = len(mats)
        P.materials = C.cast(self.mats, C.POINTER(Material))
        self.params = P
        pt = scene["particles"]
        n = len(pt["mass"])
        self.keep = {k: _rows(k, pt[k], n, np.float64, 3) for k in ("pos", "vel", "wall_velocity")}
        self.keep.update({k: _rows(k, pt[k], n, np.float64) for k in
                          ("mass", "density", "temperature", "wall_temperature")})
        if "concentration" in pt:
            self.keep["concentration"] = _rows("concentration", pt["concentration"], n, np.float64)
        self.keep["material"] = _rows("material", pt["material"], n, np.int32)
        self.keep["body"] = _rows("body", pt["body"], n, np.int32)
        self.n = n
        PI = ParticlesIn()
        PI.n = n
        for k in self.keep:
            setattr(PI, k, self.keep[k].ctypes.data)
        self.parts = PI
        bd = scene["bodies"]
        K = len(bd["quat"])
        self.bkeep = {k: _rows("bodies." + k, bd[k], K, np.float64, c).reshape(-1)
                      for k, c in (("quat", 4), ("vel", 3), ("omega", 3))}
        BI = BodiesIn()
        BI.k = K
        for k in self.bkeep:
            setattr(BI, k, self.bkeep[k].ctypes.data)
        self.bodies = BI


def _alloc_field(name, n):
    if name in _INT:
        return np.empty(n, dtype=np.int32)
    if name in _VEC:
        return np.empty((n, 3), dtype=np.float64)
    return np.empty(n, dtype=np.float64)


class Scene:
    """One simulation scene resident on the current CUDA device."""

    def __init__(self, scene, precision=None, stream=None, **overrides):
        L = lib()
        self._in = _Inputs(scene, precision, overrides)
        h = C.c_void_p()
        st = L.sph_create_scene(C.byref(self._in.params), C.byref(self._in.parts), C.byref(self._in.bodies),
                                C.c_void_p(stream) if stream else None, C.byref(h))
        _check(st)
        self.h = h
        self.n = self._in.n
        self.dim = self._in.params.dim
        self.precision = self._in.params.precision

    def step(self, n=1, sync=True):
        _check((lib().sph_step if sync else lib().sph_step_async)(self.h, n))

    def read(self, *names, original_order=True, out=None):
        """Fields as numpy arrays (input order by default); ``out`` may supply
        preallocated (e.g. pinned) arrays keyed by field name."""
        out = {nm: _out_field(nm, a, self.n) for nm, a in (out or {}).items()}
        for nm in names:
            if nm not in out:
                out[nm] = _alloc_field(nm, self.n)
        dst = (C.c_void_p * len(FIELDS))()
        mask = 0
        for nm, a in out.items():
            f = FIELDS[nm]
            mask |= 1 << f
            dst[f] = a.ctypes.data
        _check(lib().sph_read_fields(self.h, mask, dst, 1 if original_order else 0))
        return out if len(names) != 1 else out[names[0]]

    def write(self, pos=None, vel=None, temp=None):
        src = (C.c_void_p * len(FIELDS))()
        mask = 0
        keep = []
        for nm, a in (("pos", pos), ("vel", vel), ("temp", temp)):
            if a is not None:
                a = _rows(nm, a, self.n, np.float64, None if nm == "temp" else 3)
                keep.append(a)
                src[FIELDS[nm]] = a.ctypes.data
                mask |= 1 << FIELDS[nm]
        _check(lib().sph_write_fields(self.h, mask, src))

    def interpolate(self, query, field, material_mask=0xFFFFFFFF):
        """Shepard-filtered field (Eq. postprocessing) at query points (nq x 3 or nq x 2)."""
        q = np.zeros((len(query), 3))
        qa = np.asarray(query, dtype=np.float64)
        q[:, : qa.shape[1]] = qa
        comps = 3 if field == "vel" else 1
        out = np.empty((len(q), comps))
        _check(lib().sph_interpolate(self.h, len(q), q.ctypes.data, FIELDS[field], C.c_uint32(material_mask),
                                     out.ctypes.data))
        return out if comps == 3 else out[:, 0]

    def bodies(self):
        k = C.c_int32()
        _check(lib().sph_read_bodies(self.h, None, C.byref(k)))
        K = k.value
        out = dict(com=np.zeros((K, 3)), quat=np.zeros((K, 4)), vel=np.zeros((K, 3)), omega=np.zeros((K, 3)),
                   mass=np.zeros(K), inertia=np.zeros((K, 3, 3)), force=np.zeros((K, 3)), torque=np.zeros((K, 3)),
                   alive=np.zeros(K, np.int32))
        if K:
            bo = BodiesOut()
            for nm, a in out.items():
                setattr(bo, nm, a.ctypes.data)
            _check(lib().sph_read_bodies(self.h, C.byref(bo), C.byref(k)))
        return out

    def diagnostics(self):
        out = np.zeros(16)
        _check(lib().sph_diagnostics(self.h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def neighbors(self):
        counts = np.zeros(self.n, dtype=np.int64)
        tot = C.c_int64()
        _check(lib().sph_neighbors(self.h, counts.ctypes.data, None, 0, C.byref(tot)))
        lst = np.zeros(max(tot.value, 1), dtype=np.int32)
        _check(lib().sph_neighbors(self.h, counts.ctypes.data, lst.ctypes.data, tot.value, C.byref(tot)))
        return counts, lst[:tot.value]

    def info(self):
        out = np.zeros(32, dtype=np.int64)
        _check(lib().sph_info(self.h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = ["n", "n_fluid", "n_rigid", "n_wall", "n_bodies", "n_cells", "cells_x", "cells_y", "cells_z",
                "steps", "kernels_per_step", "bytes", "groups", "cells_per_group", "key_order", "pairs_total",
                "rebuilds", "list_capacity", "relabelled", "sweep_block", "sweep_blocks_per_sm",
                "search_blocks_per_sm"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def set_launch(self, sweep_block=256, sweep_waves=0, search_waves=0):
        """Launch shape of the pair sweeps and the search (see sph_set_launch)."""
        cfg = (C.c_int32 * 3)(sweep_block, sweep_waves, search_waves)
        _check(lib().sph_set_launch(self.h, cfg, 3))

    def time_steps(self, n):
        """Device time (ms) of n steps, measured with CUDA events; the scene advances."""
        ms = C.c_double()
        _check(lib().sph_time_steps(self.h, n, C.byref(ms)))
        return ms.value

    def profile(self, reps=3):
        """Mean device time per stage (ms) over reps steps launched kernel by kernel."""
        ms = np.zeros(PROFILE_STAGES)
        _check(lib().sph_profile(self.h, reps, ms.ctypes.data_as(C.POINTER(C.c_double))))
        return {lib().sph_profile_stage_name(i).decode(): float(ms[i]) for i in range(PROFILE_STAGES)}

    def close(self):
        if getattr(self, "h", None):
            lib().sph_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many scenes advanced together (continuous batching under a memory cap)."""

    def __init__(self, capacity=256, hbm_cap_bytes=150 << 30, precision=32, stream=None):
        h = C.c_void_p()
        _check(lib().sph_batch_create(capacity, hbm_cap_bytes, precision, C.c_void_p(stream) if stream else None,
                                      C.byref(h)))
        self.h = h
        self.precision = precision
        self._n = {}

    @staticmethod
    def footprint(scene, nsteps_total=1, precision=32):
        inp = _Inputs(scene, precision)
        jd = JobDesc(C.pointer(inp.params), C.pointer(inp.parts), C.pointer(inp.bodies), nsteps_total)
        b = C.c_size_t()
        _check(lib().sph_job_footprint(C.byref(jd), C.byref(b)))
        return b.value

    def admit(self, scene, nsteps_total, **overrides):
        """Returns the job id, or None when the job does not fit now."""
        inp = _Inputs(scene, self.precision, overrides)
        jd = JobDesc(C.pointer(inp.params), C.pointer(inp.parts), C.pointer(inp.bodies), nsteps_total)
        jid = C.c_int64()
        st = lib().sph_batch_admit(self.h, C.byref(jd), C.byref(jid))
        if st == -6:
            return None
        _check(st)
        self._n[jid.value] = inp.n
        return jid.value

    def step(self, n):
        _check(lib().sph_batch_step(self.h, n))

    def set_launch(self, dim, sweep_block=256, sweep_waves=0, search_waves=0):
        cfg = (C.c_int32 * 3)(sweep_block, sweep_waves, search_waves)
        _check(lib().sph_batch_set_launch(self.h, dim, cfg, 3))

    def time_steps(self, n):
        """Device time (ms) of step(n), measured with CUDA events."""
        ms = C.c_double()
        _check(lib().sph_batch_time_steps(self.h, n, C.byref(ms)))
        return ms.value

    def poll(self, max_done=4096):
        ids = np.zeros(max_done, dtype=np.int64)
        nd = C.c_int32()
        _check(lib().sph_batch_poll(self.h, ids.ctypes.data, max_done, C.byref(nd)))
        return [int(x) for x in ids[:nd.value]]

    def state(self, job_id):
        """'advancing', 'finished' or 'failed' (non-finite velocities, or a relabel that could
        not be applied: body capacity exhausted or the union-find retry cap reached)."""
        st = C.c_int32()
        _check(lib().sph_batch_job_state(self.h, job_id, C.byref(st)))
        return ("advancing", "finished", "failed")[st.value]

    def read(self, job_id, *names):
        n = self._n[job_id]
        out = {nm: _alloc_field(nm, n) for nm in names}
        dst = (C.c_void_p * len(FIELDS))()
        mask = 0
        for nm, a in out.items():
            dst[FIELDS[nm]] = a.ctypes.data
            mask |= 1 << FIELDS[nm]
        _check(lib().sph_batch_read_fields(self.h, job_id, mask, dst))
        return out if len(names) != 1 else out[names[0]]

    def diagnostics(self, job_id):
        out = np.zeros(16)
        _check(lib().sph_batch_job_diagnostics(self.h, job_id, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def release(self, job_id):
        _check(lib().sph_batch_release(self.h, job_id))
        self._n.pop(job_id, None)

    def info(self):
        out = np.zeros(8, dtype=np.int64)
        _check(lib().sph_batch_info(self.h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return dict(jobs=int(out[0]), particles=int(out[1]), bytes=int(out[2]), steps=int(out[3]),
                    active=int(out[4]), kernels_per_step=int(out[5]), pairs_total=int(out[6]))

    def close(self):
        if getattr(self, "h", None):
            lib().sph_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def density_static(dim, n, pos_ptr, mass_ptr, h, kernel_support, box_min, box_max, rho_ptr, stream=None):
    """Density summation into caller-owned device buffers without any device allocation
    (device addresses as integers; see sph_density_static in include/sph.h)."""
    lo = (C.c_double * 3)(*[float(v) for v in box_min])
    hi = (C.c_double * 3)(*[float(v) for v in box_max])
    _check(lib().sph_density_static(dim, n, C.c_void_p(pos_ptr), C.c_void_p(mass_ptr), h, kernel_support, lo, hi,
                                    C.c_void_p(rho_ptr), C.c_void_p(stream) if stream else None))


def fp32_peak(iters=20000):
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, SM count, ms)."""
    tf, ms = C.c_double(), C.c_double()
    sms = C.c_int32()
    _check(lib().sph_fp32_peak(iters, C.byref(tf), C.byref(sms), C.byref(ms)))
    return tf.value, sms.value, ms.value
