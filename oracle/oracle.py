"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It accepts the plain scene dictionaries of
``paper_2103_07925_gb300.scenes`` (passed in by the caller; this module does
not import the product package).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

ORC_MAXMAT = 32
FIELDS = dict(pos=0, vel=1, acc=2, rho=3, pres=4, temp=5, dtemp=6, mat=7, body=8, force=9,
              vext=10, cell=11, enth=12, bacc=13, conc=14, dconc=15)
_VEC = {"pos", "vel", "acc", "force", "vext", "bacc"}
_INT = {"mat", "body", "cell"}


class _Mat(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rho0", C.c_double), ("c", C.c_double), ("eta", C.c_double),
                ("cp", C.c_double), ("kappa", C.c_double), ("T_transition", C.c_double),
                ("transitions_to", C.c_int32), ("latent_heat", C.c_double),
                ("mushy_width", C.c_double), ("diffusivity", C.c_double), ("C_transition", C.c_double),
                ("C_fixed", C.c_double), ("transition_by", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("dx", C.c_double), ("h", C.c_double),
                ("kernel_support", C.c_double), ("box_min", C.c_double * 3),
                ("box_max", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("gravity", C.c_double * 3), ("dt_mode", C.c_int32), ("dt_fixed", C.c_double),
                ("k_contact", C.c_double), ("d_contact", C.c_double), ("n_materials", C.c_int32),
                ("materials", _Mat * ORC_MAXMAT), ("body_capacity", C.c_int32),
                ("src_power", C.c_double), ("src_radius", C.c_double), ("src_speed", C.c_double * 3),
                ("src_origin", C.c_double * 3), ("src_depth", C.c_double), ("src_ztop", C.c_double),
                ("skin", C.c_double), ("force_brute", C.c_int32), ("p_background", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params), C.c_int64, dp, dp, dp, dp, dp, ip, ip, dp, dp,
                                 C.c_int32, dp, dp, dp, dp]
        L.orc_interpolate.argtypes = [C.c_void_p, C.c_int64, dp, C.c_int32, C.c_uint32, dp]
        L.orc_interpolate.restype = C.c_int
        L.orc_error.restype = C.c_char_p
        L.orc_step.argtypes = [C.c_void_p, C.c_int32]
        L.orc_step.restype = C.c_int
        L.orc_get.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.orc_n.argtypes = [C.c_void_p]
        L.orc_n.restype = C.c_int64
        L.orc_nbodies.argtypes = [C.c_void_p]
        L.orc_nbodies.restype = C.c_int32
        L.orc_get_bodies.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, dp, dp, ip]
        L.orc_neighbors.argtypes = [C.c_void_p, lp, ip, C.c_int64]
        L.orc_neighbors.restype = C.c_int64
        L.orc_diagnostics.argtypes = [C.c_void_p, dp]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_kernel_w.argtypes = [C.c_int32, C.c_double, C.c_double]
        L.orc_kernel_w.restype = C.c_double
        L.orc_kernel_dw.argtypes = [C.c_int32, C.c_double, C.c_double]
        L.orc_kernel_dw.restype = C.c_double
        L.orc_body_mass_chunked.argtypes = [C.c_int32, C.c_double, C.c_int64, dp, dp, C.c_int64, dp, dp, dp]
        L.orc_quat_mul.argtypes = [dp, dp, dp]
        L.orc_quat_rot.argtypes = [dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _params(scene, force_brute=False):
    p = scene["params"]
    P = _Params()
    P.dim = p["dim"]
    P.dx = p["dx"]
    P.h = p["h"]
    P.kernel_support = p["kernel_support"]
    for d in range(3):
        P.box_min[d] = p["box_min"][d]
        P.box_max[d] = p["box_max"][d]
        P.periodic[d] = int(p["periodic"][d])
        P.gravity[d] = p["gravity"][d]
        P.src_speed[d] = p["src_speed"][d]
        P.src_origin[d] = p["src_origin"][d]
    P.dt_mode = p["dt_mode"]
    P.dt_fixed = p["dt_fixed"]
    P.k_contact = p["k_contact"]
    P.d_contact = p["d_contact"]
    mats = scene["materials"]
    P.n_materials = len(mats)
    for q, m in enumerate(mats):
        M = P.materials[q]
        for k in ("kind", "rho0", "c", "eta", "cp", "kappa", "T_transition", "transitions_to",
                  "latent_heat", "mushy_width"):
            setattr(M, k, m[k])
        M.diffusivity = m.get("diffusivity", 0.0)
        M.C_transition = m.get("C_transition", float("nan"))
        M.C_fixed = m.get("C_fixed", float("nan"))
        M.transition_by = m.get("transition_by", 0)
    P.body_capacity = p.get("body_capacity", 0)
    P.src_power = p["src_power"]
    P.src_radius = p["src_radius"]
    P.src_depth = p["src_depth"]
    P.src_ztop = p.get("src_ztop", 0.0)
    P.skin = p.get("skin", 0.0)
    P.force_brute = 1 if force_brute else 0
    P.p_background = p.get("p_background", 0.0)
    return P


class OracleScene:
    """One scene advanced by the FP64 oracle."""

    def __init__(self, scene, force_brute=False):
        L = lib()
        pt = scene["particles"]
        bd = scene["bodies"]
        self._keep = [np.ascontiguousarray(pt[k], dtype=np.float64) for k in
                      ("pos", "vel", "mass", "density", "temperature", "wall_velocity", "wall_temperature")]
        self._keep += [np.ascontiguousarray(pt[k], dtype=np.int32) for k in ("material", "body")]
        self._keep += [np.ascontiguousarray(bd[k], dtype=np.float64).reshape(-1) for k in ("quat", "vel", "omega")]
        conc = np.ascontiguousarray(pt["concentration"] if "concentration" in pt else np.zeros(len(pt["mass"])),
                                    dtype=np.float64)
        self._keep.append(conc)
        pos, vel, mass, dens, temp, wv, wt, mat, body, q, bv, bw, conc = self._keep
        self.n = len(mass)
        self.P = _params(scene, force_brute)
        k = len(bd["quat"])
        h = L.orc_create(C.byref(self.P), self.n, _dp(pos), _dp(vel), _dp(mass), _dp(dens), _dp(temp),
                         _ip(mat), _ip(body), _dp(wv), _dp(wt), k, _dp(q), _dp(bv), _dp(bw), _dp(conc))
        if not h:
            raise RuntimeError(L.orc_error().decode())
        self.h = h

    def step(self, n=1):
        rc = lib().orc_step(self.h, n)
        if rc:
            raise RuntimeError("oracle step failed (%d): %s" % (rc, lib().orc_error().decode()))

    def get(self, name):
        f = FIELDS[name]
        if name in _INT:
            out = np.empty(self.n, dtype=np.int32)
        elif name in _VEC:
            out = np.empty((self.n, 3), dtype=np.float64)
        else:
            out = np.empty(self.n, dtype=np.float64)
        lib().orc_get(self.h, f, out.ctypes.data_as(C.c_void_p))
        return out

    def bodies(self):
        k = lib().orc_nbodies(self.h)
        out = dict(com=np.empty((k, 3)), quat=np.empty((k, 4)), vel=np.empty((k, 3)),
                   omega=np.empty((k, 3)), mass=np.empty(k), inertia=np.empty((k, 3, 3)),
                   force=np.empty((k, 3)), torque=np.empty((k, 3)), alive=np.empty(k, np.int32))
        if k:
            lib().orc_get_bodies(self.h, _dp(out["com"]), _dp(out["quat"]), _dp(out["vel"]),
                                 _dp(out["omega"]), _dp(out["mass"]), _dp(out["inertia"]),
                                 _dp(out["force"]), _dp(out["torque"]), _ip(out["alive"]))
        return out

    def neighbors(self):
        """(counts, flat list): neighbour sets of every particle, ascending indices."""
        counts = np.empty(self.n, dtype=np.int64)
        tot = lib().orc_neighbors(self.h, counts.ctypes.data_as(C.POINTER(C.c_int64)), None, 0)
        lst = np.empty(max(tot, 1), dtype=np.int32)
        lib().orc_neighbors(self.h, counts.ctypes.data_as(C.POINTER(C.c_int64)), _ip(lst), tot)
        return counts, lst[:tot]

    def interpolate(self, query, field, material_mask=0xFFFFFFFF):
        """Shepard-filtered field (Eq. postprocessing) at query points (nq x 3)."""
        q = np.ascontiguousarray(query, dtype=np.float64).reshape(-1, 3)
        comps = 3 if field == "vel" else 1
        out = np.empty((len(q), comps))
        rc = lib().orc_interpolate(self.h, len(q), _dp(q), FIELDS[field], C.c_uint32(material_mask), _dp(out))
        if rc:
            raise ValueError("field %s cannot be interpolated" % field)
        return out if comps == 3 else out[:, 0]

    def diagnostics(self):
        out = np.empty(16)
        lib().orc_diagnostics(self.h, _dp(out))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_w(dim, r, h):
    return lib().orc_kernel_w(dim, r, h)


def kernel_dw(dim, r, h):
    return lib().orc_kernel_dw(dim, r, h)


def body_mass_chunked(dim, dx, pos, mass, chunk):
    pos = np.ascontiguousarray(pos, np.float64)
    mass = np.ascontiguousarray(mass, np.float64)
    m = np.zeros(1)
    c = np.zeros(3)
    I = np.zeros(9)
    lib().orc_body_mass_chunked(dim, dx, len(mass), _dp(pos), _dp(mass), chunk, _dp(m), _dp(c), _dp(I))
    return m[0], c, I.reshape(3, 3)


def quat_mul(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    o = np.zeros(4)
    lib().orc_quat_mul(_dp(a), _dp(b), _dp(o))
    return o


def quat_rot(q):
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().orc_quat_rot(_dp(q), _dp(R))
    return R.reshape(3, 3)

