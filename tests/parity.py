"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

FLOAT_FIELDS = ["pos", "vel", "acc", "rho", "pres", "temp", "dtemp", "force", "vext"]
INT_FIELDS = ["mat", "body", "cell"]


def rel_err(a, b, mask=None):
    """max |a - b| / max(|b|, s) with s the RMS of b (NaN positions must agree)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[mask]
        b = b[mask]
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return np.inf
    a = a[~na]
    b = b[~nb]
    if b.size == 0:
        return 0.0
    s = np.sqrt(np.mean(b * b))
    den = np.maximum(np.abs(b), max(s, 1e-300))
    return float(np.max(np.abs(a - b) / den))


def compare_fields(gpu, orc, fields=FLOAT_FIELDS, ints=INT_FIELDS):
    """Returns {field: error} for float fields and asserts integer fields are equal."""
    errs = {}
    for f in ints:
        g, o = gpu.read(f), orc.get(f)
        assert np.array_equal(g, o), "%s differs at %d of %d rows" % (f, int(np.sum(g != o)), len(o))
    for f in fields:
        errs[f] = rel_err(gpu.read(f), orc.get(f))
    return errs


def compare_bodies(gpu, orc):
    g, o = gpu.bodies(), orc.bodies()
    k = len(o["mass"])
    errs = {}
    assert len(g["mass"]) == k
    if k == 0:
        return errs
    assert np.array_equal(g["alive"], o["alive"])
    alive = o["alive"] == 1
    for f in ("com", "quat", "vel", "omega", "mass", "inertia", "force", "torque"):
        errs[f] = rel_err(g[f][alive], o[f][alive])
    return errs


def state_scene(sc, orc):
    """A scene dictionary holding the current state of an oracle scene (same inputs
    otherwise), to restart both sides from a shared state."""
    import copy
    s2 = copy.deepcopy(sc)
    p = s2["particles"]
    p["pos"] = orc.get("pos")
    v = orc.get("vel")
    p["vel"] = v
    p["temperature"] = orc.get("temp")
    mat = orc.get("mat")
    p["material"] = mat
    p["body"] = orc.get("body")
    # wall temperatures stay the prescribed ones
    b = orc.bodies()
    alive = b["alive"] == 1
    # renumber live bodies densely
    ids = np.cumsum(alive) - 1
    body = p["body"]
    p["body"] = np.where(body >= 0, ids[np.maximum(body, 0)], -1).astype(np.int32)
    s2["bodies"] = dict(quat=b["quat"][alive], vel=b["vel"][alive], omega=b["omega"][alive])
    return s2
