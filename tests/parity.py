"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

from paper_2103_07925_gb300.errors import body_errors, field_scales, rel_err  # noqa: F401 (re-exported)

FLOAT_FIELDS = ["pos", "vel", "acc", "rho", "pres", "temp", "dtemp", "force", "vext"]
INT_FIELDS = ["mat", "body", "cell"]


def compare_fields(gpu, orc, fields=FLOAT_FIELDS, ints=INT_FIELDS, scales=None):
    """Returns {field: error} for float fields and asserts integer fields are equal."""
    errs = {}
    for f in ints:
        g, o = gpu.read(f), orc.get(f)
        assert np.array_equal(g, o), "%s differs at %d of %d rows" % (f, int(np.sum(g != o)), len(o))
    for f in fields:
        errs[f] = rel_err(gpu.read(f), orc.get(f), scale=(scales or {}).get(f, 0.0))
    return errs


def compare_bodies(gpu, orc, sc=None):
    """Body state errors of a GPU scene against the oracle (see errors.body_errors)."""
    return body_errors(gpu.bodies(), orc.bodies(), sc, orc.get("body"))


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
