"""Error measures of a GPU result against a reference (the FP64 oracle or the FP64 path).

Errors are |x - y| / max(|y|, RMS(y), s_f): relative where a value is large, and measured
against the scale s_f of the terms that make up the field where the field is a small
difference of large terms.  No method arithmetic: only the term scales, from the scene's
parameters.
"""
import numpy as np


def rel_err(a, b, mask=None, scale=0.0):
    """max |a - b| / max(|b|, RMS(b), scale); NaN positions must agree."""
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
    s = max(np.sqrt(np.mean(b * b)), scale, 1e-300)
    den = np.maximum(np.abs(b), s)
    return float(np.max(np.abs(a - b) / den))


# Achieved bounds of the FP32 path against FP64, one step from the same state, relative to the
# field itself, max(|y|, RMS(y)) (no term scale); pressure and extrapolated velocity without
# the boundary particles whose fluid neighbours all sit at the support edge.  The rigid
# particle force is a small net of pressure terms of order p0 h^(d-1) and keeps the relative
# rounding of p0; the force on a body, its sum, keeps the precision of the other fields.
PLAIN32 = dict(pos=1e-7, rho=1e-6, pres=5e-5, acc=3e-5, vel=3e-5, vext=5e-4, force=3e-2, body_force=5e-5)


def field_scales(sc):
    """Magnitude of the terms that make up each field at the scene's reference state.

    The weakly compressible pressure p = c^2 (rho - rho0) is a small difference of large
    numbers, so its rounding error is relative to p0 = rho0 c^2, not to p; the same
    conditioning carries into accelerations (p0 / (rho0 h)), rigid forces (p0 h^(d-1)),
    one step of velocity change (dt c^2 / h) and, for heat, temperature differences
    (kappa T / (rho c_p h^2)).
    """
    p = sc["params"]
    mats = sc["materials"]
    h, d = p["h"], p["dim"]
    fl = [m for m in mats if m["kind"] == 0]
    c = max([m["c"] for m in fl] or [0.0])
    p0 = max([m["rho0"] * m["c"] ** 2 for m in fl] or [0.0])
    rho0 = min([m["rho0"] for m in fl] or [1.0])
    dt = p["dt_fixed"] if p["dt_mode"] == 0 else 0.25 * h / max(c, 1e-300)
    T = float(np.sqrt(np.mean(np.asarray(sc["particles"]["temperature"]) ** 2)))
    kap = max([m["kappa"] / (m["rho0"] * m["cp"]) for m in mats if m["kind"] != 2 and m["cp"] > 0] or [0.0])
    acc = p0 / (rho0 * h)
    return {"pres": p0, "acc": acc, "force": p0 * h ** (d - 1), "vel": dt * acc, "vext": dt * acc,
            "dtemp": kap * T / (h * h), "pos": 0.0, "rho": 0.0, "temp": 0.0}


def body_errors(g, o, sc=None, body_ids=None):
    """Body state errors of g against the reference o (dicts of com, quat, vel, omega, mass,
    inertia, force, torque, alive).  With the scene given, force and torque are measured
    against the pressure-force scale of the body's particles (N_k p0 h^(d-1), and times the
    radius of gyration for torques) and velocities against one step of that acceleration;
    body_ids (particle -> body of the reference) gives N_k."""
    k = len(o["mass"])
    errs = {}
    assert len(g["mass"]) == k
    if k == 0:
        return errs
    assert np.array_equal(g["alive"], o["alive"])
    alive = o["alive"] == 1
    if not alive.any():
        return errs
    fs = np.zeros(k)
    ts = np.zeros(k)
    vs = np.zeros(k)
    ws = np.zeros(k)
    if sc is not None:
        sca = field_scales(sc)
        p = sc["params"]
        dt = p["dt_fixed"] if p["dt_mode"] == 0 else sca["vel"] / max(sca["acc"], 1e-300)
        body = np.asarray(body_ids)
        nk = np.bincount(body[body >= 0], minlength=k).astype(float)
        rg = np.sqrt(np.maximum(np.trace(o["inertia"], axis1=1, axis2=2), 0) / np.maximum(o["mass"], 1e-300))
        fs = nk * sca["force"]
        ts = fs * rg
        lam = np.array([max(np.linalg.eigvalsh(I).min(), 1e-300) for I in o["inertia"]])
        vs = dt * fs / np.maximum(o["mass"], 1e-300)
        ws = dt * ts / lam
    sc_of = {"force": fs, "torque": ts, "vel": vs, "omega": ws}
    for f in ("com", "quat", "vel", "omega", "mass", "inertia", "force", "torque"):
        a, b = g[f][alive], o[f][alive]
        s = sc_of.get(f)
        if s is None:
            errs[f] = rel_err(a, b)
        else:
            s = s[alive].reshape((-1,) + (1,) * (b.ndim - 1))
            den = np.maximum(np.maximum(np.abs(b), np.sqrt(np.mean(b * b))), s)
            errs[f] = float(np.max(np.abs(a - b) / np.maximum(den, 1e-300)))
    return errs


def edge_only_boundary(sc, pos, material, rel=1e-5):
    """Mask of the particles that were wall or rigid (by ``material``, the kinds during the
    step) and whose nearest fluid neighbour lies within rel * r_c of the support radius r_c.
    Their extrapolated pressure and velocity (weighted means over fluid neighbours, Sec.
    3.3.4) rest on weights of about (3 - q)^5 ~ 0 and on whether r < r_c, which FP32 and
    FP64 may decide differently within rounding; these values act on no particle (every
    pair they enter has a vanishing kernel gradient)."""
    from scipy.spatial import cKDTree
    p = sc["params"]
    kinds = np.array([m["kind"] for m in sc["materials"]])
    rc = p["kernel_support"] * p["h"]
    lo, hi = np.array(p["box_min"]), np.array(p["box_max"])
    box = np.where(np.array(p["periodic"]) == 1, hi - lo, 1e6)
    x = np.asarray(pos) - lo
    fl = kinds[np.asarray(material)] == 0
    out = np.zeros(len(x), bool)
    if fl.any() and (~fl).any():
        tree = cKDTree(np.mod(x[fl], box), boxsize=box)
        r, _ = tree.query(np.mod(x[~fl], box), k=1)
        out[np.nonzero(~fl)[0]] = np.abs(r - rc) < rel * rc
    return out
