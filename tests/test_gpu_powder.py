"""The powder-bed scene (gas, metal grains on a cold substrate, a moving surface heat
source, melting and solidification with latent heat) on the GPU against the oracle, from
a state where grains melt and liquid metal solidifies in the first step."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from tests.parity import compare_bodies, field_scales

pytestmark = pytest.mark.gpu


def _bed(precision=64):
    sc = S.powder_bed(dx=0.02, n_grains=60, r_median=0.05, r_clip=(0.04, 0.08), Q0=2e7, precision=precision)
    p = sc["particles"]
    b = p["body"]
    rig = p["material"] == 2
    # every third grain starts molten below T_t (solidifies), the next one just above T_t
    # (melts), the rest stays solid; the gas is hot
    K = len(sc["bodies"]["quat"])
    liquid = rig & (b % 3 == 0)
    p["material"] = np.where(liquid, 3, p["material"]).astype(np.int32)
    # the liquid metal has moved off the lattice (no exactly tied distances)
    rng = np.random.default_rng(11)
    dx = sc["params"]["dx"]
    p["pos"] = np.where(liquid[:, None], p["pos"] + rng.uniform(-1e-3 * dx, 1e-3 * dx, p["pos"].shape), p["pos"])
    p["density"] = np.where(liquid, 1000.0, p["density"])
    p["temperature"] = np.where(liquid, 1695.0, p["temperature"])
    p["temperature"] = np.where(rig & (b % 3 == 1), 1712.0, p["temperature"])
    p["temperature"] = np.where(rig & (b % 3 == 2), 1650.0, p["temperature"])
    p["temperature"] = np.where(p["material"] == 0, 1500.0, p["temperature"])
    keep = np.array([k % 3 != 0 for k in range(K)])
    ids = np.cumsum(keep) - 1
    p["body"] = np.where(p["material"] == 2, ids[np.maximum(b, 0)], -1).astype(np.int32)
    for f in ("quat", "vel", "omega"):
        sc["bodies"][f] = sc["bodies"][f][keep]
    return sc


FIELDS = ["pos", "vel", "acc", "rho", "pres", "temp", "dtemp", "force", "vext", "enth"]


def _joins_valid(sc, g, o):
    """Body ids may differ only for solidifying particles, and only where the GPU's body is
    a nearest rigid neighbour's within the FP32 position tolerance.  Returns the mask of
    particles outside every body involved in a difference."""
    mat0 = sc["particles"]["material"]
    mo = o.get("mat")
    bg, bo = g.read("body"), o.get("body")
    diff = np.nonzero(bg != bo)[0]
    joiners = (mat0 == 3) & (mo == 2)
    assert np.all(joiners[diff]), "only solidifying particles may join a different body"
    pos = o.get("pos")
    p = sc["params"]
    rc = p["kernel_support"] * p["h"]
    L = np.array(p["box_max"]) - np.array(p["box_min"])
    stay = np.nonzero((mat0 == 2) & (mo == 2))[0]  # rigid before and after: join candidates
    for i in diff:
        d = pos[stay] - pos[i]
        for q in range(3):
            if p["periodic"][q]:
                d[:, q] -= L[q] * np.round(d[:, q] / L[q])
        r = np.linalg.norm(d, axis=1)
        near = r < rc
        assert near.any()
        rmin = r[near].min()
        ok = set(bo[stay[near & (r <= rmin * (1 + 1e-6))]].tolist())
        assert int(bg[i]) in ok, (int(i), int(bg[i]), ok)
    involved = set(bg[diff].tolist()) | set(bo[diff].tolist())
    return ~np.isin(bo, list(involved)) & ~np.isin(bg, list(involved)), len(diff)


def _edge_only_boundary(sc, o):
    """Wall and rigid particles during the step (before its relabel) whose fluid neighbours
    all sit at the support edge (positions do not change at the relabel)."""
    from paper_2103_07925_gb300.errors import edge_only_boundary
    return edge_only_boundary(sc, o.get("pos"), sc["particles"]["material"])


def _compare(sc, precision, tol):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    from tests.parity import rel_err
    g = Scene(sc, precision=precision)
    o = OracleScene(sc)
    g.step(1)
    o.step(1)
    assert g.info()["relabelled"] > 0
    assert np.array_equal(g.read("mat"), o.get("mat"))
    if precision == 64:
        assert np.array_equal(g.read("body"), o.get("body"))
        mask, nd = np.ones(len(sc["particles"]["mass"]), bool), 0
    else:
        mask, nd = _joins_valid(sc, g, o)
        assert nd <= 0.01 * g.info()["relabelled"], nd
    sca = dict(field_scales(sc), enth=0.0)
    ext = mask
    if precision == 32:
        # FP32 decides r < r_c like FP64 except within rounding of r_c (W = 0 there); a wall or
        # rigid particle whose fluid neighbours all sit at the support edge has its weighted
        # means of Sec. 3.3.4 decided by that rounding alone, and they act on no particle
        ext = mask & ~_edge_only_boundary(sc, o)
    errs = {f: rel_err(g.read(f), o.get(f), mask=ext if f in ("pres", "vext") else mask, scale=sca.get(f, 0.0))
            for f in FIELDS}
    bad = {f: e for f, e in errs.items() if not e < tol}
    assert not bad, bad
    return g, o


def test_powder_bed_fp64_step_with_melting_and_solidification():
    g, o = _compare(_bed(64), 64, 1e-12)
    be = compare_bodies(g, o, _bed(64))
    bad = {f: e for f, e in be.items() if not e < 1e-12}
    assert not bad, bad


def test_powder_bed_fp32_step_with_melting_and_solidification():
    _compare(_bed(32), 32, 1e-5)


def test_powder_bed_fp64_enthalpy_follows_oracle_over_steps():
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = _bed(64)
    g = Scene(sc, precision=64)
    o = OracleScene(sc)
    for _ in range(5):
        g.step(1)
        o.step(1)
        assert np.array_equal(g.read("mat"), o.get("mat"))
    m = sc["particles"]["mass"]
    hg, ho = np.sum(m * g.read("enth")), np.sum(m * o.get("enth"))
    assert abs(hg - ho) <= 1e-10 * abs(ho)
