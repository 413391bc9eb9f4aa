"""Concentration diffusion and concentration-driven transitions (the paper's remark on
chemically induced phase transitions, gastric example of Sec. 4.5) on the GPU against the
oracle: fields, labels and body ids from the first step, where bolus particles already
above the transition concentration turn into chyme."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from paper_2103_07925_gb300.errors import edge_only_boundary
from tests.parity import compare_bodies, compare_fields, field_scales, rel_err

pytestmark = pytest.mark.gpu
FIELDS = ["pos", "vel", "acc", "rho", "pres", "temp", "force", "vext", "conc", "dconc"]


def _gastric(tvf=False):
    sc = S.gastric2d(dx=0.1, n_boluses=4, p_background=(5 * 50.0 ** 2 if tvf else 0.0))
    p = sc["particles"]
    bol = p["material"] == 2
    rng = np.random.default_rng(2)
    # outer bolus particles start beyond C_t, the rest below it
    p["concentration"] = np.where(bol, rng.uniform(0.0, 0.9, len(p["mass"])), p["concentration"])
    return sc


def _scales(sc):
    D = max(m.get("diffusivity", 0.0) for m in sc["materials"])
    return dict(field_scales(sc), conc=1.0, dconc=D / (sc["params"]["h"] ** 2))


@pytest.mark.parametrize("tvf", [False, True])
@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_gastric_one_step_matches_oracle(tvf, precision, tol):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = _gastric(tvf)
    g = Scene(sc, precision=precision)
    o = OracleScene(sc)
    g.step(1)
    o.step(1)
    assert g.info()["relabelled"] > 0
    assert np.array_equal(g.read("mat"), o.get("mat"))
    assert np.array_equal(g.read("body"), o.get("body"))
    edge = np.zeros(len(sc["particles"]["mass"]), bool)
    if precision == 32:  # boundary particles whose fluid neighbours all sit at the support edge
        edge = edge_only_boundary(sc, o.get("pos"), sc["particles"]["material"])
    sca = _scales(sc)
    errs = {f: rel_err(g.read(f), o.get(f), mask=~edge if f in ("pres", "vext") else None, scale=sca.get(f, 0.0))
            for f in FIELDS}
    bad = {f: e for f, e in errs.items() if not e < tol}
    assert not bad, bad
    if precision == 64:
        be = compare_bodies(g, o, sc)
        bad = {f: e for f, e in be.items() if not e < tol}
        assert not bad, bad


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_concentration_slab_matches_oracle(precision, tol):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = S.conc_slab(dim=3, n=(24, 9, 9), dx=1.0 / 24)
    g = Scene(sc, precision=precision)
    o = OracleScene(sc)
    g.step(5)
    o.step(5)
    errs = compare_fields(g, o, fields=["conc", "dconc", "rho"], ints=["mat"], scales=_scales(sc))
    bad = {f: e for f, e in errs.items() if not e < tol}
    assert not bad, bad


def test_gastric_fp64_over_steps_follows_oracle():
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = S.gastric2d(dx=0.1, n_boluses=3)
    g = Scene(sc, precision=64)
    o = OracleScene(sc)
    g.step(60)
    o.step(60)
    assert np.array_equal(g.read("mat"), o.get("mat"))
    assert np.abs(g.read("conc") - o.get("conc")).max() < 1e-10
