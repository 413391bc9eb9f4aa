"""Moving boundary particles on the GPU (plane Couette channel): wall particles translate
with their prescribed velocity, and the flow they drive matches the oracle."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from tests.parity import compare_fields, field_scales

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol,skin", [(64, 1e-12, 0.0), (64, 1e-12, 0.3), (32, 1e-5, 0.3)])
def test_couette_one_step_matches_oracle(precision, tol, skin):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = S.couette2d(jitter=0.05)
    g = Scene(sc, precision=precision, skin=skin * sc["params"]["h"])
    o = OracleScene(sc)
    g.step(1)
    o.step(1)
    ints = ["mat", "body", "cell"] if (precision == 64 and skin == 0.0) else ["mat", "body"]
    errs = compare_fields(g, o, ints=ints, scales=field_scales(sc))
    bad = {f: e for f, e in errs.items() if not e < tol}
    assert not bad, bad


def test_couette_trajectory_fp64_follows_oracle():
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = S.couette2d()
    g = Scene(sc, precision=64, skin=0.3 * sc["params"]["h"])
    o = OracleScene(sc)
    g.step(200)
    o.step(200)
    vg, vo = g.read("vel"), o.get("vel")
    assert np.abs(vg - vo).max() < 1e-9
    pg, po = g.read("pos"), o.get("pos")
    mat = o.get("mat")
    top = (mat == 1) & (po[:, 1] > 0.2)
    np.testing.assert_allclose(pg[top], po[top], rtol=0, atol=1e-12)
    x0 = sc["particles"]["pos"][top, 0]
    assert np.allclose(np.mod(pg[top, 0] - x0, 0.1), np.mod(200 * sc["params"]["dt_fixed"], 0.1), atol=1e-12)
