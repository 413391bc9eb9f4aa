"""Post-processing on the GPU (Eq. postprocessing): Shepard-filtered fields at query points
against the oracle's brute-force filter, after a few steps (particles off their lattice,
lists with a skin)."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from tests.parity import field_scales, rel_err

pytestmark = pytest.mark.gpu


def _queries(sc, nq=600, seed=0):
    p = sc["params"]
    lo, hi = np.array(p["box_min"]), np.array(p["box_max"])
    q = np.zeros((nq, 3))
    d = p["dim"]
    q[:, :d] = np.random.default_rng(seed).uniform(lo[:d], hi[:d], (nq, d))
    return q


CASES = {
    "tank2d": lambda: S.tank2d_disc(dx=0.025),
    "tank3d": lambda: S.tank3d_spheres(dx=0.05, n_spheres=3, r_range=(0.1, 0.15), size=(1.0, 1.0, 1.5), fill=0.8),
    "box3d": lambda: S.periodic_box(dim=3, n=10, bodies=2, body_radius=0.2, vel_amp=0.2, jitter=0.1, T_amp=5.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_interpolation_matches_oracle(name, precision, tol):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = CASES[name]()
    g = Scene(sc, precision=precision, skin=0.3 * sc["params"]["h"])
    o = OracleScene(sc)
    g.step(3)
    o.step(3)
    q = _queries(sc)
    sca = field_scales(sc)
    for f in ("vel", "rho", "pres", "temp"):
        a, b = g.interpolate(q, f), o.interpolate(q, f)
        e = rel_err(a, b, scale=sca.get(f, 0.0))
        assert e < tol, (f, e)
    fl = 1 << 0  # the fluid material only
    a, b = g.interpolate(q, "vel", fl), o.interpolate(q, "vel", fl)
    assert rel_err(a, b, scale=sca["vel"]) < tol
    assert np.isnan(a).any() == np.isnan(b).any()


def test_bad_field_is_rejected():
    from paper_2103_07925_gb300.sph import Scene, SphError
    g = Scene(S.periodic_box(dim=2, n=12), precision=32)
    with pytest.raises(SphError):
        g.interpolate(np.zeros((3, 3)), "acc")
