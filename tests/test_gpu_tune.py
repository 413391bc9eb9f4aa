"""Launch shapes and the autotuner: the shape of a launch never changes a result, and the
tuner returns a layout and shape that run the scene correctly."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S

pytestmark = pytest.mark.gpu
FIELDS = ("pos", "vel", "rho", "pres", "temp", "dtemp", "force", "vext", "mat", "body")


def _run(sc, precision, steps, launch=None, **kw):
    from paper_2103_07925_gb300.sph import Scene
    g = Scene(sc, precision=precision, **kw)
    if launch:
        g.set_launch(**launch)
    g.step(steps)
    out = g.read(*FIELDS)
    info = g.info()
    g.close()
    return out, info


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("launch", [dict(sweep_block=64, sweep_waves=1, search_waves=1),
                                    dict(sweep_block=128, sweep_waves=2, search_waves=4),
                                    dict(sweep_block=32, sweep_waves=0, search_waves=2)])
def test_launch_shape_does_not_change_results(precision, launch):
    sc = S.tank3d_spheres(dx=0.05, n_spheres=3, r_range=(0.1, 0.15), size=(1.0, 1.0, 1.5), fill=0.8)
    ref, _ = _run(sc, precision, 6)
    got, info = _run(sc, precision, 6, launch=launch)
    assert info["sweep_block"] == launch["sweep_block"]
    for f in FIELDS:
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)


def test_bad_launch_shape_is_rejected():
    from paper_2103_07925_gb300.sph import Scene, SphError
    g = Scene(S.periodic_box(dim=2, n=12), precision=32)
    for bad in (dict(sweep_block=48), dict(sweep_block=512), dict(sweep_waves=-1)):
        with pytest.raises(SphError):
            g.set_launch(**bad)
    g.close()


def test_tuner_picks_a_valid_configuration():
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.tune import tune_scene
    from tests.parity import compare_fields, field_scales
    sc = S.tank2d_disc(dx=0.025)
    t = tune_scene(sc, precision=32, steps=4, warmup=2, skins_h=(0.0, 0.3), use_cache=False)
    assert t.ms_per_step > 0 and len(t.table) >= 8
    assert t.launch["sweep_block"] in (64, 128, 256)
    # the tuned scene still matches the oracle after one step
    from paper_2103_07925_gb300.sph import Scene
    g = Scene(sc, precision=32, **t.params)
    g.set_launch(**t.launch)
    g.step(1)
    o = OracleScene(sc)
    o.step(1)
    errs = compare_fields(g, o, fields=["pos", "vel", "rho", "pres"], ints=["mat", "body"], scales=field_scales(sc))
    assert max(errs.values()) < 1e-5, errs
    g.close()
