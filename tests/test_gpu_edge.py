"""Particles at the edge of the kernel support: a wall particle whose only fluid neighbour
sits a hair inside r_c has a weight sum far below the FP32 normal range.  The extrapolated
pressure and velocity (weighted means) must stay finite in FP32 and match the oracle in
FP64."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from tests.parity import compare_fields, field_scales

pytestmark = pytest.mark.gpu


def _edge_scene(eps, dim=3):
    dx = 0.05
    h = dx
    b = S._Builder(dim)
    mats = [S.material(S.FLUID, 1.0, c=10.0, eta=0.01), S.material(S.WALL, 1.0)]
    # a small fluid block near the origin, one wall particle far from it, and one fluid
    # particle at distance 3h (1 - eps) from the wall particle along x
    blk = S.lattice([0.0] * dim, [4] * dim, dx)
    b.add(S._pad3(blk), 0, dx ** dim, 1.0, 300.0)
    w = np.zeros((1, 3))
    w[0, :dim] = 0.7
    b.add(w, 1, dx ** dim, 1.0, 300.0)
    f = w.copy()
    f[0, 0] -= 3.0 * h * (1.0 - eps)
    b.add(f, 0, dx ** dim, 1.0, 300.0, vel=[0.3, -0.2, 0.1 if dim == 3 else 0.0])
    p = S.default_params(dim, dx, [-0.1] * dim, [1.0] * dim, gravity=[0.0, 0.0, -1.0] if dim == 3 else [0.0, -1.0, 0.0],
                         dt_mode=0, dt_fixed=1e-4)
    return b.finish(p, mats)


@pytest.mark.parametrize("eps", [1e-9, 1e-8, 3e-7, 1e-6, 1e-4])
@pytest.mark.parametrize("dim", [2, 3])
def test_edge_neighbour_keeps_fp32_finite_and_fp64_exact(eps, dim):
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = _edge_scene(eps, dim)
    g32 = Scene(sc, precision=32)
    g32.step(3)
    f = g32.read("pres", "vext", "vel", "acc")
    for k, v in f.items():
        assert np.isfinite(v).all(), k
    g32.close()
    g64 = Scene(sc, precision=64)
    g64.step(1)
    o = OracleScene(sc)
    o.step(1)
    errs = compare_fields(g64, o, scales=field_scales(sc))
    bad = {k: e for k, e in errs.items() if not e < 1e-12}
    assert not bad, bad
    g64.close()
