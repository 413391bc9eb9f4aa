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


def _clump_scene(n_rigid=20, seed=4):
    """3D: a lattice block of fluid and, more than r_c away from it, a dense clump: the sites
    of a lattice of spacing 0.37 dx inside a ball of radius 0.45 r_c (jittered by 1e-3 of
    that spacing), the n_rigid sites nearest its centre rigid (one body), the others fluid.
    Every clump particle has every other one inside the support: more neighbours than the
    in-range list of the FP32 sweeps holds (the list capacity at r_c), while its full
    neighbour list (radius r_c + 0.3 h) still fits."""
    rng = np.random.default_rng(seed)
    dx = 0.05
    h = dx
    rc = 3 * h
    b = S._Builder(3)
    mats = [S.material(S.FLUID, 1.0, c=10.0, eta=0.01), S.material(S.RIGID, 2.0)]
    b.add(S.lattice([0.0] * 3, [4] * 3, dx), 0, dx ** 3, 1.0, 300.0)
    s = 0.37 * dx
    g = (np.arange(-8, 9) + 0.5) * s
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    pts = pts[r < 0.45 * rc]
    pts = pts[np.argsort(np.linalg.norm(pts, axis=1), kind="stable")]
    pts = pts + 0.7 + rng.uniform(-1e-3 * s, 1e-3 * s, pts.shape)
    b.add(pts[n_rigid:], 0, dx ** 3, 1.0, 300.0)
    kb = b.add_body(vel=(0.05, 0.0, 0.0))
    b.add(pts[:n_rigid], 1, 2.0 * dx ** 3, 2.0, 300.0, body=kb)
    p = S.default_params(3, dx, [-0.1] * 3, [1.0] * 3, dt_mode=0, dt_fixed=1e-5, skin=0.3 * h)
    return b.finish(p, mats)


def test_dense_clump_beyond_the_in_range_capacity():
    """Targets whose neighbours inside the support exceed the in-range list capacity (the
    list capacity at r_c): the FP32 force sweep walks their full list with the distance test
    instead; both precisions against the oracle after one step."""
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = _clump_scene()
    o = OracleScene(sc)
    counts, _ = o.neighbors()
    clump = np.arange(len(counts)) >= 4 ** 3
    nb = int(clump.sum()) - 1
    assert counts[clump].min() == nb
    g0 = Scene(sc, precision=32, skin=0.0)
    cap_rc = g0.info()["list_capacity"]  # the in-range capacity: the list capacity at r_c
    g0.close()
    assert nb > cap_rc
    for precision, tol in ((64, 1e-12), (32, 1e-5)):
        g = Scene(sc, precision=precision)
        assert g.info()["list_capacity"] >= nb  # the full list (radius r_c + 0.3 h) holds them
        g.step(1)
        o2 = OracleScene(sc)
        o2.step(1)
        errs = compare_fields(g, o2, ints=["mat", "body"], scales=field_scales(sc))
        bad = {k: e for k, e in errs.items() if not e < tol}
        assert not bad, (precision, bad)
        g.close()


def _two_columns_scene():
    """3D periodic box of 8 x 8 x 8 cells whose edge exceeds r_c + skin by a relative 1e-6,
    holding two fluid particles: one at the top corner of cell (1, 0, 0), the first particle
    of the sorted order, and one at the bottom corner of cell (3, 1, 1), a cell edge plus
    2e-5 of it away along x.  With two cells per search group the second is the second
    column of its group and the first sits in the column left of the group: two columns
    apart, farther than r_c + skin, yet inside the search pre-test's margin."""
    dx = 0.1
    h = dx
    skin = dx
    rl = 3.0 * h + skin
    L = 8 * rl * (1.0 + 1e-6)
    ell = L / 8
    eps, eta = 1e-5 * ell, 2.5e-6 * ell
    b = S._Builder(3)
    mats = [S.material(S.FLUID, 1.0, c=10.0, eta=0.01)]
    b.add(np.array([[2 * ell - eps, ell - eta, ell - eta]]), 0, dx ** 3, 1.0, 300.0)
    b.add(np.array([[3 * ell + eps, ell + eta, ell + eta]]), 0, dx ** 3, 1.0, 300.0)
    p = S.default_params(3, dx, [0.0] * 3, [L] * 3, periodic=[1, 1, 1], dt_mode=0, dt_fixed=1e-5,
                         skin=skin, key_order=1, cells_per_group=2)
    return b.finish(p, mats)


def test_search_hit_two_columns_from_its_target():
    """The pair of _two_columns_scene passes the search's pre-test through its margin.  Its
    list entry would carry a column offset of -2, outside the two bits of the entry's x
    field: the field would borrow from the index, which for the first sorted particle
    wraps past the end of the arrays.  The search leaves such hits out; both precisions
    step and match the oracle (two isolated particles: no neighbour inside r_c)."""
    from oracle.oracle import OracleScene
    from paper_2103_07925_gb300.sph import Scene
    sc = _two_columns_scene()
    x = sc["particles"]["pos"]
    r = np.linalg.norm(x[1] - x[0])
    rl = sc["params"]["kernel_support"] * sc["params"]["h"] + sc["params"]["skin"]
    assert rl < r < rl * (1.0 + 5e-5)
    o = OracleScene(sc)
    assert np.array_equal(o.get("cell"), [1, 3 + 8 + 64])
    o.step(1)
    for precision, tol in ((64, 1e-12), (32, 1e-5)):
        g = Scene(sc, precision=precision)
        g.step(1)
        errs = compare_fields(g, o, fields=["pos", "vel", "acc", "rho", "pres"], ints=["mat", "cell"],
                              scales=field_scales(sc))
        bad = {k: e for k, e in errs.items() if not e < tol}
        assert not bad, (precision, bad)
        g.close()
