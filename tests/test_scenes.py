"""Scene generators reproduce the particle counts the paper prints and the sizes of
the benchmark workloads."""
import json
import os

import numpy as np

from paper_2103_07925_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_strong_scaling_scene_counts_match_paper():
    g = json.load(open(os.path.join(GOLD, "strong_scaling_scene.json")))
    sc = S.strong_scaling_cube()
    mat = sc["particles"]["material"]
    kinds = np.array([m["kind"] for m in sc["materials"]])[mat]
    assert len(mat) == g["n_total"]
    assert np.sum(kinds == S.FLUID) == g["n_fluid"]
    assert np.sum(kinds == S.RIGID) == g["n_rigid"]
    assert np.sum(kinds == S.WALL) == g["n_boundary"]
    # 48 cells of edge 0.65 span the walled box (156 sites of 0.2)
    span = sc["params"]["box_max"][0] - sc["params"]["box_min"][0]
    assert abs(span - g["cells_per_axis"] * g["cell_edge"]) < 1e-9


def test_tank2d_disc_sizes():
    sc = S.tank2d_disc()
    mat = sc["particles"]["material"]
    assert np.bincount(mat).tolist() == [3952, 996, 208]


def test_tank3d_spheres_sizes_and_seed():
    sc = S.tank3d_spheres()
    p = sc["particles"]
    kinds = np.array([m["kind"] for m in sc["materials"]])[p["material"]]
    assert np.sum(kinds == S.WALL) == 280908
    n_f, n_r = np.sum(kinds == S.FLUID), np.sum(kinds == S.RIGID)
    assert n_f + n_r == 1_000_000
    assert len(sc["bodies"]["quat"]) == 64
    per = np.bincount(p["body"][p["body"] >= 0])
    assert per.min() >= 200 and per.max() <= 2300
    sc2 = S.tank3d_spheres()
    assert np.array_equal(sc2["particles"]["pos"], p["pos"])


def _kinds(sc):
    return np.array([m["kind"] for m in sc["materials"]])[sc["particles"]["material"]]


def test_dx_for_count_gives_the_requested_size():
    for dim, n in ((2, 2e4), (2, 3e5), (3, 2e4), (3, 4e5)):
        dx = S.dx_for_count(dim, n)
        sc = S.tank2d_discs(dx=dx, n_discs=0) if dim == 2 else S.tank3d_spheres(dx=dx, n_spheres=0)
        m = len(sc["particles"]["mass"])
        assert 0.8 * n < m < 1.25 * n, (dim, n, m)
    assert S.dx_for_count(3, 1e5) > S.dx_for_count(3, 4e5)


def test_batch_mix_spread_dims_bodies_and_seed():
    mix = S.batch_mix(count=12, seed=7, n_lo=1e4, n_hi=6e4, max_bodies=5)
    specs = [s for _, s in mix]
    assert [s["index"] for s in specs] == list(range(12))
    assert {s["dim"] for s in specs} == {2, 3}
    for sc, s in mix:
        assert sc["params"]["dim"] == s["dim"]
        assert 1e4 <= s["target"] <= 6e4
        assert 0.7 * s["target"] < s["n"] < 1.4 * s["target"]
        assert len(sc["bodies"]["quat"]) == s["bodies"] <= 5
        assert sc["params"]["precision"] == 32
    again = S.batch_mix(count=12, seed=7, n_lo=1e4, n_hi=6e4, max_bodies=5)
    for (a, _), (b, _) in zip(mix, again):
        assert np.array_equal(a["particles"]["pos"], b["particles"]["pos"])


def test_powder_bed_structure():
    sc = S.powder_bed(dx=0.02, n_grains=40)
    k = _kinds(sc)
    p = sc["particles"]
    mats = sc["materials"]
    assert set(np.unique(k)) == {S.FLUID, S.RIGID, S.WALL}
    # gas (density 1) and solid metal (density 1000) present; solid melts into liquid metal
    rho0 = np.array([m["rho0"] for m in mats])[p["material"]]
    assert np.any((k == S.FLUID) & (rho0 == 1.0)) and np.any((k == S.RIGID) & (rho0 == 1000.0))
    solid = [i for i, m in enumerate(mats) if m["kind"] == S.RIGID]
    assert all(mats[i]["transitions_to"] >= 0 and mats[mats[i]["transitions_to"]]["kind"] == S.FLUID
               for i in solid)
    # one body per grain, every rigid particle belongs to one, periodic in x and y
    nb = len(sc["bodies"]["quat"])
    assert 0 < nb <= 40
    assert np.all(p["body"][k == S.RIGID] >= 0) and np.all(p["body"][k != S.RIGID] < 0)
    assert list(sc["params"]["periodic"][:2]) == [1, 1]
    # the substrate lies below z = 0, the grains above it
    z = p["pos"][:, 2]
    assert z[k == S.WALL].min() < 0.0 < z[k == S.RIGID].min()
