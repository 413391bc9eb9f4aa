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
