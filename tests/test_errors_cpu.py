"""The error measures the parity tests decide with: relative error with a floor (the RMS of
the reference, or the scale of the terms of a field), NaN agreement, the term scales of a
scene, and the mask of boundary particles whose nearest fluid neighbour sits on the edge
of the support."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from paper_2103_07925_gb300.errors import edge_only_boundary, field_scales, rel_err


def test_relative_where_large_absolute_against_the_floor_where_small():
    b = np.array([100.0, 1e-9, -50.0])
    a = b + np.array([1e-3, 1e-3, 0.0])
    # the floor is RMS(b) = 64.5...: the small entry's error 1e-3 counts against it
    rms = np.sqrt(np.mean(b * b))
    assert rel_err(a, b) == pytest.approx(1e-3 / rms)
    # a larger term scale takes over from the RMS
    assert rel_err(a, b, scale=1e3) == pytest.approx(1e-3 / 1e3)
    # relative where |b| dominates
    assert rel_err(np.array([101.0]), np.array([100.0])) == pytest.approx(0.01)


def test_nan_positions_must_agree():
    b = np.array([1.0, np.nan, 3.0])
    assert rel_err(np.array([1.0, np.nan, 3.0]), b) == 0.0
    assert rel_err(np.array([1.0, 2.0, 3.0]), b) == np.inf
    assert rel_err(np.array([np.nan, np.nan, 3.0]), b) == np.inf


def test_mask_and_empty_input():
    b = np.array([1.0, 2.0, 3.0])
    a = np.array([1.0, 5.0, 3.0])
    assert rel_err(a, b, mask=np.array([True, False, True])) == 0.0
    assert rel_err(a[:0], b[:0]) == 0.0


def test_term_scales_follow_the_scene_parameters():
    sc = S.periodic_box(dim=3, n=6, dx=0.1, c=10.0, rho0=2.0, kappa=0.5, cp=4.0, T_amp=0.0)
    s = field_scales(sc)
    p0 = 2.0 * 10.0 ** 2
    h = sc["params"]["h"]
    assert s["pres"] == pytest.approx(p0)
    assert s["acc"] == pytest.approx(p0 / (2.0 * h))
    assert s["force"] == pytest.approx(p0 * h ** 2)
    T = np.sqrt(np.mean(np.asarray(sc["particles"]["temperature"]) ** 2))
    assert s["dtemp"] == pytest.approx(0.5 / (2.0 * 4.0) * T / h ** 2)
    assert s["pos"] == s["rho"] == s["temp"] == 0.0


def _two_particle_scene(dist, periodic):
    sc = S.periodic_box(dim=3, n=6, dx=0.1)
    p = sc["params"]
    p["periodic"] = [1, 1, 1] if periodic else [0, 0, 0]
    rc = p["kernel_support"] * p["h"]
    lo = np.array(p["box_min"])
    L = np.array(p["box_max"]) - lo
    fluid = [m["kind"] for m in sc["materials"]].index(0)
    sc["materials"].append(S.material(2, 1.0))
    wall = len(sc["materials"]) - 1
    # a fluid particle near the lower x face, a wall particle dist * r_c away from it (across
    # the periodic face when periodic)
    xf = lo + np.array([0.01, 0.5, 0.5]) * L
    xw = xf - np.array([dist * rc, 0.0, 0.0])
    if periodic:
        xw = lo + np.mod(xw - lo, L)
    return sc, np.array([xf, xw]), np.array([fluid, wall])


@pytest.mark.parametrize("periodic", [False, True])
def test_edge_only_boundary_marks_walls_on_the_support_edge(periodic):
    sc, pos, mat = _two_particle_scene(1.0 - 1e-7, periodic)
    m = edge_only_boundary(sc, pos, mat)
    assert m.tolist() == [False, True]
    sc, pos, mat = _two_particle_scene(0.5, periodic)
    assert edge_only_boundary(sc, pos, mat).tolist() == [False, False]
    sc, pos, mat = _two_particle_scene(1.5, periodic)
    assert edge_only_boundary(sc, pos, mat).tolist() == [False, False]
