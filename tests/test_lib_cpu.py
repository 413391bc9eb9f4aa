"""The CUDA library builds for sm_103a, loads without a GPU, and exports every symbol
that include/sph.h declares (no compute call: there is no device here)."""
import ctypes
import os
import re

from paper_2103_07925_gb300 import build as B
from paper_2103_07925_gb300 import sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "sph.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_header_symbols():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(sph.EXPORTS) == names


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(sph, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(sph, "_lib", None)
    try:
        sph.lib()
    except sph.SphError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected SphError")


def test_no_cpu_fallback_without_a_device():
    """Without a GPU every entry point that needs the device reports a CUDA error: there is
    no host path that would compute the sweep instead."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2103_07925_gb300 import scenes as S
    sc = S.periodic_box(dim=3, n=6, dx=0.1)
    for make in (lambda: sph.Scene(sc, precision=32), lambda: sph.Scene(sc, precision=64),
                 lambda: sph.Batch(capacity=4)):
        with pytest.raises(sph.SphError) as e:
            make()
        assert e.value.status == -3  # SPH_ERR_CUDA


def test_binding_tables_match_the_header():
    """Field bits, their widths and types, status codes and the profile stage count of the
    binding are the header's."""
    txt = open(os.path.join(ROOT, "include", "sph.h")).read()
    fields = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"SPH_F_([A-Z]+) = (\d+),", txt)}
    assert fields == sph.FIELDS
    assert int(re.search(r"SPH_F_COUNT = (\d+)", txt).group(1)) == len(sph.FIELDS)
    typed = list(re.finditer(r"SPH_F_([A-Z]+) = \d+,\s*/\*\s*n(\*3)?\s+(double|int32)", txt))
    assert len(typed) == len(sph.FIELDS)
    for m in typed:
        nm = m.group(1).lower()
        assert (nm in sph._VEC) == (m.group(2) is not None), nm
        assert (nm in sph._INT) == (m.group(3) == "int32"), nm
    status = {int(v): "SPH_" + k for k, v in re.findall(r"SPH_(OK|ERR_[A-Z]+) = (-?\d+)", txt)}
    assert status == sph.STATUS
    assert int(re.search(r"#define SPH_PROFILE_STAGES (\d+)", txt).group(1)) == sph.PROFILE_STAGES


def test_job_footprint_follows_the_list_capacity_and_rejects_bad_jobs():
    """The footprint estimate is host arithmetic (no device call): it grows with the Verlet
    skin by the neighbour-list capacity, ceil(1.3 * 4/3 pi ((r_c + skin) / dx)^3 / 32) * 32
    entries of 4 bytes per particle in 3D, and it refuses a job whose particle material is
    out of range or whose dx is not positive."""
    import math
    from paper_2103_07925_gb300 import scenes
    sph._lib = None
    sc = scenes.periodic_box(dim=3, n=10, dx=0.1, bodies=0)
    h, dx = sc["params"]["h"], sc["params"]["dx"]
    rc = sc["params"]["kernel_support"] * h

    def cap(r):
        return max(32, math.ceil(1.3 * 4.0 / 3.0 * math.pi * r ** 3 / 32.0) * 32)

    fp = {}
    for skin in (0.0, 0.5, 1.0):
        sc["params"]["skin"] = skin * h
        fp[skin] = sph.Batch.footprint(sc, precision=32)
    n = len(sc["particles"]["mass"])
    for s0, s1 in ((0.0, 0.5), (0.5, 1.0)):
        grow = cap((rc + s1 * h) / dx) - cap((rc + s0 * h) / dx)
        assert fp[s1] - fp[s0] == 4 * grow * n, (s0, s1)
    bad = dict(sc, particles=dict(sc["particles"]))
    bad["particles"]["material"] = sc["particles"]["material"].copy()
    bad["particles"]["material"][3] = len(sc["materials"])
    try:
        sph.Batch.footprint(bad, precision=32)
    except sph.SphError as e:
        assert "out of range" in str(e)
    else:
        raise AssertionError("expected SphError")
    bad = dict(sc, params=dict(sc["params"], dx=0.0))
    try:
        sph.Batch.footprint(bad, precision=32)
    except sph.SphError as e:
        assert "positive" in str(e)
    else:
        raise AssertionError("expected SphError")


def test_binding_checks_array_shapes_before_the_library_sees_them():
    """The library reads and writes whole rows of the arrays it is given, unchecked: the
    binding refuses inputs and caller-supplied outputs of any other shape, dtype or layout
    (and pads an n x 2 vector field of a 2D caller with zeros)."""
    import numpy as np
    import pytest
    from paper_2103_07925_gb300 import scenes
    n = 5
    a = sph._rows("pos", np.ones((n, 2)), n, np.float64, 3)
    assert a.shape == (n, 3) and a.flags["C_CONTIGUOUS"] and np.all(a[:, 2] == 0.0)
    for bad in (np.ones((n, 4)), np.ones((n + 1, 3)), np.ones(3 * n)):
        with pytest.raises(ValueError):
            sph._rows("pos", bad, n, np.float64, 3)
    with pytest.raises(ValueError):
        sph._rows("mass", np.ones(n - 1), n, np.float64)
    ok = np.empty((n, 3))
    assert sph._out_field("pos", ok, n) is ok
    for nm, bad in (("pos", np.empty((n, 3), dtype=np.float32)), ("pos", np.empty((n, 2))),
                    ("pos", np.empty((3, n)).T), ("rho", np.empty((n, 3))), ("mat", np.empty(n)),
                    ("rho", [0.0] * n)):
        with pytest.raises(ValueError):
            sph._out_field(nm, bad, n)
    ro = np.empty(n)
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        sph._out_field("rho", ro, n)
    sc = scenes.periodic_box(dim=3, n=6, dx=0.1, bodies=1, body_radius=0.15)
    sph._Inputs(sc, 32)  # a well-formed scene passes
    sc["particles"]["mass"] = sc["particles"]["mass"][:-1]
    with pytest.raises(ValueError):
        sph._Inputs(sc, 32)
    sc = scenes.periodic_box(dim=3, n=6, dx=0.1, bodies=1, body_radius=0.15)
    sc["bodies"]["quat"] = np.asarray(sc["bodies"]["quat"])[:, :3]
    with pytest.raises(ValueError):
        sph._Inputs(sc, 32)
