"""Failure paths of the library, reached from the host without any GPU fault.

* A NaN in one particle's input velocity: ``sph_step`` returns SPH_ERR_NONFINITE; in a
  batch that job is reported finished with state 2 (failed) and stops, while the other
  jobs advance bitwise as they would alone.
* Solidification that needs more new bodies than the body capacity: the relabel of that
  step is not applied and ``sph_step`` returns SPH_ERR_CAPACITY (a batch job fails).
* The bounded retries of the union-find hooking of new bodies (Sec. 3.6, new bodies by
  connected components): a build of the library with the retry cap lowered to zero makes
  every hook give up; ``sph_step`` returns SPH_ERR_TIMEOUT and the relabel is not applied.
* A particle count past the 26 bits of a neighbour index: ``sph_create_scene`` rejects it
  before it reads any particle array.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _solidify(body_capacity=0):
    """A body at 900 in fluid at 1100 (T_t = 1000), a ring of fluid around it and two
    separate cold patches at 900: the ring joins the body, each patch forms a new body."""
    sc = S.periodic_box(dim=2, n=16, dx=0.1, bodies=1, body_radius=0.35, vel_amp=0.0, kappa=0.0)
    mats = sc["materials"]
    mats[0].update(T_transition=1000.0, transitions_to=1)
    mats[1].update(T_transition=1000.0, transitions_to=0)
    p = sc["particles"]
    x = p["pos"]
    rig = p["material"] == 1
    c = x[rig].mean(0)
    ring = (~rig) & (np.linalg.norm(x - c, axis=1) < 0.5)
    far1 = (~rig) & (np.linalg.norm(x - (c + [0.75, 0.75, 0]), axis=1) < 0.15)
    far2 = (~rig) & (np.linalg.norm(x - (c + [-0.7, 0.6, 0]), axis=1) < 0.12)
    p["temperature"] = np.where(rig, 900.0, 1100.0)
    p["temperature"][ring | far1 | far2] = 900.0
    sc["params"]["body_capacity"] = body_capacity
    return sc


def _two_new_bodies(body_capacity=0):
    """As _solidify, with two cold patches more than r_c apart from each other and from the
    body: the step creates two new bodies (one body at start)."""
    sc = _solidify(body_capacity)
    p = sc["particles"]
    x = p["pos"]
    rig = p["material"] == 1
    c = x[rig].mean(0)
    p["temperature"] = np.where(rig, 900.0, 1100.0)
    ring = (~rig) & (np.linalg.norm(x - c, axis=1) < 0.5)
    far1 = (~rig) & (np.linalg.norm(x - (c + [0.75, 0.75, 0]), axis=1) < 0.15)
    far2 = (~rig) & (np.linalg.norm(x - (c + [0.78, -0.02, 0]), axis=1) < 0.1)
    p["temperature"][ring | far1 | far2] = 900.0
    return sc


def _with_nan_velocity(sc, i):
    import copy
    s2 = copy.deepcopy(sc)
    s2["particles"]["vel"][i, 0] = np.nan
    return s2


@pytest.mark.parametrize("precision", [64, 32])
def test_nan_input_velocity_gives_nonfinite(precision):
    from paper_2103_07925_gb300.sph import Scene, SphError
    sc = S.tank2d_disc(dx=0.025)
    fl = np.nonzero(sc["particles"]["material"] == 0)[0]
    g = Scene(_with_nan_velocity(sc, int(fl[len(fl) // 2])), precision=precision)
    with pytest.raises(SphError) as e:
        g.step(1)
    assert e.value.status == -4
    g.close()


def test_batch_job_with_nan_input_fails_alone():
    from paper_2103_07925_gb300.sph import Batch
    scs = [S.tank2d_disc(dx=0.025), S.tank2d_discs(dx=0.02, n_discs=3, seed=5), S.tank2d_disc(dx=0.02, seed=9)]
    fl = np.nonzero(scs[1]["particles"]["material"] == 0)[0]
    bad = _with_nan_velocity(scs[1], int(fl[7]))
    B = Batch(capacity=4, precision=64)
    ids = [B.admit(scs[0], 5), B.admit(bad, 5), B.admit(scs[2], 5)]
    done = set()
    for _ in range(5):
        B.step(1)
        done |= set(B.poll())
    assert ids[1] in done and B.state(ids[1]) == "failed"
    assert B.state(ids[0]) == "finished" and B.state(ids[2]) == "finished"
    for k in (0, 2):  # the other jobs, bitwise as alone
        A = Batch(capacity=1, precision=64)
        j = A.admit(scs[k], 5)
        A.step(5)
        A.poll()
        for f in ("pos", "vel", "rho", "pres"):
            assert np.array_equal(A.read(j, f), B.read(ids[k], f)), (k, f)
        A.close()
    B.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_body_capacity_exhausted_by_solidification(precision):
    """One body at start and capacity 2: the step needs two new bodies (K + 2 > 2)."""
    from paper_2103_07925_gb300.sph import Scene, SphError
    sc = _two_new_bodies(body_capacity=2)
    g = Scene(sc, precision=precision)
    mat0, body0 = g.read("mat"), g.read("body")
    with pytest.raises(SphError) as e:
        g.step(1)
    assert e.value.status == -6
    assert np.array_equal(g.read("mat"), mat0) and np.array_equal(g.read("body"), body0)
    g.close()
    ok = Scene(_two_new_bodies(body_capacity=3), precision=precision)  # room for both: relabels
    ok.step(1)
    assert ok.info()["relabelled"] > 0 and ok.bodies()["alive"].sum() == 3
    ok.close()


def test_batch_job_over_body_capacity_fails():
    from paper_2103_07925_gb300.sph import Batch
    B = Batch(capacity=2, precision=64)
    good = B.admit(S.tank2d_disc(dx=0.025), 3)
    bad = B.admit(_two_new_bodies(body_capacity=2), 3)
    for _ in range(3):
        B.step(1)
        B.poll()
    assert B.state(bad) == "failed" and B.state(good) == "finished"
    B.close()


_TIMEOUT_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_2103_07925_gb300.sph import Scene, SphError, LIB_PATH
from tests.test_gpu_failures import _solidify
assert LIB_PATH == sys.argv[2], LIB_PATH
g = Scene(_solidify(body_capacity=8), precision=64)
mat0, body0 = g.read("mat"), g.read("body")
try:
    g.step(1)
    print("NO-ERROR")
except SphError as e:
    same = np.array_equal(g.read("mat"), mat0) and np.array_equal(g.read("body"), body0)
    print("STATUS", e.status, "UNCHANGED" if same else "CHANGED", str(e))
"""


def test_union_find_retry_cap_gives_timeout_and_skips_the_relabel():
    """Build of the library with SPH_RL_HOOK_TRIES=0 (no hook ever succeeds), loaded in a
    child process: the step that needs new bodies returns SPH_ERR_TIMEOUT and leaves the
    materials and body ids as they were.  The in-tree build relabels the same scene."""
    from paper_2103_07925_gb300 import build
    lib = build.build(extra=["-DSPH_RL_HOOK_TRIES=0"], variant="hook_tries_0")
    env = dict(os.environ, SPH_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_CHILD, ROOT, lib], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "STATUS -5 UNCHANGED" in r.stdout, r.stdout + r.stderr[-2000:]
    from paper_2103_07925_gb300.sph import Scene
    g = Scene(_solidify(body_capacity=8), precision=64)
    g.step(1)
    assert g.info()["relabelled"] > 0
    g.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_particle_count_beyond_the_list_index_is_rejected(precision):
    """n = 2^26 + 1 with the arrays of a 256-particle scene: SPH_ERR_INVALID from the count
    check, which comes before any array is read; 2^26 itself passes that check."""
    import ctypes as C
    from paper_2103_07925_gb300.sph import _Inputs, lib
    inp = _Inputs(S.periodic_box(dim=2, n=16, bodies=0), precision)
    inp.parts.n = (1 << 26) + 1
    h = C.c_void_p()
    L = lib()
    st = L.sph_create_scene(C.byref(inp.params), C.byref(inp.parts), C.byref(inp.bodies), None, C.byref(h))
    assert st == -1 and not h.value
    assert b"2^26" in L.sph_last_error()
