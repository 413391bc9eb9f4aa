"""Writing fluid positions, velocities and temperatures into a resident scene (the host
path of the end-to-end benchmark): writing the state a scene already holds changes
nothing, bit for bit; a particle written across the box forces a list rebuild."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S

pytestmark = pytest.mark.gpu
FIELDS = ("pos", "vel", "acc", "rho", "pres", "temp")


def _pair(precision):
    from paper_2103_07925_gb300.sph import Scene
    sc = S.periodic_box(dim=3, n=14, dx=0.1, vel_amp=0.2, kappa=0.05, T_amp=3.0)
    h = sc["params"]["h"]
    a = Scene(sc, precision=precision, skin=0.3 * h)
    b = Scene(sc, precision=precision, skin=0.3 * h)
    a.step(3)
    b.step(3)
    return sc, a, b


@pytest.mark.parametrize("precision", [64, 32])
def test_writing_the_held_state_changes_nothing(precision):
    sc, a, b = _pair(precision)
    st = b.read("pos", "vel", "temp")
    r0 = b.info()["rebuilds"]
    b.write(pos=st["pos"], vel=st["vel"], temp=st["temp"])
    a.step(4)
    b.step(4)
    ra, rb = a.read(*FIELDS), b.read(*FIELDS)
    for f in FIELDS:
        np.testing.assert_array_equal(ra[f], rb[f], err_msg=f)
    assert b.info()["rebuilds"] == a.info()["rebuilds"] >= r0


@pytest.mark.parametrize("precision", [64, 32])
def test_particle_written_across_the_box_forces_a_rebuild(precision):
    sc, a, b = _pair(precision)
    st = b.read("pos", "vel", "temp")
    L = np.array(sc["params"]["box_max"]) - np.array(sc["params"]["box_min"])
    pos = st["pos"].copy()
    pos[7] = np.mod(pos[7] + 0.5 * L, L)
    r0 = b.info()["rebuilds"]
    b.write(pos=pos)
    b.step(1)
    assert b.info()["rebuilds"] == r0 + 1
    # the moved particle's neighbours are those of its new place (lists rebuilt)
    cnt, lst = b.neighbors()
    got = b.read("rho")
    assert np.isfinite(got).all()
    assert cnt[7] > 0


@pytest.mark.parametrize("precision", [64, 32])
def test_page_locked_source_reads_like_a_staged_one(precision):
    """A page-locked source is read in place by the import kernel, a pageable one through a
    staging copy: the same values give the same state, bit for bit."""
    torch = pytest.importorskip("torch")
    sc, a, b = _pair(precision)
    st = a.read("pos", "vel", "temp")
    dx = sc["params"]["dx"]
    pos = st["pos"] + 0.01 * dx * np.cos(np.arange(st["pos"].size)).reshape(st["pos"].shape)
    vel, temp = 0.9 * st["vel"], st["temp"] + 1.0
    pinned = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy()
              for k, v in (("pos", pos), ("vel", vel), ("temp", temp))}
    pinned["pos"][:] = pos
    pinned["vel"][:] = vel
    pinned["temp"][:] = temp
    a.write(pos=pos, vel=vel, temp=temp)
    b.write(pos=pinned["pos"], vel=pinned["vel"], temp=pinned["temp"])
    a.step(3)
    b.step(3)
    ra, rb = a.read(*FIELDS), b.read(*FIELDS)
    for f in FIELDS:
        np.testing.assert_array_equal(ra[f], rb[f], err_msg=f)
