"""The autotuner's choices on the CPU: a stand-in scene whose step time is a known function
of the knobs (cell layout, skin, launch shape) replaces the library, so the search logic
(every layout x skin timed, invalid layouts skipped, coordinate descent on the launch shape,
the cache per size class, per-dimension batch tuning) is checked without a GPU."""
import pytest

from paper_2103_07925_gb300 import scenes as S
from paper_2103_07925_gb300 import sph
from paper_2103_07925_gb300 import tune


def _cost(knobs, launch):
    # a bowl with its minimum at row-major keys, two cells per group, skin 0.2 h, blocks of
    # 128, two sweep waves and search waves 4 (h = 1 in the scenes below)
    c = 10.0
    c += 0.0 if knobs["key_order"] == 1 else 3.0
    c += abs(knobs["cells_per_group"] - 2) * 0.5 if knobs["cells_per_group"] > 0 else 1.5
    c += abs(knobs["skin"] - 0.2) * 4.0
    c += {64: 0.4, 128: 0.0, 256: 0.2}[launch["sweep_block"]]
    c += {0: 0.3, 1: 0.2, 2: 0.0, 4: 0.1}[launch["sweep_waves"]]
    c += {0: 0.2, 1: 0.3, 2: 0.1, 4: 0.0}[launch["search_waves"]]
    return c


class FakeScene:
    created = []

    def __init__(self, scene, precision=32, key_order=0, cells_per_group=0, skin=0.0):
        if key_order == 0 and skin == 0.5:
            raise sph.SphError(-1, "layout not valid for this box")
        self.knobs = dict(key_order=key_order, cells_per_group=cells_per_group, skin=skin)
        self.launch = dict(sweep_block=256, sweep_waves=0, search_waves=0)
        self.closed = False
        FakeScene.created.append(self)

    def step(self, n=1):
        pass

    def set_launch(self, sweep_block=256, sweep_waves=0, search_waves=0):
        self.launch = dict(sweep_block=sweep_block, sweep_waves=sweep_waves, search_waves=search_waves)

    def time_steps(self, n):
        return n * _cost(self.knobs, self.launch)

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self):
        self.launch = {2: dict(sweep_block=256, sweep_waves=0, search_waves=0),
                       3: dict(sweep_block=256, sweep_waves=0, search_waves=0)}

    def step(self, n=1):
        pass

    def set_launch(self, dim, sweep_block=256, sweep_waves=0, search_waves=0):
        self.launch[dim] = dict(sweep_block=sweep_block, sweep_waves=sweep_waves, search_waves=search_waves)

    def time_steps(self, n):
        # dimension 2 prefers blocks of 64, dimension 3 the bowl of _cost
        k3 = dict(key_order=1, cells_per_group=2, skin=0.2)
        c3 = _cost(k3, self.launch[3])
        c2 = {64: 0.0, 128: 0.5, 256: 1.0}[self.launch[2]["sweep_block"]]
        return n * (c3 + c2)


def _scene(n=8):
    sc = S.periodic_box(dim=3, n=n, dx=1.0 / n)
    sc["params"]["h"] = 1.0
    return sc


@pytest.fixture(autouse=True)
def fake_library(monkeypatch):
    monkeypatch.setattr(sph, "Scene", FakeScene)
    FakeScene.created = []
    tune._cache.clear()
    yield
    tune._cache.clear()


def test_layout_and_launch_shape_reach_the_minimum():
    t = tune.tune_scene(_scene(), use_cache=False)
    assert t.params == dict(key_order=1, cells_per_group=2, skin=0.2)
    assert t.launch == dict(sweep_block=128, sweep_waves=2, search_waves=4)
    assert t.ms_per_step == pytest.approx(10.0)
    # every valid layout x skin was timed once, then the launch knobs one at a time
    n_layouts = len(tune.LAYOUTS) * len(tune.SKINS_H) - 1  # one combination is refused
    n_launch = (len(tune.SWEEP_BLOCKS) - 1) + 2 * (len(tune.WAVES) - 1)
    assert len(t.table) == n_layouts + n_launch
    assert all(g.closed for g in FakeScene.created)


def test_refused_layouts_are_skipped_not_fatal():
    t = tune.tune_scene(_scene(), use_cache=False)
    assert not any(k["key_order"] == 0 and k.get("skin") == 0.5 for k, _ in t.table)


def test_result_is_cached_per_size_class():
    a = tune.tune_scene(_scene(8))
    n = len(FakeScene.created)
    b = tune.tune_scene(_scene(8))
    assert b is a and len(FakeScene.created) == n
    # another size class is tuned anew
    tune.tune_scene(_scene(16))
    assert len(FakeScene.created) > n


def test_size_class_separates_dimension_precision_size_and_bodies():
    a = _scene(8)
    assert tune.size_class(a) != tune.size_class(_scene(16))
    b = dict(a, params=dict(a["params"], precision=32))
    assert tune.size_class(b) != tune.size_class(dict(a, params=dict(a["params"], precision=64)))


def test_batch_launch_shape_per_dimension():
    sc2 = S.periodic_box(dim=2, n=8, dx=1.0 / 8)
    sc2["params"]["h"] = 1.0
    out = tune.tune_batch(FakeBatch(), [_scene(), sc2], steps=2, warmup=1, use_cache=False)
    assert set(out) == {2, 3}
    assert out[2].launch["sweep_block"] == 64
    assert out[3].launch == dict(sweep_block=128, sweep_waves=2, search_waves=4)
