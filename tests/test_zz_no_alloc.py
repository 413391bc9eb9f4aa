"""The allocation-free density entry point (sph_density_static) against the scene path.

It serves callers that cannot allocate device memory: they pass their own device
buffers, and the library's cell-list scratch lives in a fixed static device array.  Two
calls in a row (different particle sets, so the second call must not see the first
call's scratch) each match the density of sph_create_scene within the FP64 tolerance of
the other parity tests.  Kept in its own file, collected last.
"""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _fluid_block(dim, n_side, dx, seed):
    rng = np.random.default_rng(seed)
    sites = S.lattice([0.0] * dim, [n_side] * dim, dx)
    sites = sites + rng.uniform(-0.2 * dx, 0.2 * dx, size=sites.shape)
    b = S._Builder(dim)
    mats = [S.material(S.FLUID, 1.0, c=10.0, eta=0.01)]
    b.add(sites, 0, dx ** dim, 1.0, 300.0)
    pad = 0.5 * dx
    L = n_side * dx
    p = S.default_params(dim, dx, [-pad] * dim, [L + pad] * dim, dt_mode=0, dt_fixed=1e-4)
    sc = b.finish(p, mats)
    # masses vary so that the output depends on the input order
    sc["particles"]["mass"] = dx ** dim * rng.uniform(0.5, 1.5, size=len(sites))
    return sc


def _scene_path_rho(sc):
    from paper_2103_07925_gb300.sph import Scene
    g = Scene(sc, precision=64)
    rho = g.read("rho")
    g.close()
    return rho


def _static_rho(sc):
    import torch
    from paper_2103_07925_gb300.sph import density_static
    p = sc["params"]
    pos = torch.tensor(np.ascontiguousarray(sc["particles"]["pos"]), dtype=torch.float64, device="cuda")
    mass = torch.tensor(np.ascontiguousarray(sc["particles"]["mass"]), dtype=torch.float64, device="cuda")
    rho = torch.full((len(mass),), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    density_static(p["dim"], len(mass), pos.data_ptr(), mass.data_ptr(), p["h"], p["kernel_support"],
                   p["box_min"], p["box_max"], rho.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return rho.cpu().numpy()


def _err(a, b):
    s = max(np.sqrt(np.mean(b * b)), 1e-300)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), s)))


def test_static_density_matches_scene_path_on_two_calls_in_a_row():
    first = _fluid_block(3, 22, 0.04, seed=11)
    second = _fluid_block(2, 90, 0.02, seed=12)
    for sc in (first, second):
        got = _static_rho(sc)
        ref = _scene_path_rho(sc)
        assert np.all(np.isfinite(got))
        assert _err(got, ref) < 1e-12
    # particles of a cell are visited in index order: a repeated call gives the same bits
    assert np.array_equal(_static_rho(first), _static_rho(first))


def test_static_density_particles_on_the_box_edge():
    """2D particles sitting exactly on box_max fall into the last cell (clamped), and their
    density still equals the scene path's."""
    sc = _fluid_block(2, 40, 0.025, seed=13)
    p = sc["params"]
    L = 40 * 0.025
    p["box_min"] = [0.0, 0.0, 0.0]
    p["box_max"] = [L, L, 0.0]
    pos = sc["particles"]["pos"]
    pos[:, :2] = np.clip(pos[:, :2], 0.0, L)
    pos[:40, 0] = L  # a column exactly on the upper x edge
    pos[40:80, 1] = L
    got = _static_rho(sc)
    ref = _scene_path_rho(sc)
    assert _err(got, ref) < 1e-12


def test_static_density_rejects_oversized_input():
    import torch
    from paper_2103_07925_gb300.sph import SphError, density_static
    n = (1 << 18) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.ones(n, dtype=torch.float64, device="cuda")
    rho = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(SphError) as e:
        density_static(3, n, pos.data_ptr(), mass.data_ptr(), 0.1, 3.0, [0, 0, 0], [1, 1, 1], rho.data_ptr())
    assert e.value.status == -6


def test_static_density_rejects_a_box_with_too_many_cells():
    """n within the limit but a box that needs more than 2^18 cells of edge >= r_c: the call
    returns SPH_ERR_CAPACITY before launching anything, and the output is untouched."""
    import torch
    from paper_2103_07925_gb300.sph import SphError, density_static
    n = 1000
    pos = torch.rand((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.ones(n, dtype=torch.float64, device="cuda")
    rho = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    h = 0.01  # r_c = 0.03: 66 cells along each edge of 2, 66^3 > 2^18
    for box_max in ([2.0, 2.0, 2.0], [1e12, 1.0, 1.0]):
        with pytest.raises(SphError) as e:
            density_static(3, n, pos.data_ptr(), mass.data_ptr(), h, 3.0, [0, 0, 0], box_max, rho.data_ptr())
        assert e.value.status == -6
    torch.cuda.synchronize()
    assert bool(torch.all(rho == 7.0))
