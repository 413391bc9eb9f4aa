"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, conservation laws of the discrete equations,
quadrature, brute force on tiny inputs, or special cases with textbook
solutions.  CPU only.
"""
import copy
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2103_07925_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- kernel (Sec. 3.1)

@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_normalisation_by_quadrature(dim):
    """Normalisation property of the kernel remark: integral of W over its support is 1."""
    h = 0.37
    area = (lambda r: 2 * math.pi * r) if dim == 2 else (lambda r: 4 * math.pi * r * r)
    tot = 0.0
    for a, b in [(0, h), (h, 2 * h), (2 * h, 3 * h)]:  # integrate piecewise between the knots
        v, _ = integrate.quad(lambda r: O.kernel_w(dim, r, h) * area(r), a, b, epsabs=1e-15, epsrel=1e-13, limit=200)
        tot += v
    assert abs(tot - 1.0) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_compact_support_positive_monotone_smooth(dim):
    h = 1.3
    rc = 3 * h
    r = np.linspace(0, rc, 3001)
    w = np.array([O.kernel_w(dim, x, h) for x in r])
    assert O.kernel_w(dim, rc, h) == 0.0 and O.kernel_w(dim, 1.01 * rc, h) == 0.0
    assert np.all(w >= 0) and np.all(np.diff(w) <= 0)
    # the derivative is the derivative of W (central differences), continuous at the knots
    for x in [0.3 * h, 0.999 * h, h, 1.5 * h, 2 * h, 2.7 * h]:
        e = 1e-6 * h
        fd = (O.kernel_w(dim, x + e, h) - O.kernel_w(dim, x - e, h)) / (2 * e)
        assert abs(O.kernel_dw(dim, x, h) - fd) < 1e-7 * abs(O.kernel_w(dim, 0, h)) / h
    assert O.kernel_dw(dim, 0.0, h) == 0.0  # smooth maximum at r = 0
    assert abs(O.kernel_dw(dim, rc, h)) == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_partition_of_unity_and_zero_gradient(dim):
    """Sum_b V_b W_ab on a regular lattice with h = dx is close to 1 and the gradient sum
    vanishes by symmetry (Sec. 3.1.1, kernel consistency)."""
    dx = 0.1
    n = 9
    g = np.arange(-n, n + 1) * dx
    pts = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)
    r = np.linalg.norm(pts, axis=1)
    w = np.array([O.kernel_w(dim, x, dx) for x in r])
    s = dx ** dim * w.sum()
    assert abs(s - 1.0) < 1e-4
    dw = np.array([O.kernel_dw(dim, x, dx) for x in r])
    with np.errstate(invalid="ignore", divide="ignore"):
        e = np.where(r[:, None] > 0, pts / r[:, None], 0.0)
    grad = (dw[:, None] * e).sum(0)
    assert np.all(np.abs(grad) < 1e-9 * np.abs(dw).sum())


# ----------------------------------------------------------------------------- neighbours (Sec. 3.2)

def _brute_sets(pos, dim, rc, box_lo=None, box_hi=None, periodic=None):
    n = len(pos)
    sets = []
    for i in range(n):
        d = pos[i] - pos
        if periodic is not None:
            for k in range(dim):
                if periodic[k]:
                    L = box_hi[k] - box_lo[k]
                    d[:, k] = np.where(d[:, k] > 0.5 * L, d[:, k] - L, np.where(d[:, k] < -0.5 * L, d[:, k] + L, d[:, k]))
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        if dim == 3:
            r2 = r2 + d[:, 2] * d[:, 2]
        m = r2 < rc * rc
        m[i] = False
        sets.append(np.nonzero(m)[0])
    return sets


@pytest.mark.parametrize("dim,periodic,n", [(2, False, 2600), (3, False, 2500), (3, True, 2500), (2, True, 2100)])
def test_neighbour_sets_equal_brute_force(dim, periodic, n):
    sc = S.random_cloud(dim=dim, n=n, L=1.0, dx=0.05 if dim == 3 else 0.03, periodic=periodic, seed=11 + n)
    o = O.OracleScene(sc)  # n > 2000: the oracle uses its cell list
    counts, lst = o.neighbors()
    p = sc["params"]
    sets = _brute_sets(sc["particles"]["pos"].copy(), dim, 3 * p["h"], p["box_min"], p["box_max"],
                       p["periodic"] if periodic else None)
    off = np.concatenate([[0], np.cumsum(counts)])
    for i in range(n):
        assert np.array_equal(lst[off[i]:off[i + 1]], sets[i]), i
    ob = O.OracleScene(sc, force_brute=True)
    c2, l2 = ob.neighbors()
    assert np.array_equal(counts, c2) and np.array_equal(lst, l2)


def test_lattice_neighbour_counts():
    """Interior lattice site with h = dx, r_c = 3 dx: 24 sites (2D) / 92 (3D) lie in the
    open disc/ball of radius 3 dx; these counts are fixed by integer geometry."""
    for dim, expect in [(2, 24), (3, 92)]:
        g = np.arange(-3, 4)
        pts = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)
        cnt = int(np.sum(np.sum(pts * pts, 1) < 9)) - 1
        assert cnt == expect
        # dx = 1/8 keeps every lattice coordinate and squared distance exact in binary
        sc = S.periodic_box(dim=dim, n=10, dx=0.125, jitter=0.0, vel_amp=0.0)
        counts, _ = O.OracleScene(sc).neighbors()
        assert np.all(counts == expect)


# ----------------------------------------------------------------------------- density (Eq. densum)

def test_density_summation_on_periodic_lattice():
    dim = 3
    sc = S.periodic_box(dim=dim, n=8, dx=0.1, jitter=0.0, vel_amp=0.0)
    o = O.OracleScene(sc)
    rho = o.get("rho")
    # independent brute-force sum with the (pinned) kernel over the lattice images
    dx = 0.1
    g = np.arange(-3, 4) * dx
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    expect = 1.0 * dx ** 3 * sum(O.kernel_w(3, x, dx) for x in r if x < 3 * dx)
    assert np.allclose(rho, expect, rtol=1e-13, atol=0)
    assert abs(expect - 1.0) < 1e-4


# ----------------------------------------------------------------------------- conservation (Eqs. conservlinmom, couplingforce)

@pytest.mark.parametrize("dim", [2, 3])
def test_linear_momentum_conserved_periodic_box(dim):
    sc = S.periodic_box(dim=dim, n=10 if dim == 3 else 20, dx=0.1, bodies=2 if dim == 3 else 3,
                        body_radius=0.16, vel_amp=0.2, jitter=0.1, seed=4)
    o = O.OracleScene(sc)
    d0 = o.diagnostics()
    scale = np.abs(sc["particles"]["mass"][:, None] * sc["particles"]["vel"]).sum()
    for _ in range(10):
        o.step(10)
        d = o.diagnostics()
        assert np.all(np.abs(d[:3] - d0[:3]) <= 1e-13 * scale), (d[:3], d0[:3])
    assert d[10] == 100


def test_angular_momentum_conserved_inviscid_fluid_cluster():
    """nu = 0, no walls, no gravity, non-periodic: every pair force is central and the
    KDK scheme conserves angular momentum of point particles exactly (rounding only)."""
    sc = S.cluster(dim=3, n=9, dx=0.1, n_bodies=0, vel_amp=0.05)
    o = O.OracleScene(sc)
    d0 = o.diagnostics()
    m = sc["particles"]["mass"]
    scale = np.sum(m * np.linalg.norm(sc["particles"]["pos"], axis=1) * np.linalg.norm(sc["particles"]["vel"], axis=1))
    o.step(60)
    d = o.diagnostics()
    assert np.linalg.norm(d[3:6] - d0[3:6]) < 1e-13 * scale, (d[3:6], d0[3:6])


def test_angular_momentum_with_isotropic_bodies():
    """Same with two spheres of isotropic inertia: the coupling forces are central too,
    so angular momentum of fluid plus bodies is kept up to the O(dt^2) time error of the
    body rotation update."""
    sc = S.cluster(dim=3, n=9, dx=0.1, n_bodies=2, vel_amp=0.05)
    o = O.OracleScene(sc)
    I = o.bodies()["inertia"]
    for k in range(2):
        assert np.allclose(I[k], I[k][0, 0] * np.eye(3), rtol=1e-12, atol=1e-16)
    d0 = o.diagnostics()
    o.step(60)
    d = o.diagnostics()
    Lscale = np.linalg.norm(d0[3:6])
    err60 = np.linalg.norm(d[3:6] - d0[3:6])
    assert err60 < 1e-6 * Lscale, (d[3:6], d0[3:6])
    assert np.all(np.abs(d[:3] - d0[:3]) < 1e-13 * (1 + np.abs(d0[:3]).max()))


def test_heat_energy_conserved_adiabatic():
    """Adiabatic closed system (periodic, no walls): sum m c_p T is constant because the
    Cleary-Monaghan pair terms are antisymmetric (Eq. heat_equation)."""
    sc = S.periodic_box(dim=3, n=8, dx=0.1, bodies=1, body_radius=0.25, vel_amp=0.05, kappa=2.0,
                        cp=1.5, T_amp=30.0)
    sc["materials"][1]["kappa"] = 7.0
    sc["materials"][1]["cp"] = 0.6
    sc["params"]["dt_fixed"] = 1e-4  # below the conduction limit 0.1 rho c_p h^2 / kappa
    o = O.OracleScene(sc)
    e0 = o.diagnostics()[7]
    for _ in range(5):
        o.step(4)
        assert abs(o.diagnostics()[7] - e0) < 1e-13 * abs(e0)
    T = o.get("temp")
    assert T.std() < sc["particles"]["temperature"].std()


# ----------------------------------------------------------------------------- rigid bodies (Sec. 3.4)

def test_disk_mass_and_inertia_converge_to_paper_values():
    gd = json.load(open(os.path.join(GOLD, "disk_mass_inertia.json")))
    R = gd["diameter"] / 2
    errs_m, errs_i = [], []
    for dx in gd["dx"]:
        n = int(np.ceil(2 * R / dx)) + 2
        ax = (np.arange(-n, n) + 0.5) * dx
        X, Y = np.meshgrid(ax, ax, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), 0 * X.ravel()], 1)
        P = P[(P[:, 0] ** 2 + P[:, 1] ** 2) <= R * R]
        m = np.full(len(P), gd["density"] * dx * dx)
        M, c, I = O.body_mass_chunked(2, dx, P, m, len(P))
        assert gd["mass_axis_range"][0] < M < gd["mass_axis_range"][1]
        assert gd["inertia_axis_range"][0] < I[2, 2] < gd["inertia_axis_range"][1]
        errs_m.append(abs(M / gd["mass_analytic"] - 1))
        errs_i.append(abs(I[2, 2] / gd["inertia_analytic"] - 1))
    assert errs_m[-1] < 1e-3 and errs_i[-1] < 1e-3
    assert errs_m[-1] < errs_m[0] / 50 and errs_i[-1] < errs_i[0] / 50


def test_two_level_mass_quantities_equal_direct_sum():
    """Eqs. procwise_* + global_* (chunks as processors) reproduce the serial result."""
    rng = np.random.default_rng(0)
    P = rng.normal(size=(997, 3))
    m = rng.uniform(0.5, 2.0, size=997)
    M1, c1, I1 = O.body_mass_chunked(3, 0.1, P, m, 997)
    for chunk in (1, 7, 64, 500):
        M2, c2, I2 = O.body_mass_chunked(3, 0.1, P, m, chunk)
        assert abs(M2 - M1) < 1e-14 * M1
        assert np.allclose(c2, c1, rtol=0, atol=1e-14 * np.abs(P).max())
        assert np.allclose(I2, I1, rtol=0, atol=1e-13 * np.abs(I1).max())
    # inertia of a point cloud = sum m (|d|^2 1 - d d^T) + sum I_r 1 (Huygens-Steiner)
    d = P - c1
    ref = np.einsum("i,ij->j", m, d * d).sum() * np.eye(3) - np.einsum("i,ij,ik->jk", m, d, d)
    Ir = 0.4 * m * ((0.75 / math.pi) ** (1 / 3) * 0.1) ** 2
    assert np.allclose(I1, ref + Ir.sum() * np.eye(3), rtol=1e-12, atol=0)


def test_quaternion_product_composes_rotations():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = rng.normal(size=4); a /= np.linalg.norm(a)
        b = rng.normal(size=4); b /= np.linalg.norm(b)
        Ra, Rb = O.quat_rot(a), O.quat_rot(b)
        assert np.allclose(Ra @ Ra.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(Ra) - 1) < 1e-14
        assert np.allclose(O.quat_rot(O.quat_mul(a, b)), Ra @ Rb, atol=1e-14)
    # rotation by angle t about z: (cos t/2, 0, 0, sin t/2) maps x to (cos t, sin t, 0)
    t = 0.7
    R = O.quat_rot([math.cos(t / 2), 0, 0, math.sin(t / 2)])
    assert np.allclose(R @ [1, 0, 0], [math.cos(t), math.sin(t), 0], atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_fall_is_exact(dim):
    """Single body, no fluid, no walls: KDK integrates constant gravity exactly,
    r_k(t) = r0 + v0 t + g t^2 / 2."""
    sc = S.free_fall(dim=dim, vel=(0.3, -0.1, 0.2) if dim == 3 else (0.3, -0.1, 0.0))
    o = O.OracleScene(sc)
    b0 = o.bodies()
    g = np.array(sc["params"]["gravity"])
    v0 = np.array(sc["bodies"]["vel"][0])
    dt = sc["params"]["dt_fixed"]
    o.step(200)
    b = o.bodies()
    t = 200 * dt
    expect = b0["com"][0] + v0 * t + 0.5 * g * t * t
    assert np.allclose(b["com"][0], expect, rtol=0, atol=1e-13 * (1 + np.abs(expect).max()))
    assert np.allclose(b["vel"][0], v0 + g * t, rtol=0, atol=1e-13)


def test_torque_free_sphere_rotates_at_constant_rate():
    w = np.array([0.3, -1.1, 0.6])
    sc = S.free_fall(dim=3, g=0.0, omega=tuple(w))
    o = O.OracleScene(sc)
    dt = sc["params"]["dt_fixed"]
    o.step(500)
    q = o.bodies()["quat"][0]
    th = np.linalg.norm(w) * 500 * dt
    ax = w / np.linalg.norm(w)
    expect = np.concatenate([[math.cos(th / 2)], math.sin(th / 2) * ax])
    assert np.allclose(q, expect, atol=1e-12)
    # rigid invariance: pairwise distances inside the body are unchanged
    x0 = sc["particles"]["pos"]
    x1 = o.get("pos")
    d0 = np.linalg.norm(x0[:, None] - x0[None], axis=-1)
    d1 = np.linalg.norm(x1[:, None] - x1[None], axis=-1)
    assert np.abs(d1 - d0).max() < 1e-13


def test_contact_elastic_head_on_swaps_velocities():
    """Two equal single-particle bodies, d_c = 0: a linear repulsive spring acting while
    r < dx returns the velocities exchanged (elastic, equal masses) and lasts half a
    period pi sqrt(m_eff / k_c) of the spring."""
    k, speed = 1e3, 0.5
    sc = S.contact_pair(dim=2, gap=0.001, speed=speed, k_contact=k, d_contact=0.0, dt=2e-5)
    o = O.OracleScene(sc)
    m = sc["particles"]["mass"][0]
    t_contact = math.pi * math.sqrt(0.5 * m / k)
    steps = int(3 * t_contact / 2e-5) + 200
    touching = 0
    fmin = 0.0
    for _ in range(steps):
        o.step(1)
        f = o.get("force")
        x = o.get("pos")
        e = (x[0] - x[1]) / np.linalg.norm(x[0] - x[1])
        fmin = min(fmin, float(f[0] @ e))  # tension cut-off: never attractive
        touching += np.linalg.norm(x[0] - x[1]) < 0.1
    v = o.bodies()["vel"]
    assert fmin >= 0.0
    assert np.allclose(v[0], [-speed, 0, 0], atol=2e-3 * speed)
    assert np.allclose(v[1], [speed, 0, 0], atol=2e-3 * speed)
    assert abs(touching * 2e-5 - t_contact) < 0.02 * t_contact


def test_contact_damping_dissipates():
    sc = S.contact_pair(dim=3, gap=0.001, speed=0.5, k_contact=1e3, d_contact=0.5, dt=2e-5)
    o = O.OracleScene(sc)
    ke0 = o.diagnostics()[6]
    o.step(4000)
    ke = o.diagnostics()[6]
    v = o.bodies()["vel"]
    assert ke < 0.9 * ke0 and v[0][0] < 0 < v[1][0]  # bounced, slower


# ----------------------------------------------------------------------------- closed forms of the fluid and heat solvers

def test_hydrostatic_pressure_closed_box():
    """Closed 2D box filled with fluid at rest under gravity: the static state has
    dp/dy = -rho0 |g| (EOS, momentum equation and wall extrapolation together; the
    closed box avoids the free surface, where the plain WCSPH density deficit pulls
    the surface rows inward)."""
    dx = 0.02
    sc = S.hydrostatic_tank2d(dx=dx, width=0.4, depth=0.56, c=10.0, eta=0.2, closed=True)
    o = O.OracleScene(sc)
    o.step(2000)
    x, p, mat, u = o.get("pos"), o.get("pres"), o.get("mat"), o.get("vel")
    f = mat == 0
    y, xx = x[f, 1], x[f, 0]
    sel = (y > 3 * dx) & (y < 0.56 - 3 * dx) & (xx > 3 * dx) & (xx < 0.4 - 3 * dx)
    A = np.stack([np.ones(sel.sum()), y[sel]], 1)
    coef = np.linalg.lstsq(A, p[f][sel], rcond=None)[0]
    rho = o.get("rho")[f][sel].mean()
    assert abs(coef[1] / (-rho * 1.0) - 1) < 5e-3, coef
    resid = p[f][sel] - A @ coef
    assert np.sqrt(np.mean(resid ** 2)) < 1e-2 * np.sqrt(np.mean((p[f][sel] - p[f][sel].mean()) ** 2))
    assert np.abs(u[f]).max() < 1e-3


@pytest.mark.parametrize("dim", [2, 3])
def test_heat_conduction_sine_decay(dim):
    """Periodic slab at rest with T = T0 + A sin(k x): the amplitude decays as
    exp(-kappa k^2 t / (rho c_p)) (1D heat equation, Eq. goveq heat)."""
    n = (48, 8) if dim == 2 else (48, 8, 8)
    dx = 1.0 / 48
    kappa, cp = 1.0, 1.0
    sc = S.heat_slab(dim=dim, n=n, dx=dx, kappa=kappa, cp=cp)
    o = O.OracleScene(sc)
    rho = o.get("rho").mean()
    x = sc["particles"]["pos"][:, 0]
    k = 2 * math.pi / 1.0
    steps = 400
    o.step(steps)
    t = steps * sc["params"]["dt_fixed"]
    T = o.get("temp")
    A = 2 * np.mean((T - 300.0) * np.sin(k * x))
    expect = 10.0 * math.exp(-kappa * k * k * t / (rho * cp))
    assert abs(A / expect - 1) < 1e-2, (A, expect)
    # particles stay at rest on the periodic lattice
    assert np.abs(o.get("pos") - sc["particles"]["pos"]).max() < 1e-12


def test_linear_temperature_field_is_stationary_in_the_interior():
    dim = 2
    sc = S.heat_slab(dim=dim, n=(20, 20), dx=0.05, A=0.0)
    sc["params"]["periodic"] = [0, 0, 0]
    sc["params"]["box_min"] = [-1.0, -1.0, 0.0]
    sc["params"]["box_max"] = [2.0, 2.0, 0.0]
    x = sc["particles"]["pos"]
    sc["particles"]["temperature"] = 300.0 + 3.0 * x[:, 0] - 2.0 * x[:, 1]
    o = O.OracleScene(sc)
    dT = o.get("dtemp")
    interior = np.all((x[:, :2] > 3.5 * 0.05) & (x[:, :2] < 1.0 - 3.5 * 0.05), axis=1)
    assert np.abs(dT[interior]).max() < 1e-9


def test_time_step_cfl_condition():
    sc = S.tank2d_disc()
    o = O.OracleScene(sc)
    o.step(1)
    d = o.diagnostics()
    # at rest the CFL term 0.25 h / c binds (viscous 0.125 h^2 / nu = 1.95e-3, body force 0.028)
    assert abs(d[11] - 0.25 * 0.0125 / 10.0) < 1e-18


# ----------------------------------------------------------------------------- phase transitions (Sec. 3.6)

def _melt_scene(T_body, T_fluid=1100.0):
    sc = S.periodic_box(dim=2, n=16, dx=0.1, bodies=1, body_radius=0.35, vel_amp=0.0, kappa=0.0)
    mats = sc["materials"]
    mats[0].update(T_transition=1000.0, transitions_to=1)
    mats[1].update(T_transition=1000.0, transitions_to=0)
    p = sc["particles"]
    p["temperature"] = np.where(p["material"] == 1, T_body, T_fluid).astype(float)
    sc["bodies"]["omega"][:] = [0, 0, 0.5]
    sc["bodies"]["vel"][:] = [0.1, 0.0, 0.0]
    return sc


def test_melting_relabels_and_retires_body():
    sc = _melt_scene(T_body=1200.0)
    o = O.OracleScene(sc)
    o.step(1)
    mat = o.get("mat")
    assert np.all(mat == 0)
    assert o.bodies()["alive"][0] == 0
    assert np.all(o.get("body") == -1)


def test_partial_melt_keeps_velocity_of_remaining_particles():
    """After a relabel the remaining particles of the body keep their velocity
    (u_k = u'_k + w x (r_k - r'_k), reading R10)."""
    sc = _melt_scene(T_body=900.0)
    p = sc["particles"]
    rig = np.nonzero(p["material"] == 1)[0]
    x = p["pos"][rig]
    hot = rig[x[:, 0] > np.median(x[:, 0])]
    p["temperature"][hot] = 1100.0
    o = O.OracleScene(sc)
    o.step(1)
    mat = o.get("mat")
    stay = rig[mat[rig] == 1]
    assert len(stay) and np.all(mat[hot] == 0)
    # reference: the rigid velocity field of the old body evaluated at the positions
    com_old_sc = O.OracleScene(_melt_scene(T_body=900.0))
    com_old_sc.step(1)
    u_ref = com_old_sc.get("vel")
    u = o.get("vel")
    assert np.allclose(u[stay], u_ref[stay], rtol=0, atol=1e-14)
    b = o.bodies()
    assert b["alive"][0] == 1 and b["mass"][0] < com_old_sc.bodies()["mass"][0]


def test_solidification_joins_nearest_body_or_forms_new_ones():
    sc = _melt_scene(T_body=900.0)
    p = sc["particles"]
    x = p["pos"]
    rig = p["material"] == 1
    c = x[rig].mean(0)
    dist = np.linalg.norm(x - c, axis=1)
    # a ring of fluid touching the body, and a separate cold patch far away
    ring = (~rig) & (dist < 0.5)
    far = (~rig) & (np.linalg.norm(x - (c + [0.75, 0.75, 0]), axis=1) < 0.15)
    p["temperature"][ring | far] = 900.0
    o = O.OracleScene(sc)
    o.step(1)
    mat, body = o.get("mat"), o.get("body")
    assert np.all(mat[ring] == 1) and np.all(body[ring] == 0)
    assert np.all(mat[far] == 1)
    newb = np.unique(body[far])
    assert len(newb) == 1 and newb[0] == 1
    b = o.bodies()
    assert b["alive"][1] == 1 and abs(b["mass"][1] - far.sum() * 0.01) < 1e-15


def test_enthalpy_balance_with_source_over_melt_and_solidify():
    """With latent heat (apparent-capacity extension) and the surface source, sum m H
    changes by exactly the integrated source power (pair terms cancel)."""
    sc = S.periodic_box(dim=2, n=16, dx=0.1, bodies=1, body_radius=0.45, vel_amp=0.0, kappa=5.0,
                        jitter=0.0)
    sc["particles"]["temperature"] = np.where(sc["particles"]["material"] == 1, 310.0, 400.0)
    mats = sc["materials"]
    for m in mats:
        m.update(T_transition=320.0, latent_heat=20.0, mushy_width=4.0)
    mats[0]["transitions_to"] = 1
    mats[1]["transitions_to"] = 0
    p = sc["params"]
    p.update(src_power=4000.0, src_radius=0.3, src_origin=[0.8, 0.0, 0.0], src_speed=[0.0, 0.0, 0.0],
             src_depth=10.0, src_ztop=5.0)
    o = O.OracleScene(sc)
    dt = p["dt_fixed"]
    e0 = o.diagnostics()[7]
    # expected source power: independent quadrature of the per-particle source terms
    melted = False
    for _ in range(40):
        mass = sc["particles"]["mass"]
        e_before = o.diagnostics()[7]
        o.step(1)
        # the source of step n+1 is evaluated at r^{n+1} with rho^{n+1}
        x = o.get("pos")
        q = 4000.0 * np.exp(-2.0 * ((x[:, 0] - 0.8) ** 2) / 0.09)
        rho1 = o.get("rho")
        expect = dt * np.sum(mass * q / rho1)
        assert abs((o.diagnostics()[7] - e_before) - expect) < 1e-10 * abs(e_before)
        melted |= bool(np.any((o.get("mat") == 0) & (sc["particles"]["material"] == 1)))
    assert melted
    assert o.diagnostics()[7] > e0


def _couette_series(y, t, U, H, nu, N=400):
    """Start-up plane Couette flow (wall at y = 0 at rest, wall at y = H moving at U from
    t = 0, fluid at rest): u = U y/H + (2U/pi) sum_n ((-1)^n / n) sin(n pi y/H) exp(-n^2 pi^2 nu t/H^2)."""
    n = np.arange(1, N + 1)[:, None]
    return U * y / H + (2 * U / np.pi) * np.sum(((-1.0) ** n / n) * np.sin(n * np.pi * y / H)
                                                 * np.exp(-(n * np.pi) ** 2 * nu * t / H ** 2), axis=0)


def test_moving_wall_couette_start_up_matches_series_and_converges():
    """Moving boundary particles (R14): the start-up of plane Couette flow follows the
    closed-form series, and the error falls as the spacing is refined."""
    errs = []
    for dx in (0.01, 0.005):
        sc = S.couette2d(dx=dx)
        o = O.OracleScene(sc)
        o.step(int(round(0.01 / sc["params"]["dt_fixed"])))
        t = o.diagnostics()[9]
        x, v, fl = o.get("pos"), o.get("vel"), o.get("mat") == 0
        errs.append(np.abs(v[fl, 0] - _couette_series(x[fl, 1], t, 1.0, 0.2, 0.1)).max())
        assert np.abs(v[fl, 1]).max() < 1e-3
    assert errs[0] < 5e-3 and errs[1] < 0.5 * errs[0], errs


def test_moving_wall_reaches_linear_profile_and_translates():
    sc = S.couette2d()
    p = sc["params"]
    tau = 0.2 ** 2 / (np.pi ** 2 * 0.1)
    n = int(round(6 * tau / p["dt_fixed"]))
    o = O.OracleScene(sc)
    o.step(n)
    x, v, mat = o.get("pos"), o.get("vel"), o.get("mat")
    fl = mat == 0
    assert np.abs(v[fl, 0] - x[fl, 1] / 0.2).max() < 2e-3
    top = (mat == 1) & (x[:, 1] > 0.2)
    x0 = sc["particles"]["pos"][top, 0]
    shift = np.mod(x[top, 0] - x0, 0.1)
    assert np.allclose(shift, np.mod(n * p["dt_fixed"], 0.1), atol=1e-12)


# --------------------------------------------------------------------------- transport velocity (R15)

def _with_pb(sc, factor=1.0):
    """The scene with the background pressure p_b = factor * p0 of its fluid."""
    fl = [m for m in sc["materials"] if m["kind"] == 0][0]
    sc["params"]["p_background"] = factor * fl["rho0"] * fl["c"] ** 2
    return sc


@pytest.mark.parametrize("dim", [2, 3])
def test_background_acceleration_vanishes_on_a_regular_lattice(dim):
    """The transport-velocity terms vanish for distributions with the kernel's partition of
    unity (Sec. 3.3.2): on a periodic lattice a~ = 0 to rounding and the lattice stays at rest."""
    sc = _with_pb(S.periodic_box(dim=dim, n=8 if dim == 3 else 16, dx=0.1, vel_amp=0.0, jitter=0.0))
    o = O.OracleScene(sc)
    fl = sc["materials"][0]
    scale = fl["rho0"] * fl["c"] ** 2 / (fl["rho0"] * 0.1)  # p_b / (rho h)
    assert np.abs(o.get("bacc")).max() < 1e-12 * scale
    o.step(20)
    assert np.abs(o.get("vel")).max() < 1e-12 * 10.0
    assert np.abs(o.get("pos") - sc["particles"]["pos"]).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_momentum_conserved_with_transport_velocity(dim):
    """1/2 (A_i + A_j) . grad W_ij is antisymmetric in i, j: total momentum stays exact."""
    sc = _with_pb(S.periodic_box(dim=dim, n=10 if dim == 3 else 20, dx=0.1, bodies=2 if dim == 3 else 3,
                                 body_radius=0.16, vel_amp=0.2, jitter=0.1, seed=4))
    o = O.OracleScene(sc)
    d0 = o.diagnostics()
    scale = np.abs(sc["particles"]["mass"][:, None] * sc["particles"]["vel"]).sum()
    for _ in range(5):
        o.step(10)
        d = o.diagnostics()
        assert np.all(np.abs(d[:3] - d0[:3]) <= 1e-13 * scale), (d[:3], d0[:3])
    assert np.abs(o.get("bacc")).max() > 0.0


def _disorder(o, sc):
    """Spread of the kernel sum sum_j V_j W_ij over fluid particles (0 on a lattice up to the
    lattice constant): the partition-of-unity defect the background pressure reduces."""
    rho, m = o.get("rho"), sc["particles"]["mass"]
    return float(np.std(rho / m))


def test_transport_velocity_regularises_a_disordered_distribution():
    """The background pressure drives a disordered distribution towards the partition of
    unity (Sec. 3.3.2): faster with p_b = p0 than without, faster still with 2 p0."""
    base = S.periodic_box(dim=2, n=24, dx=0.1, vel_amp=0.0, jitter=0.3, eta=0.05, seed=9)
    runs = {}
    for pb in (0.0, 1.0, 2.0):
        sc = _with_pb(copy.deepcopy(base), pb)
        o = O.OracleScene(sc)
        d0 = _disorder(o, sc)
        o.step(100)
        runs[pb] = _disorder(o, sc) / d0
    assert runs[1.0] < 0.9 * runs[0.0] and runs[2.0] < 0.95 * runs[1.0], runs


def test_couette_with_transport_velocity_keeps_the_linear_profile():
    sc = _with_pb(S.couette2d())
    tau = 0.2 ** 2 / (np.pi ** 2 * 0.1)
    o = O.OracleScene(sc)
    o.step(int(round(6 * tau / sc["params"]["dt_fixed"])))
    x, v, fl = o.get("pos"), o.get("vel"), o.get("mat") == 0
    assert np.abs(v[fl, 0] - x[fl, 1] / 0.2).max() < 5e-3


# --------------------------------------------------------------------------- concentration (R16)

@pytest.mark.parametrize("dim", [2, 3])
def test_concentration_sine_decay(dim):
    """C = C0 + A sin(k x) on a periodic lattice at rest decays as exp(-D k^2 t / rho)."""
    n = (48, 8) if dim == 2 else (48, 8, 8)
    sc = S.conc_slab(dim=dim, n=n, D=1.0)
    o = O.OracleScene(sc)
    rho = o.get("rho").mean()
    x = sc["particles"]["pos"][:, 0]
    k = 2 * math.pi
    o.step(400)
    t = 400 * sc["params"]["dt_fixed"]
    A = 2 * np.mean((o.get("conc") - 0.5) * np.sin(k * x))
    assert abs(A / (0.2 * math.exp(-k * k * t / rho)) - 1) < 1e-2


def test_concentration_sum_conserved_in_a_closed_box():
    sc = S.periodic_box(dim=3, n=10, dx=0.1, bodies=2, body_radius=0.2, vel_amp=0.1, jitter=0.1, seed=3)
    rng = np.random.default_rng(1)
    sc["particles"]["concentration"] = rng.uniform(0, 1, len(sc["particles"]["mass"]))
    for m in sc["materials"]:
        m["diffusivity"] = 0.5
    o = O.OracleScene(sc)
    m = sc["particles"]["mass"]
    s0 = np.sum(m * o.get("conc"))
    o.step(50)
    assert abs(np.sum(m * o.get("conc")) - s0) < 1e-13 * s0
    assert np.std(o.get("conc")) < np.std(sc["particles"]["concentration"])


def test_reservoir_bounds_and_concentration_driven_transition():
    """Juice held at C = 1 around boluses at C = 0: the concentration stays in [0, 1], rises
    in the boluses from their surface inwards, and bolus particles above C_t turn into chyme."""
    sc = S.gastric2d(dx=0.1, n_boluses=3)
    o = O.OracleScene(sc)
    mat0 = o.get("mat").copy()
    n_bolus = int(np.sum(mat0 == 2))
    nsteps = 0
    for _ in range(40):
        o.step(50)
        nsteps += 50
        C = o.get("conc")
        assert C.min() >= -1e-12 and C.max() <= 1 + 1e-12
        if np.sum(o.get("mat") == 3) > 0:
            break
    mat = o.get("mat")
    chyme = mat == 3
    assert chyme.any(), "no bolus particle reached C_t"
    assert np.all(mat0[chyme] == 2)                      # chyme comes from boluses only
    assert np.all(o.get("conc")[chyme] > 0.0)
    assert np.sum(mat == 2) == n_bolus - int(chyme.sum())
    assert np.all(o.get("body")[chyme] == -1)


# --------------------------------------------------------------------------- post-processing (Eq. postprocessing)

def test_shepard_filter_reproduces_constants_everywhere():
    """The Shepard normalisation makes the filtered field of a constant exactly that constant,
    next to walls and bodies too."""
    sc = S.tank2d_disc(dx=0.025)
    sc["particles"]["temperature"][:] = 123.25
    sc["particles"]["wall_temperature"] = np.full(len(sc["particles"]["mass"]), 123.25)
    o = O.OracleScene(sc)
    rng = np.random.default_rng(0)
    q = np.zeros((500, 3))
    q[:, :2] = rng.uniform(-0.05, 1.05, (500, 2))
    T = o.interpolate(q, "temp")
    ok = ~np.isnan(T)
    assert ok.sum() > 400
    assert np.abs(T[ok] - 123.25).max() < 1e-12


def test_shepard_filter_converges_at_second_order():
    errs = []
    for n, dx in ((24, 0.1), (48, 0.05), (96, 0.025)):
        sc = S.periodic_box(dim=2, n=n, dx=dx, vel_amp=0.0, jitter=0.0)
        x, L = sc["particles"]["pos"], n * dx
        f = lambda y: 300 + np.sin(2 * np.pi * y[:, 0] / L) * np.cos(2 * np.pi * y[:, 1] / L)
        sc["particles"]["temperature"] = f(x)
        o = O.OracleScene(sc)
        q = np.zeros((400, 3))
        q[:, :2] = np.random.default_rng(0).uniform(0, L, (400, 2))
        errs.append(np.abs(o.interpolate(q, "temp") - f(q)).max())
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5, errs


def test_shepard_filter_without_contributing_particles_is_nan():
    sc = S.tank2d_disc(dx=0.025)
    o = O.OracleScene(sc)
    q = np.array([[0.5, 0.4, 0.0], [0.1, 0.9, 0.0]])  # disc centre; far from the disc
    v = o.interpolate(q, "vel", material_mask=1 << 2)  # the disc's material only
    assert np.isfinite(v[0]).all() and np.isnan(v[1]).all()


# --------------------------------------------------------------------------- Dirichlet walls (Sec. 2.3, Eq. heat_equation)

@pytest.mark.parametrize("dim", [2, 3])
def test_linear_temperature_with_dirichlet_walls_on_its_extension_is_stationary(dim):
    """Walls hold the straight-line temperature of the fluid's profile, extended into the
    wall block.  Wall neighbours take kappa_b := kappa_a (the wall material's own kappa,
    set to 0 here, must not enter), so every fluid particle, including those next to the
    walls, sees a complete lattice of equal pair weights on a linear field: dT/dt = 0 to
    rounding.  The wall density is set to the fluid's lattice density so that V_b is
    equal on both sides.  A wrong wall conductance, a wrong sign of T_ab against a wall, or
    the wall material's kappa would each leave the near-wall particles with a rate."""
    dx = 1.0 / 24
    sc = S.dirichlet_slab(dim=dim, nx=24, ny=6, dx=dx, linear=True, wall_kappa=0.0)
    f = sc["particles"]["material"] == 0
    rho = O.OracleScene(sc).get("rho")[f]
    # the interior lattice density of the kernel remark (the partition-of-unity values)
    assert abs(rho.mean() - (1.0000632246 if dim == 2 else 0.9999799597)) < 1e-10
    sc["particles"]["density"][~f] = rho.mean()
    dT = O.OracleScene(sc).get("dtemp")[f]
    scale = 1.0 * 100.0 / (rho.mean() * 1.0 * 1.0 * dx)  # kappa (T2 - T1) / (rho c_p L dx)
    assert np.abs(dT).max() < 1e-12 * scale


def _dirichlet_series(x, t, T0, T1, T2, L, alpha, N=2000):
    """Start-up of 1D conduction between walls held at T1 (x = 0) and T2 (x = L), uniform T0
    at t = 0: T = T1 + (T2 - T1) x / L + sum_n B_n sin(n pi x / L) exp(-alpha (n pi / L)^2 t),
    B_n = 2 / (n pi) [(T0 - T1)(1 - (-1)^n) + (T2 - T1)(-1)^n]."""
    n = np.arange(1, N + 1)[:, None]
    B = 2.0 / (n * np.pi) * ((T0 - T1) * (1 - (-1.0) ** n) + (T2 - T1) * (-1.0) ** n)
    return T1 + (T2 - T1) * x / L + np.sum(B * np.sin(n * np.pi * x / L) * np.exp(-alpha * (n * np.pi / L) ** 2 * t),
                                           axis=0)


def test_dirichlet_walls_start_up_follows_the_series_and_converges():
    """Fluid at T0 between walls at T1 = T0 and T2 = T0 + 100 (Dirichlet, Sec. 2.3): the
    temperature at t = 0.02 follows the closed-form series of the 1D heat equation, with an
    error that halves with dx (the wall temperature acts at the first wall row, dx/2 from
    the fluid edge, which shifts the boundary by O(dx))."""
    errs = []
    for nx in (20, 40):
        dx = 1.0 / nx
        sc = S.dirichlet_slab(dim=2, nx=nx, ny=6, dx=dx, T_left=300.0, T_right=400.0, T0=300.0)
        o = O.OracleScene(sc)
        f = sc["particles"]["material"] == 0
        alpha = 1.0 / o.get("rho")[f].mean()  # kappa / (rho c_p)
        steps = int(round(0.02 / sc["params"]["dt_fixed"]))
        o.step(steps)
        x, T = o.get("pos")[f, 0], o.get("temp")[f]
        errs.append(np.abs(T - _dirichlet_series(x, steps * sc["params"]["dt_fixed"], 300.0, 300.0, 400.0, 1.0,
                                                 alpha)).max() / 100.0)
    assert errs[0] < 0.12 and errs[1] < 0.06, errs
    assert errs[0] / errs[1] > 1.8, errs


def test_dirichlet_walls_steady_profile_is_linear_with_the_boundary_at_the_first_wall_row():
    """Steady state between walls at T1 and T2: linear in x, and the line reaches T1 and T2
    half a spacing outside the fluid (at the first row of wall particles, which carry the
    prescribed temperature), for every dx.  A wall pair weight other than the fluid's
    (kappa_b := kappa_a) moves this point by more than a spacing."""
    for nx in (10, 20):
        dx = 1.0 / nx
        sc = S.dirichlet_slab(dim=2, nx=nx, ny=6, dx=dx, T_left=300.0, T_right=400.0, T0=350.0, dt=0.2 * dx * dx)
        o = O.OracleScene(sc)
        f = sc["particles"]["material"] == 0
        o.step(int(round(0.8 / sc["params"]["dt_fixed"])))
        x, T = o.get("pos")[f, 0], o.get("temp")[f]
        A = np.stack([np.ones_like(x), x], 1)
        c = np.linalg.lstsq(A, T, rcond=None)[0]
        assert np.abs(T - A @ c).max() < 0.02 * 100.0 * dx
        lo, hi = (300.0 - c[0]) / c[1], (400.0 - c[0]) / c[1]
        assert abs(lo / dx + 0.5) < 0.1 and abs((hi - 1.0) / dx - 0.5) < 0.1, (lo / dx, (hi - 1.0) / dx)


# --------------------------------------------------------------------------- moving rigid boundaries (R4)

def test_free_falling_fluid_filled_container_keeps_uniform_pressure():
    """A closed rigid container (one body) full of fluid, in free fall: container and fluid
    share the acceleration g, so in the extrapolation of Sec. 3.3.4 (g - a_w) vanishes and
    the fluid stays at uniform pressure with no motion relative to the container.  A wrong
    sign of a_w doubles the effective gravity seen by the walls; a_w = 0 keeps it."""
    g = -1.0
    sc = S.rigid_container2d(dx=0.01, inner=0.2, g=g, eta=0.01)
    o = O.OracleScene(sc)
    f = sc["particles"]["material"] == 0
    dt = sc["params"]["dt_fixed"]
    for k in range(1, 7):
        o.step(100)
        p, u = o.get("pres")[f], o.get("vel")[f]
        b = o.bodies()
        assert (p.max() - p.min()) < 2e-3 * 1.0 * abs(g) * 0.2  # of rho |g| H
        assert np.abs(u - b["vel"][0]).max() < 2e-5
        # the body follows g t (up to the start-up, where a_w of the initial evaluation is 0)
        assert abs(b["vel"][0][1] - g * 100 * k * dt) < 1e-5


def test_spinning_container_pushes_the_adjacent_fluid_towards_its_centre():
    """A closed rigid container spinning at w with the fluid in solid-body rotation (no
    gravity, inviscid), initial evaluation: the fluid has uniform pressure, so only the
    walls act, and they must supply a centripetal force, a_w = w x (w x r) entering
    (g - a_w) of the extrapolation.  Fluid in the row next to the container accelerates
    towards the centre at a fraction of w^2 r; the interior does not accelerate.  The
    opposite sign of the term pulls the row outwards; without the term it stays put."""
    w = 4.0
    sc = S.rigid_container2d(dx=0.01, inner=0.2, g=0.0, eta=0.0, omega=w)
    o = O.OracleScene(sc)
    f = sc["particles"]["material"] == 0
    x, a = o.get("pos")[f][:, :2], o.get("acc")[f][:, :2]
    r = np.linalg.norm(x, axis=1)
    ar = np.sum(a * x, 1) / r / (w * w * r)  # radial acceleration in units of w^2 r
    dwall = 0.1 - np.abs(x).max(1)
    first = dwall < 0.01
    interior = dwall > 0.02
    assert np.all(ar[first] < -0.2) and np.all(ar[first] > -1.0), (ar[first].min(), ar[first].max())
    assert np.abs(ar[interior]).max() < 1e-9


def test_melted_particle_takes_the_acceleration_of_its_material_point():
    """A spinning rigid sphere pressed by one wall particle (contact force and torque), hot
    enough to melt in its first step: each particle leaves the body with the acceleration
    its material point had in the rigid motion, a_k + alpha_k x r + w_k x (w_k x r) (rigid
    body kinematics; reading R10), with a_k = f_k / m_k and alpha_k = I_k^-1 m_k of the
    step's evaluation.  The same helper gives a_w in the extrapolation of Sec. 3.3.4."""
    sc = S.free_fall(dim=3, dx=0.1, radius=0.35, density=3.0, g=-9.81, omega=(1.5, -2.0, 3.0))
    mats = sc["materials"]
    mats[1].update(T_transition=1000.0, transitions_to=0)
    mats.append(S.material(S.WALL, 1.0))
    p = sc["particles"]
    p["temperature"][:] = 1200.0
    x = p["pos"]
    top = int(np.argmax(x[:, 0] + 0.3 * x[:, 1]))  # an off-centre particle on the surface
    wall = x[top] + np.array([0.09, 0.0, 0.0])
    for k in p:
        a = np.asarray(p[k])
        p[k] = np.concatenate([a, a[top:top + 1]], axis=0)
    p["pos"][-1] = wall
    p["material"][-1] = 2
    p["body"][-1] = -1
    p["vel"][-1] = 0.0
    p["wall_velocity"][-1] = 0.0
    sc["params"]["k_contact"] = 50.0
    sc["params"]["d_contact"] = 0.5
    o = O.OracleScene(sc)
    o.step(1)
    b = o.bodies()
    assert b["alive"][0] == 0 and np.all(o.get("mat")[:-1] == 0)
    ak = b["force"][0] / b["mass"][0]
    al = np.linalg.solve(b["inertia"][0], b["torque"][0])
    assert np.linalg.norm(b["torque"][0]) > 1e-3 and np.linalg.norm(al) > 1e-2  # the contact acts
    w = b["omega"][0]
    r = o.get("pos")[:-1] - b["com"][0]
    expect = ak + np.cross(al, r) + np.cross(w, np.cross(w, r))
    acc = o.get("acc")[:-1]
    assert np.abs(acc - expect).max() < 1e-12 * np.abs(expect).max()


# --------------------------------------------------------------------------- anisotropic inertia (Eq. angularmomentum)

def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_frame_rotation_covariance_with_an_anisotropic_body():
    """Rotating a whole scene (positions, velocities, gravity, body velocity and angular
    velocity, and the body orientation q -> q_R o q) by a fixed rotation R maps every output
    to R applied to the unrotated output (scalars unchanged), to rounding.  The body is an
    ellipsoid with distinct principal moments spinning about a non-principal axis in a
    viscous fluid (torque from the fluid), so alpha = R(q) I_body^-1 R(q)^T m: using the
    body-frame inertia in place of the world inertia, or a transposed rotation, breaks it."""
    sc = S.ellipsoid_in_fluid()
    ax = np.array([0.3, -0.8, 0.5])
    ax /= np.linalg.norm(ax)
    ang = 1.1
    qR = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax])
    R = O.quat_rot(qR)
    c = 0.5
    rot = copy.deepcopy(sc)
    rp, rb = rot["particles"], rot["bodies"]
    rp["pos"] = (sc["particles"]["pos"] - c) @ R.T + c
    rp["vel"] = sc["particles"]["vel"] @ R.T
    rot["params"]["gravity"] = list(R @ np.asarray(sc["params"]["gravity"]))
    rb["vel"] = sc["bodies"]["vel"] @ R.T
    rb["omega"] = sc["bodies"]["omega"] @ R.T
    rb["quat"] = np.array([_qmul(qR, q) for q in sc["bodies"]["quat"]])
    for s in (sc, rot):
        s["params"]["box_min"] = [c - 1.0] * 3
        s["params"]["box_max"] = [c + 1.0] * 3
    oa, ob = O.OracleScene(sc), O.OracleScene(rot)
    oa.step(30)
    ob.step(30)
    assert np.abs((oa.get("pos") - c) @ R.T + c - ob.get("pos")).max() < 1e-12
    for f in ("vel", "acc", "force", "vext"):
        B = ob.get(f)
        assert np.abs(oa.get(f) @ R.T - B).max() < 1e-12 * np.abs(B).max(), f
    for f in ("rho", "pres"):
        B = ob.get(f)
        assert np.abs(oa.get(f) - B).max() < 1e-12 * np.abs(B).max(), f
    ba, bb = oa.bodies(), ob.bodies()
    ev = np.linalg.eigvalsh(ba["inertia"][0])
    assert ev[1] / ev[0] > 1.5 and ev[2] / ev[1] > 1.1  # anisotropic
    for f in ("omega", "torque", "vel", "force"):
        assert np.abs(ba[f] @ R.T - bb[f]).max() < 1e-12 * np.abs(bb[f]).max(), f
    assert np.abs((ba["com"] - c) @ R.T + c - bb["com"]).max() < 1e-12
    assert np.abs(np.array([_qmul(qR, q) for q in ba["quat"]]) - bb["quat"]).max() < 1e-12
    assert np.abs(R @ ba["inertia"][0] @ R.T - bb["inertia"][0]).max() < 1e-12 * ev[2]


# --------------------------------------------------------------------------- apparent capacity (R11)

def test_temperature_of_grains_heated_through_the_mushy_interval():
    """Isolated single-particle grains of a melting material under a uniform source: the
    specific energy E(t) = sum dt q / rho they receive raises T at 1/c_s below the interval,
    at w / (c_s w + L) inside it (the interval absorbs the latent heat L on top of c_s w)
    and at 1 / c_l above it, with melting at T_t (apparent-capacity extension of the remark
    on latent heat).  Grains start below, inside and just under T_t."""
    T0 = np.array([250.0, 290.0, 305.0, 309.0])
    Tt, w, L, cs, cl, Q = 310.0, 8.0, 40.0, 1.0, 2.0, 2.0e3
    sc = S.heated_grains(T0=tuple(T0), T_t=Tt, mushy=w, latent=L, cp_s=cs, cp_l=cl, Q0=Q)
    o = O.OracleScene(sc)
    dt = sc["params"]["dt_fixed"]
    Tlo = Tt - 0.5 * w
    e1 = np.maximum(cs * (Tlo - T0), 0.0)                      # sensible heat up to the interval
    e2 = cs * w + L - np.where(T0 > Tlo, (T0 - Tlo) * (cs + L / w), 0.0)  # what is left of it
    E = np.zeros(len(T0))
    melted = np.zeros(len(T0), bool)
    for _ in range(200):
        o.step(1)
        E = E + dt * Q / o.get("rho")  # the source of the step at the step's density
        T = o.get("temp")
        expect = np.where(E <= e1, T0 + E / cs,
                          np.where(E <= e1 + e2, np.maximum(T0, Tlo) + (E - e1) * w / (cs * w + L),
                                   Tlo + w + (E - e1 - e2) / cl))
        assert np.abs(T - expect).max() < 1e-9, (T, expect)
        mat = o.get("mat")
        assert np.all((mat == 1) == (melted | (T > Tt)))  # melt at the end of the step that crosses T_t
        melted |= mat == 1
    assert np.all(melted) and np.all(T > Tlo + w)


# --------------------------------------------------------------------------- time step (Eq. timestepcond)

def _dt_of(sc):
    o = O.OracleScene(sc)
    o.step(1)
    return o.diagnostics()[11]


def test_time_step_velocity_condition_with_moving_fluid():
    """0.25 h / (c + |u|max): |u|max is the largest fluid speed at the step's start."""
    sc = S.heat_slab(dim=2, n=(12, 12), dx=0.1, A=0.0, kappa=0.0, c=2.0, dt=1e-3)
    sc["params"]["dt_mode"] = 1
    u = np.zeros((144, 3))
    u[:, 0] = 0.3
    u[17] = [0.6, -0.8, 0.0]  # speed 1
    sc["particles"]["vel"] = u
    assert abs(_dt_of(sc) - 0.25 * 0.1 / (2.0 + 1.0)) < 1e-17


def test_time_step_viscous_condition_takes_the_largest_kinematic_viscosity():
    """0.125 h^2 / nu with nu = eta / rho0 of the most viscous fluid phase."""
    sc = S.heat_slab(dim=2, n=(12, 12), dx=0.1, A=0.0, kappa=0.0, c=0.1, dt=1e-3)
    sc["params"]["dt_mode"] = 1
    sc["materials"][0]["eta"] = 0.5
    sc["materials"].append(S.material(S.FLUID, 2.0, c=0.1, eta=3.0))  # nu = 1.5
    sc["particles"]["material"][::7] = 1
    assert abs(_dt_of(sc) - 0.125 * 0.01 / 1.5) < 1e-18


def test_time_step_body_force_condition():
    """0.25 sqrt(h / |b|max) with the body force of gravity."""
    sc = S.heat_slab(dim=2, n=(12, 12), dx=0.1, A=0.0, kappa=0.0, c=0.01, dt=1e-3)
    sc["params"]["dt_mode"] = 1
    sc["params"]["periodic"] = [1, 0, 0]
    sc["params"]["box_min"][1] = -10.0
    sc["params"]["box_max"][1] = 10.0
    sc["params"]["gravity"] = [0.0, -30.0, 40.0 * 0.0]
    assert abs(_dt_of(sc) - 0.25 * math.sqrt(0.1 / 30.0)) < 1e-17


def test_time_step_contact_condition_takes_the_lightest_rigid_particle():
    """0.22 sqrt(m_r / k_c) with the smallest rigid particle mass."""
    sc = S.contact_pair(dim=2, dx=0.1, k_contact=1e6, d_contact=0.0)
    sc["params"]["dt_mode"] = 1
    sc["particles"]["mass"][1] = 0.5 * sc["particles"]["mass"][0]
    mr = sc["particles"]["mass"][1]
    assert abs(_dt_of(sc) - 0.22 * math.sqrt(mr / 1e6)) < 1e-18


def test_time_step_heat_condition_takes_the_smallest_diffusion_time():
    """0.1 rho c_p h^2 / kappa, minimised over the conducting phases (fluid and rigid)."""
    sc = S.heat_slab(dim=2, n=(12, 12), dx=0.1, A=0.0, kappa=2.0, cp=3.0, c=0.01)
    sc["params"]["dt_mode"] = 1
    sc["materials"].append(S.material(S.RIGID, 5.0, cp=0.2, kappa=10.0))  # rho c_p / kappa = 0.1
    assert abs(_dt_of(sc) - 0.1 * 0.1 * 0.01) < 1e-18
