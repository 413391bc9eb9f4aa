"""Seeded synthetic scene generators.

This module builds the *inputs* of a simulation: lattice sites, particle
masses assigned from a reference density and the lattice volume (the initial
discretisation of Sec. 3.1.2), materials, wall shells and rigid-body
membership.  It holds none of the SPH arithmetic (no kernel, no sums, no
integration) and imports nothing else from this package, so that both the
CUDA path and the FP64 CPU checker can be fed from it.

A scene is a plain ``dict``::

    {"params": {...}, "materials": [ {...}, ... ],
     "particles": {"pos": (n,3) f64, "vel": (n,3), "mass": (n,), "density": (n,),
                   "temperature": (n,), "material": (n,) i32, "body": (n,) i32,
                   "wall_velocity": (n,3), "wall_temperature": (n,)},
     "bodies": {"quat": (k,4), "vel": (k,3), "omega": (k,3)}}

Positions are always stored with three components (z = 0 in 2D).
Lattice sites sit at ``lo + (i + 1/2) dx`` (Sec. 3.1.2, Sec. 3.3.4 for the
wall layers at distance dx/2 outside the fluid).
"""
from __future__ import annotations

import math
import numpy as np

FLUID, RIGID, WALL = 0, 1, 2
NAN = float("nan")


def material(kind, rho0, c=0.0, eta=0.0, cp=1.0, kappa=0.0,
             T_transition=NAN, transitions_to=-1, latent_heat=0.0, mushy_width=0.0,
             diffusivity=0.0, C_transition=NAN, C_fixed=NAN, transition_by=0):
    """One material (phase) record; ``eta`` is the dynamic viscosity rho0*nu; the
    concentration fields follow the paper's remark on chemically induced transitions."""
    return dict(kind=int(kind), rho0=float(rho0), c=float(c), eta=float(eta), cp=float(cp),
                kappa=float(kappa), T_transition=float(T_transition),
                transitions_to=int(transitions_to), latent_heat=float(latent_heat),
                mushy_width=float(mushy_width), diffusivity=float(diffusivity),
                C_transition=float(C_transition), C_fixed=float(C_fixed), transition_by=int(transition_by))


def default_params(dim, dx, box_min, box_max, **kw):
    p = dict(dim=int(dim), dx=float(dx), h=float(dx), kernel_support=3.0,
             box_min=[float(v) for v in box_min] + [0.0] * (3 - len(box_min)),
             box_max=[float(v) for v in box_max] + [0.0] * (3 - len(box_max)),
             periodic=[0, 0, 0], gravity=[0.0, 0.0, 0.0],
             dt_mode=0, dt_fixed=1e-4, k_contact=0.0, d_contact=-1.0,
             precision=64, skin=0.0, rebin_interval=1, key_order=0, cells_per_group=0,
             body_capacity=0,
             src_power=0.0, src_radius=0.05, src_speed=[0.0, 0.0, 0.0],
             src_origin=[0.0, 0.0, 0.0], src_depth=0.0, src_ztop=0.0)
    if dim == 2:
        p["box_min"][2] = 0.0
        p["box_max"][2] = 0.0
    p.update(kw)
    return p


# --------------------------------------------------------------------------- lattices

def lattice(lo, n, dx):
    """Sites lo + (i+1/2) dx for i in [0, n) per axis; returns (N, len(n)) array."""
    axes = [lo[d] + (np.arange(n[d]) + 0.5) * dx for d in range(len(n))]
    grids = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel(order="F") for g in grids], axis=1)


def _pad3(p):
    if p.shape[1] == 3:
        return p
    out = np.zeros((p.shape[0], 3))
    out[:, : p.shape[1]] = p
    return out


def wall_shell(dim, n_in, dx, layers=3, open_top=False, top_extra=0):
    """Boundary particles in ``layers`` rows around the interior box of n_in sites.

    The interior occupies [0, n_in*dx) per axis.  With ``open_top`` the shell has no
    top layer on the last axis, and the side walls extend ``top_extra`` sites above
    the interior.
    """
    lo_i = [-layers] * dim
    hi_i = [n_in[d] + layers for d in range(dim)]
    if open_top:
        hi_i[-1] = n_in[-1] + top_extra
    idx = [np.arange(lo_i[d], hi_i[d]) for d in range(dim)]
    grids = np.meshgrid(*idx, indexing="ij")
    ijk = np.stack([g.ravel(order="F") for g in grids], axis=1)
    inside = np.ones(len(ijk), dtype=bool)
    for d in range(dim):
        hi_lim = n_in[d] if not (open_top and d == dim - 1) else hi_i[d]
        inside &= (ijk[:, d] >= 0) & (ijk[:, d] < hi_lim)
    ijk = ijk[~inside]
    return (ijk + 0.5) * dx


# --------------------------------------------------------------------------- assembly

class _Builder:
    def __init__(self, dim):
        self.dim = dim
        self.parts = []  # list of dict chunks
        self.bodies = []

    def add(self, pos, mat, mass, density, T, body=-1, vel=None, wall_T=NAN, wall_vel=None, conc=0.0):
        pos = np.asarray(pos, dtype=np.float64)
        if pos.ndim == 1:
            pos = pos.reshape(1, -1)
        pos = _pad3(pos)
        n = len(pos)
        ch = dict(pos=pos,
                  vel=np.zeros((n, 3)) if vel is None else np.broadcast_to(np.asarray(vel, float), (n, 3)).copy(),
                  mass=np.full(n, float(mass)) if np.isscalar(mass) else np.asarray(mass, float),
                  density=np.full(n, float(density)) if np.isscalar(density) else np.asarray(density, float),
                  temperature=np.full(n, float(T)) if np.isscalar(T) else np.asarray(T, float),
                  material=np.full(n, int(mat), dtype=np.int32),
                  body=np.full(n, int(body), dtype=np.int32) if np.isscalar(body) else np.asarray(body, np.int32),
                  wall_velocity=np.zeros((n, 3)) if wall_vel is None else np.broadcast_to(np.asarray(wall_vel, float), (n, 3)).copy(),
                  wall_temperature=np.full(n, float(wall_T)) if np.isscalar(wall_T) else np.asarray(wall_T, float),
                  concentration=np.full(n, float(conc)) if np.isscalar(conc) else np.asarray(conc, float))
        self.parts.append(ch)
        return n

    def add_body(self, vel=(0, 0, 0), omega=(0, 0, 0), quat=(1, 0, 0, 0)):
        self.bodies.append((list(quat), list(vel), list(omega)))
        return len(self.bodies) - 1

    def finish(self, params, materials):
        keys = ["pos", "vel", "mass", "density", "temperature", "material", "body",
                "wall_velocity", "wall_temperature", "concentration"]
        parts = {k: np.concatenate([c.get(k, np.zeros(len(c["mass"]))) for c in self.parts], axis=0) for k in keys}
        parts["material"] = parts["material"].astype(np.int32)
        parts["body"] = parts["body"].astype(np.int32)
        k = len(self.bodies)
        bodies = dict(quat=np.array([b[0] for b in self.bodies], float).reshape(k, 4),
                      vel=np.array([b[1] for b in self.bodies], float).reshape(k, 3),
                      omega=np.array([b[2] for b in self.bodies], float).reshape(k, 3))
        return dict(params=params, materials=materials, particles=parts, bodies=bodies)


def _jitter(rng, pos, amp, dim):
    if amp <= 0:
        return pos
    j = np.zeros_like(pos)
    j[:, :dim] = rng.uniform(-amp, amp, size=(len(pos), dim))
    return pos + j


# --------------------------------------------------------------------------- workloads

def tank2d_disc(dx=0.0125, seed=2103, steps_dt=None, jitter=1e-3, fill=0.65,
                disc_center=(0.5, 0.4), disc_radius=0.1, disc_density=2.0,
                c=10.0, rho0=1.0, eta=0.01, g=-1.0, precision=64):
    """2D unit box, fluid to height ``fill``, one rigid disc, 3-layer closed wall shell.

    Default sizes: 3,952 fluid, 208 rigid, 996 wall particles (dx = 0.0125).
    dt from the CFL-type conditions of Eq. (timestep) (dt_mode = 1).
    """
    rng = np.random.default_rng(seed)
    n = int(round(1.0 / dx))
    nf = int(round(fill / dx))
    sites = lattice([0.0, 0.0], [n, nf], dx)
    dc = np.linalg.norm(sites - np.asarray(disc_center), axis=1)
    in_disc = dc <= disc_radius
    b = _Builder(2)
    mats = [material(FLUID, rho0, c=c, eta=eta, cp=1.0, kappa=0.0),
            material(WALL, rho0),
            material(RIGID, disc_density)]
    fl = _jitter(rng, _pad3(sites[~in_disc]), jitter * dx, 2)
    b.add(fl, 0, rho0 * dx * dx, rho0, 300.0)
    kb = b.add_body()
    b.add(sites[in_disc], 2, disc_density * dx * dx, disc_density, 300.0, body=kb)
    w = wall_shell(2, [n, n], dx, layers=3)
    b.add(w, 1, rho0 * dx * dx, rho0, 300.0)
    lo = -3 * dx
    hi = n * dx + 3 * dx
    p = default_params(2, dx, [lo, lo], [hi, hi], gravity=[0.0, g, 0.0], dt_mode=1,
                       precision=precision)
    return b.finish(p, mats)


def tank3d_spheres(dx=0.01, n_spheres=64, seed=7925, r_range=(0.04, 0.08),
                   dens_range=(1.5, 3.0), c=45.0, rho0=1.0, nu=1e-3, g=-9.81,
                   size=(1.0, 1.0, 2.0), fill=1.0, gap=2.0, jitter=1e-3,
                   precision=64, dt_mode=1, allow_fewer=False, max_tries=200000):
    """3D tank (1 x 1 x 2), fluid to z = 1, ``n_spheres`` rigid spheres, walls open-top.

    At dx = 0.01: 1,000,000 fluid lattice sites minus the spheres, 280,908 wall
    particles (floor and four sides up to z = 2, three layers).  Sphere radii are
    uniform in ``r_range``, density ratios uniform in ``dens_range``,
    centres seeded and non-overlapping with a surface gap of ``gap``*dx.
    With ``allow_fewer`` the
    placement stops after ``max_tries`` attempts with the spheres placed so far.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz_tank = (int(round(s / dx)) for s in size)
    nzf = int(round(fill / dx))
    r_lo, r_hi = r_range
    centers, radii = [], []
    tries = 0
    while len(centers) < n_spheres:
        tries += 1
        if tries > max_tries:
            if allow_fewer:
                break
            raise RuntimeError("could not place spheres")
        r = rng.uniform(r_lo, r_hi)
        m = r + gap * dx
        cpos = np.array([rng.uniform(m, nx * dx - m), rng.uniform(m, ny * dx - m),
                         rng.uniform(m, nzf * dx - m)])
        ok = all(np.linalg.norm(cpos - c2) >= r + r2 + gap * dx for c2, r2 in zip(centers, radii))
        if ok:
            centers.append(cpos)
            radii.append(r)
    n_spheres = len(centers)
    dens = rng.uniform(dens_range[0], dens_range[1], size=n_spheres) * rho0
    sites = lattice([0.0, 0.0, 0.0], [nx, ny, nzf], dx)
    owner = np.full(len(sites), -1, dtype=np.int64)
    for k, (cc, r) in enumerate(zip(centers, radii)):
        # only test sites in the sphere's bounding box
        lo = np.maximum(((cc - r) / dx - 1).astype(int), 0)
        hi = np.minimum(((cc + r) / dx + 1).astype(int), [nx - 1, ny - 1, nzf - 1])
        ii, jj, kk = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                                 np.arange(lo[2], hi[2] + 1), indexing="ij")
        lin = (ii + nx * (jj + ny * kk)).ravel()
        d2 = np.sum((sites[lin] - cc) ** 2, axis=1)
        owner[lin[d2 <= r * r]] = k
    mats = [material(FLUID, rho0, c=c, eta=rho0 * nu, cp=1.0, kappa=0.0),
            material(WALL, rho0),
            material(RIGID, rho0 * 2.0)]
    b = _Builder(3)
    fl = _jitter(rng, sites[owner < 0], jitter * dx, 3)
    b.add(fl, 0, rho0 * dx ** 3, rho0, 300.0)
    for k in range(n_spheres):
        kb = b.add_body()
        s = sites[owner == k]
        b.add(s, 2, dens[k] * dx ** 3, dens[k], 300.0, body=kb)
    w = wall_shell(3, [nx, ny, nz_tank], dx, layers=3, open_top=True, top_extra=0)
    b.add(w, 1, rho0 * dx ** 3, rho0, 300.0)
    lo = [-3 * dx] * 3
    hi = [nx * dx + 3 * dx, ny * dx + 3 * dx, nz_tank * dx]
    p = default_params(3, dx, lo, hi, gravity=[0.0, 0.0, g], dt_mode=dt_mode, precision=precision)
    return b.finish(p, mats)


def periodic_box(dim=3, n=8, dx=0.1, seed=1, vel_amp=0.1, jitter=0.05, c=10.0, rho0=1.0,
                 eta=0.01, bodies=0, body_radius=None, body_density=2.0, kappa=0.0, cp=1.0,
                 T_amp=0.0, precision=64):
    """Fully periodic box of n^dim lattice sites, seeded jitter and random velocities.

    No walls and no gravity: the harness for linear-momentum conservation
    (Eq. (conservlinmom)).  Optional spherical/disc rigid bodies carved out of the
    lattice on a regular arrangement.
    """
    rng = np.random.default_rng(seed)
    sites = lattice([0.0] * dim, [n] * dim, dx)
    L = n * dx
    owner = np.full(len(sites), -1)
    centers = []
    if bodies:
        rad = body_radius if body_radius is not None else 1.6 * dx
        per = int(math.ceil(bodies ** (1.0 / dim)))
        for k in range(bodies):
            idx = np.unravel_index(k, [per] * dim)
            cc = np.array([(idx[d] + 0.5) * L / per for d in range(dim)])
            centers.append(cc)
            d2 = np.sum((sites - cc) ** 2, axis=1)
            owner[(d2 <= rad * rad) & (owner < 0)] = k
    mats = [material(FLUID, rho0, c=c, eta=eta, cp=cp, kappa=kappa),
            material(RIGID, body_density, cp=cp, kappa=kappa)]
    b = _Builder(dim)
    fl = sites[owner < 0]
    nfl = len(fl)
    fl = _jitter(rng, _pad3(fl), jitter * dx, dim)
    vel = np.zeros((nfl, 3))
    vel[:, :dim] = rng.uniform(-vel_amp, vel_amp, size=(nfl, dim))
    T = 300.0 + T_amp * rng.uniform(-1, 1, size=nfl)
    b.add(fl, 0, rho0 * dx ** dim, rho0, T, vel=vel)
    for k in range(len(centers)):
        v = np.zeros(3)
        v[:dim] = rng.uniform(-vel_amp, vel_amp, size=dim)
        w = np.zeros(3)
        if dim == 3:
            w = rng.uniform(-1, 1, size=3)
        else:
            w[2] = rng.uniform(-1, 1)
        kb = b.add_body(vel=v, omega=w)
        s = sites[owner == k]
        T = 300.0 + T_amp * rng.uniform(-1, 1, size=len(s))
        b.add(s, 1, body_density * dx ** dim, body_density, T, body=kb)
    p = default_params(dim, dx, [0.0] * dim, [L] * dim, periodic=[1] * dim + [0] * (3 - dim),
                       dt_mode=0, dt_fixed=0.1 * dx / c, precision=precision)
    if dim == 2:
        p["periodic"] = [1, 1, 0]
    return b.finish(p, mats)


def cluster(dim=3, n=10, dx=0.1, seed=3, vel_amp=0.05, c=10.0, rho0=1.0, n_bodies=2,
            body_radius=None, body_density=2.0, precision=64):
    """Wall-free, non-periodic fluid block with spherical bodies, inviscid (eta = 0).

    All pair forces are central, so total angular momentum is conserved by the
    pair sums; the harness for the angular-momentum check.  Body centres sit on
    lattice sites so that each body is symmetric under the cube group and its
    inertia tensor is isotropic.
    """
    rng = np.random.default_rng(seed)
    sites = lattice([0.0] * dim, [n] * dim, dx)
    rad = body_radius if body_radius is not None else 1.6 * dx
    owner = np.full(len(sites), -1)
    centers = []
    mid = (n // 2 + 0.5) * dx
    for k in range(n_bodies):
        cc = np.full(dim, mid)
        cc[0] = (int(n * (k + 1) / (n_bodies + 1)) + 0.5) * dx
        centers.append(cc)
        d2 = np.sum((sites - cc) ** 2, axis=1)
        owner[(d2 <= rad * rad) & (owner < 0)] = k
    mats = [material(FLUID, rho0, c=c, eta=0.0), material(RIGID, body_density)]
    b = _Builder(dim)
    fl = sites[owner < 0]
    vel = np.zeros((len(fl), 3))
    vel[:, :dim] = rng.uniform(-vel_amp, vel_amp, size=(len(fl), dim))
    b.add(_pad3(fl), 0, rho0 * dx ** dim, rho0, 300.0, vel=vel)
    for k in range(n_bodies):
        w = np.zeros(3)
        w[2] = rng.uniform(-1, 1)
        if dim == 3:
            w = rng.uniform(-1, 1, size=3)
        v = np.zeros(3)
        v[:dim] = rng.uniform(-vel_amp, vel_amp, size=dim)
        kb = b.add_body(vel=v, omega=w)
        b.add(sites[owner == k], 1, body_density * dx ** dim, body_density, 300.0, body=kb)
    pad = 4 * dx
    L = n * dx
    p = default_params(dim, dx, [-pad] * dim, [L + pad] * dim, dt_mode=0,
                       dt_fixed=0.05 * dx / c, precision=precision)
    return b.finish(p, mats)


def hydrostatic_tank2d(dx=0.02, width=0.4, depth=0.4, c=10.0, rho0=1.0, eta=0.05, g=-1.0,
                       closed=False, precision=64):
    """2D tank at rest under gravity.

    ``closed=False``: fluid of depth ``depth`` below a free surface, tank walls 4 rows
    higher.  ``closed=True``: the fluid fills a closed box of height ``depth`` (no free
    surface), walls on all four sides.
    """
    nx = int(round(width / dx))
    nd = int(round(depth / dx))
    ntank = nd if closed else nd + 4
    b = _Builder(2)
    mats = [material(FLUID, rho0, c=c, eta=eta), material(WALL, rho0)]
    b.add(lattice([0.0, 0.0], [nx, nd], dx), 0, rho0 * dx * dx, rho0, 300.0)
    b.add(wall_shell(2, [nx, ntank], dx, 3), 1, rho0 * dx * dx, rho0, 300.0)
    p = default_params(2, dx, [-3 * dx, -3 * dx], [(nx + 3) * dx, (ntank + 3) * dx],
                       gravity=[0.0, g, 0.0], dt_mode=1, precision=precision)
    return b.finish(p, mats)


def free_fall(dim=3, dx=0.1, radius=0.35, density=3.0, g=-9.81, omega=(0.0, 0.0, 0.0),
              vel=(0.0, 0.0, 0.0), precision=64, dt=1e-3):
    """A single rigid sphere (disc) alone in a large box: no fluid, no walls."""
    n = int(math.ceil(2 * radius / dx)) + 2
    sites = lattice([-(n * dx) / 2] * dim, [n] * dim, dx)
    keep = np.sum(sites ** 2, axis=1) <= radius * radius
    b = _Builder(dim)
    mats = [material(FLUID, 1.0, c=1.0), material(RIGID, density)]
    kb = b.add_body(vel=vel, omega=omega)
    b.add(_pad3(sites[keep]), 1, density * dx ** dim, density, 300.0, body=kb)
    L = 50.0
    gv = [0.0, 0.0, 0.0]
    gv[dim - 1] = g
    p = default_params(dim, dx, [-L] * dim, [L] * dim, gravity=gv, dt_mode=0, dt_fixed=dt,
                       precision=precision)
    return b.finish(p, mats)


def heat_slab(dim=2, n=(40, 4), dx=0.025, T0=300.0, A=10.0, kappa=1.0, cp=1.0, rho0=1.0,
              c=1.0, precision=64, dt=None):
    """Periodic fluid lattice at rest, T = T0 + A sin(2 pi x / Lx): 1D conduction check."""
    sites = lattice([0.0] * dim, list(n), dx)
    Lx = n[0] * dx
    T = T0 + A * np.sin(2 * np.pi * sites[:, 0] / Lx)
    b = _Builder(dim)
    mats = [material(FLUID, rho0, c=c, eta=0.0, cp=cp, kappa=kappa)]
    b.add(_pad3(sites), 0, rho0 * dx ** dim, rho0, T)
    L = [n[d] * dx for d in range(dim)]
    if dt is None:
        dt = 0.05 * rho0 * cp * dx * dx / kappa
    p = default_params(dim, dx, [0.0] * dim, L, periodic=[1] * dim + [0] * (3 - dim),
                       dt_mode=0, dt_fixed=dt, precision=precision)
    return b.finish(p, mats)


def contact_pair(dim=2, dx=0.1, gap=-0.02, speed=0.5, density=2.0, k_contact=1e3,
                 d_contact=1.0, precision=64, dt=1e-4):
    """Two single-particle rigid bodies approaching head-on along x (no fluid)."""
    b = _Builder(dim)
    mats = [material(FLUID, 1.0, c=1.0), material(RIGID, density)]
    x0 = -(dx + gap) / 2
    k0 = b.add_body(vel=(speed, 0, 0))
    b.add(np.array([[x0, 0.0, 0.0]]), 1, density * dx ** dim, density, 300.0, body=k0)
    k1 = b.add_body(vel=(-speed, 0, 0))
    b.add(np.array([[-x0, 0.0, 0.0]]), 1, density * dx ** dim, density, 300.0, body=k1)
    p = default_params(dim, dx, [-2.0] * dim, [2.0] * dim, dt_mode=0, dt_fixed=dt,
                       k_contact=k_contact, d_contact=d_contact, precision=precision)
    return b.finish(p, mats)


def random_cloud(dim=3, n=500, L=1.0, dx=0.1, seed=5, kinds=(0.6, 0.25, 0.15), n_bodies=3,
                 periodic=False, precision=64):
    """Random (non-lattice) particle cloud of mixed kinds, for brute-force neighbour checks."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    pos[:, :dim] = rng.uniform(0, L, size=(n, dim))
    u = rng.uniform(size=n)
    kind = np.where(u < kinds[0], 0, np.where(u < kinds[0] + kinds[1], 1, 2))
    mats = [material(FLUID, 1.0, c=5.0, eta=0.01, kappa=0.5, cp=1.0),
            material(RIGID, 2.0, kappa=1.0, cp=0.5),
            material(WALL, 1.0)]
    b = _Builder(dim)
    vel = np.zeros((n, 3))
    vel[:, :dim] = rng.uniform(-0.1, 0.1, size=(n, dim))
    T = 300.0 + 20.0 * rng.uniform(-1, 1, size=n)
    body = np.full(n, -1, dtype=np.int32)
    rig = np.nonzero(kind == 1)[0]
    for k in range(n_bodies):
        b.add_body(omega=(0, 0, 0.1 * (k + 1)))
    if len(rig):
        body[rig] = np.arange(len(rig)) % n_bodies
    m = dx ** dim
    mat = np.where(kind == 0, 0, np.where(kind == 1, 1, 2)).astype(np.int32)
    dens = np.where(kind == 1, 2.0, 1.0)
    mass = dens * m
    wall_T = np.where(kind == 2, np.where(rng.uniform(size=n) < 0.5, 310.0, NAN), NAN)
    # assemble directly (mixed kinds in one chunk, in random order)
    ch = dict(pos=pos, vel=np.where((kind == 0)[:, None], vel, 0.0), mass=mass, density=dens,
              temperature=T, material=mat, body=np.where(kind == 1, body, -1).astype(np.int32),
              wall_velocity=np.zeros((n, 3)), wall_temperature=wall_T)
    b.parts.append(ch)
    margin = 0.0 if periodic else 0.05
    p = default_params(dim, dx, [-margin] * dim, [L + margin] * dim, dt_mode=0, dt_fixed=1e-4,
                       precision=precision)
    if periodic:
        p["periodic"] = [1] * dim + [0] * (3 - dim)
    return b.finish(p, mats)


def strong_scaling_cube(dx=0.2, L=30.0, D=2.5, per_axis=6, rho_s=10.0, rho_f=1.0, c=50.0, nu=1.0,
                        g=-1.0, precision=64, dt=1e-3):
    """Sec. 4.6 scene: 6^3 = 216 spheres of diameter D on a regular grid in a cube of edge L,
    fluid elsewhere, three wall layers; dt = 1e-3 as in the paper."""
    n = int(round(L / dx))
    sites = lattice([0.0] * 3, [n] * 3, dx)
    R = 0.5 * D
    pitch = L / per_axis
    owner = np.full(len(sites), -1, dtype=np.int64)
    # each site belongs to at most one sphere; index the candidate sphere by position
    idx = np.minimum((sites // pitch).astype(int), per_axis - 1)
    cc = (idx + 0.5) * pitch
    inside = np.sum((sites - cc) ** 2, axis=1) <= R * R
    sid = idx[:, 0] + per_axis * (idx[:, 1] + per_axis * idx[:, 2])
    owner[inside] = sid[inside]
    mats = [material(FLUID, rho_f, c=c, eta=rho_f * nu), material(WALL, rho_f),
            material(RIGID, rho_s)]
    b = _Builder(3)
    b.add(sites[owner < 0], 0, rho_f * dx ** 3, rho_f, 300.0)
    order = np.argsort(owner[owner >= 0], kind="stable")
    rig = sites[owner >= 0][order]
    rid = owner[owner >= 0][order]
    for k in range(per_axis ** 3):
        b.add_body()
    b.add(rig, 2, rho_s * dx ** 3, rho_s, 300.0, body=rid.astype(np.int32))
    b.add(wall_shell(3, [n, n, n], dx, 3), 1, rho_f * dx ** 3, rho_f, 300.0)
    p = default_params(3, dx, [-3 * dx] * 3, [L + 3 * dx] * 3, gravity=[0.0, 0.0, g],
                       dt_mode=0, dt_fixed=dt, precision=precision)
    return b.finish(p, mats)


# --------------------------------------------------------------------------- batched mix

def tank2d_discs(dx=0.0125, n_discs=1, seed=2103, r_range=(0.03, 0.06), dens_range=(1.5, 3.0),
                 jitter=1e-3, fill=0.65, c=10.0, rho0=1.0, eta=0.01, g=-1.0, precision=64):
    """The 2D tank of ``tank2d_disc`` with ``n_discs`` seeded, non-overlapping discs in the
    fluid (radii uniform in ``r_range`` but at least 2 dx, density ratios in ``dens_range``)."""
    rng = np.random.default_rng(seed)
    n = int(round(1.0 / dx))
    nf = int(round(fill / dx))
    sites = lattice([0.0, 0.0], [n, nf], dx)
    owner = np.full(len(sites), -1, dtype=np.int64)
    centers, radii = [], []
    tries = 0
    while len(centers) < n_discs and tries < 100000:
        tries += 1
        r = max(rng.uniform(*r_range), 2.0 * dx)
        m = r + 2 * dx
        if nf * dx - 2 * m <= 0:
            break
        cpos = np.array([rng.uniform(m, n * dx - m), rng.uniform(m, nf * dx - m)])
        if all(np.linalg.norm(cpos - c2) >= r + r2 + 2 * dx for c2, r2 in zip(centers, radii)):
            centers.append(cpos)
            radii.append(r)
    for k, (cc, r) in enumerate(zip(centers, radii)):
        owner[np.sum((sites - cc) ** 2, axis=1) <= r * r] = k
    dens = rng.uniform(dens_range[0], dens_range[1], size=len(centers)) * rho0
    mats = [material(FLUID, rho0, c=c, eta=eta), material(WALL, rho0), material(RIGID, 2.0 * rho0)]
    b = _Builder(2)
    b.add(_jitter(rng, _pad3(sites[owner < 0]), jitter * dx, 2), 0, rho0 * dx * dx, rho0, 300.0)
    for k in range(len(centers)):
        kb = b.add_body()
        b.add(sites[owner == k], 2, dens[k] * dx * dx, dens[k], 300.0, body=kb)
    b.add(wall_shell(2, [n, n], dx, layers=3), 1, rho0 * dx * dx, rho0, 300.0)
    lo, hi = -3 * dx, n * dx + 3 * dx
    p = default_params(2, dx, [lo, lo], [hi, hi], gravity=[0.0, g, 0.0], dt_mode=1, precision=precision)
    return b.finish(p, mats)


def _count_2d(dx, fill=0.65):
    n, nf = int(round(1.0 / dx)), int(round(fill / dx))
    return n * nf + (n + 6) ** 2 - n * n


def _count_3d(dx):
    n, nz = int(round(1.0 / dx)), int(round(2.0 / dx))
    return n ** 3 + (n + 6) ** 2 * (nz + 3) - n * n * nz


def dx_for_count(dim, n_target):
    """Lattice spacing at which the cfg-1 (2D) or cfg-2 (3D) template holds about n_target
    particles (bisection on the exact site count of the template)."""
    f = _count_2d if dim == 2 else _count_3d
    lo, hi = 1e-4, 0.2
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if f(mid) > n_target:
            lo = mid
        else:
            hi = mid
    return hi


def batch_mix(count=256, seed=2103, n_lo=1e4, n_hi=5e5, max_bodies=50, precision=32):
    """Independent scenes of uneven size for the batched form: log N normal around
    sqrt(n_lo n_hi) with sigma ln(n_hi/n_lo)/4, clipped to [n_lo, n_hi]; 2D or 3D by a seeded
    coin; 0..max_bodies bodies; each scene is the 2D disc tank or the 3D sphere tank at the
    spacing that gives its N.  Returns a list of (scene, spec) pairs."""
    rng = np.random.default_rng(seed)
    mu, sig = math.log(math.sqrt(n_lo * n_hi)), math.log(n_hi / n_lo) / 4.0
    out = []
    for q in range(count):
        n_t = float(np.clip(math.exp(rng.normal(mu, sig)), n_lo, n_hi))
        dim = 2 if rng.uniform() < 0.5 else 3
        nb = int(rng.integers(0, max_bodies + 1))
        dx = dx_for_count(dim, n_t)
        s = int(rng.integers(0, 2 ** 31 - 1))
        if dim == 2:
            sc = tank2d_discs(dx=dx, n_discs=nb, seed=s, precision=precision)
        else:
            r_lo, r_hi = max(0.04, 1.5 * dx), max(0.08, 2.0 * dx)
            sc = tank3d_spheres(dx=dx, n_spheres=nb, seed=s, r_range=(r_lo, r_hi), precision=precision,
                                allow_fewer=True, max_tries=20000)
            nb = len(sc["bodies"]["quat"])
        out.append((sc, dict(index=q, dim=dim, bodies=nb, dx=dx, target=n_t,
                             n=int(len(sc["particles"]["mass"])))))
    return out


# --------------------------------------------------------------------------- powder bed

def powder_bed(dx=0.005, size=(1.0, 0.5, 0.5), n_grains=2000, r_median=0.02, r_sigma=0.3,
               r_clip=(0.01, 0.05), bed_frac=0.8, seed=2103, T0=300.0, T_melt=1700.0, mushy=20.0,
               c_metal=1.0, nu=1e-3, Q0=1e10, src_radius=0.05, src_speed=0.5, src_depth=None,
               g=-9.81, max_tries=4, preheat=None, precision=32):
    """Powder bed with melting grains (the shape of Sec. 4.4 in 3D).

    Box ``size`` (periodic in x and y) filled on a dx lattice: a three-layer wall slab
    below z = 0 held at T0 (Dirichlet), an adiabatic three-layer lid above the box, metal
    grains (rigid, density 1000): ``n_grains`` lognormal radii (median ``r_median``, log-sigma
    ``r_sigma``, clipped to ``r_clip``) placed largest first by random sequential addition
    (surface gap dx) in the lower ``bed_frac`` of the box; a grain that finds no room in
    ``max_tries`` batches of 256 candidate centres is left out,
    and gas (fluid, density 1) everywhere else.  Solid metal melts into liquid metal
    (fluid, density 1000) at T_melt with latent heat L = 0.25 c_p (T_melt - T0) over a mushy
    interval of width ``mushy``, and back.  Property ratios of the paper's example: metal
    c_p = 1, kappa = 10; gas c_p = 0.01, kappa = 0.1.  Both fluids share p0 = rho0 c^2
    (c_gas = c_metal sqrt(1000)).  A Gaussian surface source of power density Q0, radius
    ``src_radius`` moves along x at ``src_speed`` over the top of the bed, heating metal
    within ``src_depth`` (default 10 dx) below the bed top.

    ``preheat=(A, wavelength)``: the grains start at T_melt + A sin(2 pi x / wavelength)
    instead of T0 (the gas at T_melt), so that every grain crossing a zero of the sine is
    part above and part below the melting temperature: the hot parts melt at the end of
    the first step, and conduction inside the grains then moves the melting fronts, which
    keeps metal melting and solidifying step after step.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(round(s / dx)) for s in size)
    Lx, Ly, Lz = nx * dx, ny * dx, nz * dx
    zb = bed_frac * Lz
    # radii drawn up front, placed largest first by random sequential addition (surface gap
    # dx, periodic in x and y); each grain gets ``tries`` batches of candidate centres
    radii_all = np.clip(r_median * np.exp(r_sigma * rng.normal(size=n_grains)), *r_clip)
    radii_all = np.sort(np.maximum(radii_all, 1.5 * dx))[::-1]
    C = np.zeros((0, 3))
    Rr = np.zeros(0)
    tries = 0
    for r in radii_all:
        if zb - 2 * r - dx <= 0:
            continue
        for _ in range(max_tries):
            tries += 1
            cand = np.column_stack([rng.uniform(0, Lx, 256), rng.uniform(0, Ly, 256),
                                    rng.uniform(r + dx, zb - r, 256)])
            if len(C):
                d = cand[:, None, :] - C[None, :, :]
                d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
                d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
                ok = np.all(np.einsum("ijk,ijk->ij", d, d) >= (r + Rr[None, :] + dx) ** 2, axis=1)
            else:
                ok = np.ones(256, dtype=bool)
            if ok.any():
                C = np.vstack([C, cand[int(np.argmax(ok))]])
                Rr = np.append(Rr, r)
                break
    centers, radii = list(C), list(Rr)
    sites = lattice([0.0, 0.0, 0.0], [nx, ny, nz], dx)
    owner = np.full(len(sites), -1, dtype=np.int64)
    for k, (c, r) in enumerate(zip(centers, radii)):
        lo = np.floor((c - r) / dx).astype(int) - 1
        hi = np.ceil((c + r) / dx).astype(int) + 1
        ii, jj, kk = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                                 np.arange(max(lo[2], 0), min(hi[2], nz - 1) + 1), indexing="ij")
        ii, jj, kk = ii.ravel() % nx, jj.ravel() % ny, kk.ravel()
        lin = ii + nx * (jj + ny * kk)
        d = sites[lin] - c
        d[:, 0] -= Lx * np.round(d[:, 0] / Lx)
        d[:, 1] -= Ly * np.round(d[:, 1] / Ly)
        inside = np.sum(d * d, axis=1) <= r * r
        owner[lin[inside & (owner[lin] < 0)]] = k
    rho_m, rho_g = 1000.0, 1.0
    c_gas = c_metal * math.sqrt(rho_m / rho_g)
    L = 0.25 * 1.0 * (T_melt - T0)
    mats = [material(FLUID, rho_g, c=c_gas, eta=rho_g * nu, cp=0.01, kappa=0.1),
            material(WALL, rho_g, cp=1.0, kappa=10.0),
            material(RIGID, rho_m, cp=1.0, kappa=10.0, T_transition=T_melt, transitions_to=3,
                     latent_heat=L, mushy_width=mushy),
            material(FLUID, rho_m, c=c_metal, eta=rho_m * nu, cp=1.0, kappa=10.0, T_transition=T_melt,
                     transitions_to=2, latent_heat=L, mushy_width=mushy)]
    b = _Builder(3)
    b.add(sites[owner < 0], 0, rho_g * dx ** 3, rho_g, T0 if preheat is None else T_melt)
    order = np.argsort(owner[owner >= 0], kind="stable")
    rig = sites[owner >= 0][order]
    rid = owner[owner >= 0][order]
    used = np.unique(rid)
    remap = np.full(len(centers), -1, dtype=np.int64)
    remap[used] = np.arange(len(used))
    for _ in range(len(used)):
        b.add_body()
    if len(rig):
        Tg = T0 if preheat is None else T_melt + preheat[0] * np.sin(2 * np.pi * rig[:, 0] / preheat[1])
        b.add(rig, 2, rho_m * dx ** 3, rho_m, Tg, body=remap[rid].astype(np.int32))
    # substrate slab (Dirichlet T0) and adiabatic lid, three layers each
    slab = lattice([0.0, 0.0, -3 * dx], [nx, ny, 3], dx)
    b.add(slab, 1, rho_g * dx ** 3, rho_g, T0, wall_T=T0)
    lid = lattice([0.0, 0.0, Lz], [nx, ny, 3], dx)
    b.add(lid, 1, rho_g * dx ** 3, rho_g, T0, wall_T=NAN)
    ztop = float(max((c[2] + r for c, r in zip(centers, radii)), default=zb))
    p = default_params(3, dx, [0.0, 0.0, -3 * dx], [Lx, Ly, Lz + 3 * dx], periodic=[1, 1, 0],
                       gravity=[0.0, 0.0, g], dt_mode=1, precision=precision,
                       src_power=Q0, src_radius=src_radius, src_speed=[src_speed, 0.0, 0.0],
                       src_origin=[0.2 * Lx, 0.5 * Ly, 0.0], src_depth=10 * dx if src_depth is None else src_depth,
                       src_ztop=ztop, body_capacity=len(used) + 4096)
    sc = b.finish(p, mats)
    sc["info"] = dict(grains=len(used), grains_requested=n_grains, rigid=int(len(rig)), tries=tries)
    return sc


# --------------------------------------------------------------------------- shear flow

def couette2d(dx=0.01, width=0.1, height=0.2, U=1.0, c=10.0, rho0=1.0, nu=0.1, jitter=0.0, seed=7,
              dt=None, precision=64):
    """Plane Couette channel (the moving-wall set-up of the paper's shear-flow examples,
    Sec. 4.2): periodic in x, fluid of height ``height`` at rest, three layers of wall
    particles below (at rest) and above (moving along x with velocity U)."""
    rng = np.random.default_rng(seed)
    nx, ny = int(round(width / dx)), int(round(height / dx))
    b = _Builder(2)
    mats = [material(FLUID, rho0, c=c, eta=rho0 * nu), material(WALL, rho0)]
    fl = lattice([0.0, 0.0], [nx, ny], dx)
    b.add(_jitter(rng, _pad3(fl), jitter * dx, 2), 0, rho0 * dx * dx, rho0, 300.0)
    b.add(lattice([0.0, -3 * dx], [nx, 3], dx), 1, rho0 * dx * dx, rho0, 300.0)
    b.add(lattice([0.0, ny * dx], [nx, 3], dx), 1, rho0 * dx * dx, rho0, 300.0, wall_vel=[U, 0.0, 0.0])
    if dt is None:  # the viscous condition of Eq. (timestepcond) binds
        dt = min(0.25 * dx / c, 0.125 * dx * dx / nu)
    p = default_params(2, dx, [0.0, -3 * dx], [nx * dx, (ny + 3) * dx], periodic=[1, 0, 0],
                       dt_mode=0, dt_fixed=dt, precision=precision)
    return b.finish(p, mats)


# --------------------------------------------------------------------------- concentration

def gastric2d(dx=0.1, width=8.0, height=4.0, n_boluses=6, d_range=(1.0, 1.6), seed=11, c=50.0,
              nu_juice=1.0, nu_chyme=2.0, D_juice=1.0, D_bolus=0.25, D_chyme=0.25, C_t=0.8,
              p_background=0.0, dt=None, precision=64):
    """Food boluses in gastric juice (the shape of Sec. 4.5, without its moving constriction):
    a closed 2D box of juice (fluid, concentration held at 1), rigid boluses (C = 0 at
    start) that turn into chyme (fluid) where their concentration exceeds C_t, all of
    density 1.  Defaults are scaled down from the paper's 40 x 16 box and 60 boluses."""
    rng = np.random.default_rng(seed)
    nx, ny = int(round(width / dx)), int(round(height / dx))
    sites = lattice([0.0, 0.0], [nx, ny], dx)
    owner = np.full(len(sites), -1, dtype=np.int64)
    centers, radii = [], []
    tries = 0
    while len(centers) < n_boluses and tries < 20000:
        tries += 1
        r = 0.5 * rng.uniform(*d_range)
        cpos = np.array([rng.uniform(r + 2 * dx, nx * dx - r - 2 * dx), rng.uniform(r + 2 * dx, ny * dx - r - 2 * dx)])
        if all(np.linalg.norm(cpos - c2) >= r + r2 + 2 * dx for c2, r2 in zip(centers, radii)):
            centers.append(cpos)
            radii.append(r)
    for k, (cc, r) in enumerate(zip(centers, radii)):
        owner[np.sum((sites - cc) ** 2, axis=1) <= r * r] = k
    mats = [material(FLUID, 1.0, c=c, eta=nu_juice, diffusivity=D_juice, C_fixed=1.0),
            material(WALL, 1.0),
            material(RIGID, 1.0, diffusivity=D_bolus, C_transition=C_t, transitions_to=3, transition_by=1),
            material(FLUID, 1.0, c=c, eta=nu_chyme, diffusivity=D_chyme)]
    b = _Builder(2)
    b.add(_pad3(sites[owner < 0]), 0, dx * dx, 1.0, 300.0, conc=1.0)
    for k in range(len(centers)):
        kb = b.add_body()
        b.add(sites[owner == k], 2, dx * dx, 1.0, 300.0, body=kb, conc=0.0)
    b.add(wall_shell(2, [nx, ny], dx, 3), 1, dx * dx, 1.0, 300.0)
    if dt is None:
        dt = min(0.25 * dx / c, 0.125 * dx * dx / max(nu_juice, nu_chyme), 0.1 * dx * dx / max(D_juice, D_bolus))
    p = default_params(2, dx, [-3 * dx, -3 * dx], [(nx + 3) * dx, (ny + 3) * dx], dt_mode=0, dt_fixed=dt,
                       precision=precision, p_background=p_background, body_capacity=len(centers) + 64)
    return b.finish(p, mats)


def conc_slab(dim=2, n=(48, 8), dx=1.0 / 48, C0=0.5, A=0.2, D=1.0, rho0=1.0, c=1.0, precision=64, dt=None):
    """Periodic fluid lattice at rest, C = C0 + A sin(2 pi x / Lx): 1D diffusion check."""
    sites = lattice([0.0] * dim, list(n), dx)
    Lx = n[0] * dx
    C = C0 + A * np.sin(2 * np.pi * sites[:, 0] / Lx)
    b = _Builder(dim)
    b.add(_pad3(sites), 0, rho0 * dx ** dim, rho0, 300.0, conc=C)
    L = [n[d] * dx for d in range(dim)]
    if dt is None:
        dt = 0.05 * rho0 * dx * dx / D
    p = default_params(dim, dx, [0.0] * dim, L, periodic=[1] * dim + [0] * (3 - dim), dt_mode=0, dt_fixed=dt,
                       precision=precision)
    return b.finish(p, [material(FLUID, rho0, c=c, diffusivity=D)])


# --------------------------------------------------------------------------- closed-form harnesses

def dirichlet_slab(dim=2, nx=40, ny=6, dx=0.025, T_left=300.0, T_right=400.0, T0=300.0, kappa=1.0,
                   cp=1.0, rho0=1.0, wall_kappa=0.0, wall_density=None, linear=False, c=1e-3, dt=None,
                   precision=64):
    """Fluid slab at rest between two blocks of Dirichlet wall particles (three layers each,
    Sec. 3.3.4) along x; periodic across (y, and z in 3D).

    The fluid fills [0, nx dx) on the dx lattice and starts at T0; the walls sit at
    [-3 dx, 0) and [nx dx, nx dx + 3 dx) with prescribed temperatures T_left and T_right.
    With ``linear`` every particle (fluid and wall) starts on the straight line through
    (0, T_left) and (nx dx, T_right).  ``wall_kappa`` is the conductivity of the wall
    material (the heat sum must not use it: walls take kappa_b = kappa_a); ``wall_density``
    is the wall particles' given density (default rho0).  A tiny sound speed keeps the
    lattice at rest.
    """
    L = nx * dx
    tr = [ny] * (dim - 1)
    fl = _pad3(lattice([0.0] * dim, [nx] + tr, dx))
    wl = _pad3(lattice([-3 * dx] + [0.0] * (dim - 1), [3] + tr, dx))
    wr = _pad3(lattice([L] + [0.0] * (dim - 1), [3] + tr, dx))
    line = lambda x: T_left + (T_right - T_left) * x / L  # noqa: E731
    rw = rho0 if wall_density is None else wall_density
    b = _Builder(dim)
    mats = [material(FLUID, rho0, c=c, eta=0.0, cp=cp, kappa=kappa), material(WALL, rho0, cp=cp, kappa=wall_kappa)]
    b.add(fl, 0, rho0 * dx ** dim, rho0, line(fl[:, 0]) if linear else T0)
    b.add(wl, 1, rho0 * dx ** dim, rw, 300.0, wall_T=line(wl[:, 0]) if linear else T_left)
    b.add(wr, 1, rho0 * dx ** dim, rw, 300.0, wall_T=line(wr[:, 0]) if linear else T_right)
    if dt is None:
        dt = 0.05 * rho0 * cp * dx * dx / kappa
    W = ny * dx
    p = default_params(dim, dx, [-3 * dx] + [0.0] * (dim - 1), [L + 3 * dx] + [W] * (dim - 1),
                       periodic=[0] + [1] * (dim - 1) + [0] * (3 - dim), dt_mode=0, dt_fixed=dt,
                       precision=precision)
    return b.finish(p, mats)


def rigid_container2d(dx=0.01, inner=0.2, layers=3, rho_f=1.0, rho_c=2.0, c=10.0, eta=0.01, g=-1.0,
                      omega=0.0, dt=None, precision=64):
    """A closed square container of inner edge ``inner`` made of ONE rigid body (``layers``
    rows of rigid particles on the dx lattice), filled with fluid, alone in open space (no
    wall particles).  The fluid starts with the container's rigid-body velocity field:
    rotation at ``omega`` about the container's centre (at the origin).  Gravity g along y."""
    n = int(round(inner / dx))
    lo = -0.5 * n * dx
    fl = _pad3(lattice([lo, lo], [n, n], dx))
    sh = wall_shell(2, [n, n], dx, layers=layers) + lo
    vel = np.zeros_like(fl)
    vel[:, 0] = -omega * fl[:, 1]
    vel[:, 1] = omega * fl[:, 0]
    b = _Builder(2)
    mats = [material(FLUID, rho_f, c=c, eta=eta), material(RIGID, rho_c)]
    b.add(fl, 0, rho_f * dx * dx, rho_f, 300.0, vel=vel)
    kb = b.add_body(omega=(0.0, 0.0, omega))
    b.add(_pad3(sh), 1, rho_c * dx * dx, rho_c, 300.0, body=kb)
    if dt is None:
        dt = 0.25 * dx / c
    p = default_params(2, dx, [-2.0, -2.0], [2.0, 2.0], gravity=[0.0, g, 0.0], dt_mode=0, dt_fixed=dt,
                       precision=precision)
    return b.finish(p, mats)


def ellipsoid_in_fluid(n=10, dx=0.1, semi_axes=(0.36, 0.24, 0.16), omega=(0.7, -0.4, 1.1), vel=(0.05, -0.02, 0.03),
                       vel_amp=0.05, c=10.0, rho0=1.0, eta=0.05, body_density=2.0, g=(0.3, -0.5, -1.0), seed=3,
                       precision=64):
    """Wall-free, non-periodic 3D block of fluid (n^3 lattice sites, seeded random
    velocities) with one rigid ellipsoid at its centre whose principal axes lie along the
    coordinate axes (an anisotropic inertia tensor); the body spins about an axis that is
    not principal.  Gravity and every vector are general, so the scene has no symmetry."""
    rng = np.random.default_rng(seed)
    sites = lattice([0.0] * 3, [n] * 3, dx)
    mid = 0.5 * n * dx
    a = np.asarray(semi_axes, float)
    inside = np.sum(((sites - mid) / a) ** 2, axis=1) <= 1.0
    mats = [material(FLUID, rho0, c=c, eta=eta), material(RIGID, body_density)]
    b = _Builder(3)
    fl = sites[~inside]
    u = rng.uniform(-vel_amp, vel_amp, size=(len(fl), 3))
    b.add(fl, 0, rho0 * dx ** 3, rho0, 300.0, vel=u)
    kb = b.add_body(vel=vel, omega=omega)
    b.add(sites[inside], 1, body_density * dx ** 3, body_density, 300.0, body=kb)
    pad = 6 * dx
    L = n * dx
    p = default_params(3, dx, [-pad] * 3, [L + pad] * 3, gravity=list(g), dt_mode=0, dt_fixed=0.05 * dx / c,
                       precision=precision)
    return b.finish(p, mats)


def heated_grains(dim=2, T0=(250.0, 290.0, 305.0, 309.0), spacing=1.0, dx=0.1, T_t=310.0, mushy=8.0,
                  latent=40.0, cp_s=1.0, cp_l=2.0, rho_s=3.0, rho_l=3.0, Q0=2.0e3, dt=1e-3, precision=64):
    """Single-particle grains of a melting material, ``spacing`` apart (no neighbour within
    r_c), each its own rigid body, heated by the surface source made uniform over them (a
    radius so large that its Gaussian factor rounds to 1, a depth that covers every grain):
    every grain receives the same power density Q0 and nothing else."""
    b = _Builder(dim)
    mats = [material(RIGID, rho_s, cp=cp_s, T_transition=T_t, transitions_to=1, latent_heat=latent,
                     mushy_width=mushy),
            material(FLUID, rho_l, c=1.0, cp=cp_l, T_transition=T_t, transitions_to=0, latent_heat=latent,
                     mushy_width=mushy)]
    for q, T in enumerate(T0):
        kb = b.add_body()
        pos = np.zeros(3)
        pos[0] = q * spacing
        b.add(pos, 0, rho_s * dx ** dim, rho_s, T, body=kb)
    lo = [-spacing] * dim
    hi = [len(T0) * spacing] + [spacing] * (dim - 1)
    p = default_params(dim, dx, lo, hi, dt_mode=0, dt_fixed=dt, precision=precision,
                       src_power=Q0, src_radius=1e9, src_speed=[0.0, 0.0, 0.0], src_origin=[0.0, 0.0, 0.0],
                       src_depth=1e12, src_ztop=1e6, body_capacity=len(T0) + 4)
    return b.finish(p, mats)
