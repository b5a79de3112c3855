"""Seeded synthetic particle bodies shaped like the paper's test cases.

This module is shared by the FP64 CPU oracle (``oracle/``) and by the CUDA
library's tests and benchmark.  It holds none of the method's arithmetic: no
kernel function, no neighbour search, no stress, no time stepping.  It only
places particles on a jittered lattice, picks boundary-condition particle sets
(clamp/grip layers, held-concentration layers, tip column) and draws the
per-run material parameters.

Recipe (all bodies):
  * lattice centres at (i + 1/2) dx per axis, then a uniform jitter of
    +-1 % dx per coordinate, drawn from NumPy PCG64 seeded with
    ``SEED_BASE + case_number`` (case numbers 1..5 follow the five workloads;
    test bodies pass their own seed);
  * particle volume dx^d and mass rho0 dx^d regardless of the jitter;
  * boundary layers are selected from the lattice indices, not from the
    jittered positions, so they are exact layer counts.

The workloads follow the paper's cases (stretching of a bar with a
displacement-controlled grip, Sec. 5.1-5.2; diffusion-driven swelling flexure
of a thin strip or membrane, Sec. 5.3-5.4) at the sizes of the benchmark
configurations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

SEED_BASE = 2309040100
JITTER = 0.01
H_OVER_DX = 1.3


@dataclasses.dataclass
class DispBC:
    """Prescribed displacement on a particle set.

    u = ramp * u_unit on the axes in ``axis_mask`` (bit k = axis k); the other
    axes stay free.  ``report_force`` marks the set whose internal force is
    reported as the end force.
    """
    ids: np.ndarray            # int64, original particle order
    axis_mask: int
    u_unit: np.ndarray         # (len(ids), dim) float64
    report_force: bool = False


@dataclasses.dataclass
class ConcBC:
    """Particles whose concentration is held at a fixed value."""
    ids: np.ndarray
    value: float


@dataclasses.dataclass
class Material:
    model: str                 # "svk" or "j2"
    rho0: float
    E: float
    nu: float
    sigma0: float = 0.0
    sigma_inf: float = 0.0
    delta: float = 0.0
    H: float = 0.0


@dataclasses.dataclass
class StepPlan:
    """How the slow (outer) steps of a run are driven.

    ``n_slow`` slow steps; load steps set ramp = l / n_ramp for l = 1..n_slow;
    diffusion runs use ``dt_slow`` (None = the stable limit the solver
    reports).  ``ke_mode`` 0 compares total kinetic energy with
    ke_tol * ke_ref, mode 1 compares kinetic energy per unit volume with
    ke_tol * ke_ref.
    """
    n_slow: int
    n_ramp: int = 0
    dt_slow: Optional[float] = 0.0
    ke_tol: float = 1e-8
    ke_ref: float = 1.0
    ke_mode: int = 0
    max_substeps: int = 2000
    t_end: float = 0.0


@dataclasses.dataclass
class Case:
    name: str
    dim: int
    X: np.ndarray              # (n, dim) float64, original order
    dx: float
    material: Material
    eta: float
    disp_bcs: List[DispBC]
    conc_bcs: List[ConcBC]
    tip_ids: np.ndarray
    plan: StepPlan
    diffusion: Optional[Tuple[float, float, float]] = None   # (D, beta, c0)
    lattice_index: Optional[np.ndarray] = None               # (n, dim) int64
    counts: Optional[Tuple[int, ...]] = None
    h_over_dx: float = H_OVER_DX
    # time-limited contact: (time after which the set is released, its ids)
    release: Optional[Tuple[float, np.ndarray]] = None
    # lattice spacing per axis (anisotropic kernel); None = dx on every axis
    dx_axis: Optional[Tuple[float, ...]] = None

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def lattice_box(counts, dx) -> Tuple[np.ndarray, np.ndarray]:
    """Cell-centred lattice (dx: one spacing, or one per axis); returns
    (positions, integer lattice indices)."""
    axes = [np.arange(c, dtype=np.int64) for c in counts]
    grids = np.meshgrid(*axes, indexing="ij")
    idx = np.stack([g.reshape(-1) for g in grids], axis=1)
    X = (idx.astype(np.float64) + 0.5) * np.asarray(dx, dtype=np.float64)
    return X, idx


def add_jitter(X: np.ndarray, dx, rng: np.random.Generator,
               frac: float = JITTER) -> np.ndarray:
    a = frac * np.asarray(dx, dtype=np.float64)
    return X + rng.uniform(-a, a, size=X.shape)


def box_body(counts, dx: float, seed: int, jitter: float = JITTER):
    X, idx = lattice_box(counts, dx)
    rng = rng_for(seed)
    if jitter > 0:
        X = add_jitter(X, dx, rng, jitter)
    return X, idx, rng


def layer_ids(idx: np.ndarray, axis: int, first: int, count: int) -> np.ndarray:
    sel = (idx[:, axis] >= first) & (idx[:, axis] < first + count)
    return np.nonzero(sel)[0].astype(np.int64)


# --------------------------------------------------------------------------
# Workload 1: 2D plane-strain elastic bar, displacement ramp to 1 % strain.
# --------------------------------------------------------------------------
def bar2d(nx: int = 100, ny: int = 20, dx: float = 1e-4, seed: int = SEED_BASE + 1,
          n_slow: int = 20, strain: float = 0.01, max_substeps: int = 2000,
          ke_tol: float = 1e-8, E: float = 210e9, nu: float = 0.3,
          rho0: float = 7850.0, eta: float = 1e4, jitter: float = JITTER) -> Case:
    X, idx, _ = box_body((nx, ny), dx, seed, jitter)
    clamp = layer_ids(idx, 0, 0, 3)
    grip = layer_ids(idx, 0, nx - 3, 3)
    L = nx * dx
    u_total = strain * L
    u_grip = np.zeros((grip.size, 2))
    u_grip[:, 0] = u_total
    bcs = [DispBC(clamp, 0b11, np.zeros((clamp.size, 2))),
           DispBC(grip, 0b11, u_grip, report_force=True)]
    # Reference energy for the kinetic-energy criterion: half the plane-strain
    # end force at full stretch times the total stretch.
    W = ny * dx
    F_ref = E / (1.0 - nu * nu) * strain * W
    ke_ref = 0.5 * F_ref * u_total
    plan = StepPlan(n_slow=n_slow, n_ramp=n_slow, dt_slow=0.0, ke_tol=ke_tol,
                    ke_ref=ke_ref, ke_mode=0, max_substeps=max_substeps)
    return Case("bar2d", 2, X, dx, Material("svk", rho0, E, nu), eta, bcs, [],
                layer_ids(idx, 0, nx - 1, 1), plan, None, idx, (nx, ny))


# --------------------------------------------------------------------------
# Workload 2: 3D cylinder, J2 plasticity with saturation hardening.
# --------------------------------------------------------------------------
J2_K = 164.21e9
J2_MU = 80.1938e9
J2_DELTA = 16.93
J2_H = 129.24e6


def moduli_from_K_mu(K: float, mu: float) -> Tuple[float, float]:
    """Young's modulus and Poisson ratio from bulk and shear moduli
    (E = 2 mu (1 + nu) = 3 K (1 - 2 nu)).  Used only to express the paper's
    material table in (E, nu) form."""
    E = 9.0 * K * mu / (3.0 * K + mu)
    nu = (3.0 * K - 2.0 * mu) / (2.0 * (3.0 * K + mu))
    return E, nu


def cylinder3d(L: float = 50e-3, R: float = 5e-3, dx: float = 0.25e-3,
               seed: int = SEED_BASE + 2, n_slow: int = 500, strain: float = 0.30,
               ke_tol: float = 5e-3, max_substeps: int = 1_000_000,
               eta: float = 1e4, jitter: float = JITTER,
               sigma0: Optional[float] = None, sigma_inf: Optional[float] = None) -> Case:
    nx = int(round(L / dx))
    nr = int(round(2 * R / dx))
    Xl, idx = lattice_box((nx, nr, nr), dx)
    yz = Xl[:, 1:] - R
    keep = (yz[:, 0] ** 2 + yz[:, 1] ** 2) <= R * R
    Xl = Xl[keep]
    idx = idx[keep]
    Xl[:, 1:] -= R
    rng = rng_for(seed)
    X = add_jitter(Xl, dx, rng, jitter) if jitter > 0 else Xl
    if sigma0 is None:
        sigma0 = float(rng.uniform(300e6, 400e6))
    if sigma_inf is None:
        sigma_inf = float(rng.uniform(500e6, 700e6))
    E, nu = moduli_from_K_mu(J2_K, J2_MU)
    mat = Material("j2", 7850.0, E, nu, sigma0, sigma_inf, J2_DELTA, J2_H)
    left = layer_ids(idx, 0, 0, 3)
    right = layer_ids(idx, 0, nx - 3, 3)
    half = 0.5 * strain * nx * dx
    ul = np.zeros((left.size, 3)); ul[:, 0] = -half
    ur = np.zeros((right.size, 3)); ur[:, 0] = half
    bcs = [DispBC(left, 0b111, ul), DispBC(right, 0b111, ur, report_force=True)]
    A = math.pi * R * R
    ke_ref = 0.5 * sigma_inf * A * (2 * half)
    plan = StepPlan(n_slow=n_slow, n_ramp=n_slow, dt_slow=0.0, ke_tol=ke_tol,
                    ke_ref=ke_ref, ke_mode=0, max_substeps=max_substeps)
    return Case("cylinder3d", 3, X, dx, mat, eta, bcs, [],
                layer_ids(idx, 0, nx - 1, 1), plan, None, idx, (nx, nr, nr))


# --------------------------------------------------------------------------
# Workloads 3/4: diffusion-swelling flexure of a strip (2D) or plate (3D).
# --------------------------------------------------------------------------
def _swelling_case(name, counts, dx, seed, E, nu, rho0, eta, D, beta, c0,
                   ke_tol, t_end, jitter) -> Case:
    dim = len(counts)
    X, idx, _ = box_body(counts, dx, seed, jitter)
    clamp = layer_ids(idx, 0, 0, 3)
    bcs = [DispBC(clamp, (1 << dim) - 1, np.zeros((clamp.size, dim)))]
    thick_axis = dim - 1
    nt = counts[thick_axis]
    top = layer_ids(idx, thick_axis, nt - 2, 2)
    bottom = layer_ids(idx, thick_axis, 0, 2)
    cbcs = [ConcBC(top, 1.0), ConcBC(bottom, 0.0)]
    K = E / (3.0 * (1.0 - 2.0 * nu))
    p_ref = 3.0 * K * beta
    plan = StepPlan(n_slow=0, n_ramp=0, dt_slow=None, ke_tol=ke_tol, ke_ref=p_ref,
                    ke_mode=1, max_substeps=1_000_000, t_end=t_end)
    return Case(name, dim, X, dx, Material("svk", rho0, E, nu), eta, bcs, cbcs,
                layer_ids(idx, 0, counts[0] - 1, 1), plan, (D, beta, c0), idx,
                tuple(counts))


# Kinetic-energy criteria of the swelling workloads.  The paper fixes its
# criterion values per case by lowering them until the result stops changing
# (Sec. 5.1 and 5.3 criterion studies); its values (0.05 % / 0.1 % of p^l)
# belong to its own beam and membrane.  The same study on the 40,000-particle
# strip (tip elongation after 30 slow steps, criterion lowered by decades from
# 5e-4) settles at 5e-8 of 3 K beta: 5e-4 -> 1.54 mm, 5e-6 -> 1.03 mm,
# 5e-8 -> 0.912 mm, 5e-10 -> 0.925 mm, 5e-12 -> 0.919 mm.  On the 2.5 M-particle
# plate the study does not settle within 3e4 substeps per slow step; its
# criterion is 1e-5, two decades below the paper's 3D value (tip elongation
# after 4 slow steps: 1e-3 -> 0.105 mm, 1e-5 -> 0.338 mm, 1e-7 -> 0.591 mm).
STRIP_KE_TOL = 5e-8
PLATE_KE_TOL = 1e-5


def strip2d(nx: int = 2000, ny: int = 20, dx: float = 1e-5, seed: int = SEED_BASE + 3,
            E: float = 200e6, nu: float = 0.4, rho0: float = 2000.0, eta: float = 1e3,
            D: float = 1e-10, beta: float = 0.1, c0: float = 0.0,
            ke_tol: float = STRIP_KE_TOL, jitter: float = JITTER) -> Case:
    H = ny * dx
    return _swelling_case("strip2d", (nx, ny), dx, seed, E, nu, rho0, eta, D, beta,
                          c0, ke_tol, 2.0 * H * H / D, jitter)


def plate3d(nx: int = 1000, ny: int = 250, nz: int = 10, dx: float = 2e-5,
            seed: int = SEED_BASE + 4, E: float = 200e6, nu: float = 0.4,
            rho0: float = 2000.0, eta: float = 1e4, D: float = 1e-10, beta: float = 0.1,
            c0: float = 0.0, ke_tol: float = PLATE_KE_TOL, jitter: float = JITTER) -> Case:
    H = nz * dx
    return _swelling_case("plate3d", (nx, ny, nz), dx, seed, E, nu, rho0, eta, D,
                          beta, c0, ke_tol, 2.0 * H * H / D, jitter)


# --------------------------------------------------------------------------
# Workload 5: many uneven 2D instances with seeded parameters.
# --------------------------------------------------------------------------
def batch_instances(count: int = 64, n_min: int = 5_000, n_max: int = 200_000,
                    seed: int = SEED_BASE + 5) -> List[Case]:
    """Half thin strips (aspect 100:1, >= 8 layers thick, swelling-driven),
    half stubby bars (aspect 5:1, J2 plasticity, stretched).  Sizes are
    log-uniform in [n_min, n_max]."""
    rng = rng_for(seed)
    cases: List[Case] = []
    for i in range(count):
        n_target = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            ny = max(8, int(round(math.sqrt(n_target / 100.0))))
            nx = max(3 * ny, int(round(n_target / ny)))
            E = float(rng.uniform(100e6, 400e6))
            D = float(np.exp(rng.uniform(np.log(1e-11), np.log(1e-9))))
            beta = float(rng.uniform(0.05, 0.2))
            c = strip2d(nx=nx, ny=ny, dx=1e-5, seed=sub_seed, E=E, D=D, beta=beta)
            c.name = f"strip{i}"
        else:
            ny = max(8, int(round(math.sqrt(n_target / 5.0))))
            nx = max(3 * ny, int(round(n_target / ny)))
            c = bar2d(nx=nx, ny=ny, dx=1e-4, seed=sub_seed, n_slow=500, strain=0.30,
                      ke_tol=5e-3, max_substeps=1_000_000)
            E, nu = moduli_from_K_mu(J2_K, J2_MU)
            s0 = float(rng.uniform(300e6, 400e6))
            sinf = float(rng.uniform(500e6, 700e6))
            c.material = Material("j2", 7850.0, E, nu, s0, sinf, J2_DELTA, J2_H)
            W = ny * 1e-4
            c.plan.ke_ref = 0.5 * sinf * W * (0.30 * nx * 1e-4)
            c.name = f"bar{i}"
        cases.append(c)
    return cases



# --------------------------------------------------------------------------
# Droplet-contact schedules (Sec. 5.3 2D beam, Sec. 5.4 3D membrane): a porous
# body clamped at its ends / sides; the centre part of its upper half is held
# at the saturation of the droplet contact (0.4 = the porosity) for a limited
# time, then released; elsewhere c starts at 0; no flux leaves the body.
# --------------------------------------------------------------------------
def _droplet_case(name, counts, dx, seed, E, nu, rho0, eta, D, beta, c_held, t_contact,
                  t_end, ke_tol, jitter, clamp_axes, dx_axis=None) -> Case:
    dim = len(counts)
    X, idx, _ = box_body(counts, dx if dx_axis is None else dx_axis, seed, jitter)
    clamp = np.unique(np.concatenate(
        [layer_ids(idx, a, 0, 3) for a in clamp_axes] +
        [layer_ids(idx, a, counts[a] - 3, 3) for a in clamp_axes]))
    bcs = [DispBC(clamp, (1 << dim) - 1, np.zeros((clamp.size, dim)))]
    thick = dim - 1
    sel = idx[:, thick] >= counts[thick] // 2                  # upper half
    for a in range(dim - 1):                                   # centre 0.3 of each long side
        lo = int(round(0.35 * counts[a]))
        hi = int(round(0.65 * counts[a]))
        sel &= (idx[:, a] >= lo) & (idx[:, a] < hi)
    contact = np.nonzero(sel)[0].astype(np.int64)
    K = E / (3.0 * (1.0 - 2.0 * nu))
    plan = StepPlan(n_slow=0, n_ramp=0, dt_slow=None, ke_tol=ke_tol, ke_ref=3.0 * K * beta,
                    ke_mode=1, max_substeps=1_000_000, t_end=t_end)
    mid = [counts[a] // 2 for a in range(dim - 1)]
    centre = np.nonzero(np.all(idx[:, :dim - 1] == mid, axis=1))[0].astype(np.int64)
    return Case(name, dim, X, dx, Material("svk", rho0, E, nu), eta, bcs,
                [ConcBC(contact, c_held)], centre, plan, (D, beta, 0.0), idx, tuple(counts),
                release=(t_contact, contact), dx_axis=dx_axis)


def beam_droplet2d(L: float = 10e-3, W: float = 0.125e-3, ny: int = 8,
                   seed: int = SEED_BASE + 6, E: float = 200e6, nu: float = 0.4,
                   rho0: float = 2000.0, eta: float = 1e4, D: float = 1e-10, beta: float = 0.1,
                   c_held: float = 0.4, t_contact: float = 10.0, t_end: float = 100.0,
                   ke_tol: float = 5e-4, jitter: float = JITTER, aniso: float = 1.0) -> Case:
    """Sec. 5.3: a 10 x 0.125 mm beam, both ends clamped, contact on the centre
    0.3 L of the upper half for 10 s of 100 s.  Spacing W/ny across the beam,
    aniso times that along it (the paper uses 4 with its anisotropic kernel)."""
    dy = W / ny
    dxa = aniso * dy
    nx = int(round(L / dxa))
    return _droplet_case("beam_droplet2d", (nx, ny), dy, seed, E, nu, rho0, eta, D, beta,
                         c_held, t_contact, t_end, ke_tol, jitter, clamp_axes=(0,),
                         dx_axis=None if aniso == 1.0 else (dxa, dy))


def membrane_droplet3d(Lx: float = 10e-3, Ly: float = 10e-3, Lz: float = 0.125e-3, nz: int = 8,
                       seed: int = SEED_BASE + 7, E: float = 200e6, nu: float = 0.4,
                       rho0: float = 2000.0, eta: float = 1e4, D: float = 1e-10,
                       beta: float = 0.1, c_held: float = 0.4, t_contact: float = 450.0,
                       t_end: float = 2500.0, ke_tol: float = 1e-3,
                       jitter: float = JITTER, aniso: float = 1.0) -> Case:
    """Sec. 5.4: a 10 x 10 x 0.125 mm membrane, four sides clamped, contact on
    the centre 0.3 Lx x 0.3 Ly of the upper half for 450 s of 2500 s.  Spacing
    Lz/nz through the thickness, aniso times that in plane (the paper uses 8)."""
    dz = Lz / nz
    dxy = aniso * dz
    nx, ny = int(round(Lx / dxy)), int(round(Ly / dxy))
    return _droplet_case("membrane_droplet3d", (nx, ny, nz), dz, seed, E, nu, rho0, eta, D,
                         beta, c_held, t_contact, t_end, ke_tol, jitter, clamp_axes=(0, 1),
                         dx_axis=None if aniso == 1.0 else (dxy, dxy, dz))

def workload(number: int, **kw) -> Case:
    """The five benchmark workloads by number (1..4; 5 is batch_instances)."""
    if number == 1:
        return bar2d(**kw)
    if number == 2:
        return cylinder3d(**kw)
    if number == 3:
        return strip2d(**kw)
    if number == 4:
        return plate3d(**kw)
    raise ValueError("workload 5 is a batch: use batch_instances()")


def random_field(n: int, dim: int, scale: float, seed: int) -> np.ndarray:
    """Seeded random vector field (tests inject it as displacement/velocity)."""
    return rng_for(seed).uniform(-scale, scale, size=(n, dim))
