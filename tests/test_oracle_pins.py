"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
invariants, brute force written independently in NumPy, or numbers printed in
the paper's tables (tests/golden/paper_tables.json).  A plausible mistake in
the oracle (a dropped term, a wrong sign or index, a transposed operand) is
meant to fail at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from synth import bodies as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


# --------------------------------------------------------------------------
# P1: kernel normalisation and derivative (Sec. 3.1 kernel function)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_unit_integral(dim):
    h = 1.3e-4
    if dim == 2:
        val, _ = integrate.quad(lambda r: O.kernel_w(2, h, r) * 2 * math.pi * r, 0, 2 * h,
                                epsabs=1e-14, epsrel=1e-13)
    else:
        val, _ = integrate.quad(lambda r: O.kernel_w(3, h, r) * 4 * math.pi * r * r, 0, 2 * h,
                                epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_matches_central_difference(dim):
    h = 0.7
    for r in np.linspace(0.05, 1.95, 23) * h:
        e = 1e-6 * h
        fd = (O.kernel_w(dim, h, r + e) - O.kernel_w(dim, h, r - e)) / (2 * e)
        assert abs(O.kernel_dwdr(dim, h, r) - fd) < 1e-7 * (abs(fd) + 1e-3)
    assert O.kernel_w(dim, h, 2 * h) == 0.0 and O.kernel_dwdr(dim, h, 2.0001 * h) == 0.0
    assert O.kernel_dwdr(dim, h, 0.5 * h) < 0.0


# --------------------------------------------------------------------------
# P12: neighbour lists and Morton order against independent NumPy brute force
# --------------------------------------------------------------------------
def _numpy_morton_perm(X, dx):
    n, dim = X.shape
    cell = np.floor((X - X.min(axis=0)) / dx).astype(np.int64)
    bits = 32 if dim == 2 else 21
    key = np.zeros(n, dtype=np.uint64)
    for bit in range(bits):
        for k in range(dim):
            key |= (((cell[:, k] >> bit) & 1).astype(np.uint64) << np.uint64(bit * dim + k))
    return np.lexsort((np.arange(n), key))


def _numpy_neighbours(Xs, cut2):
    n, dim = Xs.shape
    rows = []
    for i in range(n):
        d2 = np.zeros(n)
        for k in range(dim):
            d = Xs[:, k] - Xs[i, k]
            d2 = d2 + d * d
        sel = np.nonzero(d2 < cut2)[0]
        rows.append(sel[sel != i])
    return rows


@pytest.mark.parametrize("dim,counts", [(2, (13, 9)), (3, (7, 6, 5))])
@pytest.mark.parametrize("jitter", [0.0, 0.01, 0.3])
def test_neighbours_match_numpy_brute_force(dim, counts, jitter):
    dx = 1e-3
    X, _, _ = B.box_body(counts, dx, seed=11 + dim, jitter=jitter)
    perm = _numpy_morton_perm(X, dx)
    for brute in (True, False):
        ob = O.OracleBody(X, dx, 1.3, brute=brute)
        assert np.array_equal(ob.perm(), perm)
        off, idx = ob.neighbors()
        h = 1.3 * dx
        w = 2.0 * h
        rows = _numpy_neighbours(X[perm], w * w)
        assert off[-1] == sum(len(r) for r in rows)
        for i, r in enumerate(rows):
            assert np.array_equal(idx[off[i]:off[i + 1]], r)


def test_neighbour_count_on_lattice():
    # interior lattice particles: offsets |o| < 2.6 -> 20 (2D), 80 (3D)
    for dim, counts in [(2, (12, 12)), (3, (9, 9, 9))]:
        X, idx, _ = B.box_body(counts, 1.0, seed=3, jitter=0.01)
        ob = O.OracleBody(X, 1.0, 1.3)
        off, _ = ob.neighbors()
        deg = np.diff(off)
        perm = ob.perm()
        interior = np.all((idx[perm] >= 2) & (idx[perm] < np.array(counts) - 2), axis=1)
        assert np.all(deg[interior] == (20 if dim == 2 else 80))


# --------------------------------------------------------------------------
# P12: colouring -- stages touch disjoint particles, every pair once
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,counts", [(2, (30, 17)), (3, (11, 9, 8))])
def test_colour_stages_are_matchings(dim, counts):
    X, _, _ = B.box_body(counts, 1.0, seed=5, jitter=0.01)
    ob = O.OracleBody(X, 1.0, 1.3)
    off, idx = ob.neighbors()
    pa, pb, col, key, sub = ob.colouring()
    # every neighbour pair exactly once, a < b
    pairs = set()
    for a in range(ob.n):
        for b in idx[off[a]:off[a + 1]]:
            if b > a:
                pairs.add((a, int(b)))
    assert len(pairs) == len(pa) and set(zip(pa.tolist(), pb.tolist())) == pairs
    assert np.all(pa < pb)
    # canonical order is sorted by (colour, block key, sub-colour)
    order = np.lexsort((pb, pa, sub, key, col))
    assert np.array_equal(order, np.arange(len(pa)))
    # within one (colour, sub-colour) stage no particle appears twice
    for c in np.unique(col):
        for s in np.unique(sub[col == c]):
            sel = (col == c) & (sub == s)
            parts = np.concatenate([pa[sel], pb[sel]])
            assert np.unique(parts).size == parts.size
    # one owner block's level holds at most 32 pairs (one warp-wide pass)
    _, counts = np.unique(np.stack([col, key, sub]), axis=1, return_counts=True)
    assert counts.max() <= 32
    # visiting the pairs by offset class keeps the level count near the degree
    nlev = {}
    for c, k, s_ in zip(col, key, sub):
        nlev[(c, k)] = max(nlev.get((c, k), 0), s_ + 1)
    deg = np.diff(off).max()
    assert max(nlev.values()) <= deg + 12
    assert len(np.unique(col)) <= 2 ** dim


# --------------------------------------------------------------------------
# P2: corrected gradient reproduces affine fields exactly (Sec. 3.1, B0)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,counts", [(2, (14, 9)), (3, (8, 7, 6))])
def test_affine_field_gives_exact_F_everywhere(dim, counts):
    dx = 2e-4
    X, _, _ = B.box_body(counts, dx, seed=21, jitter=0.01)
    ob = O.OracleBody(X, dx)
    G = np.random.default_rng(4).uniform(-0.05, 0.05, size=(dim, dim))
    ob.write(O.F_U, X @ G.T)
    F = ob.read(O.F_DEFGRAD).reshape(-1, 3, 3)
    want = np.eye(3)
    want[:dim, :dim] += G
    assert np.max(np.abs(F - want)) < 1e-13
    B0 = ob.b0()
    assert np.max(np.abs(B0 - np.transpose(B0, (0, 2, 1)))) < 1e-9 * np.max(np.abs(B0))


def test_rigid_rotation_is_stress_free_and_force_free():
    dx = 1e-4
    X, _, _ = B.box_body((9, 8, 7), dx, seed=8, jitter=0.01)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
    th = 0.4
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    ob.write(O.F_U, X @ (R - np.eye(3)).T)
    ob.substep_partial(1e-9, 2)
    PB = ob.read(O.F_PB)
    acc = ob.read(O.F_ACC)
    assert np.max(np.abs(PB)) < 1e-12 * 210e9
    assert np.max(np.abs(acc)) < 1e-12 * 210e9 / (7850 * dx)


# --------------------------------------------------------------------------
# P3/P4: force divergence and momentum conservation (Sec. 3.1 momentum eq.)
# --------------------------------------------------------------------------
def test_uniform_stress_gives_zero_force_on_lattice_interior():
    dx = 1e-4
    counts = (16, 15, 14)
    X, idx, _ = B.box_body(counts, dx, seed=1, jitter=0.0)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
    G = np.array([[1e-3, 2e-4, 0], [0, -4e-4, 1e-4], [3e-4, 0, 5e-4]])
    ob.write(O.F_U, X @ G.T)
    ob.substep_partial(1e-9, 2)
    acc = ob.read(O.F_ACC)
    scale = 210e9 * 1e-3 / (7850 * dx)
    deep = np.all((idx >= 4) & (idx < np.array(counts) - 4), axis=1)
    assert np.max(np.abs(acc[deep])) < 1e-9 * scale
    # near the surface the force is not zero (the surface is not traction free)
    assert np.max(np.abs(acc[~deep])) > 1e-3 * scale


@pytest.mark.parametrize("dim,counts", [(2, (17, 11)), (3, (9, 8, 7))])
def test_free_body_momentum_conserved(dim, counts):
    dx = 1e-4
    X, _, _ = B.box_body(counts, dx, seed=2, jitter=0.01)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
    ob.write(O.F_U, B.random_field(X.shape[0], dim, 1e-6, 9))
    ob.substep_partial(1e-9, 2)
    acc = ob.read(O.F_ACC)
    m = 7850.0 * dx ** dim
    total = (m * acc).sum(axis=0)
    assert np.all(np.abs(total) < 1e-13 * np.abs(m * acc).sum())


# --------------------------------------------------------------------------
# P5: pairwise implicit damping (Sec. 4.3)
# --------------------------------------------------------------------------
def _damping_body(dim, counts, eta, seed=3):
    dx = 1e-4
    X, _, _ = B.box_body(counts, dx, seed=seed, jitter=0.01)
    bodies = []
    for _ in range(2):
        ob = O.OracleBody(X, dx)
        ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
        ob.set_damping(eta)
        ob.write(O.F_V, B.random_field(X.shape[0], dim, 1.0, 17))
        bodies.append(ob)
    return X, dx, bodies


@pytest.mark.parametrize("dim,counts", [(2, (15, 12)), (3, (8, 7, 6))])
def test_damping_conserves_momentum_and_dissipates(dim, counts):
    X, dx, (b2, b3) = _damping_body(dim, counts, eta=1e4)
    dt = 2e-8
    b2.substep_partial(dt, 2)     # u = 0 -> F = I -> P = 0: no kick
    b3.substep_partial(dt, 3)     # plus the damping sweep
    v0, v1 = b2.read(O.F_V), b3.read(O.F_V)
    assert np.max(np.abs(v0 - B.random_field(X.shape[0], dim, 1.0, 17))) == 0.0
    p0, p1 = v0.sum(axis=0), v1.sum(axis=0)
    assert np.all(np.abs(p1 - p0) < 1e-13 * np.abs(v0).sum())
    assert (v1 ** 2).sum() < (v0 ** 2).sum()


def _explicit_damping_accel(X, v, dx, h, eta, rho0):
    """(2 eta / m_a) sum_b V_a V_b (v_a - v_b) W'(r)/r, with W' from the
    Wendland C2 formula written here independently (NumPy brute force)."""
    n, dim = X.shape
    V = dx ** dim
    m = rho0 * V
    ad = 7 / (4 * math.pi * h * h) if dim == 2 else 21 / (16 * math.pi * h ** 3)
    out = np.zeros_like(v)
    for a in range(n):
        d = X[a] - X
        r = np.sqrt((d * d).sum(axis=1))
        sel = (r < 2 * h) & (r > 0)
        q = r[sel] / h
        dw_over_r = -5 * ad * (1 - q / 2) ** 3 / (h * h)
        out[a] = (2 * eta / m) * (V * V * (v[a] - v[sel]) * dw_over_r[:, None]).sum(axis=0)
    return out


@pytest.mark.parametrize("dim,counts", [(2, (12, 10)), (3, (7, 6, 6))])
def test_damping_sweep_is_consistent_with_viscous_term(dim, counts):
    eta, rho0 = 1e4, 7850.0
    X, dx, (b2, b3) = _damping_body(dim, counts, eta=eta)
    dt = 1e-13     # first order in dt: (v_new - v)/dt -> f_v
    b2.substep_partial(dt, 2)
    b3.substep_partial(dt, 3)
    v0, v1 = b2.read(O.F_V), b3.read(O.F_V)
    fv = _explicit_damping_accel(X, v0, dx, 1.3 * dx, eta, rho0)
    got = (v1 - v0) / dt
    assert np.max(np.abs(got - fv)) < 1e-4 * np.max(np.abs(fv))


def test_damping_uniform_velocity_is_fixed_point():
    X, dx, (b2, b3) = _damping_body(2, (10, 9), eta=1e5)
    vel = np.tile([0.3, -1.2], (X.shape[0], 1))
    b3.write(O.F_V, vel)
    b3.substep_partial(3e-8, 3)
    assert np.max(np.abs(b3.read(O.F_V) - vel)) < 1e-14


def test_damping_pair_against_fixed_partner_closed_form():
    # 3-particle right triangle; particles 1 and 2 fully constrained, v = 0.
    # Then only the pairs (0,1) and (0,2) act on particle 0, each an implicit
    # decay  v0 <- v0 / (1 + dt B/m)  of the pair ODE m dv/dt = -B v, applied
    # with dt/2 in the forward and again in the reverse half sweep.
    dx = 1e-4
    X = np.array([[0.0, 0.0], [dx, 0.0], [0.0, dx]])
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 1000.0, 1e6, 0.25)
    eta = 3e3
    ob.set_damping(eta)
    ob.set_bc_displacement(np.array([1, 2]), 0b11)
    ob.write(O.F_V, np.array([[1.0, -2.0], [0, 0], [0, 0]]))
    dt = 1e-7
    ob.substep_partial(dt, 3)
    h = 1.3 * dx
    ad = 7 / (4 * math.pi * h * h)
    V, m = dx * dx, 1000.0 * dx * dx

    def Bcoef(r):
        q = r / h
        return -2 * eta * V * V * (-5 * ad * q * (1 - q / 2) ** 3 / h) / r

    # symmetric sweep: each active pair twice with dt/2
    fac = 1.0 / (1 + 0.5 * dt * Bcoef(dx) / m) ** 4
    assert np.allclose(ob.read(O.F_V)[0], np.array([1.0, -2.0]) * fac, rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# moduli and elastic law: the paper's material table (golden)
# --------------------------------------------------------------------------
def test_moduli_from_paper_table_via_stress_probe():
    g = json.load(open(GOLDEN))["necking_material"]
    K, mu = g["bulk_modulus_pa"], g["shear_modulus_pa"]
    E = 9 * K * mu / (3 * K + mu)
    nu = (3 * K - 2 * mu) / (2 * (3 * K + mu))
    for model in (O.SVK, O.J2):
        kw = dict(sigma0=1e30, sigma_inf=1e30, delta=1.0, H=0.0) if model == O.J2 else {}
        gam = 1e-7
        F = np.eye(3)
        F[0, 1] = gam
        P, *_ = O.stress_point(model, 7850.0, E, nu, F, **kw)
        assert abs(P[0, 1] / gam - mu) < 1e-5 * mu
        e = 1e-7
        P, *_ = O.stress_point(model, 7850.0, E, nu, (1 + e) * np.eye(3), **kw)
        assert abs(P[0, 0] / (3 * e) - K) < 1e-5 * K


# --------------------------------------------------------------------------
# P7: return mapping (App. A, Alg. 1)
# --------------------------------------------------------------------------
def _j2_params():
    g = json.load(open(GOLDEN))["necking_material"]
    K, mu = g["bulk_modulus_pa"], g["shear_modulus_pa"]
    E = 9 * K * mu / (3 * K + mu)
    nu = (3 * K - 2 * mu) / (2 * (3 * K + mu))
    return dict(rho0=7850.0, E=E, nu=nu, sigma0=g["initial_flow_stress_pa"],
                sigma_inf=g["saturation_flow_stress_pa"], delta=g["saturation_exponent"],
                H=g["linear_hardening_pa"]), K, mu


def _uniaxial_F(p, ex, cpinv, alpha):
    """F = diag(1+ex, s, s) with s chosen so that the lateral Kirchhoff stress
    vanishes (bisection on the oracle's material point)."""
    lo, hi = 0.5, 1.5
    for _ in range(200):
        s = 0.5 * (lo + hi)
        P, cp, al, pl, res = O.stress_point(O.J2, p["rho0"], p["E"], p["nu"],
                                            np.diag([1 + ex, s, s]), cpinv, alpha,
                                            p["sigma0"], p["sigma_inf"], p["delta"], p["H"])
        tau = P @ np.diag([1 + ex, s, s]).T
        if tau[1, 1] > 0:
            hi = s
        else:
            lo = s
    return np.diag([1 + ex, s, s]), tau, cp, al, pl, res


def test_uniaxial_yield_onset_at_initial_flow_stress():
    p, K, mu = _j2_params()
    lo, hi = 0.0, 0.01
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        _, tau, _, _, pl, _ = _uniaxial_F(p, mid, None, 0.0)
        if pl:
            hi = mid
        else:
            lo = mid
    _, tau, _, _, _, _ = _uniaxial_F(p, lo, None, 0.0)
    assert abs(tau[0, 0] - p["sigma0"]) < 1e-6 * p["sigma0"]


def test_return_mapping_consistency_and_hardening_curve():
    p, K, mu = _j2_params()
    cp, al = None, 0.0
    k = lambda a: (p["sigma0"] + (p["sigma_inf"] - p["sigma0"]) * (1 - math.exp(-p["delta"] * a))
                   + p["H"] * a)
    for ex in np.linspace(0.002, 0.2, 60):
        F, tau, cp, al, pl, res = _uniaxial_F(p, ex, cp, al)
        if pl:
            s = tau - np.trace(tau) / 3 * np.eye(3)
            # after the return the stress lies on the yield surface
            assert abs(np.linalg.norm(s) - math.sqrt(2 / 3) * k(al)) < 1e-8 * k(al)
            assert abs(res) < 1e-6 * k(al)
            # uniaxial: tau_xx = k(alpha), alpha ~ plastic log strain
            assert abs(tau[0, 0] - k(al)) < 1e-8 * k(al)
    e_el = tau[0, 0] / p["E"]
    assert abs(al - (math.log(1.2) - e_el)) < 5e-3 * al


# --------------------------------------------------------------------------
# P6: elastic closed form -- the analytic uniaxial state is a discrete
# equilibrium with the right modulus (plane strain in 2D, 3D uniaxial)
# --------------------------------------------------------------------------
def _uniaxial_state(dim, lat_coef, eps=1e-5):
    dx = 1e-4
    counts = (20, 8) if dim == 2 else (14, 6, 6)
    X, idx, _ = B.box_body(counts, dx, seed=4, jitter=0.0)
    E, nu, rho0 = 210e9, 0.3, 7850.0
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, rho0, E, nu)
    G = np.zeros((dim, dim))
    G[0, 0] = eps
    for k in range(1, dim):
        G[k, k] = lat_coef * eps
    ob.write(O.F_U, X @ G.T)
    ob.substep_partial(1e-12, 2)
    body = (idx[:, 0] >= 4) & (idx[:, 0] < counts[0] - 4)
    return ob, idx, body, E, nu, rho0, dx


@pytest.mark.parametrize("dim", [2, 3])
def test_uniaxial_closed_form_is_discrete_equilibrium(dim):
    nu = 0.3
    lat = -nu / (1 - nu) if dim == 2 else -nu
    eps = 1e-5
    ob, idx, body, E, nu, rho0, dx = _uniaxial_state(dim, lat, eps)
    Ep = E / (1 - nu * nu) if dim == 2 else E
    scale = Ep * eps / (rho0 * dx)
    acc = ob.read(O.F_ACC)
    # traction-free lateral surfaces included: no force anywhere away from the ends
    assert np.max(np.abs(acc[body])) < 1e-4 * scale
    PB = ob.read(O.F_PB).reshape(-1, dim, dim)
    P = np.einsum("nij,njk->nik", PB, np.linalg.inv(np.transpose(ob.b0(), (0, 2, 1))))
    assert np.max(np.abs(P[:, 0, 0] - Ep * eps)) < 1e-4 * Ep * eps
    for k in range(1, dim):
        assert np.max(np.abs(P[:, k, k])) < 1e-4 * Ep * eps
    # a wrong lateral contraction leaves unbalanced surface forces
    wrong = -nu if dim == 2 else -nu / (1 - nu)
    ob2, _, body2, *_ = _uniaxial_state(dim, wrong, eps)
    assert np.max(np.abs(ob2.read(O.F_ACC)[body2])) > 1e-2 * scale


# --------------------------------------------------------------------------
# P10: free swelling (App. B.2 pressure coupling)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_free_swelling_strain(dim):
    dx = 1e-5
    counts = (10, 8) if dim == 2 else (7, 6, 5)
    X, _, _ = B.box_body(counts, dx, seed=6, jitter=0.01)
    E, nu, beta = 200e6, 0.4, 1e-4
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 2000.0, E, nu)
    # damping sized to this 0.1 mm body: larger eta over-damps its slowest
    # flexural mode (relaxation rate omega^2/gamma) and it would need 1e4+ substeps
    ob.set_damping(3.0)
    ob.set_diffusion(1e-10, beta, 0.0)
    ob.write(O.F_C, np.ones(X.shape[0]))
    ob.advance(ramp=0.0, ke_tol=-1.0, max_substeps=2000)
    F = ob.read(O.F_DEFGRAD).reshape(-1, 3, 3)
    e_want = (1 + nu) * beta if dim == 2 else beta
    diag = np.array([F[:, k, k] for k in range(dim)]).T - 1
    assert np.max(np.abs(diag - e_want)) < 2e-3 * e_want
    off = F[:, :dim, :dim] - np.diag(np.diag(np.ones((dim, dim))))[None] - \
        np.einsum("ni,ij->nij", diag, np.eye(dim))
    assert np.max(np.abs(off)) < 2e-3 * e_want
    if dim == 2:
        assert np.all(F[:, 2, 2] == 1.0)


# --------------------------------------------------------------------------
# P8/P9: diffusion (Sec. 2.2 Fick's law, Sec. 4.1 dt_d)
# --------------------------------------------------------------------------
def _slab(nx=16, ny=24, dx=1e-5, D=1e-10, jitter=0.0, seed=7):
    X, idx, _ = B.box_body((nx, ny), dx, seed=seed, jitter=jitter)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob.set_diffusion(D, 0.0, 0.0)
    return X, idx, ob


def test_diffusion_linear_profile_is_fixed_point():
    X, idx, ob = _slab(jitter=0.0)
    c = 3.0 + 2.0 * X[:, 1] / 1e-4 - 0.5 * X[:, 0] / 1e-4
    ny, nx = 24, 16
    edge = (idx[:, 1] < 2) | (idx[:, 1] >= ny - 2) | (idx[:, 0] < 2) | (idx[:, 0] >= nx - 2)
    for val, ids in [(None, np.nonzero(edge)[0])]:
        for i in ids:
            ob.set_bc_concentration(np.array([i]), c[i])
    ob.write(O.F_C, c)
    dtp, dts = ob.diffusion_dt()
    for _ in range(5):
        ob.diffusion_step(dts)
    assert np.max(np.abs(ob.read(O.F_C) - c)) < 1e-12


def test_diffusion_conserves_mass_and_max_principle():
    X, idx, ob = _slab(jitter=0.01)
    c0 = np.random.default_rng(3).uniform(0, 1, X.shape[0])
    ob.write(O.F_C, c0)
    dtp, dts = ob.diffusion_dt()
    # the paper's 0.5 h^2/D exceeds the stable bound at h = 1.3 dx
    assert dtp > dts
    for _ in range(40):
        ob.diffusion_step(dts)
        c = ob.read(O.F_C)
        assert c.min() >= -1e-14 and c.max() <= 1 + 1e-14
    assert abs(c.sum() - c0.sum()) < 1e-12 * c0.sum()
    assert c.std() < 0.3 * c0.std()


def _lattice_second_moment(h_over_dx):
    """-sum_j dx^2 y_j^2 W'(r_j)/r_j over a 2D unit lattice: the factor by which
    the one-pass pairwise Laplacian scales D for fields c(y) (1 in the continuum
    limit).  Written here independently of the oracle."""
    h = h_over_dx
    ad = 7 / (4 * math.pi * h * h)
    R = int(2 * h) + 2
    S = 0.0
    for i in range(-R, R + 1):
        for j in range(-R, R + 1):
            r = math.hypot(i, j)
            if r == 0 or r >= 2 * h:
                continue
            q = r / h
            S += -(j * j) * (-5 * ad * (1 - q / 2) ** 3 / (h * h))
    return S


def test_lattice_second_moment_tends_to_one():
    assert abs(_lattice_second_moment(3.0) - 1) < 2e-4
    assert abs(_lattice_second_moment(1.3) - 1) < 0.03


def _slab_error(ny, target, dx=1e-5, D0=1e-10):
    """Max error of the oracle's slab diffusion against the Fourier series of
    c_t = D c_yy, c(0) = 0, c(H) = 1, c(y, 0) = 0, in the two middle columns of a
    wide slab (the x-edges have incomplete kernel support)."""
    nx = max(60, 3 * ny)
    X, idx, _ = B.box_body((nx, ny), dx, seed=7, jitter=0.0)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob.set_diffusion(D0, 0.0, 0.0)
    Hc = ny - 3.0                     # layer 1 at c = 0, layer ny-2 at c = 1
    j = idx[:, 1]
    lin = (j - 1) / Hc
    for layer in (0, 1, ny - 2, ny - 1):
        ids = np.nonzero(j == layer)[0]
        ob.set_bc_concentration(ids, float(lin[ids[0]]))
    ob.write(O.F_C, np.where((j <= 1) | (j >= ny - 2), lin, 0.0))
    _, dts = ob.diffusion_dt()
    H = Hc * dx
    m = nx // 2 - 1
    mid = (idx[:, 0] >= m) & (idx[:, 0] <= m + 1) & (j >= 2) & (j < ny - 2)
    t_end = target * H * H / D0
    nsteps = int(math.ceil(t_end / dts))
    for _ in range(nsteps):
        ob.diffusion_step(t_end / nsteps)
    D = D0 * _lattice_second_moment(1.3)      # effective diffusivity of the lattice
    y = (j[mid] - 1) * dx
    n = np.arange(1, 600)[:, None]
    exact = y / H + (2 * (-1.0) ** n / (n * math.pi) * np.sin(n * math.pi * y / H)
                     * np.exp(-D * n * n * math.pi ** 2 * t_end / (H * H))).sum(axis=0)
    return np.max(np.abs(ob.read(O.F_C)[mid] - exact))


def test_diffusion_slab_matches_fourier_series():
    e21 = _slab_error(24, 0.1)
    e41 = _slab_error(44, 0.1)
    assert e21 < 2.5e-3 and e41 < 1.3e-3
    assert e41 < 0.65 * e21           # first order in dx/H (held-layer boundary)
    assert _slab_error(24, 0.3) < 2.5e-3


# --------------------------------------------------------------------------
# P14: energy sanity without damping (force sign)
# --------------------------------------------------------------------------
def test_undamped_oscillation_keeps_energy_bounded():
    dx = 1e-4
    X, _, _ = B.box_body((12, 8), dx, seed=9, jitter=0.01)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
    ob.write(O.F_V, B.random_field(X.shape[0], 2, 0.1, 5))
    m = 7850.0 * dx * dx
    ke0 = 0.5 * m * (ob.read(O.F_V) ** 2).sum()
    kes = []
    for _ in range(1500):
        ke, vm, am = ob.substep(1.2e-8)
        kes.append(ke)
    kes = np.array(kes)
    assert kes.max() < 1.05 * ke0
    assert kes[-500:].max() > 0.05 * ke0


# --------------------------------------------------------------------------
# slow-step driver: stop rule and time step (Sec. 4.1, Sec. 4.2)
# --------------------------------------------------------------------------
def test_slow_step_stops_at_kinetic_energy_criterion():
    c = B.bar2d(nx=30, ny=8, n_slow=4)
    ob = O.body_from_case(c)
    tol = 1e-4
    r = ob.advance(ramp=0.25, ke_tol=tol, ke_ref=c.plan.ke_ref, max_substeps=100000)
    assert r.converged == 1 and r.ke_final <= tol * c.plan.ke_ref
    ob2 = O.body_from_case(c)
    r2 = ob2.advance(ramp=0.25, ke_tol=-1, ke_ref=c.plan.ke_ref, max_substeps=r.substeps - 1)
    assert r2.ke_final > tol * c.plan.ke_ref
    m = c.material
    K = m.E / (3 * (1 - 2 * m.nu))
    ob3 = O.body_from_case(c)
    r3 = ob3.advance(ramp=0.25, ke_tol=-1, max_substeps=1)
    g = json.load(open(GOLDEN))["time_step_rules"]
    assert r3.dt_last == pytest.approx(g["solid_cfl_factor"] * 1.3 * c.dx / math.sqrt(K / m.rho0),
                                       rel=1e-15)


def test_errors_are_reported():
    with pytest.raises(O.OracleError):
        O.OracleBody(np.zeros((1, 2)), 1e-3)
    X = np.array([[0.0, 0.0], [1.0, 0.0]])
    with pytest.raises(O.OracleError) as e:
        O.OracleBody(X, 1.0)            # collinear pair: singular correction matrix
    assert e.value.status == O.ERR_SINGULAR


# --------------------------------------------------------------------------
# Stability of the substep map (reading of the damping order, Sec. 4.3)
# --------------------------------------------------------------------------
def _step_matrix(X, dx, dim, eta, dt):
    n = X.shape[0]
    cols = []
    eps = 1e-6
    for k in range(2 * n * dim):
        ob = O.OracleBody(X, dx)
        ob.set_material(O.SVK, 7850.0, 210e9, 0.3)
        ob.set_damping(eta)
        z = np.zeros(2 * n * dim)
        z[k] = eps
        ob.write(O.F_U, z[:n * dim].reshape(n, dim) * dx)
        ob.write(O.F_V, z[n * dim:].reshape(n, dim))
        ob.substep(dt, 0.0)
        cols.append(np.concatenate([ob.read(O.F_U).reshape(-1) / dx,
                                    ob.read(O.F_V).reshape(-1)]) / eps)
    return np.array(cols).T


@pytest.mark.parametrize("dim,counts", [(2, (10, 6)), (3, (5, 4, 4))])
@pytest.mark.parametrize("eta", [1e3, 1e4, 1e5, 1e6])
def test_linearised_substep_is_stable(dim, counts, eta):
    """Spectral radius of the linearised kick/damp/drift map at the Sec. 4.1
    time step stays at 1 (rigid modes) for the whole damping range."""
    dx = 1e-4
    X, _, _ = B.box_body(counts, dx, seed=4, jitter=0.01)
    K = 210e9 / (3 * (1 - 0.6))
    dt = 0.6 * 1.3 * dx / math.sqrt(K / 7850.0)
    rho = np.max(np.abs(np.linalg.eigvals(_step_matrix(X, dx, dim, eta, dt))))
    assert rho < 1 + 1e-6


# --------------------------------------------------------------------------
# P7 (body path): homogeneous SPH body under affine F == material point
# --------------------------------------------------------------------------
def test_j2_body_matches_material_point_under_affine_F():
    p, K, mu = _j2_params()
    dx = 1e-4
    X, _, _ = B.box_body((7, 6, 6), dx, seed=12, jitter=0.01)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.J2, p["rho0"], p["E"], p["nu"], p["sigma0"], p["sigma_inf"], p["delta"],
                    p["H"])
    G = np.array([[0.01, 0.002, 0.0], [0.0, -0.004, 0.001], [0.0, 0.0, -0.004]])
    ob.write(O.F_U, X @ G.T)
    ob.substep_partial(1e-15, 1)
    PB = ob.read(O.F_PB).reshape(-1, 3, 3)
    P = np.einsum("nij,njk->nik", PB, np.linalg.inv(np.transpose(ob.b0(), (0, 2, 1))))
    Pw, cpw, alw, plw, _ = O.stress_point(O.J2, p["rho0"], p["E"], p["nu"], np.eye(3) + G, None,
                                          0.0, p["sigma0"], p["sigma_inf"], p["delta"], p["H"])
    assert plw
    assert np.max(np.abs(P - Pw[None])) < 1e-9 * np.max(np.abs(Pw))
    assert np.max(np.abs(ob.read(O.F_ALPHA) - alw)) < 1e-12
    assert np.max(np.abs(ob.read(O.F_CPINV) - cpw[None])) < 1e-12


# --------------------------------------------------------------------------
# P12: the greedy sub-colours, recomputed independently from the definition
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,counts", [(2, (21, 13)), (3, (9, 8, 7))])
def test_colouring_matches_independent_greedy(dim, counts):
    dx = 1.0
    X, _, _ = B.box_body(counts, dx, seed=15, jitter=0.01)
    ob = O.OracleBody(X, dx)
    perm = ob.perm()
    Xs = X[perm]
    cell = np.floor((Xs - Xs.min(axis=0)) / dx).astype(np.int64)
    shift = 0
    while (1 << shift) < int(math.floor(2 * 1.3)) + 1:
        shift += 1
    assert shift == ob.blk_shift == 2
    blk = cell >> shift
    off, idx = ob.neighbors()

    def mkey(c):
        key = 0
        for bit in range(21):
            for k in range(dim):
                key |= ((int(c[k]) >> bit) & 1) << (bit * dim + k)
        return key

    R = int(math.floor(2 * 1.3)) + 1

    def oclass(a, b):
        o = cell[b] - cell[a]
        nz = [int(x) for x in o[::-1] if x != 0]      # first nonzero from the top axis
        sg = 1 if (not nz or nz[0] > 0) else -1
        c = 0
        for k in range(dim - 1, -1, -1):
            c = c * (2 * R + 1) + (sg * int(o[k]) + R)
        return c

    recs = []
    for a in range(len(Xs)):
        for b in idx[off[a]:off[a + 1]]:
            if b > a:
                owner = np.minimum(blk[a], blk[b])
                col = sum(int(owner[k] & 1) << k for k in range(dim))
                # classes visited in descending order
                recs.append([col, mkey(owner), -oclass(a, int(b)), a, int(b)])
    recs.sort()
    recs = [[r[0], r[1], r[3], r[4]] for r in recs]
    used = {}
    count = {}
    subs = []
    for i, (col, key, a, b) in enumerate(recs):
        if i == 0 or (col, key) != (recs[i - 1][0], recs[i - 1][1]):
            used, count = {}, {}
        ua, ub = used.setdefault(a, set()), used.setdefault(b, set())
        c = 0
        while c in ua or c in ub or count.get(c, 0) >= 32:   # at most 32 pairs per level
            c += 1
        ua.add(c)
        ub.add(c)
        count[c] = count.get(c, 0) + 1
        subs.append(c)
    want = sorted((r[0], r[1], s, r[2], r[3]) for r, s in zip(recs, subs))
    pa, pb, col, key, sub = ob.colouring()
    got = list(zip(col.tolist(), key.tolist(), sub.tolist(), pa.tolist(), pb.tolist()))
    assert got == want


# --------------------------------------------------------------------------
# end force of the report: uniaxial state, grip reaction = sigma_xx * area
# --------------------------------------------------------------------------
def test_end_force_equals_stress_times_area():
    dx, E, nu, rho0, eps = 1e-4, 210e9, 0.3, 7850.0, 1e-5
    counts = (20, 8)
    X, idx, _ = B.box_body(counts, dx, seed=4, jitter=0.0)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, rho0, E, nu)
    G = np.diag([eps, -nu / (1 - nu) * eps])
    U = X @ G.T
    ob.write(O.F_U, U)
    grip = B.layer_ids(idx, 0, counts[0] - 3, 3)
    ob.set_bc_displacement(grip, 0b11, U[grip], report_force=True)
    r = ob.advance(ramp=1.0, ke_tol=-1, max_substeps=1, dt_sub=1e-16)
    Ep = E / (1 - nu * nu)
    area = counts[1] * dx
    assert abs(r.end_force[0] - Ep * eps * area) < 0.03 * Ep * eps * area
    assert abs(r.end_force[1]) < 0.03 * Ep * eps * area


# ----------------------------------------------------------------------------
# P17: time-limited contact (Sec. 5.3-5.4 droplet schedule): released particles
# rejoin the diffusion, and with nothing held the step conserves sum V c
# ----------------------------------------------------------------------------
def test_released_contact_rejoins_diffusion_and_conserves_mass():
    c = B.beam_droplet2d(L=1e-3, W=0.125e-3, ny=8)
    ob = O.body_from_case(c)
    dts = ob.diffusion_dt()[1]
    for _ in range(3):
        ob.diffusion_step(dts)
    cc = ob.read(O.F_C)
    held = c.release[1]
    assert np.all(cc[held] == 0.4) and cc.sum() > 0.4 * held.size
    ob.release_bc_concentration(held)
    m0 = cc.sum()
    for _ in range(5):
        ob.diffusion_step(dts)
    c2 = ob.read(O.F_C)
    assert abs(c2.sum() - m0) <= 1e-12 * m0            # no held particles left: conservative
    assert np.max(c2[held]) < 0.4                     # the released set drains
    assert c2.min() >= 0.0 and c2.max() <= 0.4        # max principle


# ----------------------------------------------------------------------------
# P18: two-stage diffusion in the deformed configuration (Sec. 3.2 form, mode 1)
# ----------------------------------------------------------------------------
def _two_stage_body(nx=36, ny=36, D=1e-10, dx=1e-5):
    X, idx, _ = B.box_body((nx, ny), dx, seed=5, jitter=0.0)
    ob = O.OracleBody(X, dx)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob.set_diffusion(D, 0.0, 0.0)
    ob.set_diffusion_mode(1)
    deep = np.all((idx >= 6) & (idx < np.array([nx, ny]) - 6), axis=1)
    return ob, X, idx, deep


def test_two_stage_linear_profile_is_steady_in_the_interior():
    ob, X, idx, deep = _two_stage_body()
    c0 = 0.3 + 0.7 * X[:, 0] / X[:, 0].max()
    ob.write(O.F_C, c0)
    ob.diffusion_step(1e-3)
    c1 = ob.read(O.F_C)
    assert np.max(np.abs(c1 - c0)[deep]) < 1e-13


@pytest.mark.parametrize("stretch", [1.0, 1.2, 0.9])
def test_two_stage_quadratic_rate_matches_closed_form(stretch):
    """c = (X/L)^2 under u = (lambda - 1) X e_x: the Piola-mapped flux is
    Q = -(2 D / lambda L^2) X e_x, so dc/dt = 2 D m / (lambda L^2) on particles
    whose whole two-stage stencil is interior (m: the lattice's second-moment
    factor, computed independently)."""
    D, dx = 1e-10, 1e-5
    ob, X, idx, deep = _two_stage_body(D=D, dx=dx)
    L = X[:, 0].max()
    u = np.zeros_like(X)
    u[:, 0] = (stretch - 1.0) * X[:, 0]
    ob.write(O.F_U, u)
    c0 = (X[:, 0] / L) ** 2
    ob.write(O.F_C, c0)
    dt = 1e-3
    ob.diffusion_step(dt)
    rate = (ob.read(O.F_C) - c0) / dt
    want = 2 * D * _lattice_second_moment(1.3) / (stretch * L * L)
    assert np.max(np.abs(rate[deep] - want)) < 1e-9 * want


def test_two_stage_rigid_rotation_changes_nothing_and_conserves_mass():
    ob, X, idx, deep = _two_stage_body(nx=20, ny=16)
    rng = np.random.default_rng(2)
    c0 = rng.uniform(0, 1, X.shape[0])
    ob.write(O.F_C, c0)
    ob.diffusion_step(2e-3)
    ref = ob.read(O.F_C)
    ob2, *_ = _two_stage_body(nx=20, ny=16)
    th = 0.4
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    ob2.write(O.F_U, X @ R.T - X)
    ob2.write(O.F_C, c0)
    ob2.diffusion_step(2e-3)
    rot = ob2.read(O.F_C)
    assert np.max(np.abs(rot - ref)) < 1e-12
    assert abs(ref.sum() - c0.sum()) < 1e-12 * c0.sum()      # no held particles


def test_two_stage_stable_step_bound_holds():
    """At the reported stable step a rough field on a jittered, sheared body
    stays bounded over many steps."""
    X, idx, _ = B.box_body((16, 12), 1e-5, seed=9, jitter=0.2)
    ob = O.OracleBody(X, 1e-5)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob.set_diffusion(1e-10, 0.0, 0.0)
    ob.set_diffusion_mode(1)
    u = np.zeros_like(X)
    u[:, 0] = 0.2 * X[:, 1]
    ob.write(O.F_U, u)
    c0 = np.random.default_rng(4).uniform(0, 1, X.shape[0])
    ob.write(O.F_C, c0)
    dt_p, dt_s = ob.diffusion_dt()
    assert 0 < dt_s < dt_p
    for _ in range(300):
        ob.diffusion_step(dt_s)
    c = ob.read(O.F_C)
    assert np.all(np.isfinite(c)) and np.max(np.abs(c - c0.mean())) <= 1.0


# ----------------------------------------------------------------------------
# P19: anisotropic kernel for thin bodies (spacing per axis; Sec. 5.3-5.4)
# ----------------------------------------------------------------------------
def _aniso_body(dim, counts, ratio, jitter=0.01, seed=31):
    d0 = 1e-5
    dxk = [ratio * d0] * (dim - 1) + [d0]                 # coarse in plane, fine across
    X, idx, _ = B.box_body(counts, dxk, seed, jitter)
    return X, idx, dxk


@pytest.mark.parametrize("dim,counts,ratio", [(2, (12, 16), 4.0), (3, (7, 6, 12), 8.0)])
def test_aniso_neighbours_are_the_ellipsoid_and_F_is_exact(dim, counts, ratio):
    X, idx, dxk = _aniso_body(dim, counts, ratio)
    ob = O.OracleBody(X, min(dxk), dx_axis=dxk)
    off, nb = ob.neighbors()
    perm = ob.perm()
    Xs = X[perm]
    h = 1.3 * min(dxk)
    s = min(dxk) / np.asarray(dxk)
    d = (Xs[:, None, :] - Xs[None, :, :]) * s          # NumPy brute force, scaled
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    for i in range(len(Xs)):
        assert np.array_equal(nb[off[i]:off[i + 1]], np.nonzero(r2[i] < (2 * h) ** 2)[0])
    G = np.random.default_rng(3).uniform(-0.05, 0.05, (dim, dim))
    ob.write(O.F_U, X @ G.T)
    F = ob.read(O.F_DEFGRAD).reshape(-1, 3, 3)
    want = np.eye(3)
    want[:dim, :dim] += G
    assert np.max(np.abs(F - want)) < 1e-12


def test_aniso_force_balance_and_momentum():
    X, idx, dxk = _aniso_body(2, (14, 20), 4.0, jitter=0.0)
    ob = O.OracleBody(X, min(dxk), dx_axis=dxk)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    G = np.array([[1e-3, 3e-4], [-2e-4, 5e-4]])
    ob.write(O.F_U, X @ G.T)
    ob.substep_partial(1e-12, 2)
    acc = ob.read(O.F_ACC)
    scale = 200e6 * 1e-3 / (2000 * min(dxk))
    deep = np.all((idx >= 4) & (idx < np.array([14, 20]) - 4), axis=1)
    assert np.max(np.abs(acc[deep])) < 1e-9 * scale          # uniform stress: no interior force
    X2, _, dxk2 = _aniso_body(2, (10, 12), 4.0, jitter=0.05)
    ob2 = O.OracleBody(X2, min(dxk2), dx_axis=dxk2)
    ob2.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob2.write(O.F_U, B.random_field(X2.shape[0], 2, 1e-2 * min(dxk2), 6))
    ob2.substep_partial(1e-12, 2)
    a2 = ob2.read(O.F_ACC)
    assert np.max(np.abs(a2.sum(0))) < 1e-10 * np.abs(a2).sum()   # pair-antisymmetric force


def test_aniso_two_stage_quadratic_rate_and_one_pass_refused():
    D, ratio = 1e-10, 4.0
    X, idx, dxk = _aniso_body(2, (20, 40), ratio, jitter=0.0)
    ob = O.OracleBody(X, min(dxk), dx_axis=dxk)
    ob.set_material(O.SVK, 2000.0, 200e6, 0.4)
    ob.set_diffusion(D, 0.0, 0.0)
    with pytest.raises(O.OracleError):
        ob.diffusion_step(1e-3)                               # one-pass form: not for this kernel
    ob.set_diffusion_mode(1)
    Ly = X[:, 1].max()
    c0 = (X[:, 1] / Ly) ** 2
    ob.write(O.F_C, c0)
    ob.diffusion_step(1e-3)
    rate = (ob.read(O.F_C) - c0) / 1e-3
    # second moment of the normalised anisotropic kernel on this lattice,
    # summed here independently: -sum_b V dy_b (d W / d y)_b
    h = 1.3 * min(dxk)
    sx = min(dxk) / dxk[0]
    ad = 7 / (4 * math.pi * h * h)
    m = 0.0
    for i in range(-4, 5):
        for j in range(-4, 5):
            if i == 0 and j == 0:
                continue
            dxv, dyv = i * dxk[0], j * dxk[1]
            rt = math.hypot(dxv * sx, dyv)
            if rt >= 2 * h:
                continue
            q = rt / h
            dw = -5 * ad * q * (1 - q / 2) ** 3 / h
            gy = sx * dw / rt * dyv                           # detS * W'/r~ * s_y^2 * dy
            m += -(dxk[0] * dxk[1]) * dyv * gy
    deep = np.all((idx >= np.array([6, 6])) & (idx < np.array([20, 40]) - 6), axis=1)
    want = 2 * D * m / Ly ** 2
    assert abs(m - 1) < 0.05
    assert np.max(np.abs(rate[deep] - want)) < 1e-9 * want


def test_aniso_with_equal_spacings_is_the_isotropic_body():
    X, _, _ = B.box_body((9, 7), 1e-5, seed=4, jitter=0.05)
    a = O.OracleBody(X, 1e-5)
    b = O.OracleBody(X, 1e-5, dx_axis=[1e-5, 1e-5])
    for o in (a, b):
        o.set_material(O.SVK, 2000.0, 200e6, 0.4)
        o.set_damping(1e3)
        o.write(O.F_U, B.random_field(X.shape[0], 2, 1e-7, 2))
        o.advance(ramp=0.0, ke_tol=-1.0, max_substeps=5)
    assert np.array_equal(a.read(O.F_U), b.read(O.F_U))
