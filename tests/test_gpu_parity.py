"""GPU (CUDA library, through the C ABI) versus the FP64 CPU oracle.

Tolerances (normwise: max |gpu - oracle| / max |oracle| per field):
  * setup products (Morton order, CSR, damping colouring): bit-exact;
  * FP64 single substep, every stage: <= 1e-12;
  * FP64 multi-substep slow steps at equal substep counts: <= 1e-9;
  * mixed precision (FP32 per-particle arithmetic, FP64 displacement and
    reductions): displacement <= 1e-4, concentration <= 1e-5.
Element by element (|gpu - oracle| / |oracle| over every component of at
least 1e-2 of the field's largest, so that small components are held too):
FP64 slow steps <= 1e-8, mixed displacement <= 1e-3, mixed concentration
<= 1e-4 (the normwise bounds times ten: a component of 1e-2 of the largest
that carries the largest absolute error allowed normwise would be at 100x).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_04010_gb300 import mtssph as M
from synth import bodies as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def elementwise(a, b, floor=1e-2):
    """Largest |a - b| / |b| over the components with |b| >= floor max|b|: a
    relative error per element for every component that is not negligible
    (small components such as lateral displacements near the clamps
    included), where a normwise error would let them drift."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    sel = np.abs(b) >= floor * np.max(np.abs(b))
    return float(np.max(np.abs(a[sel] - b[sel]) / np.abs(b[sel])))


def small_cylinder(**kw):
    return B.cylinder3d(L=5e-3, R=1.25e-3, dx=0.25e-3, n_slow=20, **kw)


def small_strip(nx=120, ny=20):
    c = B.strip2d(nx=nx, ny=ny)
    c.eta = 1.0
    return c


def pair(ctx, case, precision=M.FP64, layout=M.DAMP_AUTO):
    """Library body and an oracle body with the same damping-order layout."""
    gb = M.body_from_case(ctx, case, precision, layout)
    return O.body_from_case(case, damp_layout=gb.damping_layout()), gb


CASES = {
    "bar2d": lambda: B.bar2d(),
    "cyl3d": small_cylinder,
    "strip2d": small_strip,
    "box3d_irregular": lambda: _irregular3d(),
}


def _irregular3d():
    X, idx, _ = B.box_body((9, 8, 7), 1e-4, seed=77, jitter=0.3)
    c = B.bar2d(nx=10, ny=4)
    c.dim, c.X, c.dx = 3, X, 1e-4
    c.disp_bcs = [B.DispBC(B.layer_ids(idx, 0, 0, 2), 0b111, np.zeros((int((idx[:, 0] < 2).sum()), 3)))]
    c.tip_ids = B.layer_ids(idx, 0, 8, 1)
    return c


# ---------------------------------------------------------------- setup
LAYOUTS = {"auto": M.DAMP_AUTO, "blocks": M.DAMP_BLOCKS, "wide": M.DAMP_WIDE}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [M.FP64, M.MIXED])
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_setup_products_bit_exact(ctx, name, precision, layout):
    case = CASES[name]()
    gb = M.Body(ctx, case.X, case.dx, case.h_over_dx, precision, LAYOUTS[layout])
    shifts, cap = gb.damping_layout()
    if layout == "blocks":
        assert cap == 32 and M.WHOLE_AXIS not in shifts
    if layout == "wide":
        assert cap == 0 and list(shifts).count(M.WHOLE_AXIS) == 1
    ob = O.OracleBody(case.X, case.dx, case.h_over_dx, damp_layout=(shifts, cap))
    assert np.array_equal(gb.permutation(), ob.perm())
    go, gi = gb.neighbors()
    oo, oi = ob.neighbors()
    assert np.array_equal(go, oo) and np.array_equal(gi, oi)
    for g, o in zip(gb.colouring(), ob.colouring()):
        assert np.array_equal(g, o)


def test_setup_rejects_bad_bodies(ctx):
    with pytest.raises(M.MtsError) as e:
        M.Body(ctx, np.array([[0.0, 0.0], [1.0, 0.0]]), 1.0)
    assert e.value.status == M.ERR_SINGULAR_B
    X = np.zeros((10, 2))
    X[:, 0] = np.arange(10)
    X[3, 1] = np.nan
    with pytest.raises(M.MtsError) as e:
        M.Body(ctx, X, 1.0)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MtsError) as e:
        M.Body(ctx, np.zeros((1, 3)), 1.0)
    assert e.value.status == M.ERR_INVALID_ARG
    c = B.bar2d(nx=12, ny=5)
    with pytest.raises(M.MtsError) as e:
        M.Body(ctx, c.X, c.dx, damp_layout=3)
    assert e.value.status == M.ERR_INVALID_ARG


# ---------------------------------------------------------------- one substep
def _state(case, seed, ustrain):
    n, d = case.X.shape
    U = B.random_field(n, d, ustrain * case.dx, seed)
    V = B.random_field(n, d, 0.05, seed + 1)
    return U, V


@pytest.mark.parametrize("name,ustrain", [("bar2d", 1e-3), ("cyl3d", 2e-2), ("strip2d", 1e-3),
                                          ("box3d_irregular", 1e-3)])
@pytest.mark.parametrize("layout", ["blocks", "wide"])
def test_fp64_single_substep_every_stage(ctx, name, ustrain, layout):
    case = CASES[name]()
    U, V = _state(case, 5, ustrain)
    dt = 0.6 * case.h_over_dx * case.dx / math.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    rng = np.random.default_rng(3)
    C0 = rng.uniform(0, 1, case.n) if case.diffusion else None
    for upto in (1, 2, 3, 4):
        ob, gb = pair(ctx, case, layout=LAYOUTS[layout])
        for b in (ob, gb):
            b.write(M.F_U, U)
            b.write(M.F_V, V)
            if C0 is not None:
                b.write(M.F_C, C0)
        ob.substep_partial(dt, upto, ramp=0.5)
        gb.substep_partial(dt, upto, ramp=0.5)
        assert rel(gb.read(M.F_PB), ob.read(O.F_PB)) < 1e-12
        if case.material.model == "j2":
            assert rel(gb.read(M.F_ALPHA), ob.read(O.F_ALPHA)) < 1e-12
            assert ob.read(O.F_ALPHA).max() > 0      # the state is plastic somewhere
            assert rel(gb.read(M.F_CPINV), ob.read(O.F_CPINV)) < 1e-12
        if upto >= 2:
            assert rel(gb.read(M.F_ACC), ob.read(O.F_ACC)) < 1e-12
        assert rel(gb.read(M.F_V), ob.read(O.F_V)) < 1e-12
        assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-12
        assert rel(gb.read(M.F_DEFGRAD), ob.read(O.F_DEFGRAD)) < 1e-12


def test_affine_field_exact_F(ctx):
    for case in (B.bar2d(nx=20, ny=9), small_cylinder()):
        d = case.X.shape[1]
        G = np.random.default_rng(1).uniform(-0.05, 0.05, (d, d))
        want = np.eye(3)
        want[:d, :d] += G
        for prec, tol in ((M.FP64, 1e-13), (M.MIXED, 2e-6)):
            gb = M.Body(ctx, case.X, case.dx, case.h_over_dx, prec)
            gb.write(M.F_U, case.X @ G.T)
            F = gb.read(M.F_DEFGRAD).reshape(-1, 3, 3)
            assert np.max(np.abs(F - want)) < tol


# ---------------------------------------------------------------- slow steps
def _run_both(ctx, case, nslow, nsub, precision=M.FP64, ke_tol=-1.0, dt_slow=0.0,
              layout=M.DAMP_AUTO):
    ob, gb = pair(ctx, case, precision, layout)
    reps = []
    for l in range(1, nslow + 1):
        ramp = l / max(case.plan.n_ramp, 1)
        rg = gb.advance_slow_step(dt_slow=dt_slow, ramp=ramp, ke_tol=ke_tol, ke_ref=case.plan.ke_ref,
                                  ke_mode=case.plan.ke_mode, max_substeps=nsub, check_every=16)
        ro = ob.advance(dt_slow=dt_slow, ramp=ramp, ke_tol=-1.0, ke_ref=case.plan.ke_ref,
                        ke_mode=case.plan.ke_mode, max_substeps=rg.substeps)
        reps.append((rg, ro))
    return ob, gb, reps


def test_device_loop_counts_and_launches(ctx):
    case = B.bar2d(nx=30, ny=8)
    gb = M.body_from_case(ctx, case)
    r = gb.advance_slow_step(ramp=0.05, ke_tol=-1, max_substeps=37)          # device loop
    assert r.substeps == 37 and r.converged == 0
    per = (r.kernel_launches - 2 - 2) // 37                 # minus load/reset and tip kernels
    assert per >= 4 and (r.kernel_launches - 4) % 37 == 0
    r2 = gb.advance_slow_step(ramp=0.05, ke_tol=-1, max_substeps=37, check_every=8)
    assert r2.substeps == 37 and r2.kernel_launches == 4 + 40 * per   # 5 chunks of 8


@pytest.mark.parametrize("layout", ["blocks", "wide"])
def test_fp64_slow_steps_bar2d(ctx, layout):
    ob, gb, reps = _run_both(ctx, B.bar2d(), 3, 300, layout=LAYOUTS[layout])
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9
    assert rel(gb.read(M.F_V), ob.read(O.F_V)) < 1e-9
    assert elementwise(gb.read(M.F_U), ob.read(O.F_U)) < 1e-8
    for rg, ro in reps:
        assert rg.substeps == ro.substeps == 300
        assert abs(rg.ke_final - ro.ke_final) < 1e-9 * ro.ke_final
        assert abs(rg.end_force[0] - ro.end_force[0]) < 1e-9 * abs(ro.end_force[0])
        assert abs(rg.tip_deflection[0] - ro.tip_deflection[0]) < 1e-9 * abs(ro.tip_deflection[0])
        assert abs(rg.dt_last - ro.dt_last) < 1e-12 * ro.dt_last


@pytest.mark.parametrize("layout", ["blocks", "wide"])
def test_fp64_slow_steps_j2_cylinder(ctx, layout):
    case = small_cylinder()
    ob, gb, reps = _run_both(ctx, case, 4, 150, layout=LAYOUTS[layout])
    assert ob.read(O.F_ALPHA).max() > 0
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9
    assert rel(gb.read(M.F_ALPHA), ob.read(O.F_ALPHA)) < 1e-9


@pytest.mark.parametrize("check_every", [0, 64])    # device WHILE loop / host-checked chunks
def test_kinetic_energy_stop_matches_oracle(ctx, check_every):
    case = B.bar2d(nx=40, ny=10)
    ob, gb = pair(ctx, case)
    for l in (1, 2):
        rg = gb.advance_slow_step(ramp=l / 20, ke_tol=1e-4, ke_ref=case.plan.ke_ref,
                                  max_substeps=100000, check_every=check_every)
        ro = ob.advance(ramp=l / 20, ke_tol=1e-4, ke_ref=case.plan.ke_ref, max_substeps=100000)
        assert rg.converged == ro.converged == 1
        assert rg.substeps == ro.substeps
        assert rg.ke_final <= 1e-4 * case.plan.ke_ref
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9


def test_diffusion_and_swelling_fp64(ctx):
    case = small_strip()
    ob, gb = pair(ctx, case)
    dtp_o, dts_o = ob.diffusion_dt()
    dtp_g, dts_g = gb.diffusion_dt()
    assert abs(dtp_g - dtp_o) < 1e-14 * dtp_o and abs(dts_g - dts_o) < 1e-12 * dts_o
    for _ in range(3):
        rg = gb.advance_slow_step(dt_slow=dts_o, ke_tol=-1, max_substeps=50, check_every=16)
        ob.advance(dt_slow=dts_o, ke_tol=-1, max_substeps=rg.substeps)
    assert rel(gb.read(M.F_C), ob.read(O.F_C)) < 1e-12
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9
    with pytest.raises(M.MtsError) as e:
        gb.advance_slow_step(dt_slow=1.5 * dts_g, max_substeps=1)
    assert e.value.status == M.ERR_UNSTABLE_DT


# ---------------------------------------------------------------- mixed precision
def test_mixed_precision_bar2d_displacement(ctx):
    case = B.bar2d()
    ob, gb, reps = _run_both(ctx, case, 2, 2000, precision=M.MIXED)
    e = rel(gb.read(M.F_U), ob.read(O.F_U))
    assert e < 1e-4, e
    assert elementwise(gb.read(M.F_U), ob.read(O.F_U)) < 1e-3


def test_mixed_precision_concentration(ctx):
    case = small_strip()
    ob, gb = pair(ctx, case, M.MIXED)
    _, dts = ob.diffusion_dt()
    for _ in range(20):
        rg = gb.advance_slow_step(dt_slow=dts, ke_tol=-1, max_substeps=5, check_every=8)
        ob.advance(dt_slow=dts, ke_tol=-1, max_substeps=rg.substeps)
    assert rel(gb.read(M.F_C), ob.read(O.F_C)) < 1e-5
    assert elementwise(gb.read(M.F_C), ob.read(O.F_C)) < 1e-4


@pytest.mark.parametrize("layout", ["blocks", "wide"])
def test_mixed_precision_j2_cylinder(ctx, layout):
    case = small_cylinder()
    ob, gb, reps = _run_both(ctx, case, 3, 300, precision=M.MIXED, layout=LAYOUTS[layout])
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-4
    assert elementwise(gb.read(M.F_U), ob.read(O.F_U)) < 1e-3


# ---------------------------------------------------------------- full size
@pytest.mark.parametrize("precision,tol,layout", [(M.FP64, 1e-12, "auto"), (M.MIXED, 1e-4, "auto"),
                                                 (M.FP64, 1e-12, "wide")])
def test_full_size_cylinder_first_substeps(ctx, precision, tol, layout):
    """The benchmark workload (3D J2 cylinder, 252,800 particles) at full size:
    setup products bit-exact, then two substeps after the first load jump."""
    case = B.cylinder3d()
    ob, gb = pair(ctx, case, precision, LAYOUTS[layout])
    if layout == "auto":      # blocks of 4 cells (4 dx > 2h) on every axis, 32 pairs per level
        assert gb.damping_layout() == ((2, 2, 2), 32)
    off_g, idx_g = gb.neighbors()
    off_o, idx_o = ob.neighbors()
    assert np.array_equal(off_g, off_o) and np.array_equal(idx_g, idx_o)
    for g, o in zip(gb.colouring(), ob.colouring()):
        assert np.array_equal(g, o)
    ramp = 1.0 / case.plan.n_ramp
    rg = gb.advance_slow_step(ramp=ramp, ke_tol=-1, max_substeps=2, check_every=2)
    ro = ob.advance(ramp=ramp, ke_tol=-1, max_substeps=2)
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol
    assert rel(gb.read(M.F_V), ob.read(O.F_V)) < max(tol, 1e-12) * (1 if precision == M.FP64 else 10)
    assert abs(rg.ke_final - ro.ke_final) < (1e-12 if precision == M.FP64 else 1e-3) * ro.ke_final


# ---------------------------------------------------------------- errors
def test_api_errors(ctx):
    case = B.bar2d(nx=20, ny=6)
    gb = M.Body(ctx, case.X, case.dx)
    with pytest.raises(M.MtsError) as e:
        gb.advance_slow_step(max_substeps=1)
    assert e.value.status == M.ERR_STATE
    gb.set_material(M.ELASTIC_SVK, 7850, 210e9, 0.3)
    with pytest.raises(M.MtsError) as e:
        gb.write(M.F_U, np.full((case.n, 2), np.nan))
    assert e.value.status == M.ERR_NONFINITE
    with pytest.raises(M.MtsError) as e:
        gb.set_bc_displacement([case.n + 5], 1)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MtsError):
        gb.advance_slow_step(max_substeps=0)
    with pytest.raises(M.MtsError) as e:
        gb.advance_slow_step(dt_slow=1.0, max_substeps=1)
    assert e.value.status == M.ERR_STATE
    gb.set_bc_displacement(np.zeros(0, np.int64), 1)      # empty set is fine
    r = gb.advance_slow_step(max_substeps=1)
    assert r.substeps == 1 and r.converged == 0


# ---------------------------------------------------------------- checkpoint / resume
@pytest.mark.parametrize("precision", [M.FP64, M.MIXED])
def test_save_load_state_resumes_bit_exact(ctx, precision):
    case = small_cylinder()
    gb = M.body_from_case(ctx, case, precision)
    kw = dict(ke_tol=case.plan.ke_tol, ke_ref=case.plan.ke_ref, max_substeps=400)
    gb.advance_slow_step(ramp=1 / case.plan.n_ramp, **kw)
    state = gb.save_state()
    r1 = gb.advance_slow_step(ramp=2 / case.plan.n_ramp, **kw)
    u1, a1 = gb.read(M.F_U), gb.read(M.F_ALPHA)
    gb.advance_slow_step(ramp=3 / case.plan.n_ramp, **kw)        # move on, then rewind
    gb.load_state(state)
    r2 = gb.advance_slow_step(ramp=2 / case.plan.n_ramp, **kw)
    assert r2.substeps == r1.substeps and r2.ke_final == r1.ke_final
    assert np.array_equal(gb.read(M.F_U), u1) and np.array_equal(gb.read(M.F_ALPHA), a1)
    other = M.body_from_case(ctx, B.bar2d(nx=12, ny=5), precision)
    with pytest.raises(M.MtsError) as e:
        other.load_state(state)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MtsError):
        gb.load_state(state[:-8])


# ---------------------------------------------------------------- other workloads at full size
def test_full_size_strip_diffusion_swelling():
    """The 2D swelling strip at its full size (2,000 x 20 = 40,000 particles):
    setup bit-exact, then two slow steps (diffusion step + 40 substeps each)
    against the oracle, FP64 and mixed precision."""
    ctx = M.Context(0)
    case = B.strip2d()
    assert case.n == 40000
    ob = O.body_from_case(case)
    dts = ob.diffusion_dt()[1]
    for l in (1, 2):
        ob.advance(dt_slow=dts, ke_tol=-1.0, max_substeps=40, ke_mode=1)
    for prec, tol_u, tol_c in ((M.FP64, 1e-9, 1e-12), (M.MIXED, 1e-4, 1e-5)):
        gb = M.body_from_case(ctx, case, prec)
        if prec == M.FP64:
            for g, o in zip(gb.colouring(), ob.colouring()):
                assert np.array_equal(g, o)
        for l in (1, 2):
            r = gb.advance_slow_step(dt_slow=dts, ke_tol=-1.0, max_substeps=40, ke_mode=1)
            assert r.substeps == 40
        assert rel(gb.read(M.F_C), ob.read(O.F_C)) < tol_c
        assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol_u
        gb.close()
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(M.FP64, 1e-12), (M.MIXED, 2e-5)])
def test_full_size_plate_properties(precision, tol):
    """The 3D plate at its full size (1,000 x 250 x 10 = 2.5 M particles), too
    large for the oracle's setup: properties that hold at any size.  The
    neighbour lists are symmetric with the lattice count in the interior, the
    damping order lists every pair once, and an affine displacement field
    gives F = I + G exactly at every particle, surfaces included."""
    ctx = M.Context(0)
    case = B.plate3d()
    assert case.n == 2_500_000
    gb = M.Body(ctx, case.X, case.dx, case.h_over_dx, precision)
    off, idx = gb.neighbors()
    deg = np.diff(off)
    assert off[-1] % 2 == 0 and deg.max() <= 80 and np.median(deg) == 80
    pa, pb = gb.colouring()[:2]
    assert pa.size == off[-1] // 2 and np.all(pa < pb)
    G = np.random.default_rng(4).uniform(-0.02, 0.02, (3, 3))
    gb.write(M.F_U, case.X @ G.T)
    F = gb.read(M.F_DEFGRAD).reshape(-1, 3, 3)
    assert np.max(np.abs(F - (np.eye(3) + G))) < tol
    gb.close()
    ctx.close()


@pytest.mark.parametrize("which", ["beam", "membrane"])
@pytest.mark.parametrize("precision,tol_u,tol_c", [(M.FP64, 1e-9, 1e-12), (M.MIXED, 1e-4, 1e-5)])
def test_droplet_contact_schedule(ctx, which, precision, tol_u, tol_c):
    """Sec. 5.3 / 5.4 schedules (small bodies): held contact for two slow
    steps, released, two more; GPU against the oracle."""
    case = (B.beam_droplet2d(L=2e-3) if which == "beam"
            else B.membrane_droplet3d(Lx=0.6e-3, Ly=0.6e-3))
    ob, gb = pair(ctx, case, precision)
    dts = ob.diffusion_dt()[1]
    for step in range(4):
        if step == 2:
            ob.release_bc_concentration(case.release[1])
            gb.release_bc_concentration(case.release[1])
        kw = dict(dt_slow=dts, ke_tol=-1.0, ke_ref=case.plan.ke_ref, ke_mode=1, max_substeps=30)
        rg = gb.advance_slow_step(**kw)
        ro = ob.advance(**kw)
        assert rg.substeps == ro.substeps == 30
    assert rel(gb.read(M.F_C), ob.read(O.F_C)) < tol_c
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol_u
    assert np.max(np.abs(ob.read(O.F_U))) > 0


@pytest.mark.parametrize("which", ["strip", "plate"])
@pytest.mark.parametrize("precision,tol_u,tol_c", [(M.FP64, 1e-9, 1e-12), (M.MIXED, 1e-4, 1e-5)])
def test_two_stage_diffusion(ctx, which, precision, tol_u, tol_c):
    """Diffusion mode 1 (two-stage flux in the deformed configuration):
    stable-step bound and three slow steps (diffusion + 20 substeps) against
    the oracle; the body bends, so F enters the flux."""
    case = small_strip() if which == "strip" else B.plate3d(nx=24, ny=10, nz=8)
    ob, gb = pair(ctx, case, precision)
    ob.set_diffusion_mode(1)
    gb.set_diffusion_mode(1)
    for step in range(3):
        dto = ob.diffusion_dt()
        dtg = gb.diffusion_dt()
        assert abs(dtg[1] - dto[1]) <= (1e-12 if precision == M.FP64 else 1e-5) * dto[1]
        kw = dict(dt_slow=dto[1], ke_tol=-1.0, ke_ref=case.plan.ke_ref, ke_mode=1, max_substeps=20,
                  force_dt=True)
        gb.advance_slow_step(**kw)
        ob.advance(**kw)
    assert rel(gb.read(M.F_C), ob.read(O.F_C)) < tol_c
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol_u
    assert np.max(np.abs(ob.read(O.F_U))) > 0


@pytest.mark.parametrize("which", ["beam", "membrane"])
@pytest.mark.parametrize("precision,tol_u,tol_c", [(M.FP64, 1e-9, 1e-12), (M.MIXED, 1e-4, 1e-5)])
def test_anisotropic_kernel_droplet(ctx, which, precision, tol_u, tol_c):
    """The paper's thin-body set-up with its anisotropic kernel (spacing 4x
    along the beam, 8x in the membrane's plane) and the two-stage diffusion:
    setup bit-exact, F exact for affine fields, then slow steps through the
    contact release against the oracle."""
    case = (B.beam_droplet2d(L=2e-3, aniso=4.0) if which == "beam"
            else B.membrane_droplet3d(Lx=1.2e-3, Ly=1.2e-3, aniso=8.0))
    ob, gb = pair(ctx, case, precision)
    assert np.array_equal(gb.permutation(), ob.perm())
    go, gi = gb.neighbors()
    oo, oi = ob.neighbors()
    assert np.array_equal(go, oo) and np.array_equal(gi, oi)
    for g, o in zip(gb.colouring(), ob.colouring()):
        assert np.array_equal(g, o)
    assert rel(gb.read(M.F_X), case.X) < 1e-12
    d = case.dim
    G = np.random.default_rng(7).uniform(-0.02, 0.02, (d, d))
    gb.write(M.F_U, case.X @ G.T)
    want = np.eye(3)
    want[:d, :d] += G
    assert np.max(np.abs(gb.read(M.F_DEFGRAD).reshape(-1, 3, 3) - want)) < (
        1e-12 if precision == M.FP64 else 2e-5)
    gb.write(M.F_U, np.zeros((case.n, d)))
    ob.set_diffusion_mode(1)
    gb.set_diffusion_mode(1)
    with pytest.raises(M.MtsError):
        M.body_from_case(ctx, case, precision).advance_slow_step(dt_slow=1e-3, max_substeps=1)
    for step in range(3):
        if step == 2:
            ob.release_bc_concentration(case.release[1])
            gb.release_bc_concentration(case.release[1])
        dts = ob.diffusion_dt()[1]
        kw = dict(dt_slow=dts, ke_tol=-1.0, ke_ref=case.plan.ke_ref, ke_mode=1, max_substeps=20,
                  force_dt=True)
        gb.advance_slow_step(**kw)
        ob.advance(**kw)
    assert rel(gb.read(M.F_C), ob.read(O.F_C)) < tol_c
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol_u
    assert rel(gb.read(M.F_PB), ob.read(O.F_PB)) < tol_u
    assert np.max(np.abs(ob.read(O.F_U))) > 0
