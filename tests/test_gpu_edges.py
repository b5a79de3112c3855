"""GPU edge cases against the FP64 oracle: no damping, a fully constrained
body, an unloaded body, and the smallest bodies (one tile, a few owner groups,
levels with a handful of pairs)."""
import dataclasses
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


def test_zero_damping_matches_oracle(ctx):
    """eta = 0: the damping stage is skipped; undamped substeps still agree."""
    case = B.bar2d(nx=20, ny=6, eta=0.0)
    ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, M.FP64)
    for l in (1, 2):
        rg = gb.advance_slow_step(ramp=l / 20, ke_tol=-1, max_substeps=40)
        ro = ob.advance(ramp=l / 20, ke_tol=-1, max_substeps=40)
        assert rg.substeps == ro.substeps == 40
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9
    assert rel(gb.read(M.F_V), ob.read(O.F_V)) < 1e-9


def test_fully_constrained_body(ctx):
    """Every particle prescribed on every axis: u is the prescribed field,
    v stays zero and the kinetic-energy stop fires at the first check."""
    case = B.bar2d(nx=12, ny=5)
    n = case.n
    ids = np.arange(n, dtype=np.int64)
    u_unit = B.random_field(n, 2, 1e-6, 11)
    case = dataclasses.replace(case, disp_bcs=[B.DispBC(ids, 0b11, u_unit, report_force=True)])
    ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, M.FP64)
    rg = gb.advance_slow_step(ramp=0.3, ke_tol=1e-9, ke_ref=case.plan.ke_ref, max_substeps=50)
    ro = ob.advance(ramp=0.3, ke_tol=1e-9, ke_ref=case.plan.ke_ref, max_substeps=50)
    assert rg.converged == ro.converged == 1
    assert rg.substeps == ro.substeps
    assert np.array_equal(gb.read(M.F_V), np.zeros((n, 2)))
    assert rel(gb.read(M.F_U), 0.3 * u_unit) < 1e-15
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-15


@pytest.mark.parametrize("precision", [M.FP64, M.MIXED])
def test_unloaded_body_does_not_move(ctx, precision):
    """No load (ramp 0): zero force everywhere, the stop fires at the first
    check and the displacement stays exactly zero."""
    case = B.bar2d(nx=30, ny=8)
    ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, precision)
    rg = gb.advance_slow_step(ramp=0.0, ke_tol=1e-12, ke_ref=case.plan.ke_ref, max_substeps=100)
    ro = ob.advance(ramp=0.0, ke_tol=1e-12, ke_ref=case.plan.ke_ref, max_substeps=100)
    assert rg.converged == ro.converged == 1
    assert rg.substeps == ro.substeps
    assert not np.any(gb.read(M.F_U))
    assert not np.any(gb.read(M.F_V))


def _tiny(dim):
    counts = (4, 3) if dim == 2 else (3, 3, 3)
    X, idx, _ = B.box_body(counts, 1e-4, seed=5, jitter=0.05)
    c = B.bar2d(nx=10, ny=4)
    clamp = B.layer_ids(idx, 0, 0, 1)
    return dataclasses.replace(
        c, dim=dim, X=X, dx=1e-4,
        disp_bcs=[B.DispBC(clamp, (1 << dim) - 1, np.zeros((clamp.size, dim)))],
        tip_ids=B.layer_ids(idx, 0, counts[0] - 1, 1), lattice_index=idx, counts=counts)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision,tol", [(M.FP64, 1e-12), (M.MIXED, 1e-4)])
def test_tiny_bodies_every_stage(ctx, dim, precision, tol):
    """12 and 27 particles: one partial tile, owner groups of a few particles
    and levels of one to a few pairs, through every stage of one substep."""
    case = _tiny(dim)
    U = B.random_field(case.n, dim, 1e-3 * case.dx, 7)
    V = B.random_field(case.n, dim, 0.05, 8)
    dt = 0.6 * case.h_over_dx * case.dx / math.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    for upto in (1, 2, 3, 4):
        ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, precision)
        for b in (ob, gb):
            b.write(M.F_U, U)
            b.write(M.F_V, V)
        ob.substep_partial(dt, upto, ramp=0.5)
        gb.substep_partial(dt, upto, ramp=0.5)
        assert rel(gb.read(M.F_PB), ob.read(O.F_PB)) < tol
        assert rel(gb.read(M.F_V), ob.read(O.F_V)) < tol
        assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol


def _roller_cylinder():
    """Small J2 cylinder held by rollers: the left end slides freely in y and
    z (x prescribed), the right end is pulled in x only, and the bottom line
    of the left end is also held in y — every constrained pair has free axes."""
    c = B.cylinder3d(L=4e-3, R=1e-3, dx=0.25e-3, n_slow=10)
    idx = c.lattice_index
    nx = c.counts[0]
    left = B.layer_ids(idx, 0, 0, 2)
    right = B.layer_ids(idx, 0, nx - 2, 2)
    low = left[idx[left, 1] == idx[left, 1].min()]
    half = 0.15 * nx * c.dx
    ul = np.zeros((left.size, 3))
    ur = np.zeros((right.size, 3))
    ur[:, 0] = 2 * half
    bcs = [B.DispBC(left, 0b001, ul), B.DispBC(right, 0b001, ur, report_force=True),
           B.DispBC(low, 0b010, np.zeros((low.size, 3)))]
    return dataclasses.replace(c, disp_bcs=bcs)


@pytest.mark.parametrize("precision,tol", [(M.FP64, 1e-12), (M.MIXED, 1e-4)])
def test_roller_bcs_every_stage(ctx, precision, tol):
    """Partially constrained particles (rollers): the per-axis constrained
    damping update and the BC drift, one substep stage by stage."""
    case = _roller_cylinder()
    U = B.random_field(case.n, 3, 1e-3 * case.dx, 21)
    V = B.random_field(case.n, 3, 0.05, 22)
    dt = 0.6 * case.h_over_dx * case.dx / math.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    for upto in (3, 4):
        gb = M.body_from_case(ctx, case, precision)
        ob = O.body_from_case(case, damp_layout=gb.damping_layout())
        for b in (ob, gb):
            b.write(M.F_U, U)
            b.write(M.F_V, V)
        ob.substep_partial(dt, upto, ramp=0.5)
        gb.substep_partial(dt, upto, ramp=0.5)
        assert rel(gb.read(M.F_V), ob.read(O.F_V)) < tol
        assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol


def test_roller_bcs_slow_steps(ctx):
    case = _roller_cylinder()
    gb = M.body_from_case(ctx, case, M.FP64)
    ob = O.body_from_case(case, damp_layout=gb.damping_layout())
    for l in (1, 2):
        rg = gb.advance_slow_step(ramp=l / 10, ke_tol=-1, max_substeps=30)
        ro = ob.advance(ramp=l / 10, ke_tol=-1, max_substeps=30)
        assert rg.substeps == ro.substeps == 30
        assert abs(rg.end_force[0] - ro.end_force[0]) <= 1e-9 * abs(ro.end_force[0])
    assert rel(gb.read(M.F_U), ob.read(O.F_U)) < 1e-9
    assert rel(gb.read(M.F_V), ob.read(O.F_V)) < 1e-9


def test_roller_bcs_adjoint_dot_product(ctx):
    """<J dtheta, lambda> (PyTorch forward mode on the oracle's set-up) equals
    <dtheta, J^T lambda> from the GPU reverse mode with roller BCs, whose
    constrained pairs take the transposed per-axis update."""
    import torch
    from oracle import adjoint as A
    case = _roller_cylinder()
    rng = np.random.default_rng(9)
    lam = rng.normal(size=(case.n, 3))
    gb = M.body_from_case(ctx, case, M.FP64)
    p = dict(dt_slow=0.0, ramp=0.1, ke_tol=-1.0, ke_ref=case.plan.ke_ref, max_substeps=2,
             check_every=0)
    ck = gb.save_state()
    gb.advance_slow_step(**p)
    gb.adjoint_enable(2)
    gb.adjoint_seed(u_bar=lam)
    gb.load_state(ck)
    th_g = gb.adjoint_slow_step(2, **p)
    ob = O.body_from_case(case, damp_layout=gb.damping_layout())
    tb = A.TorchBody(case, ob)
    th0 = tb.theta0()
    dth = torch.from_numpy(rng.normal(size=7)) * th0.abs()
    dth[5] = dth[6] = 0.0

    def f(th):
        st, _, _, _ = tb.slow_step(tb.initial_state(), th, p["ramp"], 2)
        return tb.to_original(st[0])

    _, jv = torch.func.jvp(f, (th0,), (dth,))
    lhs = float((jv.numpy() * lam).sum())
    rhs = float((dth.numpy() * th_g).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_misaligned_allocator_is_refused():
    """An allocator hook whose pointers are off the 16-byte grid: body creation
    fails with an invalid-argument status and every block is given back."""
    import ctypes as C
    import torch
    live = {}

    def _alloc(nbytes, user):
        t = torch.empty(int(nbytes) + 16, dtype=torch.uint8, device="cuda")
        p = t.data_ptr() + 8
        live[p] = t
        return p

    def _release(ptr, nbytes, user):
        live.pop(ptr, None)

    cb = (M.Allocator.ALLOC(_alloc), M.Allocator.RELEASE(_release))
    al = M.Allocator(cb[0], cb[1], None)
    st = torch.cuda.Stream()
    h = C.c_void_p()
    assert M.lib().mts_ctx_create(0, C.c_void_p(st.cuda_stream), C.byref(al), C.byref(h)) == M.OK
    case = B.bar2d(nx=12, ny=4)
    X = np.ascontiguousarray(case.X, dtype=np.float64)
    desc = M.BodyDesc(2, M.MIXED, case.n, X.ctypes.data, case.dx, case.h_over_dx,
                      M.DAMP_AUTO, 0, (C.c_double * 3)(0.0, 0.0, 0.0))
    hb = C.c_void_p()
    s = M.lib().mts_body_create(h, C.byref(desc), C.byref(hb))
    st.synchronize()
    M.lib().mts_ctx_destroy(h)
    assert s == M.ERR_INVALID_ARG
    assert not live


@pytest.mark.parametrize("precision,tol", [(M.FP64, 1e-12), (M.MIXED, 3e-4)])
def test_wide_support_every_stage(ctx, precision, tol):
    """h = 1.8 dx in 3D: interior particles have up to 185 neighbours, more
    than the bank-balanced visiting order handles, so the tiles keep the CSR
    order for them; every stage of one substep still matches the oracle.
    FP64 at 1e-12 checks that every neighbour is visited exactly once.  Mixed
    precision: F = I + grad u held in FP32 has an absolute error of a few
    1e-8 per entry, i.e. about 1e-4 of grad u at these 1e-3 strains, before
    the rounding of sums 2.4 times longer than at h = 1.3 dx; hence 3e-4."""
    counts = (7, 7, 7)
    X, idx, _ = B.box_body(counts, 1e-4, seed=6, jitter=0.05)
    c = B.bar2d(nx=10, ny=4)
    clamp = B.layer_ids(idx, 0, 0, 1)
    case = dataclasses.replace(
        c, dim=3, X=X, dx=1e-4, h_over_dx=1.8,
        disp_bcs=[B.DispBC(clamp, 0b111, np.zeros((clamp.size, 3)))],
        tip_ids=B.layer_ids(idx, 0, counts[0] - 1, 1), lattice_index=idx, counts=counts)
    ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, precision)
    off, _ = ob.neighbors()
    assert np.diff(off).max() > 128
    U = B.random_field(case.n, 3, 1e-3 * case.dx, 17)
    V = B.random_field(case.n, 3, 0.05, 18)
    dt = 0.6 * case.h_over_dx * case.dx / math.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    for upto in (1, 2, 4):
        ob, gb = O.body_from_case(case), M.body_from_case(ctx, case, precision)
        for b in (ob, gb):
            b.write(M.F_U, U)
            b.write(M.F_V, V)
        ob.substep_partial(dt, upto, ramp=0.5)
        gb.substep_partial(dt, upto, ramp=0.5)
        assert rel(gb.read(M.F_PB), ob.read(O.F_PB)) < tol
        assert rel(gb.read(M.F_V), ob.read(O.F_V)) < tol
        assert rel(gb.read(M.F_U), ob.read(O.F_U)) < tol


def test_write_rejects_one_nonfinite_value(ctx):
    """A single infinity deep inside an otherwise finite field is found (its
    index is reported) and the field is left as it was."""
    case = B.bar2d(nx=200, ny=20)         # 8,000 values
    gb = M.body_from_case(ctx, case, M.MIXED)
    before = gb.read(M.F_U)
    U = B.random_field(case.n, 2, 1e-6, 31)
    k = 2 * case.n - 7                    # flat index, near the end of the field
    U.reshape(-1)[k] = -np.inf
    with pytest.raises(M.MtsError) as e:
        gb.write(M.F_U, U)
    assert e.value.status == M.ERR_NONFINITE
    assert f"at {k}" in str(e.value)
    assert np.array_equal(gb.read(M.F_U), before)
    U.reshape(-1)[k] = 0.0
    gb.write(M.F_U, U)
    assert np.array_equal(gb.read(M.F_U), U)


def test_integer_conversions_match_hardware(ctx):
    """The mixed-precision drift and force kernels convert between FP32 and
    FP64 with integer operations (IEEE 754 formats, round to nearest even);
    on 16 M hashed bit patterns steered into subnormals, zeros, infinities,
    NaNs, overflow and exact ties they give the hardware's bits."""
    for seed in (1, 2):
        assert M.selftest_conversions(ctx, 1 << 24, seed) == (0, 0)
