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
