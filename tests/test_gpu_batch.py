"""Batched advance (many bodies, one graph launch per slow step) on the GPU:
every body of a batch computes exactly what it computes alone (bit-exact),
and a batch member matches the FP64 oracle like a single body does."""
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


def _cases():
    """Uneven members: small strips (diffusion + swelling) and J2 bars from the
    batched-workload generator, plus a 3D J2 cylinder."""
    cs = B.batch_instances(count=4, n_min=400, n_max=3000, seed=B.SEED_BASE + 50)
    cs.append(B.cylinder3d(L=4e-3, R=1e-3, dx=0.25e-3, n_slow=10))
    return cs


def _params(case, l):
    p = dict(ramp=l / max(case.plan.n_ramp, 1), ke_tol=case.plan.ke_tol, ke_ref=case.plan.ke_ref,
             ke_mode=case.plan.ke_mode, max_substeps=300)
    if case.diffusion is not None:
        p.update(dt_slow=None)
    return p


def _fill_dt(body, p):
    if p.get("dt_slow", 0.0) is None:
        p["dt_slow"] = body.diffusion_dt()[1]
    return p


@pytest.mark.parametrize("precision", [M.FP64, M.MIXED])
def test_batch_equals_single_bodies(ctx, precision):
    cases = _cases()
    solo = [M.body_from_case(ctx, c, precision) for c in cases]
    mem = [M.body_from_case(ctx, c, precision) for c in cases]
    bt = M.Batch(ctx, mem)
    for l in (1, 2, 3):
        ps = [_fill_dt(b, _params(c, l)) for b, c in zip(mem, cases)]
        reps = bt.advance(ps)
        for b, c, p, r in zip(solo, cases, ps, reps):
            rs = b.advance_slow_step(**p)
            assert r.substeps == rs.substeps and r.converged == rs.converged
            assert r.ke_final == rs.ke_final and r.dt_last == rs.dt_last
            assert list(r.end_force) == list(rs.end_force)
            assert list(r.tip_deflection) == list(rs.tip_deflection)
    sub = [r.substeps for r in reps]
    assert len(set(sub)) > 1            # members stopped on their own criteria
    for a, b in zip(mem, solo):
        assert np.array_equal(a.read(M.F_U), b.read(M.F_U))
        assert np.array_equal(a.read(M.F_V), b.read(M.F_V))
        assert np.array_equal(a.read(M.F_C), b.read(M.F_C))
    bt.close()


def test_batch_member_matches_oracle(ctx):
    cases = _cases()
    mem = [M.body_from_case(ctx, c, M.FP64) for c in cases]
    bt = M.Batch(ctx, mem)
    k = len(cases) - 1                                  # the 3D cylinder
    ob = O.body_from_case(cases[k], damp_layout=mem[k].damping_layout())
    for l in (1, 2):
        ps = [_fill_dt(b, _params(c, l)) for b, c in zip(mem, cases)]
        reps = bt.advance(ps)
        ob.advance(ramp=ps[k]["ramp"], ke_tol=-1.0, max_substeps=reps[k].substeps)
    u_o = ob.read(O.F_U)
    assert np.max(np.abs(mem[k].read(M.F_U) - u_o)) / np.max(np.abs(u_o)) < 1e-9
    bt.close()


def test_batch_rejects_bad_members(ctx):
    c = B.bar2d(nx=12, ny=5)
    a, b = M.body_from_case(ctx, c), M.body_from_case(ctx, c)
    with pytest.raises(M.MtsError):
        M.Batch(ctx, [a, a])
    other = M.Context(0)
    z = M.body_from_case(other, c)
    with pytest.raises(M.MtsError):
        M.Batch(ctx, [a, z])
    with pytest.raises(M.MtsError):
        M.Batch(ctx, [])
    bt = M.Batch(ctx, [a, b])
    with pytest.raises(ValueError):
        bt.advance([{}])
    bt.close()
    other.close()
