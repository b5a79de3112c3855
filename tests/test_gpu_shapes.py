"""Launch shapes and their autotuner: damping warps per CTA never change the
results; other tile sizes still match the oracle and give the same results
however they were set; the autotuner restores the state, and a body created
with its choice reproduces the tuned body bit for bit (also in a batch)."""
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


def small_cylinder():
    return B.cylinder3d(L=5e-3, R=1.25e-3, dx=0.25e-3, n_slow=20)


def _slow_steps(gb, case, n=2, sub=25):
    for l in range(1, n + 1):
        gb.advance_slow_step(ramp=l / case.plan.n_ramp, ke_tol=-1, ke_ref=case.plan.ke_ref,
                             max_substeps=sub)
    return gb.read(M.F_U), gb.read(M.F_V)


@pytest.mark.parametrize("precision", [M.FP64, M.MIXED])
def test_damping_warps_do_not_change_results(ctx, precision):
    case = small_cylinder()
    ref = None
    for w in (1, 2, 4):
        gb = M.body_from_case(ctx, case, precision)
        gb.set_shapes(0, w)
        assert gb.shapes()["damp_warps"] == w
        u, v = _slow_steps(gb, case)
        if ref is None:
            ref = (u, v)
        else:
            assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1])
        gb.close()


@pytest.mark.parametrize("precision,tiles,tol", [(M.FP64, (64, 128), 1e-9),
                                                 (M.MIXED, (256, 512), 1e-4)])
def test_tile_sizes_match_oracle_and_each_other(ctx, precision, tiles, tol):
    case = small_cylinder()
    ob = O.body_from_case(case)
    for l in (1, 2):
        ob.advance(ramp=l / case.plan.n_ramp, ke_tol=-1, max_substeps=25)
    for t in tiles:
        made = M.body_from_case(ctx, case, precision, tile=t)        # chosen at creation
        assert made.shapes()["tile"] == t
        reset = M.body_from_case(ctx, case, precision)                # re-tiled afterwards
        reset.set_shapes(t, 0)
        assert reset.shapes()["tile"] == t
        u1, v1 = _slow_steps(made, case)
        u2, v2 = _slow_steps(reset, case)
        assert np.array_equal(u1, u2) and np.array_equal(v1, v2)
        assert rel(u1, ob.read(O.F_U)) < tol
        made.close()
        reset.close()


def test_shapes_reject_bad_values(ctx):
    case = small_cylinder()
    g64 = M.body_from_case(ctx, case, M.FP64)
    g32 = M.body_from_case(ctx, case, M.MIXED)
    for b, t, w in ((g32, 100, 0), (g32, 1024, 0), (g32, 0, 3), (g64, 256, 0)):
        with pytest.raises(M.MtsError) as e:
            b.set_shapes(t, w)
        assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MtsError) as e:
        g32.autotune(substeps=0)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MtsError) as e:
        M.Body(ctx, case.X, case.dx, precision=M.FP64, tile=512)
    assert e.value.status == M.ERR_INVALID_ARG


def test_autotune_restores_state_and_is_reproducible(ctx):
    case = small_cylinder()
    tuned = M.body_from_case(ctx, case, M.MIXED)
    _slow_steps(tuned, case, n=1)
    u0, v0 = tuned.read(M.F_U), tuned.read(M.F_V)
    choice = tuned.autotune(substeps=6, ramp=2 / case.plan.n_ramp)
    assert choice["tile"] in (256, 512) and choice["damp_warps"] in (1, 2, 4) and choice["ms"] > 0
    assert tuned.shapes() == {"tile": choice["tile"], "damp_warps": choice["damp_warps"]}
    assert np.array_equal(tuned.read(M.F_U), u0) and np.array_equal(tuned.read(M.F_V), v0)
    other = M.body_from_case(ctx, case, M.MIXED)          # the same history, then the choice
    _slow_steps(other, case, n=1)
    other.set_shapes(choice["tile"], choice["damp_warps"])
    for g in (tuned, other):
        g.advance_slow_step(ramp=2 / case.plan.n_ramp, ke_tol=-1, max_substeps=25)
    assert np.array_equal(tuned.read(M.F_U), other.read(M.F_U))
    assert np.array_equal(tuned.read(M.F_V), other.read(M.F_V))


def test_batch_autotune_matches_single_bodies(ctx):
    cases = [B.bar2d(nx=40, ny=8), B.bar2d(nx=64, ny=12), small_cylinder()]
    bodies = [M.body_from_case(ctx, c, M.MIXED) for c in cases]
    bt = M.Batch(ctx, bodies)
    shapes = bt.autotune(substeps=4, ramp=0.05)
    assert len(shapes) == 3
    params = [dict(ramp=0.05, ke_tol=-1, max_substeps=30) for _ in cases]
    bt.advance(params)
    for c, b, sh in zip(cases, bodies, shapes):
        single = M.body_from_case(ctx, c, M.MIXED, tile=sh["tile"])
        single.set_shapes(0, sh["damp_warps"])
        single.advance_slow_step(ramp=0.05, ke_tol=-1, max_substeps=30)
        assert np.array_equal(single.read(M.F_U), b.read(M.F_U))
        single.close()
    bt.close()


def test_one_launch_damping_equals_multi_launch():
    """A body with many damping groups per SM (the 2.5 M-particle plate) runs
    its damping sweep as one launch with a task queue; the same body with the
    multi-launch form (MTS_DAMP_MULTILAUNCH=1) gives the same bits: every task
    computes what its group computes in its colour launch."""
    import os
    ctx = M.Context(0)
    case = B.plate3d()
    out = []
    for multi in (False, True):
        if multi:
            os.environ["MTS_DAMP_MULTILAUNCH"] = "1"
        try:
            gb = M.body_from_case(ctx, case, M.MIXED)
            dts = gb.diffusion_dt()[1]
            for _ in range(2):
                r = gb.advance_slow_step(dt_slow=dts, ke_tol=-1.0, ke_ref=case.plan.ke_ref,
                                         ke_mode=1, max_substeps=12)
                assert r.substeps == 12
            out.append((gb.read(M.F_U), gb.read(M.F_V), r.kernel_launches))
            gb.close()
        finally:
            os.environ.pop("MTS_DAMP_MULTILAUNCH", None)
    (u1, v1, k1), (u2, v2, k2) = out
    assert k1 < k2                     # the one-launch form really ran
    assert np.array_equal(u1, u2) and np.array_equal(v1, v2)
    ctx.close()
