"""Reverse mode on the GPU (FP64) against the reverse-mode oracle
(oracle/adjoint.py, itself pinned to the C oracle by central differences):
parameter gradients and initial-state adjoints of an objective of the tip
deflection, the end force and the final displacement, over slow steps with
the substep sizes of the forward run held fixed."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import adjoint as A
from paper_2309_04010_gb300 import mtssph as M
from synth import bodies as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def small_cylinder():
    return B.cylinder3d(L=4e-3, R=1e-3, dx=0.25e-3, n_slow=10)


def small_strip():
    c = B.strip2d(nx=36, ny=10, dx=1e-5)
    c.eta = 1.0
    return c


def small_bar():
    return B.bar2d(nx=24, ny=6, n_slow=4)


CASES = {"cyl3d_j2": (small_cylinder, 2, 8), "strip2d_swelling": (small_strip, 2, 6),
         "bar2d_svk": (small_bar, 2, 12)}


def _weights(case, seed=11):
    rng = np.random.default_rng(seed)
    d = case.dim
    return rng.normal(size=d), rng.normal(size=d), rng.normal(size=(case.n, d))


def _steps(case, gb, nslow, nsub):
    dts = gb.diffusion_dt()[1] if case.diffusion is not None else 0.0
    return [dict(dt_slow=dts, ramp=l / max(case.plan.n_ramp, 1), ke_tol=-1.0,
                 ke_ref=case.plan.ke_ref, max_substeps=nsub, check_every=0)
            for l in range(1, nslow + 1)]


def _gpu_gradient(ctx, case, nslow, nsub, w_tip, w_f, r, precision=M.FP64):
    gb = M.body_from_case(ctx, case, precision)
    steps = _steps(case, gb, nslow, nsub)
    ckpts, counts = [], []
    for p in steps:
        ckpts.append(gb.save_state())
        counts.append(gb.advance_slow_step(**p).substeps)
    u_end = gb.read(M.F_U)
    gb.adjoint_enable(max(counts))
    gb.adjoint_seed(u_bar=r, tip_bar=w_tip, force_bar=w_f)
    th = np.zeros(7)
    for p, ck, k in zip(reversed(steps), reversed(ckpts), reversed(counts)):
        gb.load_state(ck)
        th += gb.adjoint_slow_step(k, **p)
    return gb, th, steps, u_end


def _oracle_gradient(case, gb, steps, nsub, w_tip, w_f, r):
    ob = O.body_from_case(case, damp_layout=gb.damping_layout())
    tb = A.TorchBody(case, ob)
    th = tb.theta0().clone().requires_grad_(True)
    st0 = list(tb.initial_state())
    u0 = st0[0].clone().requires_grad_(True)
    st = (u0, *st0[1:])
    ef = tip = None
    for p in steps:
        st, ef, tip, _ = tb.slow_step(st, th, p["ramp"], nsub, dt_slow=p["dt_slow"])
    L = (torch.from_numpy(w_tip) * tip).sum() + (torch.from_numpy(w_f) * ef).sum() + (
        torch.from_numpy(r) * tb.to_original(st[0])).sum()
    g_th, g_u0 = torch.autograd.grad(L, (th, u0))
    return g_th.numpy(), tb.to_original(g_u0).numpy(), tb.to_original(st[0]).detach().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_reverse_mode_oracle(ctx, name):
    make, nslow, nsub = CASES[name]
    case = make()
    w_tip, w_f, r = _weights(case)
    gb, th_g, steps, u_end = _gpu_gradient(ctx, case, nslow, nsub, w_tip, w_f, r)
    th_o, u0_o, u_o = _oracle_gradient(case, gb, steps, nsub, w_tip, w_f, r)
    assert np.max(np.abs(u_end - u_o)) <= 1e-11 * np.max(np.abs(u_o))   # same forward run
    used = [0] if case.material.model == "svk" else [0, 1, 2, 3, 4]
    if case.diffusion is not None:
        used += [5, 6]
    for k in used:
        assert abs(th_g[k] - th_o[k]) <= 1e-8 * max(abs(th_o[k]), 1e-300), (
            A.THETA_NAMES[k], th_g[k], th_o[k])
        assert th_o[k] != 0.0, A.THETA_NAMES[k]
    u0_g = gb.read_adjoint(M.F_U)
    assert np.max(np.abs(u0_g - u0_o)) <= 1e-8 * np.max(np.abs(u0_o))


def test_adjoint_dot_product_one_substep(ctx):
    """<J dtheta, lambda> from the oracle's forward-mode derivative equals
    <dtheta, J^T lambda> from the GPU reverse mode, for one substep of the
    J2 cylinder (lambda on the final displacement)."""
    case = small_cylinder()
    rng = np.random.default_rng(5)
    lam = rng.normal(size=(case.n, case.dim))
    gb = M.body_from_case(ctx, case, M.FP64)
    p = _steps(case, gb, 1, 1)[0]
    ck = gb.save_state()
    gb.advance_slow_step(**p)
    gb.adjoint_enable(1)
    gb.adjoint_seed(u_bar=lam)
    gb.load_state(ck)
    th_g = gb.adjoint_slow_step(1, **p)
    ob = O.body_from_case(case, damp_layout=gb.damping_layout())
    tb = A.TorchBody(case, ob)
    th0 = tb.theta0()
    dth = torch.from_numpy(rng.normal(size=7)) * th0.abs()
    dth[5] = dth[6] = 0.0

    def f(th):
        st, _, _, _ = tb.slow_step(tb.initial_state(), th, p["ramp"], 1)
        return tb.to_original(st[0])

    _, jv = torch.func.jvp(f, (th0,), (dth,))
    lhs = float((jv.numpy() * lam).sum())
    rhs = float((dth.numpy() * th_g).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_adjoint_central_differences_on_gpu(ctx):
    """The GPU's own forward runs, differenced in E and sigma_inf with fixed
    substep size, against the GPU reverse mode."""
    case = small_cylinder()
    w_tip, w_f, r = _weights(case, seed=3)
    gb0 = M.body_from_case(ctx, case, M.FP64)
    dt_sub = 0.5 * 0.6 * case.h_over_dx * case.dx / np.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    steps = [dict(ramp=l / case.plan.n_ramp, ke_tol=-1.0, max_substeps=6, dt_sub=dt_sub)
             for l in (1, 2)]

    def objective(theta):
        gb = M.body_from_case(ctx, case, M.FP64)
        gb.set_parameters(theta)
        rep = None
        for p in steps:
            rep = gb.advance_slow_step(**p)
        d = case.dim
        return (w_tip @ np.array(rep.tip_deflection[:d]) + w_f @ np.array(rep.end_force[:d]) +
                float((r * gb.read(M.F_U)).sum()))

    ckpts = []
    for p in steps:
        ckpts.append(gb0.save_state())
        gb0.advance_slow_step(**p)
    gb0.adjoint_enable(6)
    gb0.adjoint_seed(u_bar=r, tip_bar=w_tip, force_bar=w_f)
    th = np.zeros(7)
    for p, ck in zip(reversed(steps), reversed(ckpts)):
        gb0.load_state(ck)
        th += gb0.adjoint_slow_step(6, **p)
    theta0 = gb0.parameters()
    for k in (0, 2):
        h = 1e-6 * abs(theta0[k])
        tp, tm = theta0.copy(), theta0.copy()
        tp[k] += h
        tm[k] -= h
        fd = (objective(tp) - objective(tm)) / (2 * h)
        assert abs(th[k] - fd) <= 2e-6 * max(abs(fd), abs(th[k])), (A.THETA_NAMES[k], th[k], fd)


def test_autograd_function_wraps_the_reverse_mode(ctx):
    case = small_bar()
    gb = M.body_from_case(ctx, case, M.FP64)
    steps = _steps(case, gb, 2, 10)
    theta = torch.tensor(gb.parameters(), dtype=torch.float64, requires_grad=True)
    ck = gb.save_state()
    out = M.slow_steps(gb, theta, steps)
    w = torch.tensor([0.3, -0.2, 1.1, 0.4], dtype=torch.float64)
    (g,) = torch.autograd.grad((out * w).sum(), theta)
    # the same through the explicit calls
    gb2 = M.body_from_case(ctx, case, M.FP64)
    ckpts, counts = [], []
    for p in steps:
        ckpts.append(gb2.save_state())
        counts.append(gb2.advance_slow_step(**p).substeps)
    gb2.adjoint_enable(max(counts))
    gb2.adjoint_seed(tip_bar=w[:2].numpy(), force_bar=w[2:].numpy())
    th = np.zeros(7)
    for p, c, k in zip(reversed(steps), reversed(ckpts), reversed(counts)):
        gb2.load_state(c)
        th += gb2.adjoint_slow_step(k, **p)
    assert np.array_equal(g.numpy(), th)
    assert g[0] != 0
    gb.load_state(ck)


def test_adjoint_errors(ctx):
    case = small_bar()
    aniso = B.beam_droplet2d(L=1e-3, aniso=4.0)
    ga = M.body_from_case(ctx, aniso, M.MIXED)
    with pytest.raises(M.MtsError) as e:
        ga.adjoint_enable(4)
    assert e.value.status == M.ERR_STATE
    gm = M.body_from_case(ctx, case, M.MIXED)
    with pytest.raises(M.MtsError) as e:
        gm.adjoint_slow_step(2, ramp=0.1)
    assert e.value.status == M.ERR_STATE
    gb = M.body_from_case(ctx, case, M.FP64)
    with pytest.raises(M.MtsError) as e:
        gb.adjoint_slow_step(2, ramp=0.1)
    assert e.value.status == M.ERR_STATE
    gb.adjoint_enable(3)
    with pytest.raises(M.MtsError) as e:
        gb.adjoint_slow_step(5, ramp=0.1)
    assert e.value.status == M.ERR_INVALID_ARG


def test_equilibrium_adjoint_matches_differences_of_equilibria(ctx):
    """Implicit-function adjoint at a relaxed equilibrium (SVK bar) against
    central differences of equilibria relaxed to machine precision."""
    case = B.bar2d(nx=24, ny=6, n_slow=4, eta=1e3)   # relaxes in ~1e4 substeps (1e4: overdamped)
    w_tip, w_f, r = _weights(case, seed=8)
    p = dict(ramp=1.0 / case.plan.n_ramp, ke_tol=1e-26, ke_ref=case.plan.ke_ref,
             max_substeps=60000)

    def objective(theta):
        gb = M.body_from_case(ctx, case, M.FP64)
        gb.set_parameters(theta)
        rep = gb.advance_slow_step(**p)
        d = case.dim
        val = (w_tip @ np.array(rep.tip_deflection[:d]) + w_f @ np.array(rep.end_force[:d]) +
               float((r * gb.read(M.F_U)).sum()))
        return val, gb

    J0, gb = objective(M.body_from_case(ctx, case, M.FP64).parameters())
    gb.adjoint_enable(1)
    gb.adjoint_seed(u_bar=r, tip_bar=w_tip, force_bar=w_f)
    th, iters = gb.adjoint_equilibrium(max_iters=100000, tol=1e-10)
    assert iters > 10
    theta0 = gb.parameters()
    h = 1e-5 * theta0[0]
    tp, tm = theta0.copy(), theta0.copy()
    tp[0] += h
    tm[0] -= h
    fd = (objective(tp)[0] - objective(tm)[0]) / (2 * h)
    assert abs(th[0] - fd) <= 1e-5 * abs(fd), (th[0], fd)


def test_equilibrium_adjoint_with_end_force_seed_only(ctx):
    """A seed on the end force alone (nothing in u-bar, v-bar at the start)
    converges and agrees with the unrolled reverse of the same relaxed step."""
    case = B.bar2d(nx=24, ny=6, n_slow=4, eta=1e3)
    gb = M.body_from_case(ctx, case, M.FP64)
    ck = gb.save_state()
    p = dict(ramp=0.25, ke_tol=1e-22, ke_ref=case.plan.ke_ref, max_substeps=60000)
    k = gb.advance_slow_step(**p).substeps
    gb.adjoint_enable(k)
    gb.adjoint_seed(force_bar=[1.0, 0.0])
    th_eq, iters = gb.adjoint_equilibrium(max_iters=200000, tol=1e-10)
    assert iters > 8
    gb.adjoint_reset()
    gb.adjoint_seed(force_bar=[1.0, 0.0])
    gb.load_state(ck)
    th_un = gb.adjoint_slow_step(k, **p)
    assert th_un[0] != 0
    assert abs(th_eq[0] - th_un[0]) <= 1e-5 * abs(th_un[0]), (th_eq[0], th_un[0])


def _oracle_relaxed_objective(case, theta, w_tip, w_f, r, relax, c_field=None):
    """The objective at the oracle's relaxed equilibrium with parameters theta
    = (E, sigma0, sigma_inf, delta, H, D, beta) (nu fixed)."""
    ob = O.body_from_case(case)
    m = case.material
    ob.set_material(O.SVK if m.model == "svk" else O.J2, m.rho0, theta[0], m.nu, theta[1],
                    theta[2], theta[3], theta[4])
    if case.diffusion is not None:
        ob.set_diffusion(theta[5], theta[6], case.diffusion[2])
    if c_field is not None:
        ob.write(O.F_C, c_field)
    rep = ob.advance(**relax)
    assert rep.converged == 1
    d = case.dim
    return (w_tip @ np.array(rep.tip_deflection[:d]) + w_f @ np.array(rep.end_force[:d]) +
            float((r * ob.read(O.F_U)).sum()))


@pytest.mark.parametrize("which", ["E", "beta"])
def test_equilibrium_adjoint_matches_oracle_differences(ctx, which):
    """The implicit-function adjoint of a relaxed equilibrium against central
    differences of the ORACLE's equilibria, relaxed to machine precision, for
    the parameters the mechanical equilibrium depends on: Young's modulus (an
    SVK bar pulled at its grip) and the swelling coefficient (a cantilever
    strip with a prescribed through-thickness concentration, damping near the
    critical value of its flexural mode).  The hardening parameters act only
    through the plastic history and D only through the diffusion step, which
    the equilibrium adjoint leaves out."""
    if which == "E":
        case = B.bar2d(nx=24, ny=6, n_slow=4, eta=1e3)
        c_field, k, rel_h, tol = None, 0, 1e-5, 1e-5
        relax = dict(ramp=1.0 / case.plan.n_ramp, ke_tol=1e-26, ke_ref=case.plan.ke_ref,
                     ke_mode=0, max_substeps=200000)
    else:
        case = B.strip2d(nx=30, ny=8, dx=1e-5, beta=1e-3, eta=1.0)
        c_field = (case.lattice_index[:, 1] + 0.5) / case.counts[1]
        k, rel_h, tol = 6, 1e-3, 1e-4          # the response is nearly linear in beta
        K = case.material.E / (3 * (1 - 2 * case.material.nu))
        relax = dict(ramp=0.0, ke_tol=1e-22, ke_ref=3 * K * case.diffusion[1], ke_mode=1,
                     max_substeps=200000)
    w_tip, w_f, r = _weights(case, seed=8)
    r *= 1e-3
    gb = M.body_from_case(ctx, case, M.FP64)
    if c_field is not None:
        gb.write(M.F_C, c_field)
    theta0 = gb.parameters()
    rep = gb.advance_slow_step(**relax)
    assert rep.converged == 1
    gb.adjoint_enable(1)
    gb.adjoint_seed(u_bar=r, tip_bar=w_tip, force_bar=w_f)
    th, iters = gb.adjoint_equilibrium(max_iters=400000, tol=1e-11)
    gb.close()
    h = rel_h * theta0[k]
    tp, tm = theta0.copy(), theta0.copy()
    tp[k] += h
    tm[k] -= h
    fd = (_oracle_relaxed_objective(case, tp, w_tip, w_f, r, relax, c_field) -
          _oracle_relaxed_objective(case, tm, w_tip, w_f, r, relax, c_field)) / (2 * h)
    assert fd != 0
    assert abs(th[k] - fd) <= tol * abs(fd), (which, th[k], fd)


# --------------------------------------------------------------------------
# Mixed precision: FP32 forward, FP64 reverse about the FP32 trajectory
# --------------------------------------------------------------------------
# Tolerance.  The mixed forward run differs from the FP64 one by the FP32
# rounding of the per-particle arithmetic: here <= 1e-5 relative in u (the
# parity tests bound it by 1e-4).  The reverse mode is the exact FP64
# transpose of the linearisation about that trajectory, so its gradient
# differs from the oracle's (the FP64 trajectory) by the change of the
# Jacobian between the two linearisation points: of the same relative order
# as the state difference times the relative curvature of the maps, well
# below 1e-3 for these small-strain steps.  1e-3 is therefore the bound
# tested, for every parameter the objective depends on and for the adjoint
# of the initial displacement.
MIXED_ADJ_TOL = 1e-3


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_adjoint_matches_reverse_mode_oracle(ctx, name):
    make, nslow, nsub = CASES[name]
    case = make()
    w_tip, w_f, r = _weights(case)
    gb, th_g, steps, u_end = _gpu_gradient(ctx, case, nslow, nsub, w_tip, w_f, r, M.MIXED)
    th_o, u0_o, u_o = _oracle_gradient(case, gb, steps, nsub, w_tip, w_f, r)
    assert np.max(np.abs(u_end - u_o)) <= 1e-4 * np.max(np.abs(u_o))   # FP32 forward run
    used = [0] if case.material.model == "svk" else [0, 1, 2, 3, 4]
    if case.diffusion is not None:
        used += [5, 6]
    for k in used:
        assert abs(th_g[k] - th_o[k]) <= MIXED_ADJ_TOL * abs(th_o[k]), (
            A.THETA_NAMES[k], th_g[k], th_o[k])
    u0_g = gb.read_adjoint(M.F_U)
    assert np.max(np.abs(u0_g - u0_o)) <= MIXED_ADJ_TOL * np.max(np.abs(u0_o))


def test_mixed_batch_members_reverse_mode(ctx):
    """Four uneven members of the batched workload (two swelling strips, two
    J2 bars) advanced together in mixed precision by batch launches, then
    each member's slow steps reversed: gradients of tip deflection and end
    force with respect to every parameter its objective depends on, against
    the reverse-mode oracle run with the members' substep counts."""
    cases = B.batch_instances(count=4, n_min=400, n_max=1500, seed=B.SEED_BASE + 51)
    for c in cases:
        c.eta = 1.0 if c.diffusion is not None else c.eta
    bodies = [M.body_from_case(ctx, c, M.MIXED) for c in cases]
    bt = M.Batch(ctx, bodies)
    nsub = 8
    ck = [[] for _ in cases]
    steps = []
    for l in (1, 2):
        ps = []
        for c, b in zip(cases, bodies):
            p = dict(dt_slow=b.diffusion_dt()[1] if c.diffusion is not None else 0.0,
                     ramp=l / max(c.plan.n_ramp, 1), ke_tol=-1.0, ke_ref=c.plan.ke_ref,
                     max_substeps=nsub, check_every=0)
            ps.append(p)
        for k, b in enumerate(bodies):
            ck[k].append(b.save_state())
        reps = bt.advance(ps)
        assert all(r.substeps == nsub for r in reps)
        steps.append(ps)
    bt.close()
    for k, (c, b) in enumerate(zip(cases, bodies)):
        w_tip, w_f, _ = _weights(c, seed=20 + k)
        r = np.zeros((c.n, c.dim))
        b.adjoint_enable(nsub)
        b.adjoint_seed(tip_bar=w_tip, force_bar=w_f)
        th = np.zeros(7)
        for l in (1, 0):
            b.load_state(ck[k][l])
            th += b.adjoint_slow_step(nsub, **steps[l][k])
        th_o, _, _ = _oracle_gradient(c, b, [steps[0][k], steps[1][k]], nsub, w_tip, w_f, r)
        used = [0] if c.material.model == "svk" else [0, 1, 2, 3, 4]
        if c.diffusion is not None:
            used += [5, 6]
        for q in used:
            assert abs(th[q] - th_o[q]) <= MIXED_ADJ_TOL * abs(th_o[q]), (
                c.name, A.THETA_NAMES[q], th[q], th_o[q])
        b.close()
