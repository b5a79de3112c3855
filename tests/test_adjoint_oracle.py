"""Pins of the reverse-mode oracle (oracle/adjoint.py) against the C oracle:
its forward restatement reproduces the C oracle's slow steps, and its
gradients with respect to the material and diffusion parameters match central
differences of the C oracle run with fixed substep sizes (frozen counts)."""
import copy
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from oracle import adjoint as A
from synth import bodies as B


def small_cylinder():
    """3D J2 cylinder, 3 % stretch per slow step: plastic from the first step."""
    return B.cylinder3d(L=4e-3, R=1e-3, dx=0.25e-3, n_slow=10)


def small_strip():
    c = B.strip2d(nx=36, ny=10, dx=1e-5)
    c.eta = 1.0
    return c


def with_theta(case, th):
    """Copy of a case with the parameters THETA_NAMES set to th."""
    c = copy.deepcopy(case)
    E, s0, sinf, delta, H, D, beta = [float(x) for x in th]
    c.material = dataclasses.replace(c.material, E=E, sigma0=s0, sigma_inf=sinf, delta=delta, H=H)
    if c.diffusion is not None:
        c.diffusion = (D, beta, c.diffusion[2])
    return c


def run_c(case, steps, nsub, dt_sub=0.0, dts=None):
    """C oracle: `steps` slow steps of nsub substeps each (diffusion steps of
    size dts, default the stable size, for swelling cases)."""
    ob = O.body_from_case(case)
    if dts is None:
        dts = ob.diffusion_dt()[1] if case.diffusion is not None else 0.0
    rep = None
    for l in range(1, steps + 1):
        rep = ob.advance(dt_slow=dts, ramp=l / max(case.plan.n_ramp, 1), ke_tol=-1.0,
                         max_substeps=nsub, dt_sub=dt_sub)
    return ob, rep, dts


def run_torch(tb, th, steps, nsub, dts_slow, dt_sub=0.0):
    st = tb.initial_state()
    out = None
    for l in range(1, steps + 1):
        st, ef, tip, _ = tb.slow_step(st, th, l / max(tb.case.plan.n_ramp, 1), nsub, dt_slow=dts_slow,
                                      dt_override=dt_sub)
        out = (ef, tip)
    return st, out


@pytest.mark.parametrize("make", [small_cylinder, small_strip])
def test_torch_restatement_matches_c_oracle(make):
    case = make()
    ob, rep, dts = run_c(case, 2, 12)
    tb = A.TorchBody(case, O.body_from_case(case))
    st, (ef, tip) = run_torch(tb, tb.theta0(), 2, 12, dts)
    u = tb.to_original(st[0]).numpy()
    uo = ob.read(O.F_U)
    assert np.max(np.abs(u - uo)) <= 1e-11 * np.max(np.abs(uo))
    assert np.max(np.abs(tb.to_original(st[3]).numpy() - ob.read(O.F_ALPHA))) <= 1e-11 * max(
        1e-30, np.max(np.abs(ob.read(O.F_ALPHA))))
    assert np.max(np.abs(tb.to_original(st[4]).numpy() - ob.read(O.F_C))) <= 1e-12
    d = case.dim
    assert np.allclose(ef.numpy(), np.array(rep.end_force[:d]), rtol=1e-10, atol=1e-12 * max(
        1.0, np.max(np.abs(rep.end_force[:d]))))
    assert np.allclose(tip.numpy(), np.array(rep.tip_deflection[:d]), rtol=1e-10, atol=1e-18)
    if case.material.model == "j2":
        assert ob.read(O.F_ALPHA).max() > 0


def _objective_weights(case, seed=7):
    rng = np.random.default_rng(seed)
    d = case.dim
    return rng.normal(size=d), rng.normal(size=d), rng.normal(size=(case.n, d))


@pytest.mark.parametrize("make,which", [(small_cylinder, (0, 1, 2, 3, 4)),
                                        (small_strip, (0, 5, 6))])
def test_torch_gradient_matches_c_oracle_differences(make, which):
    """d/d theta of w_tip . tip + w_f . end_force + sum r . u after two slow
    steps, fixed substep and diffusion step sizes (so the C oracle's counts and
    sizes do not move under the perturbation)."""
    case = make()
    steps, nsub = 2, 10
    probe = O.body_from_case(case)
    dt_sub = 0.5 * 0.6 * case.h_over_dx * case.dx / np.sqrt(
        case.material.E / (3 * (1 - 2 * case.material.nu)) / case.material.rho0)
    # half the stable diffusion step: stays stable under the perturbation of D
    dts = 0.5 * probe.diffusion_dt()[1] if case.diffusion is not None else 0.0
    w_tip, w_f, r = _objective_weights(case)
    tb = A.TorchBody(case, probe)
    th = tb.theta0().clone().requires_grad_(True)
    st, (ef, tip) = run_torch(tb, th, steps, nsub, dts, dt_sub)
    u_orig = tb.to_original(st[0])
    L = (torch.from_numpy(w_tip) * tip).sum() + (torch.from_numpy(w_f) * ef).sum() + (
        torch.from_numpy(r) * u_orig).sum()
    (grad,) = torch.autograd.grad(L, th)

    def objective(thv):
        ob, rep, _ = run_c(with_theta(case, thv), steps, nsub, dt_sub, dts)
        d = case.dim
        return (w_tip @ np.array(rep.tip_deflection[:d]) + w_f @ np.array(rep.end_force[:d]) +
                float((r * ob.read(O.F_U)).sum()))

    th0 = tb.theta0().numpy()
    for k in which:
        hstep = 1e-6 * abs(th0[k])
        tp, tm = th0.copy(), th0.copy()
        tp[k] += hstep
        tm[k] -= hstep
        fd = (objective(tp) - objective(tm)) / (2 * hstep)
        scale = max(abs(fd), abs(float(grad[k])), 1e-300)
        assert abs(float(grad[k]) - fd) <= 2e-6 * scale, (A.THETA_NAMES[k], float(grad[k]), fd)
        assert abs(fd) > 0, A.THETA_NAMES[k]
