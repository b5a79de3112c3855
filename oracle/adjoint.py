"""Reverse-mode derivatives of the slow step, in plain PyTorch float64 on the
CPU.  Test infrastructure only: the library never imports this module; the
tests compare the library's adjoint with it.

The slow step (Sec. 4.2: load jump or one diffusion step, then damped
substeps) is restated with vectorised PyTorch operations in the order of the
C oracle (mts_oracle.c), on that oracle's setup products (Morton order,
neighbour lists, B0, canonical damping order); torch.autograd then gives the
vector-Jacobian products exactly.  The substep sizes are inputs: the size rule
(Sec. 4.1) and the kinetic-energy stop (Sec. 4.2) are piecewise constant or
non-smooth in the state, so a derivative holds them fixed at the values of the
run being differentiated (frozen sizes and counts).

Parameters, in this order (THETA_NAMES): Young's modulus E (with Poisson's
ratio fixed, so mu = E/(2(1+nu)), K = E/(3(1-2nu)), lambda = K - 2mu/3,
App. A.2 / B.2), the hardening parameters sigma_0, sigma_inf, delta, H of
k(alpha) (App. A.3), the diffusivity D (Sec. 2.2) and the swelling
coefficient beta (App. B.2).

Pinned by tests/test_adjoint_oracle.py against the C oracle: the forward
restatement reproduces it, and its gradients match central differences of the
C oracle run with fixed substep sizes.
"""
import math

import numpy as np
import torch

from . import J2, OracleBody

THETA_NAMES = ("E", "sigma0", "sigma_inf", "delta", "H", "D", "beta")
R23 = math.sqrt(2.0 / 3.0)


def _alpha(dim, h):
    return 7.0 / (4.0 * math.pi * h * h) if dim == 2 else 21.0 / (16.0 * math.pi * h ** 3)


def _dwdr(dim, h, r):
    """W'(r) of the Wendland C2 kernel (Sec. 3.1), r < 2h."""
    q = r / h
    t = 1.0 - 0.5 * q
    return -5.0 * _alpha(dim, h) * q * t ** 3 / h


class TorchBody:
    """A synth Case on the C oracle's setup products, with differentiable
    slow steps.  Index space: the oracle's sorted (Morton) order."""

    def __init__(self, case, ob: OracleBody):
        self.case = case
        n, d = case.X.shape
        self.n, self.dim = n, d
        perm = ob.perm()
        rank = np.empty(n, np.int64)
        rank[perm] = np.arange(n)
        self.perm, self.rank = perm, rank
        X = case.X[perm]
        self.h = case.h_over_dx * case.dx
        self.V = case.dx ** d
        m = case.material
        self.model, self.rho0, self.nu = m.model, m.rho0, m.nu
        self.mass = self.rho0 * self.V
        self.eta = case.eta
        off, idx = ob.neighbors()
        ea = np.repeat(np.arange(n), np.diff(off))
        eb = idx.astype(np.int64)
        dv = X[ea] - X[eb]
        r = np.sqrt((dv * dv).sum(1))
        self.ea, self.eb = torch.from_numpy(ea), torch.from_numpy(eb)
        # grad_a W_ab = W'(r) (X_a - X_b) / r
        self.g = torch.from_numpy(_dwdr(d, self.h, r)[:, None] * dv / r[:, None])
        self.dwr = torch.from_numpy(_dwdr(d, self.h, r) / r)            # W'(r)/r per edge
        self.B0 = torch.from_numpy(ob.b0()[perm])                        # (n, d, d)
        # boundary conditions in sorted order
        fix = np.zeros((n, d), bool)
        u_unit = np.zeros((n, d))
        fgrp = np.zeros(n, bool)
        for bc in case.disp_bcs:
            s = rank[np.asarray(bc.ids, np.int64)]
            for k in range(d):
                if bc.axis_mask & (1 << k):
                    fix[s, k] = True
                    if bc.u_unit is not None:
                        u_unit[s, k] = np.asarray(bc.u_unit).reshape(-1, d)[:, k]
            if bc.report_force:
                fgrp[s] = True
        self.fix = torch.from_numpy(fix)
        self.u_unit = torch.from_numpy(u_unit)
        self.fgrp = torch.from_numpy(fgrp)
        tg = np.zeros(n, bool)
        if case.tip_ids is not None and len(case.tip_ids):
            tg[rank[np.asarray(case.tip_ids, np.int64)]] = True
        self.tgrp = torch.from_numpy(tg)
        held = np.zeros(n, bool)
        held_val = np.zeros(n)
        for cb in case.conc_bcs:
            s = rank[np.asarray(cb.ids, np.int64)]
            held[s] = True
            held_val[s] = cb.value
        self.cheld = torch.from_numpy(held)
        self.cheld_val = torch.from_numpy(held_val)
        self.has_diff = case.diffusion is not None
        self.c0 = case.diffusion[2] if self.has_diff else 0.0
        # damping stages: the canonical order is (colour, owner block, sub-colour,
        # a, b); owner blocks of one colour touch disjoint particles, so the
        # pairs of one (colour, sub-colour) form one stage of disjoint pairs
        pa, pb, col, key, sub = ob.colouring()
        self.stages = []
        if len(pa):
            sk = col.astype(np.int64) * 4096 + sub
            for k in np.unique(sk):
                sel = np.nonzero(sk == k)[0]
                a, b = pa[sel].astype(np.int64), pb[sel].astype(np.int64)
                dvp = X[a] - X[b]
                rp = np.sqrt((dvp * dvp).sum(1))
                coef = -2.0 * self.V * self.V * _dwdr(d, self.h, rp) / rp   # B_ab / eta
                self.stages.append((torch.from_numpy(a), torch.from_numpy(b),
                                    torch.from_numpy(coef)))

    # ------------------------------------------------------------ parameters
    def theta0(self) -> torch.Tensor:
        m = self.case.material
        D, beta = (self.case.diffusion[0], self.case.diffusion[1]) if self.has_diff else (0.0, 0.0)
        return torch.tensor([m.E, m.sigma0, m.sigma_inf, m.delta, m.H, D, beta],
                            dtype=torch.float64)

    def initial_state(self):
        n, d = self.n, self.dim
        z = torch.zeros((n, d), dtype=torch.float64)
        cp = torch.zeros((n, 6), dtype=torch.float64)
        cp[:, :3] = 1.0
        c = torch.where(self.cheld, self.cheld_val, torch.full((n,), self.c0, dtype=torch.float64))
        return (z, z.clone(), cp, torch.zeros(n, dtype=torch.float64), c)

    # ------------------------------------------------------------ stress
    def _stress(self, F, cp, al, c, th):
        """P (n,3,3), new C-bar_p^-1 (n,6) and alpha (App. A Alg. 1 / B.2)."""
        E, s0, sinf, delta, H, _, beta = th
        mu = E / (2.0 * (1.0 + self.nu))
        K = E / (3.0 * (1.0 - 2.0 * self.nu))
        I = torch.eye(3, dtype=torch.float64).expand_as(F)
        if self.model == "svk":
            Eg = 0.5 * (F.transpose(1, 2) @ F - I)
            tr = Eg.diagonal(dim1=1, dim2=2).sum(-1)
            lam = K - 2.0 * mu / 3.0
            S = lam * tr[:, None, None] * I + 2.0 * mu * Eg
            P = F @ S
            cp2, al2 = cp, al
        else:
            def kfun(a):
                return s0 + (sinf - s0) * (1.0 - torch.exp(-delta * a)) + H * a

            def dkfun(a):
                return (sinf - s0) * delta * torch.exp(-delta * a) + H

            J = torch.linalg.det(F)
            Fb = F * (1.0 / torch.pow(J, 1.0 / 3.0))[:, None, None]
            Cp = torch.stack([torch.stack([cp[:, 0], cp[:, 3], cp[:, 5]], -1),
                              torch.stack([cp[:, 3], cp[:, 1], cp[:, 4]], -1),
                              torch.stack([cp[:, 5], cp[:, 4], cp[:, 2]], -1)], 1)
            bpre = Fb @ Cp @ Fb.transpose(1, 2)
            trb = bpre.diagonal(dim1=1, dim2=2).sum(-1)
            spre = mu * (bpre - (trb / 3.0)[:, None, None] * I)
            ss = (spre * spre).sum((1, 2))
            one = torch.ones_like(ss)
            # |s_pre| with a finite derivative where s_pre = 0 (undeformed)
            s = torch.where(ss > 0, torch.sqrt(torch.where(ss > 0, ss, one)), torch.zeros_like(ss))
            kal = kfun(al)
            plastic = (s - R23 * kal) > 0
            s_safe = torch.where(plastic, s, one)
            mubar = mu * trb / 3.0
            dg = torch.zeros_like(s)
            active = plastic.clone()
            for _ in range(30):
                g = s - R23 * kfun(al + R23 * dg) - 2.0 * mubar * dg
                active = active & ~(torch.abs(g) <= 1e-13 * R23 * kal)
                if not bool(active.any()):
                    break
                dgd = -(2.0 / 3.0) * dkfun(al + R23 * dg) - 2.0 * mubar
                dg = torch.where(active, dg - g / torch.where(active, dgd, one), dg)
            fac = torch.where(plastic, 1.0 - 2.0 * mubar * dg / s_safe, one)
            snew = spre * fac[:, None, None]
            al2 = torch.where(plastic, al + R23 * dg, al)
            be = snew / mu + (trb / 3.0)[:, None, None] * I
            Fbi = torch.linalg.inv(Fb)
            Cn = Fbi @ be @ Fbi.transpose(1, 2)
            cpn = torch.stack([Cn[:, 0, 0], Cn[:, 1, 1], Cn[:, 2, 2],
                               0.5 * (Cn[:, 0, 1] + Cn[:, 1, 0]), 0.5 * (Cn[:, 1, 2] + Cn[:, 2, 1]),
                               0.5 * (Cn[:, 0, 2] + Cn[:, 2, 0])], -1)
            cp2 = torch.where(plastic[:, None], cpn, cp)
            tau = snew + (0.5 * K * (J * J - 1.0))[:, None, None] * I
            P = tau @ torch.linalg.inv(F).transpose(1, 2)
        if self.has_diff and float(beta.detach()) != 0.0:
            J = torch.linalg.det(F)
            p = 3.0 * K * beta * (c - self.c0)
            P = P - (p * J)[:, None, None] * torch.linalg.inv(F).transpose(1, 2)
        return P, cp2, al2

    # ------------------------------------------------------------ substep pieces
    def defgrad(self, u):
        d = self.dim
        du = u[self.eb] - u[self.ea]
        G = torch.zeros((self.n, d, d), dtype=torch.float64).index_add(
            0, self.ea, self.V * du[:, :, None] * self.g[:, None, :])
        F = torch.eye(3, dtype=torch.float64).repeat(self.n, 1, 1)
        Fd = torch.eye(d, dtype=torch.float64) + G @ self.B0
        if d == 3:
            return Fd
        top = torch.cat([Fd, torch.zeros((self.n, 2, 1), dtype=torch.float64)], 2)
        return torch.cat([top, F[:, 2:3, :]], 1)

    def force(self, PB):
        s = ((PB[self.ea] + PB[self.eb]) @ self.g[:, :, None]).squeeze(-1)
        return torch.zeros((self.n, self.dim), dtype=torch.float64).index_add(
            0, self.ea, self.V * s) / self.rho0

    def damp(self, v, dt):
        if self.eta == 0.0 or not self.stages:
            return v
        hdt = 0.5 * dt
        free = (~self.fix).to(torch.float64) / self.mass

        def apply(v, a, b, coef):
            B = (self.eta * coef)[:, None]
            ima, imb = free[a], free[b]
            w = v[a] - v[b]
            wn = w / (1.0 + hdt * B * (ima + imb))
            va = v[a] - hdt * B * wn * ima
            vb = v[b] + hdt * B * wn * imb
            return v.index_copy(0, a, va).index_copy(0, b, vb)

        for a, b, coef in self.stages:
            v = apply(v, a, b, coef)
        for a, b, coef in reversed(self.stages):
            v = apply(v, a, b, coef)
        return v

    def substep(self, state, th, dt, ramp):
        """One substep (Sec. 4.2 inner loop) of size dt; returns the new state
        and the acceleration of its force stage."""
        u, v, cp, al, c = state
        d = self.dim
        F = self.defgrad(u)
        P, cp2, al2 = self._stress(F, cp, al, c, th)
        PB = P[:, :d, :d] @ self.B0.transpose(1, 2)      # P B0^T (the C oracle's form)
        acc = self.force(PB)
        free = ~self.fix
        v = v + dt * acc * free
        v = self.damp(v, dt)
        u = torch.where(self.fix, ramp * self.u_unit, u + dt * v)
        v = torch.where(self.fix, torch.zeros_like(v), v)
        return (u, v, cp2, al2, c), acc

    def diffusion(self, c, th, dt):
        """Explicit step of the pairwise Laplacian (Sec. 3.2 reading), held
        particles reset."""
        D = th[5]
        s = torch.zeros(self.n, dtype=torch.float64).index_add(
            0, self.ea, 2.0 * D * self.V * (c[self.ea] - c[self.eb]) * self.dwr)
        return torch.where(self.cheld, self.cheld_val, c + dt * s)

    def substep_dt(self, state, acc, dt_override=0.0):
        """The next substep size (Sec. 4.1) from a state (no gradient)."""
        if dt_override > 0:
            return dt_override
        m = self.case.material
        K = m.E / (3.0 * (1.0 - 2.0 * self.nu))
        cs = math.sqrt(K / self.rho0)
        v = state[1].detach()
        vmax = float(torch.sqrt((v * v).sum(1)).max())
        a = (acc.detach() * (~self.fix)).double()
        amax = float(torch.sqrt((a * a).sum(1)).max())
        t1 = self.h / (cs + vmax)
        t2 = math.sqrt(self.h / amax) if amax > 0 else math.inf
        return 0.6 * min(t1, t2)

    def slow_step(self, state, th, ramp, nsub, dt_slow=0.0, dts=None, dt_override=0.0):
        """Load jump, optional diffusion step, nsub substeps.  dts: the substep
        sizes (computed by the Sec. 4.1 rule, without gradient, when None).
        Returns (state, end force, tip deflection, sizes used)."""
        u, v, cp, al, c = state
        u = torch.where(self.fix, ramp * self.u_unit, u)
        v = torch.where(self.fix, torch.zeros_like(v), v)
        if dt_slow > 0:
            c = self.diffusion(c, th, dt_slow)
        state = (u, v, cp, al, c)
        m = self.case.material
        K = m.E / (3.0 * (1.0 - 2.0 * self.nu))
        dt = dt_override if dt_override > 0 else 0.6 * self.h / math.sqrt(K / self.rho0)
        used = []
        acc = None
        for k in range(nsub):
            if dts is not None:
                dt = dts[k]
            used.append(dt)
            state, acc = self.substep(state, th, dt, ramp)
            if dts is None:
                dt = self.substep_dt(state, acc, dt_override)
        end_force = -(self.mass * acc * self.fgrp[:, None]).sum(0)
        nt = int(self.tgrp.sum())
        tip = (state[0] * self.tgrp[:, None]).sum(0) / max(nt, 1)
        return state, end_force, tip, used

    def to_original(self, x):
        """Rows of a sorted-order array in original particle order."""
        out = torch.empty_like(x)
        out[torch.from_numpy(self.perm)] = x
        return out
