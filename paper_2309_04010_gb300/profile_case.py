"""Run a few substeps of a workload through the library (for ncu captures).

    python -m paper_2309_04010_gb300.profile_case --workload cylinder3d \
        --precision mixed --substeps 2

Builds the body (setup), applies the first load increment (or, for the
diffusion workloads, one diffusion step of the stable size) and runs the given
number of substeps with the kinetic-energy stop disabled, then prints one line
with the substep count and the setup products' sizes.  --diffusion-mode 1
takes the two-stage diffusion form; --reverse runs the reverse mode of the
last slow step (FP64).  Used as the command under `ncu` so that a capture
covers a known, small number of launches.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cylinder3d",
                    choices=["bar2d", "cylinder3d", "strip2d", "plate3d", "membrane_droplet3d"])
    ap.add_argument("--diffusion-mode", type=int, default=0)
    ap.add_argument("--reverse", action="store_true")
    ap.add_argument("--membrane-mm", type=float, default=10.0,
                    help="in-plane size of the membrane workload (the paper's is 10 mm)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--substeps", type=int, default=2)
    ap.add_argument("--slow-steps", type=int, default=1)
    args = ap.parse_args()

    from paper_2309_04010_gb300 import mtssph as M
    from synth import bodies as B

    if args.workload == "membrane_droplet3d":
        case = B.membrane_droplet3d(Lx=args.membrane_mm * 1e-3, Ly=args.membrane_mm * 1e-3)
    else:
        case = getattr(B, args.workload)()
    ctx = M.Context(0)
    prec = M.MIXED if args.precision == "mixed" else M.FP64
    gb = M.body_from_case(ctx, case, prec)
    if args.diffusion_mode:
        gb.set_diffusion_mode(args.diffusion_mode)
    off, _ = gb.neighbors()
    total = 0
    p = None
    ck = None
    for l in range(1, args.slow_steps + 1):
        ramp = l / case.plan.n_ramp if case.plan.n_ramp else 0.0
        p = dict(ramp=ramp, ke_tol=-1.0, max_substeps=args.substeps, check_every=args.substeps)
        if case.diffusion is not None:
            p.update(dt_slow=gb.diffusion_dt()[1], ke_mode=1, force_dt=True)
        ck = gb.save_state()
        r = gb.advance_slow_step(**p)
        total += r.substeps
    if args.reverse:
        gb.adjoint_enable(args.substeps)
        gb.adjoint_seed(tip_bar=[1.0] * case.dim, force_bar=[1.0] * case.dim)
        gb.load_state(ck)
        gb.adjoint_slow_step(args.substeps, **p)
    print(f"profile_case workload={args.workload} n={case.n} nnz={int(off[-1])} "
          f"precision={args.precision} substeps={total}")
    gb.close()
    ctx.close()


if __name__ == "__main__":
    main()
