"""Run a few substeps of a workload through the library (for ncu captures).

    python -m paper_2309_04010_gb300.profile_case --workload cylinder3d \
        --precision mixed --substeps 2

Builds the body (setup), applies the first load increment and runs the given
number of substeps with the kinetic-energy stop disabled, then prints one line
with the substep count and the setup products' sizes.  Used as the command
under `ncu` so that a capture covers a known, small number of launches.
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
                    choices=["bar2d", "cylinder3d", "strip2d", "plate3d"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--substeps", type=int, default=2)
    ap.add_argument("--slow-steps", type=int, default=1)
    args = ap.parse_args()

    from paper_2309_04010_gb300 import mtssph as M
    from synth import bodies as B

    case = getattr(B, args.workload)()
    ctx = M.Context(0)
    prec = M.MIXED if args.precision == "mixed" else M.FP64
    gb = M.body_from_case(ctx, case, prec)
    off, _ = gb.neighbors()
    total = 0
    for l in range(1, args.slow_steps + 1):
        ramp = l / case.plan.n_ramp if case.plan.n_ramp else 0.0
        r = gb.advance_slow_step(ramp=ramp, ke_tol=-1.0, max_substeps=args.substeps,
                                 check_every=args.substeps)
        total += r.substeps
    print(f"profile_case workload={args.workload} n={case.n} nnz={int(off[-1])} "
          f"precision={args.precision} substeps={total}")
    gb.close()
    ctx.close()


if __name__ == "__main__":
    main()
