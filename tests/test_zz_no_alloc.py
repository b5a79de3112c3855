"""The allocation-free kinetic-energy entry point (mts_kinetic_energy_noalloc).

It serves callers that cannot allocate device memory where they need the
number (device memory owned by another allocator, latency-critical paths that
cannot afford cudaMalloc's device-wide synchronisation, code that must not hit
out-of-memory after set-up).  This test calls it through the C ABI on
caller-owned buffers and checks its result against the kinetic energy and
maximum speed that the slow-step entry point reports for the same velocities,
and against a plain FP64 NumPy sum over the velocities read back, on two calls
in a row (the second call reuses the library's static scratch).  Kept in its
own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_noalloc_kinetic_energy_matches_slow_step_report(precision):
    import torch

    from paper_2309_04010_gb300 import mtssph as M
    from synth import bodies as B

    prec = M.MIXED if precision == "mixed" else M.FP64
    tdtype = torch.float32 if precision == "mixed" else torch.float64
    ctx = M.Context(0)
    try:
        for case in (B.bar2d(nx=60, ny=12), B.cylinder3d(L=4e-3, R=1e-3, n_slow=10)):
            gb = M.body_from_case(ctx, case, prec)
            rep = gb.advance_slow_step(ramp=1.0 / case.plan.n_ramp, ke_tol=-1.0,
                                       max_substeps=25)
            V = gb.read(M.F_V)                     # velocities after the last substep
            assert rep.ke_final > 0 and rep.max_v > 0
            v_dev = torch.tensor(V, dtype=tdtype, device="cuda").contiguous()
            out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
            dim = V.shape[1]
            mass = case.material.rho0 * case.dx ** dim
            stream = torch.cuda.current_stream().cuda_stream
            # independent FP64 values from the velocities as read back; in mixed
            # precision each |v|^2 is formed in FP32 by the library, so the two
            # agree to FP32 rounding of the squares
            v2 = (V.astype(np.float64) ** 2).sum(axis=1)
            ke_np, vmax_np = 0.5 * mass * v2.sum(), float(np.sqrt(v2.max()))
            tol_np = 1e-12 if precision == "fp64" else 1e-6
            for _ in range(2):                     # two calls in a row share the scratch
                M.kinetic_energy_noalloc(v_dev.data_ptr(), prec, dim, case.n, mass,
                                         out.data_ptr(), stream)
                torch.cuda.synchronize()
                ke, vmax = out.cpu().numpy()
                assert abs(ke - rep.ke_final) <= 1e-12 * rep.ke_final
                assert abs(vmax - rep.max_v) <= 1e-12 * rep.max_v
                assert abs(ke - ke_np) <= tol_np * ke_np
                assert abs(vmax - vmax_np) <= tol_np * vmax_np
                out.fill_(-1.0)
            gb.close()
    finally:
        ctx.close()


def test_noalloc_rejects_bad_arguments():
    import torch

    from paper_2309_04010_gb300 import mtssph as M

    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = M.lib()
    assert L.mts_kinetic_energy_noalloc(None, M.FP64, 2, 8, 1.0, out.data_ptr(), None) == \
        M.ERR_INVALID_ARG
    assert L.mts_kinetic_energy_noalloc(buf.data_ptr(), M.FP64, 2, 0, 1.0, out.data_ptr(),
                                        None) == M.ERR_INVALID_ARG
    assert L.mts_kinetic_energy_noalloc(buf.data_ptr(), M.FP64, 2, 1 << 40, 1.0, out.data_ptr(),
                                        None) == M.ERR_INVALID_ARG
    assert b"outside" in L.mts_last_error()
    assert L.mts_kinetic_energy_noalloc(buf.data_ptr(), M.FP64, 4, 8, 1.0, out.data_ptr(),
                                        None) == M.ERR_INVALID_ARG
