"""The allocation-free entry point, pcv_cv_loss_fp64_static.

Some callers cannot call cudaMalloc (a host application that owns all device
memory through its own pool, or a latency-critical loop where the device-wide
synchronisation of cudaMalloc/cudaFree is not acceptable).  For them the library
offers one entry point whose work memory is a fixed static device array.  This
test calls it through the C ABI and checks, on two calls in a row (the second
finds the first call's leftovers in the shared array), that it gives the same
losses as the regular entry point pcv_cv_loss_device in FP64, within the FP64
parity tolerance.  The file is named to run last in the suite.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1912_13132_gb300 import datagen

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _device_inputs(ctx, w, torch):
    dev = "cuda"
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    V_idx = ctx.V_idx
    return dict(d_x=f64(w.xy[:, 0]), d_y=f64(w.xy[:, 1]), d_v=f64(w.v),
                d_T_idx=torch.tensor(ctx.T_idx.astype(np.int32), device=dev),
                d_Vx=f64(w.xy[V_idx, 0]), d_Vy=f64(w.xy[V_idx, 1]), d_Vv=f64(w.v[V_idx]))


def test_static_scratch_matches_regular_entry(gpu_lib):
    import torch

    pcv = gpu_lib
    w = datagen.make_uniform(1500, 700, 3, 0.06, seed=4242, name="noalloc")
    P1 = np.array([[1.0, 0.1, 0.05], [2.0, 0.05, 0.02], [0.5, 0.2, 0.1]])
    P2 = np.array([[1.3, 0.07, 0.03], [1.0, 0.15, 0.01]])
    with pcv.Context(w.xy, w.v, w.role, w.layout) as ctx:
        inp = _device_inputs(ctx, w, torch)
        for P in (P1, P2):
            d_p = torch.tensor(P, dtype=torch.float64, device="cuda")
            B = len(P)
            ref_sspe = torch.empty(B, dtype=torch.float64, device="cuda")
            ref_z = torch.empty((B, ctx.N), dtype=torch.float64, device="cuda")
            ctx.cv_loss_device(d_p, ref_sspe, precision="fp64", d_z=ref_z)
            sspe = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
            z = torch.full((B, ctx.N), -1.0, dtype=torch.float64, device="cuda")
            st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
            rc = pcv.pcv_cv_loss_fp64_static(inp["d_x"], inp["d_y"], inp["d_v"], ctx.T_off, inp["d_T_idx"],
                                             ctx.V_off, inp["d_Vx"], inp["d_Vy"], inp["d_Vv"], d_p, sspe,
                                             d_sspe_per_subset=z, d_status=st)
            assert rc == pcv.PCV_OK
            torch.cuda.synchronize()
            a, r = sspe.cpu().numpy(), ref_sspe.cpu().numpy()
            assert np.all(st.cpu().numpy() == 0)
            assert np.all(np.abs(a - r) <= TOL * np.abs(r)), (a, r)
            za, zr = z.cpu().numpy(), ref_z.cpu().numpy()
            assert np.all(np.abs(za - zr) <= TOL * np.abs(zr) + 1e-300)


def test_static_scratch_bad_row_optional_outputs_and_no_validation(gpu_lib):
    """An invalid configuration row gives its own PCV_ERR_ARG status and a NaN loss while
    the others evaluate; the optional outputs may be NULL; a layout whose cores hold no
    validation data runs no task and returns zero losses -- each as the regular entry
    point does."""
    import torch

    pcv = gpu_lib
    w = datagen.make_uniform(900, 400, 3, 0.06, seed=4243, name="noalloc-bad")
    P = np.array([[1.0, 0.1, 0.05], [1.0, -0.1, 0.05], [0.7, 0.08, 0.02]])
    d_p = torch.tensor(P, dtype=torch.float64, device="cuda")
    with pcv.Context(w.xy, w.v, w.role, w.layout) as ctx:
        inp = _device_inputs(ctx, w, torch)
        ref = torch.empty(3, dtype=torch.float64, device="cuda")
        ref_st = torch.empty(3, dtype=torch.int32, device="cuda")
        ctx.cv_loss_device(d_p, ref, precision="fp64", d_status=ref_st)
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        rc = pcv.pcv_cv_loss_fp64_static(inp["d_x"], inp["d_y"], inp["d_v"], ctx.T_off, inp["d_T_idx"],
                                         ctx.V_off, inp["d_Vx"], inp["d_Vy"], inp["d_Vv"], d_p, out,
                                         d_status=st)
        assert rc == pcv.PCV_OK
        out2 = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        rc = pcv.pcv_cv_loss_fp64_static(inp["d_x"], inp["d_y"], inp["d_v"], ctx.T_off, inp["d_T_idx"],
                                         ctx.V_off, inp["d_Vx"], inp["d_Vy"], inp["d_Vv"], d_p, out2)
        assert rc == pcv.PCV_OK
        torch.cuda.synchronize()
        a, a2, r = out.cpu().numpy(), out2.cpu().numpy(), ref.cpu().numpy()
        assert st.cpu().numpy().tolist() == ref_st.cpu().numpy().tolist() == [0, pcv.PCV_ERR_ARG, 0]
        assert np.isnan(a[1]) and np.isnan(a2[1]) and np.isnan(r[1])
        for x in (a, a2):
            assert np.all(np.abs(x[[0, 2]] - r[[0, 2]]) <= TOL * np.abs(r[[0, 2]])), (x, r)
    # no validation data anywhere: every subset is skipped (Sec. 4.3.1)
    role = np.zeros_like(w.role)
    with pcv.Context(w.xy, w.v, role, w.layout) as ctx:
        inp = _device_inputs(ctx, w, torch)
        assert ctx.V_off[-1] == 0
        for key in ("d_Vx", "d_Vy", "d_Vv"):      # no validation points: a placeholder, never read
            inp[key] = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref = torch.empty(3, dtype=torch.float64, device="cuda")
        ref_st = torch.empty(3, dtype=torch.int32, device="cuda")
        ctx.cv_loss_device(d_p, ref, precision="fp64", d_status=ref_st)
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        rc = pcv.pcv_cv_loss_fp64_static(inp["d_x"], inp["d_y"], inp["d_v"], ctx.T_off, inp["d_T_idx"],
                                         ctx.V_off, inp["d_Vx"], inp["d_Vy"], inp["d_Vv"], d_p, out,
                                         d_status=st)
        assert rc == pcv.PCV_OK
        torch.cuda.synchronize()
        a, r = out.cpu().numpy(), ref.cpu().numpy()
        assert st.cpu().numpy().tolist() == ref_st.cpu().numpy().tolist()
        assert a[0] == r[0] == 0.0 and a[2] == r[2] == 0.0 and np.isnan(a[1]) == np.isnan(r[1])


def test_static_scratch_rejects_oversized(gpu_lib):
    import torch

    pcv = gpu_lib
    N = 1
    T_off = np.array([0, 4000], dtype=np.int64)      # one training set too large for the array
    V_off = np.array([0, 10], dtype=np.int64)
    d = torch.zeros(4000, dtype=torch.float64, device="cuda")
    idx = torch.arange(4000, dtype=torch.int32, device="cuda")
    P = torch.tensor([[1.0, 0.1, 0.05]], dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = pcv.pcv_cv_loss_fp64_static(d, d, d, T_off, idx, V_off, d, d, d, P, out)
    assert rc == pcv.PCV_ERR_ARG
    # offsets that would index before the caller's arrays
    rc = pcv.pcv_cv_loss_fp64_static(d, d, d, np.array([-5, 10], dtype=np.int64), idx, V_off, d, d, d, P, out)
    assert rc == pcv.PCV_ERR_ARG
    rc = pcv.pcv_cv_loss_fp64_static(d, d, d, np.array([0, 10], dtype=np.int64), idx,
                                     np.array([-1, 5], dtype=np.int64), d, d, d, P, out)
    assert rc == pcv.PCV_ERR_ARG
