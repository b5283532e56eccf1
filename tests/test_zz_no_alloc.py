"""The allocation-free energy entry point (for callers that cannot call
cudaMalloc) against the regular context-based reduction of the same state
and against the CPU oracle, on two calls in a row; that a warm call
allocates no device memory; its size limit and the binding's argument
checks."""
import ctypes
import os

import numpy as np
import pytest

import paper_2404_02950_gb300 as slh
from oracle import energy as oenergy
from paper_2404_02950_gb300 import inputs
from tests.helpers import oparams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(slh.LIB_PATH):
        from paper_2404_02950_gb300 import build
        build.build()
    return slh.lib()


@pytest.mark.parametrize("prec,order,tol", [("f64", 4, 1e-12), ("f32", 6, 5e-6)])
def test_noalloc_energy_matches_context_reduction_twice(prec, order, tol):
    import torch
    n, dx, eta = 40, 0.125, 2.5
    p = slh.EOMParams(order=order, a=0.1)
    y = inputs.gaussian_field(n, 5.0, seed=8)
    y = (y[0], y[1], 0.5 * y[0], -0.25 * y[1])
    h = slh.Hierarchy(n, dx, nghost=3, bf=8, prec=prec)
    boxes = [((0, 0, 0), (n - 1, n - 1, n - 1))]
    h.init_level(0, boxes)
    h.set_state(0, slh.dense_from_boxes(y, boxes))
    h.set_eta(eta)
    ref = h.reduce_energy(p)
    dt = torch.float64 if prec == "f64" else torch.float32
    fields = torch.from_numpy(np.stack(y)).to(dt).cuda().contiguous()
    # the oracle on the state as stored (FP32 values widened exactly)
    orc = oenergy.energy_periodic([a.astype(np.float64) for a in fields.cpu().numpy()], eta, dx, oparams(p))
    outs = [torch.full((5,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            # a warm call allocates nothing: neither through torch nor on the device
            alloc0 = torch.cuda.memory_allocated()
            free0, _ = torch.cuda.mem_get_info()
        slh.slh_energy_noalloc(fields, n, dx, eta, p, outs[call])
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        got = outs[call].cpu().numpy()
        for k in range(4):
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1.0), (call, k, got[k], ref[k])
            assert abs(got[k] - orc[k]) <= tol * max(abs(orc[k]), 1.0), (call, k, got[k], orc[k])
        assert got[4] == ref[4], (call, got[4], ref[4])
        assert got[4] == orc[4], (call, got[4], orc[4])
    h.close()


def test_noalloc_binding_rejects_bad_buffers():
    import torch
    n = 8
    p = slh.EOMParams()
    good = torch.zeros(4 * n ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    bad_calls = [
        (good.cpu(), out),                                                  # host tensor
        (good.to(torch.bfloat16), out),                                     # unsupported dtype
        (good[: 4 * n ** 3 - 1], out),                                      # too short
        (good.view(4, n ** 3).t(), out),                                    # not contiguous
        (good, torch.zeros(5, dtype=torch.float32, device="cuda")),          # out not float64
        (good, torch.zeros(4, dtype=torch.float64, device="cuda")),          # out too short
    ]
    for f, o in bad_calls:
        with pytest.raises(ValueError):
            slh.slh_energy_noalloc(f, n, 1.0, 1.0, p, o)


def test_noalloc_rejects_lattice_beyond_scratch_limit():
    import torch
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    fields = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = slh.EOMParams().c()
    st = slh.lib().slh_energy_noalloc(ctypes.c_void_p(fields.data_ptr()), 4097, slh.SLH_F64, 1.0, 1.0,
                                      ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), None)
    assert st == -2
    assert b"scratch limit" in slh.lib().slh_last_error()
