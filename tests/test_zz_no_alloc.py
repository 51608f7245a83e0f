"""imrt_eval_csr_noalloc: the allocation-free evaluation for callers that cannot allocate
device memory (graph capture, fixed device budgets). Called through the C ABI and checked
against plan_eval, the allocating path, on two calls in a row. This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_0908_4421_gb300 import Options, Plan, phantom
from paper_0908_4421_gb300 import _lib as L

pytestmark = pytest.mark.gpu

DOSE_RTOL = 1e-5   # the tolerance of the other parity tests
OBJ_RTOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    return torch


def _device_inputs(torch, case):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(case.row_ptr), t(case.col), t(case.val), t(case.mask)


def _noalloc(lib, torch, case, dev, x, stream):
    rp, col, val, mask = dev
    csr = L.imrt_csr(case.m, case.n, case.nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1)
    thr = np.ascontiguousarray(case.thresholds, np.float32)
    w = np.ascontiguousarray(case.weights, np.float32)
    z = torch.empty(case.m, dtype=torch.float32, device="cuda")
    G = ctypes.c_double()
    st = lib.imrt_eval_csr_noalloc(ctypes.byref(csr), mask.data_ptr(), case.n_structures, thr.ctypes.data,
                                   w.ctypes.data, x.data_ptr(), z.data_ptr(), ctypes.addressof(G), stream)
    assert st == L.IMRT_OK, lib.imrt_last_error().decode()
    return G.value, z.cpu().numpy()


@pytest.mark.parametrize("name", ["tiny", "ragged"])
def test_noalloc_matches_plan_eval_twice(torch_cuda, name):
    torch = torch_cuda
    lib = L.load()
    case = (phantom.make_case(phantom.TINY_5MM_5BEAM) if name == "tiny"
            else phantom.random_case(3, m=3001, n=57, density=0.15, n_structures=3, empty_rows=40, long_rows=3))
    dev = _device_inputs(torch, case)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.Generator(np.random.PCG64(11))
    with Plan.from_case(case, Options(stream=stream), device=True) as plan:
        for call in range(2):  # two calls in a row share (and must re-clear) the scratch array
            x = rng.uniform(0.0, 2.0, case.n).astype(np.float32)
            G_ref, z_ref, _ = plan.eval(x)
            G, z = _noalloc(lib, torch, case, dev, torch.from_numpy(x).cuda(), stream)
            assert np.linalg.norm(z - z_ref) <= DOSE_RTOL * np.linalg.norm(z_ref), call
            assert abs(G - G_ref) <= OBJ_RTOL * abs(G_ref), (call, G, G_ref)


def test_noalloc_rejects_sizes_beyond_its_limit(torch_cuda):
    torch = torch_cuda
    lib = L.load()
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    csr = L.imrt_csr(16_777_217, 4, 0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1)
    thr = np.zeros(2, np.float32)
    G = ctypes.c_double()
    st = lib.imrt_eval_csr_noalloc(ctypes.byref(csr), buf.data_ptr(), 1, thr.ctypes.data, thr.ctypes.data,
                                   buf.data_ptr(), None, ctypes.addressof(G), None)
    assert st == L.IMRT_EUNSUPPORTED
    assert "allocation-free limit" in lib.imrt_last_error().decode()
