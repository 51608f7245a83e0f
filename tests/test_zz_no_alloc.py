"""imrt_eval_csr_noalloc: the allocation-free evaluation, for callers that cannot allocate
device memory when they evaluate a plan (delivery controllers whose device memory is
reserved once at start-up, frameworks that own every allocation). Called through the C
ABI on two calls in a row and checked against plan_eval (the allocating entry point) and
the FP64 oracle; malformed CSR inputs must come back as IMRT_EINVAL without a fault. This
file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
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


def _device_inputs(torch, row_ptr, col, val, mask):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(row_ptr), t(col), t(val), t(mask)


def _noalloc(lib, torch, case, dev, x, stream, m=None, n=None, nnz=None):
    rp, col, val, mask = dev
    m = case.m if m is None else m
    csr = L.imrt_csr(m, case.n if n is None else n, case.nnz if nnz is None else nnz, rp.data_ptr(),
                     col.data_ptr(), val.data_ptr(), 1)
    thr = np.ascontiguousarray(case.thresholds, np.float32)
    w = np.ascontiguousarray(case.weights, np.float32)
    z = torch.empty(m, dtype=torch.float32, device="cuda")
    G = ctypes.c_double()
    st = lib.imrt_eval_csr_noalloc(ctypes.byref(csr), mask.data_ptr(), case.n_structures, thr.ctypes.data,
                                   w.ctypes.data, x.data_ptr(), z.data_ptr(), ctypes.addressof(G), stream)
    torch.cuda.synchronize()
    return st, G.value, z.cpu().numpy()


@pytest.mark.parametrize("name", ["tiny", "ragged"])
def test_noalloc_matches_plan_eval_and_oracle_twice(torch_cuda, name):
    torch = torch_cuda
    lib = L.load()
    orc = oracle.get()
    case = (phantom.make_case(phantom.TINY_5MM_5BEAM) if name == "tiny"
            else phantom.random_case(3, m=3001, n=57, density=0.15, n_structures=3, empty_rows=40, long_rows=3))
    dev = _device_inputs(torch, case.row_ptr, case.col, case.val, case.mask)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.Generator(np.random.PCG64(11))
    with Plan.from_case(case, Options(stream=stream), device=True) as plan:
        for call in range(2):  # two calls in a row share (and must re-clear) the scratch array
            x = rng.uniform(0.0, 2.0, case.n).astype(np.float32)
            G_ref, z_ref, _ = plan.eval(x)
            st, G, z = _noalloc(lib, torch, case, dev, torch.from_numpy(x).cuda(), stream)
            assert st == L.IMRT_OK, lib.imrt_last_error().decode()
            # against the allocating entry point
            assert np.linalg.norm(z - z_ref) <= DOSE_RTOL * np.linalg.norm(z_ref), call
            assert abs(G - G_ref) <= OBJ_RTOL * abs(G_ref), (call, G, G_ref)
            # against the FP64 oracle, voxel by voxel
            G_o, z_o, _, _ = orc.eval(case, x.astype(np.float64), gradient=False)
            assert np.linalg.norm(z - z_o) <= DOSE_RTOL * np.linalg.norm(z_o), call
            np.testing.assert_allclose(z, z_o, rtol=0, atol=DOSE_RTOL * np.abs(z_o).max())
            assert abs(G - G_o) <= OBJ_RTOL * abs(G_o), (call, G, G_o)


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


@pytest.mark.parametrize("fault", ["column_equals_n", "negative_column", "decreasing_row_ptr", "row_ptr_end"])
def test_noalloc_rejects_malformed_csr(torch_cuda, fault):
    """A malformed CSR made on the host: the kernel reads only inside the arrays (it skips the bad
    rows and entries) and the call returns IMRT_EINVAL; a valid call afterwards still matches."""
    torch = torch_cuda
    lib = L.load()
    case = phantom.random_case(5, m=700, n=31, density=0.2, n_structures=2, empty_rows=5)
    row_ptr, col = case.row_ptr.copy(), case.col.copy()
    if fault == "column_equals_n":
        col[col.size // 2] = case.n
    elif fault == "negative_column":
        col[7] = -3
    elif fault == "decreasing_row_ptr":
        j = int(np.argmax(np.diff(row_ptr) > 2)) + 1  # a row with entries: its start moves past its end
        row_ptr[j] = row_ptr[j + 1] + 1
    else:
        row_ptr[-1] = row_ptr[-1] - 1  # row_ptr[m] != nnz
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.from_numpy(np.full(case.n, 0.5, np.float32)).cuda()
    st, _, _ = _noalloc(lib, torch, case, _device_inputs(torch, row_ptr, col, case.val, case.mask), x, stream)
    assert st == L.IMRT_EINVAL, st
    assert "invalid CSR" in lib.imrt_last_error().decode()
    st, G, z = _noalloc(lib, torch, case, _device_inputs(torch, case.row_ptr, case.col, case.val, case.mask), x,
                        stream)
    assert st == L.IMRT_OK
    G_o, z_o, _, _ = oracle.get().eval(case, np.full(case.n, 0.5), gradient=False)
    assert abs(G - G_o) <= OBJ_RTOL * abs(G_o)


def test_noalloc_rejects_bad_weights(torch_cuda):
    torch = torch_cuda
    lib = L.load()
    case = phantom.random_case(6, m=100, n=9, density=0.3)
    dev = _device_inputs(torch, case.row_ptr, case.col, case.val, case.mask)
    x = torch.ones(case.n, dtype=torch.float32, device="cuda")
    rp, col, val, mask = dev
    csr = L.imrt_csr(case.m, case.n, case.nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1)
    thr = np.ascontiguousarray(case.thresholds, np.float32)
    for bad in (-1.0, np.inf):
        w = np.ascontiguousarray(case.weights, np.float32)
        w[0, 0] = bad
        G = ctypes.c_double()
        st = lib.imrt_eval_csr_noalloc(ctypes.byref(csr), mask.data_ptr(), case.n_structures, thr.ctypes.data,
                                       w.ctypes.data, x.data_ptr(), None, ctypes.addressof(G), None)
        assert st == L.IMRT_EINVAL
