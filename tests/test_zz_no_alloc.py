"""dsc_compute_dij_noalloc: the entry point for callers that may not allocate
device memory (pre-reserved treatment loops, fixed GPU memory quotas, code
where cudaMalloc is not allowed).  Its working memory is a fixed array inside
the library; the test allocates the inputs and outputs itself and checks two
calls in a row against dsc_compute_dij, the allocating entry point.

This file is collected last so that a failure here comes after every other
test has run.
"""
import numpy as np
import pytest

from paper_0908_4417_gb300 import phantoms as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def dsc():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc as D
    D.lib()
    return D


def reference(dsc, w):
    csr, res, g = dsc.compute_workload(w, value_dtype=P.VALUE_F32)
    dsc.dsc_release_result(res)
    dsc.dsc_destroy_geometry(g)
    return csr


def noalloc(dsc, w, capacity):
    dev = torch.device("cuda", 0)
    rho = torch.from_numpy(np.ascontiguousarray(w.density)).to(dev)
    row_ptr = torch.full((w.nrows + 1,), -1, dtype=torch.int64, device=dev)
    col = torch.full((capacity,), -1, dtype=torch.int32, device=dev)
    val = torch.full((capacity,), -1.0, dtype=torch.float32, device=dev)
    flags = dsc.DSC_FLAG_TRILINEAR_TABLE if getattr(w, "table_mode", 0) == P.TABLE_TRILINEAR else 0
    opts = dsc.compute_opts(w.tau, P.VALUE_F32, w.h_frac, flags)
    stream = torch.cuda.current_stream(dev)
    nnz = dsc.dsc_compute_dij_noalloc(w.grid, rho.data_ptr(), w.model, w.beams, opts, row_ptr.data_ptr(),
                                      col.data_ptr(), val.data_ptr(), capacity, stream.cuda_stream)
    torch.cuda.synchronize()
    return nnz, row_ptr.cpu().numpy(), col[:nnz].cpu().numpy(), val[:nnz].cpu().numpy()


def test_two_calls_in_a_row_match_compute_dij(dsc):
    # the second call (a larger problem) runs on the array the first one left behind
    for w in (P.water_32(), P.slabs_128(value_dtype=P.VALUE_F32)):
        ref = reference(dsc, w)
        nnz, row_ptr, col, val = noalloc(dsc, w, ref.nnz + 1000)
        assert nnz == ref.nnz
        assert np.array_equal(row_ptr, ref.row_ptr)
        assert np.array_equal(col, ref.col)
        rel = np.abs(val.astype(np.float64) - ref.val) / ref.val
        assert rel.max() <= TOL


def test_smaller_problem_after_a_larger_one(dsc):
    """The array keeps the previous call's contents: a small problem after a
    large one (the reverse of the order above) must not pick up any of it --
    the same CSR as the allocating entry point, bit for bit."""
    for w in (P.slabs_128(value_dtype=P.VALUE_F32), P.water_32()):
        ref = reference(dsc, w)
        nnz, row_ptr, col, val = noalloc(dsc, w, ref.nnz + 64)
        assert nnz == ref.nnz
        assert np.array_equal(row_ptr, ref.row_ptr) and np.array_equal(col, ref.col)
        assert np.array_equal(val, ref.val.astype(np.float32))


def test_trilinear_table_and_logistic_profile(dsc):
    """The option flags and the model's profile reach the fixed-memory path
    too: same CSR as the allocating entry point."""
    import dataclasses
    w = dataclasses.replace(P.slabs_128(value_dtype=P.VALUE_F32), table_mode=P.TABLE_TRILINEAR)
    w = dataclasses.replace(w, model=dataclasses.replace(w.model, profile=P.PROFILE_LOGISTIC))
    ref = reference(dsc, w)
    nnz, row_ptr, col, val = noalloc(dsc, w, ref.nnz + 16)
    assert nnz == ref.nnz
    assert np.array_equal(row_ptr, ref.row_ptr) and np.array_equal(col, ref.col)
    assert np.array_equal(val, ref.val.astype(np.float32))


def test_rejects_requests_beyond_the_fixed_memory(dsc):
    w = P.prostate_256()
    with pytest.raises(dsc.DscError) as e:
        noalloc(dsc, w, 16)
    assert e.value.status == 1 and "fixed maximum" in str(e.value)
    w = P.water_32()
    with pytest.raises(dsc.DscError) as e:
        noalloc(dsc, w, 10)
    assert e.value.status == 1 and "capacity" in str(e.value)
