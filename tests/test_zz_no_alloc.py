"""The allocation-free entry point, vdmc_count_csr_noalloc.

Callers that cannot allocate device memory while they count -- a serving
loop that reserved a fixed device-memory budget at start-up, or a host
application whose own allocator owns the device -- use this entry point with
CSR buffers they own; the library's scratch is a fixed device array.  This
test calls it through the C ABI, twice in a row on the same output buffer,
and checks the counts against vdmc_count's bit for bit (the counts are exact
integers; the tolerance is zero).  It also checks that a repeated call leaves
the device's free memory unchanged, and that a call without a status word is
refused.  It lives in a file that pytest collects last, and passes both alone
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import to_numpy_u64
from paper_2201_11655_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11655_b300 import build, vdmc
    build.build()
    L = vdmc.load()
    vp = ctypes.c_void_p
    L.vdmc_count_csr_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp]
    L.vdmc_count_csr_noalloc.restype = ctypes.c_int
    return L


def device_csr(g):
    """The graph's CSR as caller-owned device tensors (the caller may allocate
    these ahead of time; the count itself allocates nothing)."""
    rowptr, col, new2old = g.export_csr()
    n = g.n
    ranks = (col >> 2).astype(np.int64)
    pbeg = np.array([rowptr[r] + np.searchsorted(ranks[rowptr[r]:rowptr[r + 1]], r, side="right")
                     for r in range(n)], dtype=np.int64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return {"rowptr": t(rowptr), "col": t(col.view(np.int32)), "pbeg": t(pbeg), "new2old": t(new2old),
            "nnz": int(col.size)}


def call(L, g, csr, k, out, status):
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    return L.vdmc_count_csr_noalloc(g.n, csr["nnz"], p(csr["rowptr"]), p(csr["col"]), p(csr["pbeg"]),
                                    p(csr["new2old"]), k, p(out), p(status), None)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_noalloc_matches_count_twice(lib, seed):
    from paper_2201_11655_b300 import vdmc
    if seed == 0:
        n, s, d = synth.gnp(100, 0.08, 0)
    elif seed == 1:
        n, s, d = synth.chung_lu(3000, 4.0, 2.2, 41, reciprocity=0.2)
    else:
        n, s, d = synth.chung_lu(20000, 5.0, 2.3, 7, reciprocity=0.2)
    with vdmc.graph_create(n, s, d) as g:
        csr = device_csr(g)
        for k in (3, 4):
            want = to_numpy_u64(vdmc.count(g, k))
            out = torch.full((n, vdmc.num_classes(k)), 12345, dtype=torch.int64, device="cuda").view(torch.uint64)
            status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
            free_before = None
            for rep in range(2):
                assert call(lib, g, csr, k, out, status) == 0
                torch.cuda.synchronize()
                assert int(status.item()) == 0
                np.testing.assert_array_equal(to_numpy_u64(out), want, err_msg="k=%d call %d" % (k, rep))
                # the first call may load the kernel's code; the second must
                # leave the device's free memory exactly where it was
                free_now = torch.cuda.mem_get_info()[0]
                if rep == 1:
                    assert free_now == free_before, "k=%d: device free memory changed by %d bytes" % (
                        k, free_now - free_before)
                free_before = free_now


def test_noalloc_rejects_oversize_and_bad_args(lib):
    big = (1 << 18) + 1
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sp = ctypes.c_void_p(st.data_ptr())
    assert lib.vdmc_count_csr_noalloc(big, 0, None, None, None, None, 4, None, sp, None) == 1
    assert lib.vdmc_count_csr_noalloc(10, 0, None, None, None, None, 5, None, sp, None) == 1
    assert lib.vdmc_count_csr_noalloc(10, 4, None, None, None, None, 3, None, sp, None) == 1


def test_noalloc_requires_status_word(lib):
    # without a status word a failed index check would go unreported
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.gnp(60, 0.1, 4)
    with vdmc.graph_create(n, s, d) as g:
        csr = device_csr(g)
        out = torch.zeros((n, vdmc.num_classes(3)), dtype=torch.int64, device="cuda").view(torch.uint64)
        p = lambda x: ctypes.c_void_p(x.data_ptr())
        rc = lib.vdmc_count_csr_noalloc(g.n, csr["nnz"], p(csr["rowptr"]), p(csr["col"]), p(csr["pbeg"]),
                                        p(csr["new2old"]), 3, p(out), None, None)
        assert rc == 1
