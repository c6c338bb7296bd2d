"""The allocation-free colouring entry point (msp_vertices_grouping_noalloc).

Some callers cannot allocate device memory (a memory pool that owns the whole GPU, code
that must not let cudaMalloc/cudaFree synchronise the device, an environment where the
CUDA allocator is replaced); this entry point serves them from a fixed file-scope
device array.  Its colouring must equal the one the solver's own setup computes
(msp_setup followed by msp_colour0), on two calls in a row, since every call reuses the
same array.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from synthetic import box_jacobian, grid_spe10

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2208_08594_gb300 as msp  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return (torch.from_numpy(np.ascontiguousarray(a.row_ptr)).to(DEV),
            torch.from_numpy(np.ascontiguousarray(a.col_idx)).to(DEV),
            torch.from_numpy(np.ascontiguousarray(a.values.reshape(-1))).to(DEV))


@pytest.mark.parametrize("make", [
    lambda: grid_spe10(nx=20, ny=18, nz=9),
    lambda: box_jacobian(30, 20, 10, 3, 7, layered=True, kz_ratio=0.1, n_wells=2),
], ids=["spe10_like_b4", "wells_b3"])
def test_noalloc_colouring_matches_setup(make):
    a = make()
    rp, ci, v = _dev(a)
    solver = msp.Solver(a.nb, a.b, rp, ci, v, coarse_max=200)
    ref, g_ref = solver.colour0()
    solver.close()
    for _ in range(2):  # the scratch array keeps the previous call's contents
        out = torch.full((a.nb,), -1, dtype=torch.int32, device=DEV)
        g = msp.msp_vertices_grouping_noalloc(a.nb, rp, ci, out)
        torch.cuda.synchronize()
        assert g == g_ref
        assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    L = msp._native.lib()
    n = msp.NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device=DEV)
    ci = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = torch.zeros(n, dtype=torch.int32, device=DEV)
    g = ctypes.c_int32()
    st = L.msp_vertices_grouping_noalloc(n, ctypes.c_void_p(rp.data_ptr()),
                                         ctypes.c_void_p(ci.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.byref(g), None)
    assert st == -1
    assert b"exceeds the maximum" in L.msp_noalloc_error()


def test_noalloc_rejects_row_pointers_outside_the_column_array():
    """A row pointer past row_ptr[n] is reported (MSP_ERR_PATTERN), never followed; col_idx
    is padded so that even a scan that followed it would stay inside the buffer."""
    a = grid_spe10(nx=8, ny=6, nz=4)
    rp = a.row_ptr.copy()
    rp[a.nb // 2] = a.nnzb + 5
    ci = np.concatenate([a.col_idx, np.arange(2 * a.nnzb + 16, dtype=np.int32) % a.nb])
    drp = torch.from_numpy(rp).to(DEV)
    dci = torch.from_numpy(ci.astype(np.int32)).to(DEV)
    out = torch.zeros(a.nb, dtype=torch.int32, device=DEV)
    L = msp._native.lib()
    g = ctypes.c_int32()
    st = L.msp_vertices_grouping_noalloc(a.nb, ctypes.c_void_p(drp.data_ptr()),
                                         ctypes.c_void_p(dci.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.byref(g), None)
    torch.cuda.synchronize()
    assert st == -2
