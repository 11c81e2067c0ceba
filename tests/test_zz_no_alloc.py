"""pic_poisson_solve_static -- the Poisson entry point for callers that cannot
allocate device memory while they run (its scratch is a fixed device array
inside the library) -- must give the same phi as pic_poisson_solve, whose
scratch the caller allocates.

Three calls in a row with different grids and data (the largest grid the
array holds, 256 x 512 cells, first) check that what one call leaves in the
shared array does not leak into the next.  The file is
named to be collected last; it builds and loads the library itself so that it
also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from parity import FIELD_TOL, field_err

pytestmark = pytest.mark.gpu

PIC_ERR_CAPACITY = -3


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_10727_gb300.pic import LIB_PATH
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, vp, vp]
    L.pic_poisson_solve.argtypes = sig + [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.pic_poisson_solve_static.argtypes = sig + [vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.pic_poisson_workspace_bytes.argtypes = [C.c_int, C.c_int]
    L.pic_poisson_workspace_bytes.restype = C.c_size_t
    return L


def _problem(nr, nz, seed):
    rng = np.random.default_rng(seed)
    R, L = 0.05, 0.05 * nz / nr
    Q = rng.normal(size=(nr + 1, nz + 1)) * 1e-15
    bc = np.zeros((nr + 1, nz + 1))
    bc[: int(0.7 * nr), 0] = -250.0 - 100.0 * rng.random()
    bc[:, nz] = rng.random(nr + 1)
    return R, L, Q, bc


def test_static_scratch_matches_caller_scratch(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for call, (nr, nz) in enumerate([(256, 512), (64, 48), (256, 256)]):
        R, L, Q, bc = _problem(nr, nz, seed=100 + call)
        Qd = torch.tensor(Q, device="cuda")
        phi_ref = torch.tensor(bc, device="cuda")
        phi_new = torch.tensor(bc, device="cuda")
        work = torch.empty(lib.pic_poisson_workspace_bytes(nr, nz), dtype=torch.uint8,
                           device="cuda")
        it_a, res_a = C.c_int(), C.c_double()
        it_b, res_b = C.c_int(), C.c_double()
        rc_a = lib.pic_poisson_solve(nr, nz, R, L, 1e-13, 500, Qd.data_ptr(), phi_ref.data_ptr(),
                                     work.data_ptr(), stream, C.byref(it_a), C.byref(res_a))
        rc_b = lib.pic_poisson_solve_static(nr, nz, R, L, 1e-13, 500, Qd.data_ptr(),
                                            phi_new.data_ptr(), stream, C.byref(it_b),
                                            C.byref(res_b))
        torch.cuda.synchronize()
        assert rc_a == 0 and rc_b == 0, (call, rc_a, rc_b)
        assert res_b.value <= 1e-13
        assert field_err(phi_new.cpu().numpy(), phi_ref.cpu().numpy()) <= FIELD_TOL
        assert it_b.value == it_a.value


def test_static_scratch_rejects_grids_above_its_maximum(lib):
    import torch
    nr = nz = 512
    Qd = torch.zeros((nr + 1, nz + 1), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(Qd)
    rc = lib.pic_poisson_solve_static(nr, nz, 0.05, 0.05, 1e-10, 100, Qd.data_ptr(), phi.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream, None, None)
    assert rc == PIC_ERR_CAPACITY
