"""Allocation-free field solve (avl_field_solve_noalloc).

It serves callers that cannot allocate device memory when they need a solve
(memory fully reserved by another allocator, or a loop that must not pay for
cudaMalloc / cudaFree).  Its scratch is a fixed device array shared by every
call, so this test runs it on consecutive calls with different grid sizes,
the largest ones included, and compares each result with the allocating
avl_field_solve.  The array and the solve's kernels are placed on the GPU by
the first call (lazy module loading), so a warm-up call comes first, as the
header asks of callers.  The file sorts last so that a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_03901_gb300 import build
    build.build()
    from paper_1804_03901_gb300 import avl
    return avl


def solve_pair(A, nx, soft, cP, seed):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(seed)
    rho = torch.tensor(rng.normal(size=nx) + 0.2, dtype=torch.float64, device="cuda")
    E_ref = torch.empty_like(rho)
    E = torch.full_like(rho, float("nan"))
    A.check(A.avl_field_solve(nx, 2.5, cP, soft, rho.data_ptr(), E_ref.data_ptr(), st))
    A.check(A.avl_field_solve_noalloc(nx, 2.5, cP, soft, rho.data_ptr(), E.data_ptr(), st))
    torch.cuda.synchronize()
    return (torch.linalg.norm(E - E_ref) / torch.linalg.norm(E_ref)).item()


def test_noalloc_matches_allocating_solve_on_consecutive_calls(A):
    # warm-up: the first call places the array and the kernels on the GPU
    assert solve_pair(A, 64, 1, 1.0, 99) < 1e-10
    # power-of-two grids with staged tables, the largest power of two (tables
    # read from the array), DFT grids up to the largest accepted nx
    cases = [(512, 1, 1.0), (96, 0, 4 * np.pi), (8192, 1, 1.0), (12288, 0, 1.0), (12798, 1, 4 * np.pi),
             (512, 1, 1.0)]
    for call, (nx, soft, cP) in enumerate(cases):
        err = solve_pair(A, nx, soft, cP, 100 + call)
        assert err < 1e-10, (call, nx, err)


def test_noalloc_rejects_grids_beyond_its_scratch(A):
    assert A.avl_field_solve_noalloc(12799, 1.0, 1.0, 1, 1, 1, None) == A.AVL_EINVAL
    assert b"12798" in A.avl_last_error(None)
