"""Stand-alone spectral Poisson solve (avl_field_solve) against the oracle."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O

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


@pytest.mark.parametrize("nx", [4, 15, 64, 512, 4096, 6000, 8192])
@pytest.mark.parametrize("soft,cP", [(1, 1.0), (0, 4 * np.pi)])
def test_field_solve_matches_oracle(A, nx, soft, cP):
    import torch
    rng = np.random.default_rng(nx)
    L = 3.7
    rho = rng.normal(size=nx) + 0.3
    r = torch.tensor(rho, dtype=torch.float64, device="cuda")
    E = torch.empty_like(r)
    st = torch.cuda.current_stream().cuda_stream
    A.check(A.avl_field_solve(nx, L, cP, soft, r.data_ptr(), E.data_ptr(), st))
    ref = O.poisson(nx, L, cP, soft, rho)
    err = np.linalg.norm(E.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-10, err


def test_field_solve_rejects_bad_arguments(A):
    assert A.avl_field_solve(2, 1.0, 1.0, 1, 1, 1, None) == A.AVL_EINVAL
    assert A.avl_field_solve(16, -1.0, 1.0, 1, 1, 1, None) == A.AVL_EINVAL
    assert A.avl_field_solve(16, 1.0, 1.0, 1, None, 1, None) == A.AVL_EINVAL
    assert b"nx" in A.avl_last_error(None) or b"NULL" in A.avl_last_error(None)
