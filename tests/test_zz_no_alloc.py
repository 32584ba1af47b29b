"""The allocation-free block product (scr_bsr_spmv_noalloc) against the
allocating one (scr_bsr_spmv), through the C ABI.

Callers that cannot let a library allocate device memory (hosts whose device
memory belongs to another allocator or is fixed at start-up, code that must
not call cudaFree, which waits for the whole device) use the allocation-free
entry point; it must give the same product.  This file is collected after
all the others so that a run stopping at the first failure has run them
before it; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

import fsi_inputs as F
from oracle.sparse import bsr_matvec_by_definition

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2206_06996_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def _random_bsr(rng, nbr, nbc, br, bc, max_per_row=15):
    rp = [0]
    cols = []
    for i in range(nbr):
        k = int(rng.integers(0, max_per_row + 1))
        cols.extend(np.sort(rng.choice(nbc, size=min(k, nbc), replace=False)).tolist())
        rp.append(len(cols))
    return F.BSR(br, bc, nbr, nbc, np.array(rp, np.int32), np.array(cols, np.int32),
                 rng.standard_normal(len(cols) * br * bc))


@pytest.mark.parametrize("br,bc", [(3, 3), (1, 3), (3, 1), (1, 1)])
def test_noalloc_matches_allocating_entry_point_twice(br, bc):
    rng = np.random.default_rng(br * 10 + bc)
    for call in range(2):  # two calls in a row share the static scratch
        M = _random_bsr(rng, 3000 + 17 * call, 2000, br, bc)
        Md = pkg.DeviceBSR.from_host(M)
        x = torch.as_tensor(rng.standard_normal(M.nb_cols * bc), device="cuda")
        y_ref = pkg.bsr_spmv(Md, x)
        y = torch.full((M.nb_rows * br,), float("nan"), dtype=torch.float64, device="cuda")
        pkg.bsr_spmv_noalloc(Md, x, y)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(b).max()))
        ref = bsr_matvec_by_definition(M, x.cpu().numpy())
        assert np.allclose(a, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_noalloc_on_the_solver_matrix():
    s = F.tube_system("tube_mini")
    Ad = pkg.DeviceBSR.from_host(s.A)
    x = torch.as_tensor(np.random.default_rng(1).standard_normal(3 * s.n_v), device="cuda")
    y = torch.empty(3 * s.n_v, dtype=torch.float64, device="cuda")
    for _ in range(2):
        pkg.bsr_spmv_noalloc(Ad, x, y)
        y_ref = pkg.bsr_spmv(Ad, x)
        assert torch.allclose(y, y_ref, rtol=1e-12, atol=1e-12 * float(y_ref.abs().max()))


def test_noalloc_rejects_matrices_beyond_its_scratch():
    nbr = 80000
    k = 3  # 80000 * 3 blocks * 9 = 2,160,000 stored scalars > 2,097,152
    rp = np.arange(0, nbr * k + 1, k, dtype=np.int32)
    col = np.tile(np.arange(k, dtype=np.int32), nbr)
    M = F.BSR(3, 3, nbr, nbr, rp, col, np.ones(nbr * k * 9))
    Md = pkg.DeviceBSR.from_host(M)
    x = torch.ones(3 * nbr, dtype=torch.float64, device="cuda")
    y = torch.empty(3 * nbr, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.ScrError) as e:
        pkg.bsr_spmv_noalloc(Md, x, y)
    assert e.value.status == 1 and "static scratch" in str(e.value)


def test_noalloc_rejects_invalid_columns():
    M = F.BSR(1, 1, 2, 2, np.array([0, 2, 3], np.int32), np.array([1, 0, 5], np.int32), np.ones(3))
    Md = pkg.DeviceBSR.from_host(M)
    x = torch.ones(2, dtype=torch.float64, device="cuda")
    y = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.ScrError) as e:
        pkg.bsr_spmv_noalloc(Md, x, y)
    assert e.value.status == 1
