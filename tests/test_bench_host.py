"""Host-side accounting of the benchmark: the algorithmic bytes of one chain step and of one
solver step, written out term by term for the benchmark workload."""
import bench


def test_chain_step_bytes():
    n, nnz, k = 1_000_000, 15_994_770, 20
    # row_ptr, col_idx, the input block read once, the output block written once (k columns)
    assert bench.spmm_bytes(n, nnz, k, 2, 2) == 4 * (n + 1) + 4 * nnz + 2 * n * k + 2 * n * k
    assert bench.spmm_bytes(n, nnz, k, 2, 2, weighted=True) == \
        bench.spmm_bytes(n, nnz, k, 2, 2) + 4 * nnz


def test_solver_step_bytes():
    n, nnz, k, ell = 1_000_000, 15_994_770, 20, 41
    chain, step = bench.step_bytes(n, nnz, k, ell)
    rp_ci = 4 * (n + 1) + 4 * nnz
    # first launch: BF16 shadow in, BF16 out; 39 middle launches BF16 -> BF16; last: F32 Y out
    want_chain = (rp_ci + 2 * n * k + 2 * n * k) * (ell - 1) + (rp_ci + 2 * n * k + 4 * n * k)
    assert chain == want_chain
    # Gram reads V and Y (F32); the update reads V and Y, writes V (F32) and its BF16 shadow
    assert step == chain + 2 * 4 * n * k + 3 * 4 * n * k + 2 * n * k
    assert round(step / 1e9, 2) == 6.55


def test_job_rate_counts_every_rank():
    assert bench._job_rate(4, 1e9, 2.0) == 4 * bench._job_rate(1, 1e9, 2.0)
