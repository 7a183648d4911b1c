"""The gather-rate probe (the benchmark's measurement library) gathers what it says it gathers:
per row the sum of the CSR neighbours' rows (mode 0) or of the next deg(r) rows (mode 2)."""
import numpy as np
import pytest
import torch

import gen
import paper_2207_14589_gb300 as sped
from paper_2207_14589_gb300 import probe
from util_gpu import DEV, host, stored, to_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [4, 20, 33])
def test_probe_sums_the_gathered_rows(k):
    g = gen.random_graph(3000, 12000, seed=61, hub=2, hub_degree=400)
    rp = torch.from_numpy(g.row_ptr).to(DEV)
    ci = torch.from_numpy(g.col_idx).to(DEV)
    X0 = gen.gaussian_block(g.n, k, seed=62)
    X = to_block(X0, torch.bfloat16)
    Xs = stored(X0, torch.bfloat16)
    deg = np.diff(g.row_ptr)
    for mode in (0, 1, 2):
        Y = sped.alloc_block(g.n, k, torch.bfloat16, DEV)
        probe.probe_gather(rp, ci, X, Y, k, mode=mode, seed=5)
        torch.cuda.synchronize()
        got = host(Y, k)
        if mode == 1:  # hashed rows: only the row sums' scale is checkable
            assert np.isfinite(got).all()
            continue
        want = np.empty_like(Xs)
        for r in range(g.n):
            if mode == 0:
                nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
            else:
                nb = (r + 1 + np.arange(deg[r])) % g.n
            want[r] = Xs[nb].sum(axis=0)
        scale = np.abs(Xs).max() * max(1, deg.max())
        assert np.abs(got - want).max() <= 2e-2 * scale
