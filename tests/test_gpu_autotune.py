"""Schedule selection for the chain step: every schedule the tuner may pick (row group, merge
path at any share size) computes the same fused step (Section 2) as the FP64 oracle, the tuner
reports its timings and keeps its choice per graph and per shape."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, DEV, TOL, host, rel, stored, to_block

pytestmark = pytest.mark.gpu


def _hub_graph():
    return gen.random_graph(3001, 12000, seed=11, hub=5, hub_degree=1200, isolated=25)


@pytest.mark.parametrize("ipg", [32, 100, 256, 1024, 65536])
@pytest.mark.parametrize("xt,yt", [(torch.float64, torch.float64),
                                   (torch.bfloat16, torch.bfloat16)])
def test_every_merge_share_matches_oracle(ipg, xt, yt):
    g = gen.uniform_edge_weights(_hub_graph(), seed=12)
    G = sped.Graph.from_csr(g)
    G.set_schedule(2, ipg)
    k = 20
    X0 = gen.gaussian_block(g.n, k, seed=13)
    X = to_block(X0, xt)
    Y = sped.alloc_block(g.n, k, yt, DEV, fill=float("nan"))
    sped.poly_step(G, X, Y, k, alpha=0.0, beta=-0.02, gamma=1.0)  # split 0: the set schedule
    torch.cuda.synchronize()
    Xs = stored(X0, xt)
    assert_close(host(Y, k), Xs - 0.02 * oracle.laplacian_apply(g, Xs), TOL[yt])


@pytest.mark.parametrize("gname", ["hub", "sbm"])
def test_autotune_reports_and_keeps_a_valid_schedule(gname):
    g = _hub_graph() if gname == "hub" else gen.sbm(5000, 5, 0.01, 0.0004, seed=14)
    G = sped.Graph.from_csr(g)
    rep = G.autotune(8, torch.float64)
    assert rep["split"] in (1, 2)
    if not rep["cached"]:
        assert len(rep["ms"]) == 5 and all(t > 0 for t in rep["ms"])
        best = int(np.argmin(rep["ms"]))
        assert rep["split"] == (1 if best == 0 else 2)
        assert rep["merge_ipg"] == (0 if best == 0 else [128, 256, 512, 1024][best - 1])
    # p(L) V under the tuned schedule against the oracle
    ell, k = 7, 8
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = gen.gaussian_block(g.n, k, seed=15)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.apply_poly(G, V, Y, k)
    torch.cuda.synchronize()
    assert_close(host(Y, k), oracle.poly_limit(g, V0, info.scale_s, ell), 1e-12)


def test_autotune_table_serves_the_same_shape():
    g = _hub_graph()
    first = sped.Graph.from_csr(g).autotune(4, torch.bfloat16)
    again = sped.Graph.from_csr(g).autotune(4, torch.bfloat16)
    assert again["cached"]
    assert (again["split"], again["merge_ipg"]) == (first["split"], first["merge_ipg"])


def test_set_schedule_rejects_bad_arguments():
    G = sped.Graph.from_csr(gen.path(50))
    for split, ipg in [(3, 0), (-1, 0), (2, 7), (2, 1 << 21)]:
        with pytest.raises(sped.SpedError):
            G.set_schedule(split, ipg)
