"""Host-side accounting of the benchmark: the algorithmic bytes of one chain step and of one
solver step, written out term by term for the benchmark workload."""
import json

import pytest

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


def _fake_full():
    arm = {"steps": 12, "ms": 1.234567, "angle": 9e-4, "ritz_value_abs_error": [1e-7] * 20,
           "ritz_vector_angle": [1e-4] * 20}
    ttk = {"reference": {"certificate": {"davis_kahan_sin_theta_bound": 3e-7}}}
    ttk.update({a: dict(arm) for a in bench.TTK_ARMS})
    ttk.update(bench.ttk_ratios(ttk))
    return {"metric": bench.METRIC, "value": 1286.8, "unit": "GB/s", "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 5.088, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "sbm_n1000000_b20_deg16_k20", "l2": "x" * 300},
            "roofline": {"bound": "hbm", "achieved": 1245.0, "peak": 6799.6, "unit": "GB/s",
                         "frac": 0.183, "traffic": 2.095e8, "traffic_source": "y" * 200,
                         "kernel": "k_step_rowgroup", "per_launch_bytes": 1.48e8,
                         "launch_us": 119.2, "peak_kind": "measured (copy, burst)"},
            "e2e": {"value": 1273.0, "unit": "GB/s", "h2d_bytes_per_step": 8e7,
                    "d2h_bytes_per_step": 8e7, "ms_per_step": 5.14, "copies": "z" * 100},
            "cpu_baseline": {"value": 4.1, "unit": "GB/s", "cores": 16, "kind": "oracle",
                             "sample": "s" * 250, "single_thread": {"value": 0.3}},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 40},
            "gpu_launches": 900, "gather_ceiling": {"x": [1.0] * 500},
            "time_to_bottom_k": {"sbm_n2000_b4_k4": ttk, "sbm_regular_n1e6_b20_k20": ttk,
                                 "sbm_n2000_b4_k4_seeds_0_1_2": {0: {}, 1: {}, 2: {}}},
            "batched": {"ms": [0.1] * 1000}}


def test_headline_is_the_last_line_and_short(capsys, tmp_path):
    out = tmp_path / "extras.json"
    bench.emit(_fake_full(), str(out))
    lines = capsys.readouterr().out.strip().split("\n")
    last = json.loads(lines[-1])
    assert len(lines[-1]) <= 4096
    for key in ("metric", "value", "unit", "ms_per_step", "roofline", "e2e", "cpu_baseline",
                "clocks", "gpu_launches", "n_gpus", "steps", "warmup", "config"):
        assert key in last
    assert last["roofline"]["frac"] == 0.183 and last["e2e"]["h2d_bytes_per_step"] == 8e7
    ttk = last["time_to_bottom_k"]["sbm_regular_n1e6_b20_k20"]
    assert ttk["same_solver_speedup_oja"] == 1.0 and ttk["reference_sin_theta_bound"] == 3e-7
    # every extra measurement is on its own earlier line and in the extras file
    extras = {json.loads(x)["extra"] for x in lines[:-1]}
    assert {"gather_ceiling", "time_to_bottom_k", "batched"} <= extras
    assert json.load(open(out))["batched"]["ms"][0] == 0.1


def test_same_solver_ratios():
    r = bench.ttk_ratios({"plain_fp64_oja": {"ms": 10.0}, "dilated_mixed_oja": {"ms": 2.0},
                          "plain_fp64_mu_eg": {"ms": 30.0}, "dilated_mixed_mu_eg": {"ms": 5.0},
                          "dilated_fp64_oja": {"ms": 4.0}})
    assert r["same_solver_speedup_oja"] == 5.0 and r["same_solver_speedup_mu_eg"] == 6.0
    assert r["dilation_only_speedup_oja_fp64"] == 2.5
    assert r["speedup_best_dilated_vs_plain_fp64"] == 5.0  # best plain 10 over best dilated 2


def test_graded_k_picks_the_nearest_clear_gap():
    theta = [0.0, 0.9] + [1.8 + 0.001 * i for i in range(30)] + [2.7, 2.8, 2.9, 3.0, 3.1]
    k, gap = bench.pick_graded_k(theta, 20)
    assert k == 32 and gap > 0.3


def test_reference_certificate_matches_the_oracle():
    # the time-to-bottom-k certificate is host FP64 code of the benchmark's own (scipy.sparse
    # Laplacian, numpy Rayleigh-Ritz); its Ritz values and residual bound must agree with the
    # oracle's Rayleigh-Ritz and residual on a weighted graph and a perturbed bottom subspace
    import numpy as np
    import gen
    import oracle
    g = gen.uniform_edge_weights(gen.sbm(400, 4, 0.1, 0.005, seed=3), seed=4)
    lam, U = np.linalg.eigh(oracle.dense_laplacian(g))
    k, kp = 4, 8
    V = U[:, :kp] + 1e-6 * np.random.default_rng(0).standard_normal((g.n, kp))
    c = bench.certify_reference(g, V, k)
    theta, W = oracle.rayleigh_ritz(g, V)
    assert np.allclose(c["ritz_values"], theta[:k + 1], rtol=1e-10, atol=1e-12)
    Uk = V @ W[:, :k]
    R = oracle.laplacian_apply(g, Uk) - Uk * theta[:k]
    assert c["residual_2norm"] == pytest.approx(np.linalg.norm(R, 2), rel=1e-8)
    # the bound holds against the dense eigendecomposition
    ang = oracle.principal_angle_max(U[:, :k], Uk)
    assert np.sin(ang) <= c["davis_kahan_sin_theta_bound"] * (1 + 1e-9)


def test_streak_helper_matches_the_oracle():
    # the benchmark's streak (torch, on whatever device holds the blocks) against the oracle's
    # definition (Section 5.2) on CPU tensors: leading run of columns within eps of their
    # eigenvector, sign ignored
    import math
    import numpy as np
    import torch
    import oracle
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((60, 5)))
    for noise, flip in ((1e-3, False), (0.3, True), (0.05, True), (1.0, False)):
        V = U + noise * rng.standard_normal(U.shape)
        if flip:
            V[:, 1] *= -1.0
        for eps in (math.pi / 8, 0.05):
            n, ang = bench._streak_device(torch, torch.from_numpy(U), torch.from_numpy(V), 5, eps)
            assert n == oracle.eigenvector_streak(V, U, eps)
            for i in range(5):
                v = V[:, i] / np.linalg.norm(V[:, i])
                want = math.asin(min(1.0, np.linalg.norm(v - (v @ U[:, i]) * U[:, i])))
                assert ang[i] == pytest.approx(want, abs=1e-12)
