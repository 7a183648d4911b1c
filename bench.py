"""Benchmark of the SPED hot path on one GB300 (or N replicas, one per GPU).

Workload (default): stochastic block model, N = 1,000,000 nodes in 20 equal blocks, mean degree
16 (14 inside the block, 2 outside), unweighted, k = 20. One step = one mixed-precision dilated
solver step: p(L) V by the limit form (I - sL)^l chained in BF16 (first step reads the F32
master, last step writes F32), the 2k x 2k Gram [V Y]^T [V Y], the k x k FP64 mu-EG algebra and the
N x k update. Value = algorithmic HBM bytes of the step / device time (GB/s).

Also measured: the dominant kernel (one chain step) against the HBM roofline and against the
gather-rate probe, the end-to-end rate through the C ABI with host buffers, the step replayed
from a CUDA graph, time-to-bottom-k (largest principal angle <= 1e-3) for the dilated
mixed-precision solver against the plain-L FP64 solver, and the FP64 CPU oracle; with the
extended measurements (default on, `--only-extra` selects): the walk estimator, edge
minibatches, the differentiable path, the batched solver, a permuted node order, the degree
threshold, the 3-room grid world and fitted polynomial coefficients.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "time-to-bottom-k (angle≤1e-3) dilated vs plain L; p(L)·V HBM GB/s vs roofline"
WORKLOAD = dict(n=1_000_000, blocks=20, p_in=14 / 49_999, p_out=2 / 950_000, k=20, ell=41)
SEED = gen.DEFAULT_SEED


def make_graph():
    w = WORKLOAD
    return gen.sbm(w["n"], w["blocks"], w["p_in"], w["p_out"], seed=SEED)


def spmm_bytes(n, nnz, k, b_in, b_out, weighted=False):
    """Algorithmic bytes of one chain step: row pointers, column indices (+ weights), the
    input block read once, the output block written once (k columns, not the padding)."""
    return 4 * (n + 1) + 4 * nnz + (4 * nnz if weighted else 0) + n * k * b_in + n * k * b_out


def step_bytes(n, nnz, k, ell, shadow=True):
    """One mixed-precision dilated solver step (F32 master V, BF16 chain, F32 Y). With the BF16
    shadow of V the first chain step reads the shadow and the update also writes it."""
    chain = spmm_bytes(n, nnz, k, 2 if shadow else 4, 2) + \
        (ell - 2) * spmm_bytes(n, nnz, k, 2, 2) + spmm_bytes(n, nnz, k, 2, 4)
    gram = n * k * 4 * 2
    update = n * k * 4 * 3 + (n * k * 2 if shadow else 0)
    return chain, chain + gram + update


# ----------------------------------------------------------------------------------------
def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_source_hash():
    """sha256 (first 16 hex digits) of the row-group chain kernel's source: spmm.cu up to its
    merge-path section, then the device helpers of sped_internal.cuh (element conversions and
    chunk loads / stores)."""
    h = hashlib.sha256()
    spmm = open(os.path.join(ROOT, "paper_2207_14589_gb300/csrc/spmm.cu"), "rb").read()
    cut = spmm.find(b"// merge path")
    h.update(spmm[:cut] if cut >= 0 else spmm)
    hdr = open(os.path.join(ROOT, "paper_2207_14589_gb300/csrc/sped_internal.cuh"), "rb").read()
    a, b = hdr.find(b"// device helpers"), hdr.find(b"// Philox4x32-10")
    h.update(hdr[a:b] if 0 <= a < b else hdr)
    return h.hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "step_rowgroup_bf16_sbm1e6_k20.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic per launch \(bytes\):\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != _kernel_source_hash():
        return None
    return float(t.group(1))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"sped_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        time.sleep(0.2)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if hasattr(self, "f"):
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                         "sw_power_cap"]
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def _max_over_ranks(x, world, device="cpu"):
    """The job's time is its slowest rank's: the largest x over the ranks (x itself on one)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(world, bytes_per_rank_step, ms_per_step):
    """Whole-job GB/s: every rank processes its own replica's bytes in the job's step time."""
    return world * bytes_per_rank_step / (ms_per_step * 1e-3) / 1e9


def _angle_and_delta(sped, Vstar, V, k):
    """Largest principal angle between span(V*) and span(V), and the subspace error of Section
    5.2, delta = 1 - tr(U* P) / k = 1 - ||Q*^T Q_V||_F^2 / k, both from their FP64 Gram."""
    G = sped.gram(Vstar, k, V, k).cpu().numpy()
    Ps, C, Pv = G[:k, :k], G[:k, k:], G[k:, k:]
    Rs = np.linalg.cholesky(Ps)
    Rv = np.linalg.cholesky(Pv)
    M = np.linalg.solve(Rs, np.linalg.solve(Rv, C.T).T)  # Q*^T Q_V
    smin = np.linalg.svd(M, compute_uv=False).min()
    ang = float(math.asin(math.sqrt(max(0.0, 1.0 - min(1.0, smin) ** 2))))
    return ang, float(max(0.0, 1.0 - np.sum(M * M) / k))


def _principal_angle(sped, Vstar, V, k):
    """Largest principal angle between span(V*) and span(V) from their FP64 Gram."""
    return _angle_and_delta(sped, Vstar, V, k)[0]


def certify_reference(g, Vs, k):
    """Davis-Kahan certificate of a reference subspace, computed on the host in FP64 with
    scipy.sparse (the Laplacian written out from the CSR arrays) and numpy, so that the reference
    the arms are graded against does not rest on the GPU path alone. Rayleigh-Ritz of L on
    span(Vs) (kp >= k + 1 columns, orthonormalised by QR) gives Ritz pairs (theta_i, u_i); the
    residual block R = L U_k - U_k Theta_k of the first k Ritz vectors and the gap
    delta = theta_{k+1} - theta_k to the first guard Ritz value bound the largest principal
    angle between span(U_k) and the bottom-k eigenvectors of L by sin(theta_max) <= ||R||_2 /
    delta (sin-theta theorem; delta stands in for lambda_{k+1} - theta_k, as the guard vectors
    estimate lambda_{k+1})."""
    import scipy.sparse as sp
    n = g.n
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    A = sp.csr_matrix((w, g.col_idx.astype(np.int64), g.row_ptr.astype(np.int64)), shape=(n, n))
    L = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    Q, _ = np.linalg.qr(np.ascontiguousarray(Vs, dtype=np.float64))
    H = Q.T @ (L @ Q)
    theta, Z = np.linalg.eigh(0.5 * (H + H.T))
    U = Q @ Z[:, :k]
    R = L @ U - U * theta[:k]
    rnorm = float(math.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ R).max())))
    gap = float(theta[k] - theta[k - 1])
    return {"by": "host FP64 (scipy.sparse Laplacian, numpy Rayleigh-Ritz and residual of the "
                  "GPU reference block)",
            "ritz_values": [float(x) for x in theta[:k + 1]],
            "residual_2norm": rnorm, "gap_theta_k1_minus_theta_k": gap,
            "davis_kahan_sin_theta_bound": rnorm / gap if gap > 0 else None}


def _eigen_errors(sped, torch, G, V, k, master, Vref, theta_ref, dense):
    """Per-eigenpair errors of an arm's result: its Ritz values of L against the reference's
    (and the dense eigendecomposition's when given), and the angle between each of its Ritz
    vectors and the matching reference Ritz vector (Vref holds the reference Ritz vectors)."""
    X = V.clone()
    theta, _ = sped.rayleigh_ritz(G, X, k, rotate=True)
    theta = theta.cpu().numpy()
    C = sped.gram(Vref, k, X.to(torch.float64) if master != torch.float64 else X, k).cpu().numpy()
    cos = np.clip(np.abs(np.diag(C[:k, k:])) / np.sqrt(np.diag(C[:k, :k]) * np.diag(C[k:, k:])),
                  0.0, 1.0)
    out = {"ritz_value_abs_error": [float(x) for x in np.abs(theta - theta_ref)],
           "ritz_vector_angle": [float(x) for x in np.arccos(cos)]}
    if dense is not None:
        lam, U = dense
        Xh = X[:, :k].double().cpu().numpy()
        Xh /= np.linalg.norm(Xh, axis=0)
        out["dense_eigenvalue_abs_error"] = [float(x) for x in np.abs(theta - lam)]
        out["dense_eigenvector_angle"] = [float(x) for x in
                                          np.arccos(np.clip(np.abs(np.sum(Xh * U, axis=0)), 0, 1))]
    return out


TTK_ARMS = {
    # name: polynomial, solver, eta (None = 2 / lambda*), chain phases, master dtype, step cap
    "dilated_mixed_mu_eg": dict(poly=("limit", 7), solver="mu_eg", eta=1.5,
                                chain=("bf16", "f32"), master="f32", cap=400),
    "dilated_mixed_oja": dict(poly=("limit", 15), solver="oja", eta=0.0,
                              chain=("bf16", "f32"), master="f32", cap=200),
    # Chebyshev filter T_15 on [(theta_k + theta_{k+1}) / 2, lambda_bound] (the reference's
    # Ritz values): damps the unwanted part of the spectrum, grows fastest below it
    "chebyshev_filter_mixed_oja": dict(poly=("cheb", 15), solver="oja", eta=0.0,
                                       chain=("bf16", "f32"), master="f32", cap=200),
    # the same solvers in FP64 on the dilated operator, then on the plain reversed Laplacian
    # lambda* I - L (Eq. reveig): same-solver ratios separate the dilation's gain from the
    # choice of solver and from the precision
    "dilated_fp64_oja": dict(poly=("limit", 15), solver="oja", eta=0.0,
                             chain=("f64",), master="f64", cap=200),
    "plain_fp64_oja": dict(poly=("shift", 1), solver="oja", eta=0.0,
                           chain=("f64",), master="f64", cap=3000),
    "plain_fp64_mu_eg": dict(poly=("shift", 1), solver="mu_eg", eta=None,
                             chain=("f64",), master="f64", cap=3000),
    "plain_fp32_mu_eg": dict(poly=("shift", 1), solver="mu_eg", eta=None,
                             chain=("f32",), master="f32", cap=3000),
}


def time_to_bottom_k(sped, torch, g, k, dev, stream, ell_ref, ref_steps=14, seed=SEED,
                     certify=True, kp=None, arms=None):
    """Time to reach a largest principal angle <= 1e-3 to the bottom-k subspace, per arm.

    Reference subspace: FP64 subspace iteration on the dilated operator (l = ell_ref) run far
    past the tolerance; its invariant-subspace residual is reported. Each arm runs twice from the
    same V0: an instrumented pass (angle after every step; the mixed-precision arms also read
    the residual statistics to decide when the BF16 chain has stalled and switch to an F32
    chain) and a timed pass that replays exactly the recorded schedule without any checks."""
    dt = {"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}
    G = sped.Graph.from_csr(g, device=dev)
    n = g.n
    V0 = torch.from_numpy(gen.gaussian_block(n, k, seed=seed)).to(dev)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell_ref)
    # reference: k + 4 vectors (the extra ones speed it up and estimate lambda_{k+1})
    kp = kp or k + 4
    Vs = sped.alloc_block(n, kp, torch.float64, dev)
    Vs[:, :kp] = torch.from_numpy(gen.gaussian_block(n, kp, seed=seed + 31)).to(dev)
    Vs[:, :k] = V0
    ref_opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    stats = torch.zeros(3 * kp, dtype=torch.float64, device=dev)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, ref_opts, kp), dtype=torch.uint8, device=dev)
    for _ in range(ref_steps):
        sped.eig_step(G, Vs, kp, ref_opts, stats=stats, scratch=scr)
    torch.cuda.synchronize()
    ref_residual = float(stats[kp:kp + k].max())  # residuals of the first k columns
    stats = stats[:3 * k]
    # reference Ritz pairs of L (rotate the reference block into its Ritz vectors, ascending: its
    # first k columns span the reference bottom-k subspace)
    theta_all, _ = sped.rayleigh_ritz(G, Vs, kp, rotate=True)
    theta_all = theta_all.cpu().numpy()
    theta_ref = theta_all[:k]
    out = {"graph": g.name, "n": n, "nnz": g.nnz, "k": k,
           "reference": {"solver": "oja_fp64_limit", "degree": ell_ref, "steps": ref_steps,
                         "vectors": kp, "ritz_value_k_plus_1": float(theta_all[k]),
                         "invariant_subspace_residual": ref_residual,
                         "ritz_values": [float(x) for x in theta_ref]}}
    if certify:
        out["reference"]["certificate"] = certify_reference(
            g, Vs[:, :kp].cpu().numpy(), k)
    dense = None
    if n <= 4000:  # small graph: also against the dense FP64 eigendecomposition of L
        Ld = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
        Ld[rows, g.col_idx] = -(g.w if g.w is not None else 1.0)
        Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
        lam, U = np.linalg.eigh(Ld)
        dense = (lam[:k], U[:, :k])
        out["reference"]["dense_eigenvalue_error_max"] = float(np.abs(theta_ref - lam[:k]).max())
    del scr
    for name, a in TTK_ARMS.items():
        if arms is not None and name not in arms:
            continue
        if a["poly"][0] == "limit":
            info = G.set_polynomial(sped.POLY_LIMIT_EXP, a["poly"][1])
        elif a["poly"][0] == "cheb":
            d = a["poly"][1]
            info = G.set_polynomial(sped.POLY_CHEBYSHEV, d,
                                    eps=0.5 * float(theta_all[k - 1] + theta_all[k]),
                                    coeffs=[0.0] * d + [1.0])
        else:
            info = G.set_polynomial(sped.POLY_SHIFT, 1)
        eta = a["eta"] if a["eta"] is not None else 2.0 / info.lambda_star
        solver = sped.MU_EG if a["solver"] == "mu_eg" else sped.OJA
        master = dt[a["master"]]
        opts = {c: sped.step_opts(solver, eta, dt[c], master) for c in a["chain"]}
        scr = torch.empty(max(sped.eig_step_scratch_bytes(G, o, k) for o in opts.values()),
                          dtype=torch.uint8, device=dev)
        V = sped.alloc_block(n, k, master, dev)
        V[:, :k] = V0.to(master)
        phase, hist, schedule, steps, ang, delta = 0, [], [], None, None, None
        for t in range(1, a["cap"] + 1):
            c = a["chain"][phase]
            sped.eig_step(G, V, k, opts[c], stats=stats, scratch=scr)
            schedule.append(c)
            if phase + 1 < len(a["chain"]):
                res = float(stats[k:2 * k].max())
                hist.append(res)
                if res <= 3e-3 or (len(hist) >= 4 and res > 0.9 * hist[-4]):
                    phase += 1
            if t <= 400 or t % 10 == 0:
                ang, delta = _angle_and_delta(sped, Vs, V, k)
                if ang <= 1e-3:
                    steps = t
                    break
        rec = {"steps": steps, "angle": ang, "subspace_error_delta": delta,
               "degree": info.degree, "eta": eta,
               "spmm": None if steps is None else steps * info.degree,
               "chain_schedule": {c: schedule.count(c) for c in a["chain"]}}
        if steps is not None:
            V[:, :k] = V0.to(master)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for c in schedule:
                sped.eig_step(G, V, k, opts[c], scratch=scr)
            e1.record(stream)
            e1.synchronize()
            rec["ms"] = e0.elapsed_time(e1)
            rec["angle_after_timed_run"] = _principal_angle(sped, Vs, V, k)
            rec.update(_eigen_errors(sped, torch, G, V, k, master, Vs, theta_ref, dense))
        out[name] = rec
        del scr, V
    out.update(ttk_ratios(out))
    return out


def ttk_ratios(out):
    """Speed-ups from the arms' device times: the same solver on the plain reversed Laplacian
    (FP64) over the dilated operator (mixed precision, and FP64 to isolate the dilation), and the
    best dilated arm over the best plain FP64 arm."""
    ms = lambda a: (out.get(a) or {}).get("ms")
    r = {}
    for key, plain, dil in (("same_solver_speedup_oja", "plain_fp64_oja", "dilated_mixed_oja"),
                            ("same_solver_speedup_mu_eg", "plain_fp64_mu_eg",
                             "dilated_mixed_mu_eg"),
                            ("dilation_only_speedup_oja_fp64", "plain_fp64_oja",
                             "dilated_fp64_oja")):
        if ms(plain) and ms(dil):
            r[key] = ms(plain) / ms(dil)
    plains = [ms(a) for a in ("plain_fp64_oja", "plain_fp64_mu_eg") if ms(a)]
    dils = [ms(a) for a in ("dilated_mixed_oja", "dilated_mixed_mu_eg") if ms(a)]
    if plains and dils:
        r["speedup_best_dilated_vs_plain_fp64"] = min(plains) / min(dils)
    if ms("plain_fp64_mu_eg") and ms("chebyshev_filter_mixed_oja"):
        r["speedup_chebyshev_filter_vs_plain_fp64"] = \
            min(plains) / ms("chebyshev_filter_mixed_oja")
    return r


def pick_graded_k(theta, k_min, rel_gap=0.05):
    """The smallest k >= k_min whose Ritz gap theta_{k+1} - theta_k is at least rel_gap of
    theta_{k+1} (a gap the solvers resolve in tens of steps), else the k with the largest
    relative gap (theta ascending, the last few values left as guards)."""
    theta = np.asarray(theta, dtype=np.float64)
    last = len(theta) - 4
    rel = [(theta[j] - theta[j - 1]) / max(abs(theta[j]), 1e-300) for j in range(1, len(theta))]
    for kk in range(k_min, last + 1):
        if rel[kk - 1] >= rel_gap:
            return kk, rel[kk - 1]
    kk = int(np.argmax(rel[k_min - 1:last])) + k_min
    return kk, rel[kk - 1]


def ttk_benchmark_graph(sped, torch, g, G, dev, stream, k_min, ell, kp=40, probe_steps=40,
                        min_rel_gap=0.02):
    """Time-to-bottom-k on the benchmark SBM itself. Its bottom-20 sits inside a cluster of
    block modes and modes localized at low-degree nodes with no clear gap after the 20th, so the
    angle is graded at the nearest k >= 20 with a clear gap: an FP64 subspace iteration with kp
    vectors on the dilated operator gives the Ritz values, pick_graded_k picks k (leaving four
    guard vectors for the reference), and the mixed-precision dilated arms race the plain-L
    FP64 arms at that k. When no gap of at least min_rel_gap exists below kp - 4 (the solver
    path takes k <= 40), the probe is reported and nothing is graded."""
    res, _ = spectrum_probe(sped, torch, G, g.n, dev, kp=kp, steps=(probe_steps,))
    theta = res[probe_steps]["ritz"]
    kk, gap = pick_graded_k(theta, k_min)
    name = f"sbm_n{g.n}_b{WORKLOAD['blocks']}_deg16_benchmark_graph"
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    if gap < min_rel_gap:
        return {name: {"graded": False, "probe_ritz_values": theta,
                       "probe_max_residual": res[probe_steps]["max_residual"],
                       "why": f"no relative Ritz gap >= {min_rel_gap} for k in [{k_min}, "
                              f"{kp - 4}] (largest {gap:.3g} at k = {kk}); the solver path "
                              f"takes k <= 40"}}
    r = time_to_bottom_k(sped, torch, g, kk, dev, stream, ell, ref_steps=40, kp=min(kk + 4, 40),
                         arms=("dilated_mixed_oja", "dilated_mixed_mu_eg", "dilated_fp64_oja",
                               "plain_fp64_oja", "plain_fp64_mu_eg"))
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    r["k_graded"] = kk
    r["why_k"] = (f"bottom-{k_min} is not separated from the next Ritz values; k = {kk} is the "
                  f"nearest with a relative gap {gap:.3g} (probe: {kp} FP64 vectors, "
                  f"{probe_steps} steps)")
    r["probe_ritz_values"] = theta
    return {name: r}


def ritz_spectrum(sped, torch, G, V, k):
    """Rayleigh-Ritz values of L on span(V) (ascending) from the FP64 Gram of [V, L V]."""
    n = V.shape[0]
    LV = sped.alloc_block(n, k, torch.float64, V.device)
    sped.poly_step(G, V, LV, k, alpha=0.0, beta=1.0, gamma=0.0)
    Gm = sped.gram(V, k, LV, k).cpu().numpy()
    P, H = Gm[:k, :k], Gm[:k, k:]
    H = 0.5 * (H + H.T)
    R = np.linalg.cholesky(P)
    Ri = np.linalg.inv(R)
    return np.linalg.eigvalsh(Ri @ H @ Ri.T)


def spectrum_probe(sped, torch, G, n, dev, kp=32, steps=(10, 20, 30)):
    """Bottom of the spectrum by FP64 subspace iteration on the dilated operator with kp
    vectors; Ritz values after each listed step count."""
    G.set_polynomial(sped.POLY_LIMIT_EXP, WORKLOAD["ell"])
    V = sped.alloc_block(n, kp, torch.float64, dev)
    V[:, :kp] = torch.from_numpy(gen.gaussian_block(n, kp, seed=SEED + 7)).to(dev)
    opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    stats = torch.zeros(3 * kp, dtype=torch.float64, device=dev)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, kp), dtype=torch.uint8, device=dev)
    out, done = {}, 0
    for s in steps:
        for _ in range(s - done):
            sped.eig_step(G, V, kp, opts, stats=stats, scratch=scr)
        done = s
        out[s] = {"ritz": [float(x) for x in ritz_spectrum(sped, torch, G, V, kp)],
                  "max_residual": float(stats[kp:2 * kp].max())}
    return out, V


def cpu_baseline(g, sample_steps=None, threads=None):
    """The FP64 oracle (as it stands) on a bounded sample of the same work: a few chain steps
    X <- X - sL X on the full graph at k = 20, run at once on `threads` host threads (default:
    all cores; the oracle's C loops release the interpreter lock), each thread on its own
    block; the single-thread figure is reported beside it."""
    import concurrent.futures as cf
    import oracle
    k = WORKLOAD["k"]
    s = 1.0 / WORKLOAD["ell"]
    V = gen.gaussian_block(g.n, k, seed=SEED)
    t0 = time.perf_counter()
    oracle.poly_limit(g, V, s, 1)
    one = time.perf_counter() - t0
    m = sample_steps or max(1, min(40, int(12.0 / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.poly_limit(g, V, s, m)
    dt1 = time.perf_counter() - t0
    b1 = m * spmm_bytes(g.n, g.nnz, k, 2, 2)
    nt = threads or os.cpu_count() or 1
    blocks = [gen.gaussian_block(g.n, k, seed=SEED + 1 + i) for i in range(nt)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        list(ex.map(lambda X: oracle.poly_limit(g, X, s, m), blocks))
    dtn = time.perf_counter() - t0
    return {"value": nt * b1 / dtn / 1e9, "unit": "GB/s", "cores": nt, "kind": "oracle",
            "sample": f"{nt} host threads each running {m} limit-form chain steps "
                      f"X <- X - sL X over the full graph (k={k}, FP64) on its own block, "
                      f"{dtn:.2f} s wall; bytes counted as one BF16 chain step of the GPU arm",
            "single_thread": {"value": b1 / dt1 / 1e9, "cores": 1, "seconds": dt1, "steps": m}}


def measure_permuted(sped, torch, dev, stream, k, ell, steps=20):
    """The benchmark step on the same SBM with its node order randomly permuted (block
    structure no longer follows node ids)."""
    w = WORKLOAD
    g = gen.sbm(w["n"], w["blocks"], w["p_in"], w["p_out"], seed=SEED, permute=True)
    G = sped.Graph.from_csr(g, device=dev)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V0 = torch.from_numpy(gen.gaussian_block(g.n, k, seed=SEED)).to(dev)
    V[:, :k] = (V0 / V0.norm(dim=0)).float()
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=dev)
    step = lambda: sped.eig_step(G, V, k, opts, scratch=scr)
    for _ in range(3):
        step()
    ms = _timed(torch, stream, step, steps)
    _, step_b = step_bytes(g.n, g.nnz, k, ell, shadow=False)
    return {"workload": f"sbm_n{g.n}_b{w['blocks']}_deg16_k{k}_permuted", "nnz": g.nnz,
            "ms_per_step": ms, "gbs": step_b / (ms * 1e-3) / 1e9}


# ----------------------------------------------------------------------------------------
def _timed(torch, stream, fn, reps):
    """Mean device time (ms) of fn() over reps calls, CUDA events on the launching stream."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_stochastic(sped, torch, g, G, dev, stream, k, ell, reps=5, err_degrees=(1, 3, 7)):
    """Sampled-term estimate of p(L)V (Section 4.3) on the benchmark graph with M = nnz
    walkers, so that M l matches the nnz l row touches of the exact chain: walk steps per
    second and effective GB/s (the exact F32 chain's algorithmic bytes over the estimate's time)
    at the benchmark degree, and the relative error of one estimate against the exact F32 chain
    at that and smaller degrees (the estimator samples the monomial expansion, whose terms grow
    like (1 + s lambda)^l against a result of size |1 - s lambda|^l, so its variance explodes
    with the degree)."""
    M = g.nnz
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(g.n, k, seed=SEED + 11)).to(dev)
    Yx = sped.alloc_block(g.n, k, torch.float32, dev)
    Y = sped.alloc_block(g.n, k, torch.float32, dev)
    scr = torch.empty(sped.apply_poly_scratch_bytes(G, k, torch.float32), dtype=torch.uint8,
                      device=dev)
    out = {"walkers": M, "degree": ell, "k": k}
    seed = [SEED]
    for deg in sorted(set(err_degrees) | {ell}):
        G.set_polynomial(sped.POLY_LIMIT_EXP, deg)
        exact = lambda: sped.apply_poly(G, V, Yx, k, chain_dtype=torch.float32, scratch=scr)
        exact()
        ynorm = float(torch.linalg.vector_norm(Yx[:, :k].double()))
        rec = {}
        if deg == ell:
            rec["exact_f32_chain_ms"] = _timed(torch, stream, exact, reps)
            rec["exact_f32_chain_bytes"] = deg * spmm_bytes(g.n, g.nnz, k, 4, 4)
        for mode, name in ((sped.STOCHASTIC_IS, "importance_weighted"),
                           (sped.STOCHASTIC_REJECT, "rejection")):
            scr_s = torch.empty(sped.apply_poly_scratch_bytes(G, k, torch.float32, mode),
                                dtype=torch.uint8, device=dev)

            def est():
                seed[0] += 1
                sped.apply_poly(G, V, Y, k, chain_dtype=torch.float32, mode=mode, walkers=M,
                                seed=seed[0], scratch=scr_s)
            est()
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm((Y[:, :k] - Yx[:, :k]).double())) / ynorm
            r = {"relative_error_vs_exact": err}
            if deg == ell:
                ms = _timed(torch, stream, est, reps)
                r.update({"ms": ms, "walk_steps_per_s": M * deg / (ms * 1e-3),
                          "effective_gbs": rec["exact_f32_chain_bytes"] / (ms * 1e-3) / 1e9})
            rec[name] = r
            del scr_s
        out[f"degree_{deg}"] = rec
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    return out


def measure_minibatch(sped, torch, g, G, dev, stream, k, ell, reps=5,
                      batches=(1 << 18, 1 << 20, 1 << 22), sbm_steps=(10, 40, 100)):
    """Edges fed in minibatches (the stochastic optimisation model of Sections 2 and 6): every
    multiplication by L in the limit-form chain uses its own estimate (|E|/B) sum_j w x x^T from
    B uniform edge draws (or, stratified, one draw per contiguous stratum of the edge order,
    weighted by the stratum's size). On the benchmark graph (F32 chain and blocks): time per
    estimate of p(L) V, edges per second and the relative error against the exact F32 chain for
    each B and both samplers;
    the two launches of one chain step at B = 2^20 timed apart (dense pass Y = X, then the edge
    scatter) with the scatter's algorithmic bytes per draw (edge id lookups 12 B, two X rows
    read, two Y rows read and written by atomics). On the small SBM (N = 2,000, 4 blocks, k = 4,
    B = |E|/4 per multiplication, FP64): mu-EG with the plain reversed Laplacian against the
    limit form of degree 7, largest principal angle to the dense bottom-k after a few step
    counts (a fixed step size stops at a noise floor set by the minibatch variance)."""
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    info = G.info()
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(g.n, k, seed=SEED + 41)).to(dev)
    Yx = sped.alloc_block(g.n, k, torch.float32, dev)
    Y = sped.alloc_block(g.n, k, torch.float32, dev)
    mode = sped.STOCHASTIC_MINIBATCH
    scr = torch.empty(max(sped.apply_poly_scratch_bytes(G, k, torch.float32),
                          sped.apply_poly_scratch_bytes(G, k, torch.float32, mode),
                          sped.apply_poly_scratch_bytes(G, k, torch.float32,
                                                        sped.STOCHASTIC_MINIBATCH_STRATIFIED)),
                      dtype=torch.uint8, device=dev)
    sped.apply_poly(G, V, Yx, k, chain_dtype=torch.float32, scratch=scr)
    ynorm = float(torch.linalg.vector_norm(Yx[:, :k].double()))
    out = {"graph_edges": info.n_edges, "degree": ell, "k": k, "dtype": "f32"}
    # the two launches of one step, timed apart
    B = 1 << 20
    a, b, wv = sped.sample_edges(G, SEED, 0, B)
    empty = a[:0]
    dense = lambda: sped.edge_step(g.n, V, Y, k, empty, empty, None, gamma=1.0)
    full = lambda: sped.edge_step(g.n, V, Y, k, a, b, wv, edge_scale=info.n_edges / B,
                                  beta=-info.scale_s, gamma=1.0)
    dense()
    full()
    ms_d = _timed(torch, stream, dense, 20)
    ms_f = _timed(torch, stream, full, 20)
    # one chain step as the chain runs it (edges drawn inside the scatter)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 1)
    one = lambda: sped.apply_poly(G, V, Y, k, chain_dtype=torch.float32, mode=mode, walkers=B,
                                  seed=SEED, scratch=scr)
    one()
    ms_one = _timed(torch, stream, one, 20)
    per_draw = 12 + 2 * k * 4 + 2 * 2 * k * 4
    scatter_ms = max(ms_f - ms_d, 1e-6)
    peak, peak_src = _peaks()
    out["step_b1048576"] = {
        "dense_ms": ms_d, "dense_gbs": 2 * g.n * k * 4 / (ms_d * 1e-3) / 1e9,
        "dense_frac": 2 * g.n * k * 4 / (ms_d * 1e-3) / 1e9 / peak,
        "peak_gbs": peak, "peak_source": peak_src,
        "scatter_ms": scatter_ms, "scatter_bytes_per_draw": per_draw,
        "scatter_gbs": B * per_draw / (scatter_ms * 1e-3) / 1e9,
        "draws_per_s": B / (scatter_ms * 1e-3),
        "chain_step_drawn_ms": ms_one,
        "drawn_scatter_ms": max(ms_one - ms_d, 1e-6)}
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    seed = [SEED]
    for md, tag in ((mode, "batch"), (sped.STOCHASTIC_MINIBATCH_STRATIFIED, "stratified_batch")):
        for B in batches:
            def est():
                seed[0] += 1
                sped.apply_poly(G, V, Y, k, chain_dtype=torch.float32, mode=md, walkers=B,
                                seed=seed[0], scratch=scr)
            est()
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm((Y[:, :k] - Yx[:, :k]).double())) / ynorm
            ms = _timed(torch, stream, est, reps)
            out[f"{tag}_{B}"] = {"ms": ms, "edges_per_s": ell * B / (ms * 1e-3),
                                 "batch_over_edges": B / info.n_edges,
                                 "relative_error_vs_exact": err}
    del scr, V, Y, Yx
    # stochastic mu-EG on the small SBM
    gs = gen.sbm(2000, 4, 0.05, 0.001, seed=SEED)
    n, ks = gs.n, 4
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(gs.row_ptr))
    Ld[rows, gs.col_idx] = -1.0
    Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
    lam, U = np.linalg.eigh(Ld)
    Ud = sped.alloc_block(n, ks, torch.float64, dev)
    Ud[:, :ks] = torch.from_numpy(U[:, :ks]).to(dev)
    Gs = sped.Graph.from_csr(gs, device=dev)
    Bs = Gs.info().n_edges // 4
    V0 = torch.from_numpy(gen.gaussian_block(n, ks, seed=SEED + 43)).to(dev)
    sb = {"graph": "sbm_n2000_b4_k4", "batch": Bs, "edges": Gs.info().n_edges}
    for name, poly, eta, md in (("plain_mu_eg", ("shift", 1), None, mode),
                                ("limit7_mu_eg", ("limit", 7), 0.5, mode),
                                ("plain_mu_eg_stratified", ("shift", 1), None,
                                 sped.STOCHASTIC_MINIBATCH_STRATIFIED),
                                ("limit7_mu_eg_stratified", ("limit", 7), 0.5,
                                 sped.STOCHASTIC_MINIBATCH_STRATIFIED)):
        inf = (Gs.set_polynomial(sped.POLY_LIMIT_EXP, 7) if poly[0] == "limit"
               else Gs.set_polynomial(sped.POLY_SHIFT, 1))
        e = eta if eta is not None else 2.0 / inf.lambda_star
        opts = sped.step_opts(sped.MU_EG, e, torch.float64, torch.float64, mode=md, walkers=Bs,
                              seed=SEED)
        scr = torch.empty(sped.eig_step_scratch_bytes(Gs, opts, ks), dtype=torch.uint8,
                          device=dev)
        Vb = sped.alloc_block(n, ks, torch.float64, dev)
        Vb[:, :ks] = V0
        rec = {"eta": e, "degree": inf.degree}
        for t in range(1, max(sbm_steps) + 1):
            opts.seed = SEED + 7919 * t
            sped.eig_step(Gs, Vb, ks, opts, scratch=scr)
            if t in sbm_steps:
                rec[f"angle_step_{t}"] = _principal_angle(sped, Ud, Vb, ks)
        rec["edges_per_step"] = Bs * inf.degree
        sb[name] = rec
    out["sbm_mu_eg"] = sb
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    return out


def measure_degree_sweep(sped, torch, dev, stream, k=4, cap=200,
                         degrees=(11, 51, 151, 251)):
    """The limit form's degree threshold (cliques graphs of Section 5.4): four 450-cliques joined
    by 25 short-circuit edges (lambda_max near 450). With the table's scale s = 1/l the factor
    |1 - s lambda| exceeds 1 on the clique modes for l = 11, 51, 151 and the dilated operator's
    dominant eigenvectors are no longer the bottom of L; at l = 251 it stays below 1. The
    automatic scale (s = 2 / lambda_bound when l < lambda_bound / 2) keeps every degree
    correct. Oja (subspace iteration, eta = 0) in FP64, steps to a largest principal angle
    <= 1e-3 against the dense eigendecomposition. The Taylor series of -e^{-L} and of
    log(L + eps) run at the same degrees (App. A.3 compares the series families)."""
    g = gen.cliques([450] * 4, short_circuit=25, seed=SEED)
    n = g.n
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    Ld[rows, g.col_idx] = -1.0
    Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
    lam, U = np.linalg.eigh(Ld)
    Ud = sped.alloc_block(n, k, torch.float64, dev)
    Ud[:, :k] = torch.from_numpy(U[:, :k]).to(dev)
    G = sped.Graph.from_csr(g, device=dev)
    V0 = torch.from_numpy(gen.gaussian_block(n, k, seed=SEED + 23)).to(dev)
    opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    out = {"graph": "cliques_4x450_sc25", "n": n, "nnz": g.nnz, "k": k,
           "lambda_max": float(lam[-1]), "eigengap_k": float(lam[k] - lam[k - 1])}
    for deg in degrees:
        for rule, scale in (("table_s_1_over_l", 1.0 / deg), ("automatic_s", 0.0)):
            info = G.set_polynomial(sped.POLY_LIMIT_EXP, deg, scale=scale)
            V = sped.alloc_block(n, k, torch.float64, dev)
            V[:, :k] = V0
            scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8,
                              device=dev)
            steps, ang = None, None
            for t in range(1, cap + 1):
                sped.eig_step(G, V, k, opts, scratch=scr)
                ang = _principal_angle(sped, Ud, V, k)
                if ang <= 1e-3:
                    steps = t
                    break
            out[f"l{deg}_{rule}"] = {"scale_s": info.scale_s, "converged": steps is not None,
                                     "steps": steps, "spmm": None if steps is None else steps * deg,
                                     "final_angle": ang}
    # App. A.3: the other series of Table 2 at the same degrees (Taylor -e^{-L} with l + 1 terms,
    # Taylor log(L + eps) around 1), Oja from the same V0
    for deg in degrees:
        for fam, kind in (("taylor_exp", sped.POLY_TAYLOR_EXP), ("taylor_log", sped.POLY_TAYLOR_LOG)):
            G.set_polynomial(kind, deg)
            V = sped.alloc_block(n, k, torch.float64, dev)
            V[:, :k] = V0
            scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8,
                              device=dev)
            steps, ang, finite = None, None, True
            for t in range(1, cap + 1):
                sped.eig_step(G, V, k, opts, scratch=scr)
                if not bool(torch.isfinite(V[:, :k]).all()):
                    finite = False  # the series' values overflowed FP64 (|p(lambda)| > 1e308)
                    break
                ang = _principal_angle(sped, Ud, V, k)
                if ang <= 1e-3:
                    steps = t
                    break
            out[f"l{deg}_{fam}"] = {"converged": steps is not None, "steps": steps,
                                    "final_angle": ang, "finite": finite, "last_step": t}
    return out


def measure_three_room(sped, torch, dev, stream, k=3, cap_plain=20000, cap_dilated=2000):
    """Solver steps to the bottom-k (k = 3: one mode per room) subspace of the 3-room grid world
    of Section 5.3 (s = 2, h = 10: 21 x 61 cells, two walls with one door each), plain reversed
    Laplacian against the dilated operator of degree 251 (limit form), for subspace iteration
    (Oja, eta = 0) and mu-EG, FP64; converged at a largest principal angle <= 1e-3 against the
    dense eigendecomposition; beside it the steps until the eigenvector streak (Section 5.2,
    eps = pi/8) covers all k eigenvectors, the measure Fig. 1 plots."""
    g = gen.three_room_grid(2, 10)
    n = g.n
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    Ld[rows, g.col_idx] = -1.0
    Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
    lam, U = np.linalg.eigh(Ld)
    Ud = sped.alloc_block(n, k, torch.float64, dev)
    Ud[:, :k] = torch.from_numpy(U[:, :k]).to(dev)
    G = sped.Graph.from_csr(g, device=dev)
    V0 = torch.from_numpy(gen.gaussian_block(n, k, seed=SEED + 29)).to(dev)
    out = {"graph": g.name, "n": n, "k": k, "lambda_k": float(lam[k - 1]),
           "lambda_k_plus_1": float(lam[k])}
    arms = {"plain_oja": ("shift", sped.OJA, 0.0, cap_plain),
            "dilated251_oja": ("limit", sped.OJA, 0.0, cap_dilated),
            "plain_mu_eg": ("shift", sped.MU_EG, None, cap_plain),
            "dilated251_mu_eg": ("limit", sped.MU_EG, 1.0, cap_dilated)}
    for name, (poly, solver, eta, cap) in arms.items():
        info = (G.set_polynomial(sped.POLY_LIMIT_EXP, 251) if poly == "limit"
                else G.set_polynomial(sped.POLY_SHIFT, 1))
        e = eta if eta is not None else 2.0 / info.lambda_star
        opts = sped.step_opts(solver, e, torch.float64, torch.float64)
        V = sped.alloc_block(n, k, torch.float64, dev)
        V[:, :k] = V0
        scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=dev)
        every = 1 if cap <= cap_dilated else 10
        steps, ang, streak_steps, streak = None, None, None, 0
        for t in range(1, cap + 1):
            sped.eig_step(G, V, k, opts, scratch=scr)
            if t % every == 0 or t == cap:
                if steps is None:
                    ang = _principal_angle(sped, Ud, V, k)
                    if ang <= 1e-3:
                        steps = t
                if streak_steps is None:
                    streak, _ = _streak_device(torch, Ud, V, k, math.pi / 8)
                    if streak == k:
                        streak_steps = t
                if steps is not None and streak_steps is not None:
                    break
        out[name] = {"steps": steps, "spmm": None if steps is None else steps * info.degree,
                     "final_angle": ang, "eta": e, "steps_to_full_streak": streak_steps,
                     "final_streak": streak}
    for sv in ("oja", "mu_eg"):
        p_, d_ = out[f"plain_{sv}"]["steps"], out[f"dilated251_{sv}"]["steps"]
        if p_ and d_:
            out[f"step_ratio_{sv}"] = p_ / d_
        p_ = out[f"plain_{sv}"]["steps_to_full_streak"]
        d_ = out[f"dilated251_{sv}"]["steps_to_full_streak"]
        if p_ and d_:
            out[f"streak_step_ratio_{sv}"] = p_ / d_
    return out


def _streak_device(torch, Ud, V, k, eps):
    """Section 5.2's eigenvector streak on the device: the length of the leading run of columns
    of V whose angle to the matching column of Ud (unit eigenvectors) is at most eps, sign
    ignored; also returns the per-column angles."""
    X = V[:, :k]
    X = X / X.norm(dim=0, keepdim=True)
    U = Ud[:, :k]
    c = (X * U).sum(dim=0, keepdim=True)
    ang = torch.asin(torch.clamp((X - c * U).norm(dim=0), max=1.0)).cpu().numpy()
    n = 0
    for a in ang:
        if a > eps:
            break
        n += 1
    return n, [float(a) for a in ang]


def measure_link_prediction(sped, torch, dev, stream, k=4, cap_plain=5000, cap_dilated=2000):
    """App. A.1 (clustering probabilistic graphs): four 250-cliques joined by 25 short-circuit
    edges (n = 1,000), each edge removed with probability 0.2 and put back with its
    common-neighbours score over the largest score as weight. Oja (eta = 0) and mu-EG in FP64,
    plain reversed Laplacian against the limit form of degree 251: steps until the eigenvector
    streak (Section 5.2, eps = pi/8) covers all k bottom eigenvectors, and the streak after 10,
    100 and 1,000 steps (the paper plots the streak over training)."""
    g, removed = gen.link_completed_cliques([250] * 4, short_circuit=25, p_remove=0.2, seed=SEED)
    n = g.n
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    Ld[rows, g.col_idx] = -g.w
    Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
    lam, U = np.linalg.eigh(Ld)
    Ud = torch.from_numpy(U[:, :k]).to(dev)
    G = sped.Graph.from_csr(g, device=dev)
    V0 = torch.from_numpy(gen.gaussian_block(n, k, seed=SEED + 31)).to(dev)
    eps = math.pi / 8
    out = {"graph": g.name, "n": n, "nnz": g.nnz, "k": k, "removed_edges": int(removed.shape[1]),
           "predicted_edges_kept": int((g.w < 1).sum() // 2),
           "lambda": [float(x) for x in lam[:k + 1]], "eps": eps}
    arms = {"plain_oja": ("shift", sped.OJA, 0.0, cap_plain),
            "dilated251_oja": ("limit", sped.OJA, 0.0, cap_dilated),
            "plain_mu_eg": ("shift", sped.MU_EG, None, cap_plain),
            "dilated251_mu_eg": ("limit", sped.MU_EG, 1.0, cap_dilated)}
    for name, (poly, solver, eta, cap) in arms.items():
        info = (G.set_polynomial(sped.POLY_LIMIT_EXP, 251) if poly == "limit"
                else G.set_polynomial(sped.POLY_SHIFT, 1))
        e = eta if eta is not None else 2.0 / info.lambda_star
        opts = sped.step_opts(solver, e, torch.float64, torch.float64)
        V = sped.alloc_block(n, k, torch.float64, dev)
        V[:, :k] = V0
        scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=dev)
        steps, at = None, {}
        streak, ang = 0, None
        for t in range(1, cap + 1):
            sped.eig_step(G, V, k, opts, scratch=scr)
            if t in (10, 100, 1000) or poly == "limit" or t % 10 == 0 or t == cap:
                streak, ang = _streak_device(torch, Ud, V, k, eps)
                if t in (10, 100, 1000):
                    at[f"streak_at_{t}"] = streak
                if streak == k:
                    steps = t
                    break
        out[name] = {"steps_to_full_streak": steps,
                     "spmm": None if steps is None else steps * info.degree,
                     "final_streak": streak, "final_angles": ang, "eta": e, **at}
    return out


def _cheb_quadratic_forms(mu, d, k, a, b):
    """From the block moments mu_l = V^T T_l V (l <= 2d + 1) of the Chebyshev basis on [a, b]:
    A[l, m] = V^T T_l T_m V = (mu_{l+m} + mu_{|l-m|}) / 2 and Bm[l, m] = V^T T_l L T_m V, with
    L = (b - a)/2 x + (a + b)/2 I and x T_m = (T_{m+1} + T_{|m-1|}) / 2, so that for Y = M V,
    M = sum c_l T_l: Y^T Y = sum c_l c_m A[l, m] and Y^T L Y = sum c_l c_m Bm[l, m]."""
    A = np.empty((d + 1, d + 1, k, k))
    X = np.empty_like(A)
    for l in range(d + 1):
        for m in range(d + 1):
            A[l, m] = 0.5 * (mu[l + m] + mu[abs(l - m)])
            X[l, m] = 0.25 * (mu[l + m + 1] + mu[abs(l - m - 1)] + mu[l + abs(m - 1)]
                              + mu[abs(l - abs(m - 1))])
    return A, 0.5 * (b - a) * X + 0.5 * (a + b) * A


def _fit_chebyshev(mu, d, k, a, b, c0):
    """Coefficients c of M = sum_l c_l T_l(x) on [a, b] minimising the sum of the Ritz values of
    L on span(M V), tr((Y^T Y)^-1 Y^T L Y) with Y = M V, from the block moments (see
    _cheb_quadratic_forms). BFGS with the analytic gradient; c is scale-free and returned with
    unit norm."""
    import scipy.optimize as so
    A, Bm = _cheb_quadratic_forms(mu, d, k, a, b)

    def f(c):
        S = np.einsum("l,m,lmij->ij", c, c, A)
        Q = np.einsum("l,m,lmij->ij", c, c, Bm)
        Si = np.linalg.inv(S)
        g1 = np.einsum("m,lmij,ji->l", c, Bm, Si)
        g2 = np.einsum("m,lmij,ji->l", c, A, Si @ Q @ Si)
        return float(np.trace(Si @ Q)), 2.0 * (g1 - g2)
    r = so.minimize(f, c0, jac=True, method="BFGS", options={"maxiter": 200, "gtol": 1e-12})
    return r.x / np.linalg.norm(r.x), float(r.fun)


def measure_fitted_poly(sped, torch, dev, stream, k=3, degree=31, cap=60):
    """Fitted polynomial coefficients (the paper names meta-learning the coefficients as future
    work, Section 6): on the 3-room grid world of Section 5.3 (k = 3), every Oja step (eta = 0,
    FP64) computes the Chebyshev block moments V^T T_l V, l <= 2d + 1, on [0, lambda_bound]
    (2d + 1 chain steps and 2d + 2 Grams on the device), fits the degree-d coefficients on the
    host to minimise the sum of the Ritz values of L on span(M V), and applies the fitted M.
    Steps and SpMMs to a largest principal angle <= 1e-3 against the dense eigendecomposition,
    beside the fixed operators of the three_room measurement."""
    g = gen.three_room_grid(2, 10)
    n = g.n
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    Ld[rows, g.col_idx] = -1.0
    Ld[np.arange(n), np.arange(n)] = -Ld.sum(axis=1)
    lam, U = np.linalg.eigh(Ld)
    Ud = sped.alloc_block(n, k, torch.float64, dev)
    Ud[:, :k] = torch.from_numpy(U[:, :k]).to(dev)
    G = sped.Graph.from_csr(g, device=dev)
    lb = G.info().lambda_bound
    d = degree
    # start: Chebyshev interpolant of exp(-2 lambda) on [0, lb]
    nodes = np.cos(np.pi * (np.arange(4 * d) + 0.5) / (4 * d))
    fx = np.exp(-2.0 * (nodes + 1.0) * lb / 2.0)
    c = np.array([(2.0 - (j == 0)) / (4 * d) * np.sum(fx * np.cos(j * np.arccos(nodes)))
                  for j in range(d + 1)])
    V = sped.alloc_block(n, k, torch.float64, dev)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(n, k, seed=SEED + 29)).to(dev)
    opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    steps, ang, fits = None, None, []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host_s = 0.0
    for t in range(1, cap + 1):
        mu = sped.poly_moments(G, V, k, 2 * d + 2, basis="chebyshev", a=0.0, b=lb)
        mu = mu.cpu().numpy()
        h0 = time.perf_counter()
        c, fval = _fit_chebyshev(mu, d, k, 0.0, lb, c)
        host_s += time.perf_counter() - h0
        fits.append(fval)
        G.set_polynomial(sped.POLY_CHEBYSHEV, d, eps=0.0, coeffs=c, lambda_star=lb)
        sped.eig_step(G, V, k, opts)
        ang = _principal_angle(sped, Ud, V, k)
        if ang <= 1e-3:
            steps = t
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"graph": g.name, "n": n, "k": k, "degree": d, "solver": "oja_fp64",
            "steps": steps, "final_angle": ang,
            "spmm": None if steps is None else steps * (2 * d + 1 + d),
            "ritz_sum_fitted_last": fits[-1], "ritz_sum_exact": float(lam[:k].sum()),
            "wall_s": wall, "host_fit_s": host_s}


def measure_batched(sped, torch, dev, stream, k=8, degree=31, steps=4, n_graphs=4096):
    """Many independent graphs in one persistent launch (Section 5 applied per graph): 4,096
    SBMs with log-uniform sizes in [200, 20,000], 2-8 blocks, mean degree 12, 87.5 % of edge
    ends inside blocks; k = 8, limit form of degree 31, BF16 chain, mu-EG."""
    gs = gen.batched_sbm(n_graphs)
    B = sped.Batch.from_graphs(gs, degree=degree, device=dev)
    n, nnz = B.n_total, int(B.col_idx.numel())
    V = sped.batch_block(n, k, device=dev)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(n, k, seed=SEED + 13)).to(dev)
    scr = torch.empty(B.scratch_bytes(k), dtype=torch.uint8, device=dev)
    ritz = torch.empty((B.n_graphs, k), dtype=torch.float64, device=dev)
    B.set_schedule(512, 2)
    run = lambda: B.eig_steps(V, k, steps=steps, eta=1.0, ritz=ritz, scratch=scr)
    run()
    ms_default = _timed(torch, stream, run, 3) / steps
    tune = B.autotune(V, k)  # picks threads per CTA and CTAs per SM for this batch
    run()
    ms = _timed(torch, stream, run, 3) / steps
    # the same call captured once in a CUDA graph and replayed
    graph_ms = None
    try:
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(cg, stream=side):
                B.eig_steps(V, k, steps=steps, eta=1.0, ritz=ritz, scratch=scr, stream=side)
        stream.wait_stream(side)
        cg.replay()
        torch.cuda.synchronize()
        graph_ms = _timed(torch, stream, cg.replay, 3) / steps
    except Exception as exc:  # capture is optional: report why it was skipped
        graph_ms = f"skipped: {type(exc).__name__}: {exc}"
    step_b = degree * spmm_bytes(n, nnz, k, 2, 2) + n * k * 4 * 2 + n * k * 4 * 3
    peak, kind = _peaks()
    return {"workload": f"batched_sbm_{B.n_graphs}graphs_n{n}_k{k}", "graphs": B.n_graphs,
            "n_total": n, "nnz_total": nnz, "k": k, "degree_l": degree,
            "ms_per_step": ms, "graph_steps_per_s": B.n_graphs / (ms * 1e-3),
            "step_bytes": step_b, "gbs": step_b / (ms * 1e-3) / 1e9,
            "frac_of_hbm": step_b / (ms * 1e-3) / 1e9 / peak, "peak_kind": kind,
            "launches_per_call": 1, "steps_per_call": steps,
            "schedule": {"threads": tune["threads"], "ctas_per_sm": tune["ctas_per_sm"],
                         "candidate_ms": tune["ms"], "default_512x2_ms_per_step": ms_default},
            "cuda_graph_replay_ms_per_step": graph_ms}


def measure_differentiable(sped, torch, dev, stream, k=10, ell=11, reps=5):
    """Forward (EigenGame utilities of the columns of V under (I - sL(w))^l) and backward
    (adjoint chain for dV, checkpointed SDDMM for dw) on an SBM with N = 200,000, 10 blocks,
    mean degree 20, 87.5 % intra-block edge ends, learnable weights U(0.5, 1.5), k = 10."""
    g = gen.uniform_edge_weights(gen.sbm_by_degree(200_000, 10, 20.0, 0.875, seed=5), seed=6)
    G = sped.Graph.from_csr(g, device=dev)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    ne = G.info().n_edges
    w = torch.from_numpy(np.random.default_rng(SEED + 17).uniform(0.5, 1.5, ne)).to(dev)
    w = w.float().requires_grad_(True)
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(g.n, k, seed=SEED + 19)).to(dev)
    V.requires_grad_(True)
    gu = torch.linspace(1.0, 0.1, k, dtype=torch.float64, device=dev)

    def fwd_bwd():
        V.grad, w.grad = None, None
        u = sped.eigengame_utilities(V, w, G, k)
        (u * gu).sum().backward()
    fwd_bwd()
    ms = _timed(torch, stream, fwd_bwd, reps)
    fwd = lambda: sped.eigengame_utilities(V.detach(), w.detach(), G, k)
    fwd()
    ms_f = _timed(torch, stream, fwd, reps)
    return {"workload": f"sbm_n{g.n}_b10_deg20_k{k}_weighted", "n": g.n, "nnz": g.nnz,
            "edges": ne, "k": k, "degree_l": ell, "dtype": "f32",
            "forward_ms": ms_f, "forward_backward_ms": ms,
            "backward_over_forward": (ms - ms_f) / ms_f}


def measure_power_law(sped, torch, dev, stream, n=16_000_000, k=32, ell=251, target_nnz=None):
    """Skewed-degree workload for the merge-path chain step: planted-cluster Chung-Lu graph
    (power law gamma = 2.5 on expected degrees [4, 10^4], 64 clusters of log-normal sizes, 90 %
    intra-cluster edge ends, weights U(0.5, 1.5)), k = 32, BF16 chain, limit form of degree
    251 with s = 2 / lambda_bound. Times one merge-path step, one row-group step on the same
    graph, and the whole p(L) V."""
    t0 = time.perf_counter()
    g = gen.chung_lu_clusters(n, target_nnz=target_nnz or None, seed=SEED, device=dev)
    gen_s = time.perf_counter() - t0
    G = sped.Graph.from_csr(g, device=dev)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    X = sped.alloc_block(g.n, k, torch.bfloat16, dev)
    X[:, :k] = torch.randn(g.n, k, generator=torch.Generator(device=dev).manual_seed(SEED),
                           device=dev).to(torch.bfloat16)
    Y = sped.alloc_block(g.n, k, torch.bfloat16, dev)
    one_b = spmm_bytes(g.n, g.nnz, k, 2, 2, weighted=True) + 4 * g.n
    out = {"workload": f"chung_lu_n{g.n}_nnz{g.nnz}_k{k}_weighted", "n": g.n, "nnz": g.nnz,
           "max_degree": int(np.max(np.diff(g.row_ptr))), "k": k, "degree_l": ell,
           "scale_s": info.scale_s, "host_generation_s": gen_s, "bytes_per_step": one_b,
           "autotune": G.autotune(k, torch.bfloat16)}
    peak, kind = _peaks()
    for split, name in ((0, "tuned"), (2, "merge_path"), (1, "row_group")):
        step = lambda: sped.poly_step(G, X, Y, k, alpha=0.0, beta=-info.scale_s, gamma=1.0,
                                      split=split)
        step()
        ms = _timed(torch, stream, step, 5)
        out[name] = {"step_ms": ms, "gbs": one_b / (ms * 1e-3) / 1e9,
                     "frac_of_hbm": one_b / (ms * 1e-3) / 1e9 / peak}
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V[:, :k] = X[:, :k].float()
    Yf = sped.alloc_block(g.n, k, torch.float32, dev)
    scr = torch.empty(sped.apply_poly_scratch_bytes(G, k, torch.bfloat16), dtype=torch.uint8,
                      device=dev)
    full = lambda: sped.apply_poly(G, V, Yf, k, chain_dtype=torch.bfloat16, scratch=scr)
    full()
    ms = _timed(torch, stream, full, 1)
    out["p_of_L_V_ms"] = ms
    out["p_of_L_V_gbs"] = ell * one_b / (ms * 1e-3) / 1e9
    out["peak_kind"] = kind
    return out


# ----------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, on the host cores. Each of the W + K
    steps is a bounded sample of the workload: every host thread runs one limit-form chain step
    X <- X - sL X over the full graph (k = 20) on its own block; the K timed steps give the rate
    (bytes counted as one BF16 chain step of the GPU arm per thread and step)."""
    if rank != 0:
        return
    import concurrent.futures as cf
    import oracle
    g = make_graph()
    k, s = WORKLOAD["k"], 1.0 / WORKLOAD["ell"]
    nt = os.cpu_count() or 1
    blocks = [gen.gaussian_block(g.n, k, seed=SEED + 1 + i) for i in range(nt)]
    per_step = nt * spmm_bytes(g.n, g.nnz, k, 2, 2)
    times = []
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            list(ex.map(lambda X: oracle.poly_limit(g, X, s, 1), blocks))
            if step >= args.warmup:
                times.append(time.perf_counter() - t0)
    total = float(sum(times))
    value = args.steps * per_step / total / 1e9
    sample = (f"{nt} host threads, each step one limit-form chain step X <- X - sL X over the "
              f"full graph (k={k}, FP64) per thread on its own block; {args.steps} timed steps "
              f"after {args.warmup} untimed, {total:.2f} s; bytes counted as one BF16 chain "
              f"step of the GPU arm per thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(g),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": nt, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(g):
    w = WORKLOAD
    return {"workload": f"sbm_n{w['n']}_b{w['blocks']}_deg16_k{w['k']}",
            "n": g.n, "nnz": g.nnz, "k": w["k"], "degree_l": w["ell"], "blocks": w["blocks"],
            "p_in": w["p_in"], "p_out": w["p_out"], "seed": SEED,
            "chain": "bf16 storage, f32 accumulate; f32 master V with a bf16 shadow; f64 k x k",
            "solver": "mu-EG, eta=1.0, limit form (I - sL)^l",
            "l2": "working set (graph 68 MB + blocks >= 200 MB) larger than L2 (129 MB)"}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2207_14589_gb300 as sped
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    g = make_graph()
    w = WORKLOAD
    k, ell = w["k"], w["ell"]
    G = sped.Graph.from_csr(g, device=dev)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = torch.from_numpy(gen.gaussian_block(g.n, k, seed=SEED + rank)).to(dev)
    V0 = V0 / V0.norm(dim=0)
    V = sped.alloc_block(g.n, k, torch.float32, dev)
    V[:, :k] = V0.float()
    # the update keeps a BF16 shadow of V that the next step's first chain launch reads
    Vb = sped.alloc_block(g.n, k, torch.bfloat16, dev)
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32, v_shadow=Vb)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=dev)
    K, W = args.steps, args.warmup
    for _ in range(W):
        sped.eig_step(G, V, k, opts, scratch=scr)
        opts.shadow_valid = 1
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for b, e in ev:  # torch creates the underlying cudaEvent_t at the first record
        b.record(stream)
        e.record(stream)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else
                os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]) as clk:
        t_start.record(stream)
        for i in range(K):
            opts.ev_chain_begin = ctypes_ptr(ev[i][0])
            opts.ev_chain_end = ctypes_ptr(ev[i][1])
            sped.eig_step(G, V, k, opts, scratch=scr)
        t_end.record(stream)
        t_end.synchronize()
    torch.cuda.synchronize()
    ms_total = t_start.elapsed_time(t_end)
    opts.ev_chain_begin = None
    opts.ev_chain_end = None
    chain_ms = [b.elapsed_time(e) for b, e in ev]
    ms_total = _max_over_ranks(ms_total, world, dev)
    chain_b, step_b = step_bytes(g.n, g.nnz, k, ell)
    ms_step = ms_total / K
    value = _job_rate(world, step_b, ms_step)
    peak, peak_kind = _peaks()
    mean_chain_ms = float(np.mean(chain_ms))
    launch_ms = mean_chain_ms / ell
    per_launch_bytes = chain_b / ell
    achieved = per_launch_bytes / (launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _ncu_traffic(),
                "traffic_source": "from profile: ncu dram bytes per launch in "
                                  "profiles/step_rowgroup_bf16_sbm1e6_k20.md, taken on this "
                                  "kernel source (null when the source changed since)",
                "kernel": "k_step_rowgroup (chain step, bf16 storage, f32 accumulate)",
                "per_launch_bytes": per_launch_bytes, "launch_us": launch_ms * 1e3,
                "peak_kind": f"{peak_kind} (copy, burst)"}

    # the chain step against the rate at which this GPU serves the same random row gathers:
    # the probe replays its access stream without arithmetic (CSR order, hashed rows,
    # consecutive rows)
    Xg = sped.alloc_block(g.n, k, torch.bfloat16, dev)
    Xg[:, :k] = V[:, :k].to(torch.bfloat16)
    Yg = sped.alloc_block(g.n, k, torch.bfloat16, dev)
    gather = {"chain_step_us": launch_ms * 1e3, "gathers_per_launch": g.nnz,
              "bytes_per_gather": sped.padded_ld(k, torch.bfloat16) * 2}
    from paper_2207_14589_gb300 import probe as gprobe
    for name, mode in gprobe.MODES.items():
        probe = lambda: gprobe.probe_gather(G.row_ptr, G.col_idx, Xg, Yg, k, mode=mode, seed=SEED)
        probe()
        us = _timed(torch, stream, probe, 20) * 1e3
        gather[f"{name}_us"] = us
        gather[f"{name}_gathers_per_s"] = g.nnz / (us * 1e-6)
    gather["chain_over_csr_order_gathers"] = gather["chain_step_us"] / gather["csr_order_us"]
    del Xg, Yg

    # end to end through the C ABI with host buffers: every step copies its V from pinned host
    # memory, runs, and copies its result back. Two device buffers and two copy streams let
    # the copies of neighbouring steps overlap the current step's kernels (each step's input
    # comes from the host, so the steps are independent calls); the timed region spans the
    # first H2D to the last D2H.
    e2e_steps = min(K, 50)
    hostV = torch.empty_like(V, device="cpu").pin_memory()
    hostV.copy_(V.cpu())
    hostOut = torch.empty_like(hostV).pin_memory()
    Vb = [V, torch.empty_like(V)]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    ev_h = [torch.cuda.Event() for _ in range(2)]
    ev_c = [torch.cuda.Event() for _ in range(2)]
    ev_d = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    opts.shadow_valid = 0  # V arrives from the host every step: the chain starts from V
    e0.record(stream)
    h2d.wait_stream(stream)
    d2h.wait_stream(stream)
    with torch.cuda.stream(h2d):
        Vb[0].copy_(hostV, non_blocking=True)
        ev_h[0].record(h2d)
    for t in range(e2e_steps):
        cur, nxt = t % 2, (t + 1) % 2
        if t + 1 < e2e_steps:
            with torch.cuda.stream(h2d):
                if t >= 1:
                    h2d.wait_event(ev_d[nxt])  # the result of step t - 1 has left that buffer
                Vb[nxt].copy_(hostV, non_blocking=True)
                ev_h[nxt].record(h2d)
        stream.wait_event(ev_h[cur])
        sped.eig_step(G, Vb[cur], k, opts, scratch=scr, stream=stream)
        ev_c[cur].record(stream)
        with torch.cuda.stream(d2h):
            d2h.wait_event(ev_c[cur])
            hostOut.copy_(Vb[cur], non_blocking=True)
            ev_d[cur].record(d2h)
    stream.wait_stream(d2h)
    stream.wait_stream(h2d)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    vb = V.numel() * V.element_size()
    e2e = {"value": _job_rate(world, step_b, e2e_ms), "unit": "GB/s",
           "h2d_bytes_per_step": vb, "d2h_bytes_per_step": vb, "ms_per_step": e2e_ms,
           "copies": "pinned host buffers, two copy streams overlapping the neighbouring steps"}
    del Vb

    # the same step captured once in a CUDA graph and replayed (launch gaps removed)
    graph_rec = None
    try:
        opts.ev_chain_begin = None
        opts.ev_chain_end = None
        sped.eig_step(G, V, k, opts, scratch=scr)  # refresh the shadow after the e2e steps
        opts.shadow_valid = 1
        cg = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            sped.eig_step(G, V, k, opts, scratch=scr)  # warm the side stream
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(cg):
            sped.eig_step(G, V, k, opts, scratch=scr)
        for _ in range(3):
            cg.replay()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(K):
            cg.replay()
        g1.record(stream)
        g1.synchronize()
        gms = g0.elapsed_time(g1) / K
        graph_rec = {"ms_per_step": gms, "value": world * step_b / (gms * 1e-3) / 1e9,
                     "unit": "GB/s", "launches_per_replay": ell + 4}
    except Exception as exc:  # capture is optional: report why it was skipped
        graph_rec = {"skipped": f"{type(exc).__name__}: {exc}"}

    extra = {}
    if rank == 0 and not args.no_extra:
        want = set(args.only_extra.split(",")) if args.only_extra else None
        runs = {
            "stochastic": lambda: measure_stochastic(sped, torch, g, G, dev, stream, k, ell),
            "minibatch": lambda: measure_minibatch(sped, torch, g, G, dev, stream, k, ell),
            "differentiable": lambda: measure_differentiable(sped, torch, dev, stream),
            "batched": lambda: measure_batched(sped, torch, dev, stream,
                                               n_graphs=args.batched_graphs),
            "permuted_node_order": lambda: measure_permuted(sped, torch, dev, stream, k, ell),
            "degree_sweep": lambda: measure_degree_sweep(sped, torch, dev, stream),
            "three_room": lambda: measure_three_room(sped, torch, dev, stream),
            "link_prediction": lambda: measure_link_prediction(sped, torch, dev, stream),
            "fitted_poly": lambda: measure_fitted_poly(sped, torch, dev, stream)}
        # gathered bytes of one chain step (every stored entry pulls one k-column row)
        extra["gather_bytes_per_launch"] = g.nnz * k * 2
        for name, fn in runs.items():
            if want is None or name in want:
                extra[name] = fn()
    if rank == 0 and not args.no_power_law:
        extra["power_law"] = measure_power_law(sped, torch, dev, stream, n=args.power_law_n,
                                               target_nnz=args.target_nnz)
    if rank == 0 and not args.no_ttk:
        # bottom-20 of this workload is not a well-conditioned subspace (Poisson low-degree
        # nodes put localized modes inside the block-mode cluster; `--spectrum` shows it), so
        # time-to-bottom-k is measured on the small SBM (N = 2,000, 4 blocks, k = 4) and on the
        # near-regular SBM of the benchmark's size, block structure and mean degree
        del scr
        g1 = gen.sbm(2000, 4, 0.05, 0.001, seed=SEED)
        g1.name = "sbm_n2000_b4_k4"
        g2 = gen.sbm_regular(w["n"], w["blocks"], 14, 2, seed=SEED)
        g2.name = f"sbm_regular_n{w['n']}_b{w['blocks']}_deg14+2"
        extra["time_to_bottom_k"] = {
            "sbm_n2000_b4_k4": time_to_bottom_k(sped, torch, g1, 4, dev, stream, 45),
            "sbm_regular_n1e6_b20_k20": time_to_bottom_k(sped, torch, g2, k, dev, stream, 41)}
        # the small workload again with seeds 0, 1, 2 (graph and V0): steps and times per arm
        per_seed = {}
        for sd in (0, 1, 2):
            gs = gen.sbm(2000, 4, 0.05, 0.001, seed=sd)
            gs.name = f"sbm_n2000_b4_k4_seed{sd}"
            r = time_to_bottom_k(sped, torch, gs, 4, dev, stream, 45, seed=sd)
            per_seed[sd] = {a: {"steps": r[a]["steps"], "ms": r[a].get("ms")}
                            for a in TTK_ARMS}
            per_seed[sd].update(ttk_ratios(r))
        extra["time_to_bottom_k"]["sbm_n2000_b4_k4_seeds_0_1_2"] = per_seed
        if args.ttk_seeds:
            # the near-regular SBM of the benchmark's size with seeds 0, 1, 2 (graph and V0)
            per_seed = {}
            for sd in (0, 1, 2):
                gs = gen.sbm_regular(w["n"], w["blocks"], 14, 2, seed=sd)
                gs.name = f"sbm_regular_n{w['n']}_b{w['blocks']}_deg14+2_seed{sd}"
                r = time_to_bottom_k(sped, torch, gs, k, dev, stream, 41, seed=sd)
                per_seed[sd] = {a: {"steps": r[a]["steps"], "ms": r[a].get("ms")}
                                for a in TTK_ARMS}
                per_seed[sd].update(ttk_ratios(r))
                per_seed[sd]["certificate_sin_bound"] = (
                    r["reference"].get("certificate", {}).get("davis_kahan_sin_theta_bound"))
            extra["time_to_bottom_k"]["sbm_regular_n1e6_b20_k20_seeds_0_1_2"] = per_seed
        # the benchmark graph itself, graded at the nearest k >= 20 whose Ritz gap is clear
        extra["time_to_bottom_k"].update(ttk_benchmark_graph(sped, torch, g, G, dev, stream,
                                                             k, ell))
    clocks = clk.summary()
    if rank != 0:
        return
    full = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": _config(g),
            "roofline": roofline, "e2e": e2e, "clocks": clocks,
            "gpu_launches": K * (ell + 4),
            "poly_gbs": chain_b / (mean_chain_ms * 1e-3) / 1e9,
            "cuda_graph_replay": graph_rec,
            "gather_ceiling": gather,
            "step_bytes": step_b}
    full.update(extra)
    if not args.no_cpu:
        full["cpu_baseline"] = cpu_baseline(g)
    emit(full, args.extras_out)


# keys of the headline line; everything else goes to the extra lines (and the extras file)
HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                 "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                 "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches")


def _round(x, digits=4):
    """Floats to `digits` significant digits, recursively (keeps the headline short)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: _round(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_round(v, digits) for v in x]
    return x


def ttk_summary(ttk):
    """Compact time-to-bottom-k figures per graph: [steps, ms] of every arm, the same-solver
    ratios (plain-L time over dilated time, same solver), and the reference's certificate."""
    out = {}
    for gname, r in ttk.items():
        if not isinstance(r, dict) or "reference" not in r:
            continue
        s = {arm: [r[arm].get("steps"), r[arm].get("ms")] for arm in TTK_ARMS if arm in r}
        for key in ("same_solver_speedup_oja", "same_solver_speedup_mu_eg",
                    "speedup_best_dilated_vs_plain_fp64"):
            if r.get(key) is not None:
                s[key] = r[key]
        cert = r["reference"].get("certificate")
        if cert:
            s["reference_sin_theta_bound"] = cert.get("davis_kahan_sin_theta_bound")
        if r.get("k_graded") is not None:
            s["k_graded"] = r["k_graded"]
        out[gname] = s
    return out


def headline(full):
    """The one JSON line the benchmark ends with: the contract's keys (with the long
    descriptions shortened) plus the time-to-bottom-k summary; a few KB at most."""
    line = {k: full[k] for k in HEADLINE_KEYS if k in full}
    rf = dict(line.get("roofline") or {})
    line["roofline"] = {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic",
                                           "traffic_source", "kernel", "per_launch_bytes",
                                           "launch_us", "peak_kind") if k in rf}
    cb = full.get("cpu_baseline")
    if cb:
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")
                                if k in cb}
    if "e2e" in line:
        line["e2e"] = {k: line["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                   "d2h_bytes_per_step", "ms_per_step")
                       if k in line["e2e"]}
    if "time_to_bottom_k" in full:
        line["time_to_bottom_k"] = ttk_summary(full["time_to_bottom_k"])
    return _round(line)


def emit(full, extras_out=None):
    """Print every extended measurement as its own JSON line ({"extra": name, "result": ...}),
    write all of them to `extras_out` when given, and end with the headline line."""
    rest = {k: v for k, v in full.items() if k not in HEADLINE_KEYS}
    for name, val in rest.items():
        print(json.dumps({"extra": name, "result": _round(val, 6)}), flush=True)
    if extras_out:
        d = os.path.dirname(os.path.abspath(extras_out))
        os.makedirs(d, exist_ok=True)
        with open(extras_out, "w") as f:
            json.dump(full, f, indent=1)
    print(json.dumps(headline(full)), flush=True)


def ctypes_ptr(event):
    return event.cuda_event


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-ttk", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the stochastic, differentiable and batched measurements")
    ap.add_argument("--only-extra", default=None,
                    help="comma list of the extra measurements to run (stochastic, minibatch, "
                         "differentiable, batched, permuted_node_order, degree_sweep, "
                         "three_room, link_prediction, fitted_poly); default all")
    ap.add_argument("--batched-graphs", type=int, default=4096,
                    help="number of graphs of the batched measurement")
    ap.add_argument("--no-power-law", action="store_true",
                    help="skip the merge-path chain on the 16M-node Chung-Lu graph")
    ap.add_argument("--power-law-n", type=int, default=16_000_000,
                    help="nodes of the Chung-Lu graph for --power-law")
    ap.add_argument("--target-nnz", type=float, default=3.2e8,
                    help="scale the Chung-Lu expected degrees to this many stored entries "
                         "(0: the degree law's own, about 1.9e8)")
    ap.add_argument("--extras-out", default=None,
                    help="also write every measurement (headline and extras) to this JSON file")
    ap.add_argument("--ttk-seeds", action="store_true",
                    help="also run time-to-bottom-k on the near-regular 1e6-node SBM with seeds "
                         "0, 1, 2 (graph and V0)")
    ap.add_argument("--spectrum", action="store_true",
                    help="print the bottom of the workload's spectrum and exit")
    args = ap.parse_args()
    if args.spectrum:
        import torch
        import paper_2207_14589_gb300 as sped
        g = make_graph()
        G = sped.Graph.from_csr(g)
        res, _ = spectrum_probe(sped, torch, G, g.n, torch.device("cuda"))
        print(json.dumps({"spectrum_probe": res}), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
