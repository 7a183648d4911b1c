"""Helpers shared by the GPU parity tests: move seeded inputs to the device, round them the way
the device stores them, and measure relative errors against the FP64 oracle."""
import numpy as np
import torch

import paper_2207_14589_gb300 as sped

DEV = "cuda"
TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 1e-2}


def to_block(A, dtype, device=DEV):
    """Padded device block holding A (n x k)."""
    n, k = A.shape
    T = sped.alloc_block(n, k, dtype, device)
    T[:, :k] = torch.from_numpy(np.ascontiguousarray(A)).to(device=device, dtype=dtype)
    return T


def stored(A, dtype):
    """A as the device stores it (rounded to dtype), back in float64."""
    return torch.from_numpy(np.ascontiguousarray(A)).to(dtype).to(torch.float64).numpy()


def host(T, k):
    return T[:, :k].to(torch.float64).cpu().numpy()


def rel(got, want):
    d = np.linalg.norm(want)
    return float(np.linalg.norm(got - want) / (d if d > 0 else 1.0))


def errors(got, want):
    """Relative errors of an n x k result (1-D: one column) against the oracle's, at four
    granularities: the whole block (Frobenius), every column, every row and every entry. Each
    is relative to the reference's own norm at that granularity, floored at the root mean
    square of that granularity over the block (so that a row, column or entry that is small
    because of cancellation is held to the accuracy of the block, not to its own size)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    if want.ndim == 1:
        got, want = got[:, None], want[:, None]
    assert got.shape == want.shape, (got.shape, want.shape)
    n, k = want.shape
    err = got - want
    fro = float(np.linalg.norm(want))
    if fro == 0.0:
        m = float(np.abs(err).max()) if err.size else 0.0
        return {"fro": m, "col": m, "row": m, "entry": m}
    col = np.linalg.norm(err, axis=0) / np.maximum(np.linalg.norm(want, axis=0), fro / np.sqrt(k))
    row = np.linalg.norm(err, axis=1) / np.maximum(np.linalg.norm(want, axis=1), fro / np.sqrt(n))
    ent = np.abs(err) / np.maximum(np.abs(want), fro / np.sqrt(n * k))
    return {"fro": float(np.linalg.norm(err)) / fro, "col": float(col.max()),
            "row": float(row.max()), "entry": float(ent.max())}


# per-granularity factors on a block tolerance: a row of k entries or a column of n entries
# spreads its rounding errors less evenly than the whole block, and a single entry least
FACTORS = {"fro": 1.0, "col": 2.0, "row": 2.0, "entry": 4.0}


def assert_close(got, want, tol):
    """Element-wise parity: the block within tol (relative Frobenius, the tolerance of the
    method's stated bound), every column and every row within 2 tol, every entry within 4 tol
    (see errors()). A wrong column, a few wrong rows or a single wrong entry of a large block
    fail here even when the block's Frobenius error stays small."""
    got = np.asarray(got, dtype=np.float64)
    assert np.isfinite(got).all(), "non-finite values in the result"
    e = errors(got, want)
    bad = {g: v for g, v in e.items() if not v <= FACTORS[g] * tol}
    assert not bad, f"tolerance {tol:g} exceeded: {bad} (all: {e})"
    return e


def assert_gram_close(got, want, tol):
    """Element-wise parity of a Gram matrix: |G_ij - W_ij| <= tol sqrt(W_ii W_jj) for every
    (i, j) (the Cauchy-Schwarz scale of the entry), exact symmetry, and the relative Frobenius
    error within tol."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.isfinite(got).all()
    assert np.array_equal(got, got.T)
    d = np.sqrt(np.maximum(np.diag(want), 0.0))
    scale = np.outer(d, d)
    scale[scale == 0.0] = 1.0
    e = float((np.abs(got - want) / scale).max())
    assert e <= tol, f"entry-wise Gram error {e:.3e} > {tol:g}"
    assert rel(got, want) <= tol
    return e


def assert_step_close(got, want, step, Y, tol, seed=0, directions=3):
    """Element-wise parity of a solver step's output whose input Y = p(L) V carries the chain's
    storage bound tol (relative Frobenius). The step maps Y to its output through the eta Y
    term and the Gram-derived coefficients, which can amplify an error in Y, unevenly across
    columns when a column nearly cancels before its normalisation. The gain is measured on the
    oracle: Y is perturbed by a relative tol in a few seeded Gaussian directions, and the
    largest errors of the perturbed steps against `want` at every granularity (errors()) set
    the bound, times 3 (a storage error can line up with the step's amplifying directions
    better than a random direction does) and 1.5 of margin; never below FACTORS * tol."""
    ep = {}
    for d in range(directions):
        D = np.random.default_rng(seed * 7919 + d).standard_normal(Y.shape)
        Yp = Y + tol * np.linalg.norm(Y) * D / np.linalg.norm(D)
        for g, v in errors(step(Yp), want).items():
            ep[g] = max(ep.get(g, 0.0), v)
    got = np.asarray(got, dtype=np.float64)
    assert np.isfinite(got).all(), "non-finite values in the result"
    e = errors(got, want)
    bound = {g: 1.5 * max(FACTORS[g] * tol, 3.0 * ep[g]) for g in e}
    bad = {g: (e[g], bound[g]) for g in e if not e[g] <= bound[g]}
    assert not bad, f"step errors above the propagated bound: {bad} (all: {e})"
    return e
