"""Tensor-core projection products (split BF16 digits, exact FP32 chunks,
FP64 combination) against their plain FP64 definition.

C = A^T B and Y - A B are checked element by element against numpy's FP64
products with the error bound of the representation: per term at most
2^-55 (max|a_col| |b_k| + max|b_col| |a_k|) from the 8 kept digits and
2^-58 max|a_col| max|b_col| from the dropped digit products, plus FP64
rounding of the chunk combination.  Sizes span several 128-row tiles,
several 256-element chunks, ragged tails (k not a multiple of 32, m and n not
multiples of 128 and 16) and columns whose scales differ by up to 1e16.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _bound(A, B):
    """Elementwise error bound for C = A^T B with A: k x m, B: k x n (numpy)."""
    aa, bb = np.abs(A), np.abs(B)
    amax, bmax = aa.max(axis=0), bb.max(axis=0)
    digits = 2.0 ** -55 * (np.outer(amax, bb.sum(axis=0)) + np.outer(aa.sum(axis=0), bmax))
    dropped = 2.0 ** -58 * A.shape[0] * np.outer(amax, bmax)
    fp64 = 2.0 ** -52 * (aa.T @ bb) * (2 + A.shape[0] / 256)
    return digits + dropped + fp64 + 1e-300


def _scaled(rng, k, m, spread):
    X = rng.standard_normal((k, m))
    X *= 10.0 ** rng.uniform(-spread, spread, size=m)
    return X


@pytest.mark.parametrize("k,m,n,spread", [(6144, 37, 20, 0), (1000, 300, 5, 8), (98304, 150, 16, 2),
                                          (8, 1, 1, 0), (4104, 129, 33, 4)])
def test_split_gemm_tn_matches_fp64(k, m, n, spread):
    torch = _torch()
    import paper_1510_02237_gb300 as P
    rng = np.random.default_rng(k + m + n)
    A = _scaled(rng, k, m, spread)
    B = _scaled(rng, k, n, spread)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()   # (m, k): column-major k x m
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Ct = torch.full((n, m), np.nan, dtype=torch.float64, device="cuda")
    P.parareal_split_gemm_tn(At, Bt, Ct)
    C = Ct.cpu().numpy().T
    ref = A.T @ B
    err = np.abs(C - ref)
    assert np.all(np.isfinite(C))
    assert np.all(err <= _bound(A, B)), float((err / _bound(A, B)).max())


@pytest.mark.parametrize("k,m,n,spread", [(6144, 37, 20, 0), (1000, 300, 5, 6), (98304, 150, 16, 2),
                                          (4104, 513, 17, 3)])
def test_split_gemm_nn_matches_fp64(k, m, n, spread):
    torch = _torch()
    import paper_1510_02237_gb300 as P
    rng = np.random.default_rng(7 * k + m + n)
    A = _scaled(rng, k, m, spread)
    Bm = _scaled(rng, m, n, spread)
    Y0 = rng.standard_normal((k, n))
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    Yt = torch.from_numpy(np.ascontiguousarray(Y0.T)).cuda()
    P.parareal_split_gemm_nn(At, Bt, Yt)
    Y = Yt.cpu().numpy().T
    ref = Y0 - A @ Bm
    # A's digits are scaled per column l (over the rows), B's folded rows
    # 2^{E_l} B[l, :] per column of B: the digit error of a term is bounded by
    # the largest (max |A[:, l]|) |B[l, j]| of its column, times 2^-52
    amax = np.abs(A).max(axis=0)
    big = (amax[:, None] * np.abs(Bm)).max(axis=0)
    bound = (2.0 ** -52 * m * big[None, :] + 2.0 ** -52 * (np.abs(A) @ np.abs(Bm)) * (2 + m / 256)
             + 2.0 ** -52 * np.abs(Y0) + 1e-300)
    err = np.abs(Y - ref)
    assert np.all(np.isfinite(Y))
    assert np.all(err <= bound), float((err / bound).max())


def test_split_gemm_exact_on_digit_representable_inputs():
    """Inputs with few significant bits are represented exactly by the digits;
    then every product is exact and only the final FP64 sums round: integer
    data whose sums stay below 2^53 must come out bit-exact."""
    torch = _torch()
    import paper_1510_02237_gb300 as P
    rng = np.random.default_rng(3)
    k, m, n = 2048, 40, 16
    A = rng.integers(-1000, 1000, size=(k, m)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(k, n)).astype(np.float64)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Ct = torch.empty((n, m), dtype=torch.float64, device="cuda")
    P.parareal_split_gemm_tn(At, Bt, Ct)
    assert np.array_equal(Ct.cpu().numpy().T, A.T @ B)


def test_split_gemm_rejects_bad_sizes():
    torch = _torch()
    import paper_1510_02237_gb300 as P
    A = torch.zeros((4, 12), dtype=torch.float64, device="cuda")   # k = 12: not a multiple of 8
    B = torch.zeros((2, 12), dtype=torch.float64, device="cuda")
    Ct = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PararealError):
        P.parareal_split_gemm_tn(A, B, Ct)
