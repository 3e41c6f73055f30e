"""The coarse factorization the GPU uses for the two-level preconditioner, restated in FP32 on
the CPU and checked against the oracle's Galerkin operator (CPU; no CUDA).

J_c = R J^pi Pr = I - gamma P_c is an M-matrix with row sums 1 - gamma: at gamma = 0.999 its
pivots arise from cancellation in a plain LU.  The elimination in the form of Grassmann, Taksar
and Heyman carries each row's sum s and forms the pivot as s plus the magnitudes of the row's
upper entries, so every quantity is a sum of terms of one sign; in FP32 the inverse stays
accurate to about 1e-6 however close J_c is to singular.  (The coarse solve's accuracy changes only
how fast the preconditioned GMRES converges, never what it converges to.)
"""
import numpy as np
import pytest

import mdp_synth
import oracle

f32 = np.float32


def gth_lu(Jc, bw, row_sums):
    """Banded LU of Jc (half-bandwidth bw) in FP32 by the GTH recurrences: the pivot is
    u_kk = s_k + sum_{j>k} |S_kj| (row sum plus the magnitudes of the row's final upper
    entries), then l_ik = S_ik / u_kk, s_i += |l_ik| s_k and S_ij -= l_ik u_kj (i != j), the
    diagonal never being formed by subtraction.  Returns unit-lower L and upper U."""
    n = Jc.shape[0]
    A = Jc.astype(f32).copy()
    s = row_sums.astype(f32).copy()
    for k in range(n):
        o = f32(0)
        for j in range(k + 1, min(n, k + bw + 1)):
            o = f32(o - A[k, j])
        u = f32(s[k] + o)
        A[k, k] = u
        for i in range(k + 1, min(n, k + bw + 1)):
            l = f32(A[i, k] / u)
            A[i, k] = l
            s[i] = f32(s[i] - l * s[k])
            for j in range(k + 1, min(n, k + bw + 1)):
                if j != i:
                    A[i, j] = f32(A[i, j] - l * A[k, j])
    L = np.tril(A, -1).astype(np.float64) + np.eye(n)
    U = np.triu(A).astype(np.float64)
    return L, U


def fp32_triangular_inverse(L, U):
    """Columns of (L U)^{-1} by forward and backward substitution in FP32, as the GPU's column
    kernel does (one recurrence per column)."""
    n = L.shape[0]
    Lf, Uf = L.astype(f32), U.astype(f32)
    X = np.zeros((n, n), dtype=f32)
    for j in range(n):
        y = np.zeros(n, dtype=f32)
        for k in range(j, n):
            y[k] = f32((1.0 if k == j else 0.0) - np.dot(Lf[k, j:k], y[j:k]))
        x = np.zeros(n, dtype=f32)
        for k in range(n - 1, -1, -1):
            x[k] = f32((y[k] - np.dot(Uf[k, k + 1:], x[k + 1:])) / Uf[k, k])
        X[:, j] = x
    return X.astype(np.float64)


@pytest.mark.parametrize("gamma", [0.99, 0.999, 0.9999])
def test_fp32_gth_inverse_of_the_galerkin_operator(gamma):
    syn = mdp_synth.ell_banded(3000, 8, 16, 200, 40, gamma, seed=21, val_dtype=np.float64)
    m = oracle.from_synth(syn)
    pi = oracle.bellman(m, np.zeros(syn.S)).pi
    block = 128
    R, Pr, Jc, _ = oracle.two_level(m, pi, block)
    n = Jc.shape[0]
    # coarse half-bandwidth: the farthest nonzero from the diagonal
    nz = np.nonzero(np.abs(Jc) > 0)
    bw = int(np.max(np.abs(nz[0] - nz[1])))
    assert bw <= 31
    # the row sums of J_c are 1 - gamma (P^pi is row-stochastic), the device's s
    rs = Jc.sum(axis=1)
    np.testing.assert_allclose(rs, 1.0 - gamma, rtol=1e-9, atol=1e-13)
    L, U = gth_lu(Jc, bw, np.full(n, 1.0 - gamma))
    X = fp32_triangular_inverse(L, U)
    exact = np.linalg.inv(Jc)
    rel = np.max(np.abs(X - exact)) / np.max(np.abs(exact))
    assert rel <= 5e-6, rel
    # the inverse of an M-matrix is entrywise nonnegative, and so is the FP32 one
    assert np.min(X) >= -1e-6 * np.max(X)
