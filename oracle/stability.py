"""Stability of the ppRPA pencil at workload sizes (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The generalised problem of Sec. ppRPA Equation, M z = omega W z with
W = diag(I_nvv, -I_noo), has real roots split by the sign of z^T W z
(Eq. xy_norm) when some shift mu makes M - mu W positive definite: then
every root is real, the nvv addition roots lie above mu and the noo removal
roots below it.  When no such mu exists the two families meet and complex
pairs can appear.  This file answers both questions for problems whose
explicit matrix fits in host memory (tens of thousands of pairs):

* ``matrix_rows`` / ``explicit_matrix_ri`` build rows of M from the
  density-fitted integrals, <ab|cd> = sum_P L^P_ac L^P_bd, one pair row at a
  time, with the spin-adapted elements of Sec. ppRPA Equation;
* ``shifted_lambda_min`` is the lowest eigenvalue of the symmetric M - mu W
  (positive exactly when mu is a definite shift);
* ``roots_near`` returns the eigenvalues of W M nearest a point by
  shift-invert Arnoldi (complex ones included), each with its normalised
  metric z^T W z / z^H z (+1 addition, -1 removal, about 0 for complex pairs).

Pinned in the tests by the element-by-element ``build_matrix`` (rows), dense
symmetric eigenvalues (lambda_min) and the dense eigenvalues of
``solve_full`` (roots near a point).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .davidson_ref import _pairs_all


def matrix_rows(eps_act, nocc_act, L_act, mult, rows):
    """Rows ``rows`` of M (len(rows), N), each from its definition (Sec. ppRPA Equation).

    Row I = (a, b): <ab|rs> = sum_P L^P_ar L^P_bs for all r, s is the product
    L[:, a, :]^T L[:, b, :]; the singlet element is
    (<ab|cd> + <ab|dc>) / sqrt((1 + d_ab)(1 + d_cd)), the triplet one
    <ab|cd> - <ab|dc>, and the diagonal adds (eps_a + eps_b) on virtual pairs
    and -(eps_i + eps_j) on occupied pairs.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    L = np.asarray(L_act, dtype=np.float64)
    n = eps.shape[0]
    P1, P2, nvv, noo = _pairs_all(n, nocc_act, mult)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    out = np.empty((len(rows), nvv + noo))
    for t, I in enumerate(rows):
        a, b = P1[I], P2[I]
        V = L[:, a, :].T @ L[:, b, :]  # V[r, s] = <ab|rs>
        if mult == 1:
            fac = 1.0 / np.sqrt((1.0 + (a == b)) * (1.0 + (P1 == P2)))
            out[t] = fac * (V[P1, P2] + V[P2, P1])
        else:
            out[t] = V[P1, P2] - V[P2, P1]
        out[t, I] += w[I] * (eps[a] + eps[b])
    return out


def explicit_matrix_ri(eps_act, nocc_act, L_act, mult):
    """The whole M (N x N) from ``matrix_rows``; returns ``(M, nvv, noo)``."""
    n = np.asarray(eps_act).shape[0]
    _, _, nvv, noo = _pairs_all(n, nocc_act, mult)
    N = nvv + noo
    M = np.empty((N, N))
    for r0 in range(0, N, 512):
        rows = np.arange(r0, min(N, r0 + 512))
        M[rows] = matrix_rows(eps_act, nocc_act, L_act, mult, rows)
    return M, nvv, noo


def shifted_lambda_min(M, nvv, noo, mu):
    """Lowest eigenvalue of the symmetric matrix M - mu W (Lanczos, ARPACK)."""
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    N = nvv + noo
    op = spla.LinearOperator((N, N), matvec=lambda x: M @ x - mu * (w * x), dtype=np.float64)
    vals = spla.eigsh(op, k=1, which="SA", tol=1e-10, maxiter=20 * N, return_eigenvectors=False)
    return float(vals[0])


def roots_near(M, nvv, noo, sigma, k=20):
    """The k eigenvalues of W M (roots of M z = omega W z) nearest ``sigma``.

    Shift-invert Arnoldi: (W M - sigma I)^-1 = (M - sigma W)^-1 W, applied
    through one dense LU factorisation of M - sigma W.  Returns
    ``(omega (complex, k), metric (k,))`` sorted by real part, metric =
    z^H W z / z^H z of each eigenvector.
    """
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    N = nvv + noo
    Ms = M.copy()
    Ms[np.diag_indices(N)] -= sigma * w
    lu = sla.lu_factor(Ms, overwrite_a=True, check_finite=False)
    del Ms
    op = spla.LinearOperator((N, N), matvec=lambda x: w * (M @ x), dtype=np.float64)
    inv = spla.LinearOperator((N, N), matvec=lambda x: sla.lu_solve(lu, w * x, check_finite=False),
                              dtype=np.float64)
    vals, vecs = spla.eigs(op, k=k, sigma=sigma, OPinv=inv, tol=1e-10, maxiter=50 * N)
    metric = np.real(np.einsum("ik,i,ik->k", vecs.conj(), w, vecs)) / np.real(
        np.einsum("ik,ik->k", vecs.conj(), vecs))
    order = np.argsort(vals.real)
    return vals[order], metric[order]


def block_shift_window(eps_act, nocc_act, L_act, mult, steps=40, seed=0):
    """Necessary condition for a definite shift, from the diagonal blocks alone.

    M - mu W positive definite needs its diagonal blocks A - mu I and C + mu I positive
    definite, i.e. -lambda_min(C) < mu < lambda_min(A).  lambda_min(C) is taken from the
    explicit occupied-pair block (``matrix_rows``); lambda_min(A) is bounded from above by
    the lowest Ritz value of ``steps`` Lanczos steps on A, applied through the
    density-fitted sigma with a zero occupied part (``ri_sigma``, virtual-pair rows).  If
    that upper bound lies below -lambda_min(C), no shift is definite and the pencil is
    proven indefinite.  Returns a dict with ``theta_A`` (>= lambda_min(A)),
    ``lambda_min_C``, ``window`` = theta_A + lambda_min(C) and ``proven_indefinite``.
    """
    from .davidson_ref import ri_sigma

    eps = np.asarray(eps_act, dtype=np.float64)
    n = eps.shape[0]
    _, _, nvv, noo = _pairs_all(n, nocc_act, mult)
    N = nvv + noo
    if noo:
        Crows = matrix_rows(eps_act, nocc_act, L_act, mult, np.arange(nvv, N))
        lam_c = float(np.linalg.eigvalsh(Crows[:, nvv:])[0])
        del Crows
    else:
        lam_c = np.inf

    def a_mul(x):
        z = np.zeros(N)
        z[:nvv] = x
        return ri_sigma(eps_act, nocc_act, L_act, mult, z[None, :])[0, :nvv]

    # plain Lanczos with full reorthogonalisation; the lowest Ritz value bounds lambda_min(A)
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(nvv)
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    for j in range(min(steps, nvv)):
        w = a_mul(Q[-1])
        alpha.append(float(Q[-1] @ w))
        for v in Q:
            w -= (v @ w) * v
        b = float(np.linalg.norm(w))
        if j + 1 == min(steps, nvv) or b < 1e-12:
            break
        beta.append(b)
        Q.append(w / b)
    T = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
    theta = float(np.linalg.eigvalsh(T)[0])
    window = theta + lam_c
    return {"theta_A": theta, "lambda_min_C": lam_c, "window": window,
            "proven_indefinite": bool(window < 0.0), "lanczos_steps": len(alpha)}


def classified_spectrum(M, nvv, noo, imag_tol=1e-9):
    """Every root of M z = omega W z (dense), sorted into the three kinds of Eq. xy_norm's
    reading: real addition roots (z^T W z > 0), real removal roots (< 0), and complex
    values (|Im| > imag_tol times the spectral scale; they come in conjugate pairs and their
    eigenvectors have z^H W z = 0).  Returns ``(addition ascending, removal ascending,
    complex (sorted by real part))``."""
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    vals, vecs = sla.eig(w[:, None] * M)
    scale = max(1.0, float(np.max(np.abs(vals)))) if vals.size else 1.0
    cplx = np.abs(vals.imag) > imag_tol * scale
    real = ~cplx
    v = vecs[:, real].real
    metric = np.einsum("ik,i,ik->k", v, w, v)
    r = vals[real].real
    add = np.sort(r[metric > 0])
    rem = np.sort(r[metric < 0])
    c = vals[cplx]
    return add, rem, c[np.argsort(c.real)]
