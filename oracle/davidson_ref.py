"""Plain CPU density-fitted sigma and Davidson solver (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's Davidson routine (Sec. Implementation Details) is cited to
earlier work and its details are not given; this file writes the standard
Davidson iteration for the generalised problem M z = omega W z of
Sec. ppRPA Equation, with the subspace problem handed to
``scipy.linalg.eig``.  It is used where the explicit matrix no longer fits
(large workloads) and as the timed CPU baseline.  It is pinned by the
explicit matrix (``ri_sigma`` against ``build_matrix``) and by full
diagonalisation (roots) in the oracle's own tests.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .pprpa_ref import pair_list


def _pair_arrays(n, offset, mult):
    pl = pair_list(n, mult)
    p = np.array([x[0] for x in pl], dtype=np.int64) + offset
    q = np.array([x[1] for x in pl], dtype=np.int64) + offset
    return p, q


def _pairs_all(n, no, mult):
    pv, qv = _pair_arrays(n - no, no, mult)
    po, qo = _pair_arrays(no, 0, mult)
    return np.concatenate([pv, po]), np.concatenate([qv, qo]), len(pv), len(po)


def ri_sigma(eps_act, nocc_act, L_act, mult, Z):
    """sigma = M z for k vectors (rows of ``Z``), from the density-fitted integrals.

    With <ab|cd> = sum_P L^P_ac L^P_bd, the two-electron part of
    sum_{c<=d} A_{ab,cd} X_cd (singlet elements, Sec. ppRPA Equation) equals
    (sum_P L^P Zt L^P)_ab / sqrt(1 + d_ab), where Zt is the symmetric matrix
    with Zt_cd = Zt_dc = X_cd (c < d) and Zt_cc = sqrt(2) X_cc.  For the
    triplet Zt is antisymmetric (Zt_cd = X_cd, Zt_dc = -X_cd) and the factor
    is 1.  The occupied block Y enters the same Zt on the occupied
    diagonal block, which gives B Y, B^T X and C Y together.  The diagonal
    term adds (eps_a + eps_b) X_ab and -(eps_i + eps_j) Y_ij.
    This identity is checked against the explicit matrix in the tests.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    L = np.asarray(L_act, dtype=np.float64)
    Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
    k = Z.shape[0]
    n = eps.shape[0]
    p, q, nvv, noo = _pairs_all(n, nocc_act, mult)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    Zt = np.zeros((k, n, n))
    if mult == 1:
        vals = np.where(p == q, np.sqrt(2.0), 1.0)[None, :] * Z
        Zt[:, p, q] = vals
        Zt[:, q, p] = vals
    else:
        Zt[:, p, q] = Z
        Zt[:, q, p] = -Z
    O = np.zeros((k, n, n))
    for P in range(L.shape[0]):
        # O_j += L^P Zt_j L^P, one auxiliary function at a time, all k vectors together
        O += L[P] @ Zt @ L[P]
    two_e = O[:, p, q]
    if mult == 1:
        two_e = two_e / np.where(p == q, np.sqrt(2.0), 1.0)[None, :]
    d = w * (eps[p] + eps[q])
    return d[None, :] * Z + two_e


def ri_sigma_rows(eps_act, nocc_act, L_act, mult, z, rows, Lrow=None):
    """Selected components sigma_I = sum_J M_IJ z_J, one row at a time.

    Each row I = (p, q) of M is formed from its definition (Sec. ppRPA
    Equation): the needed <pq|rs> = sum_P L^P_pr L^P_qs for all r, s is one
    product of the P-columns of orbitals p and q.  Used to check sampled
    outputs at sizes where the full matrix does not fit.  ``Lrow(p)`` may
    supply L^P_{p, :} as an (naux, n) array instead of ``L_act``.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    if Lrow is None:
        L = np.asarray(L_act, dtype=np.float64)

        def Lrow(p):
            return L[:, p, :]
    n = eps.shape[0]
    P1, P2, nvv, noo = _pairs_all(n, nocc_act, mult)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    out = np.zeros(len(rows))
    for t, I in enumerate(rows):
        a, b = P1[I], P2[I]
        V = Lrow(a).T @ Lrow(b)  # V[r, s] = <ab|rs>
        direct = V[P1, P2]
        exch = V[P2, P1]
        if mult == 1:
            fac = 1.0 / np.sqrt((1.0 + (a == b)) * (1.0 + (P1 == P2)))
            row = fac * (direct + exch)
        else:
            row = direct - exch
        row = row.copy()
        row[I] += w[I] * (eps[a] + eps[b])
        out[t] = row @ z
    return out


def davidson(sigma_fn, diag, nvv, noo, nroots, tol=1e-6, max_iter=200, max_space=None,
             nguess=None, imag_tol=1e-8):
    """Lowest ``nroots`` two-electron addition roots by Davidson iteration.

    Standard Davidson for M z = omega W z, W = diag(I_nvv, -I_noo):
    unit-vector guesses at the lowest diagonal entries of the A block; the
    subspace problem (V^T M V) c = omega (V^T W V) c solved by
    ``scipy.linalg.eig``; roots selected by positive norm c^T (V^T W V) c
    (Eq. xy_norm), lowest first; residual r = M z - omega W z for
    W-normalised z; diagonal-preconditioned correction r / (D - omega w);
    two passes of classical Gram-Schmidt; collapse to the current Ritz
    vectors when the subspace is full.  Converged when every target root
    has ||r||_2 <= tol.

    ``sigma_fn(Zrows) -> sigma rows`` applies M to k vectors (k, N).
    Returns a dict with ``omega`` (nroots,), ``z`` (N, nroots), ``resid``,
    ``iters``, ``n_sigma`` (number of single-vector sigma applications),
    ``converged``.
    """
    N = nvv + noo
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    diag = np.asarray(diag, dtype=np.float64)
    if nguess is None:
        nguess = min(nvv, max(2 * nroots, nroots + 8))
    if max_space is None:
        max_space = max(8 * nroots, nguess + 4 * nroots)
    idx = np.argsort(diag[:nvv], kind="stable")[:nguess]
    V = np.zeros((N, nguess))
    V[idx, np.arange(nguess)] = 1.0
    Sig = sigma_fn(V.T).T
    n_sigma = nguess
    omega = None
    resid = None
    Zr = None
    for it in range(1, max_iter + 1):
        G = V.T @ Sig
        G = 0.5 * (G + G.T)
        S = V.T @ (w[:, None] * V)
        vals, C = sla.eig(G, S)
        ok = np.isfinite(vals) & (np.abs(vals.imag) <= imag_tol * np.maximum(1.0, np.abs(vals.real)))
        vals = vals.real
        C = C.real
        nrm = np.einsum("ik,ij,jk->k", C, S, C)
        sel = np.where(ok & (nrm > 0))[0]
        sel = sel[np.argsort(vals[sel])]
        tgt = sel[:nroots]
        if len(tgt) < nroots:
            raise RuntimeError("subspace holds fewer positive-norm roots than requested")
        Ct = C[:, tgt] / np.sqrt(nrm[tgt])[None, :]
        omega = vals[tgt]
        Zr = V @ Ct
        R = Sig @ Ct - omega[None, :] * (w[:, None] * Zr)
        resid = np.linalg.norm(R, axis=0)
        if np.all(resid <= tol):
            return {"omega": omega, "z": Zr, "resid": resid, "iters": it,
                    "n_sigma": n_sigma, "converged": True}
        todo = np.where(resid > tol)[0]
        T = []
        for j in todo:
            den = diag - omega[j] * w
            den = np.where(np.abs(den) < 1e-4, np.where(den < 0, -1e-4, 1e-4), den)
            T.append(R[:, j] / den)
        T = np.array(T).T
        if V.shape[1] + T.shape[1] > max_space:
            keep = sel[: min(len(sel), max(nguess, nroots))]
            Ck = C[:, keep]
            Q, Rq = np.linalg.qr(Ck)
            V = V @ Q
            Sig = Sig @ Q
        newv = []
        for j in range(T.shape[1]):
            t = T[:, j]
            t0 = np.linalg.norm(t)
            for _ in range(2):
                t = t - V @ (V.T @ t)
                for u in newv:
                    t = t - u * (u @ t)
            tn = np.linalg.norm(t)
            if tn > 1e-10 * max(t0, 1e-300):
                newv.append(t / tn)
        if not newv:
            break
        Vn = np.array(newv).T
        Sn = sigma_fn(Vn.T).T
        n_sigma += Vn.shape[1]
        V = np.hstack([V, Vn])
        Sig = np.hstack([Sig, Sn])
    return {"omega": omega, "z": Zr if omega is not None else None, "resid": resid,
            "iters": max_iter, "n_sigma": n_sigma, "converged": False}
