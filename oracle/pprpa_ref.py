"""Spin-adapted ppRPA by definition: explicit matrix, dense diagonalisation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: i, j, k, l occupied; a, b, c, d virtual;
p, q, r, s general orbitals.  Active orbitals are ordered occupied first,
then virtual.  Density fitting writes <pq|rs> = (pr|qs) = sum_P L^P_pr L^P_qs.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def active_orbitals(occ, nocc_act, nvir_act):
    """Indices of the active orbitals: the highest ``nocc_act`` occupied and
    the lowest ``nvir_act`` virtual ones (orbital energies sorted ascending).

    The paper's active-space formalism uses canonical orbitals near the gap
    (Sec. ppRPA Equation, active-space paragraph; Sec. Implementation
    Details); it does not fix the selection rule, so this reading is the
    one stated here.
    """
    occ = np.asarray(occ, dtype=np.float64)
    nocc = int(np.count_nonzero(occ > 0.5))
    nmo = occ.shape[0]
    if not (0 <= nocc_act <= nocc and 0 <= nvir_act <= nmo - nocc):
        raise ValueError("active space larger than the orbital space")
    return np.concatenate([np.arange(nocc - nocc_act, nocc), np.arange(nocc, nocc + nvir_act)])


def fractional_slots(occ, nocc_act, nvir_act):
    """Active slots for fractional occupations (Sec. ppRPA for Fractional Charge Systems).

    With occupation numbers n_p in [0, 1] per spatial orbital (equal for both spins),
    non-increasing in orbital order, the hole slots are the highest ``nocc_act`` orbitals
    with n > 0 and the particle slots the lowest ``nvir_act`` orbitals with n < 1, so that
    a fractionally occupied orbital is both.  The paper's matrix elements carry
    sqrt((1-n_a)(1-n_b)(1-n_c)(1-n_d)), sqrt((1-n_a)(1-n_b) n_k n_l) and sqrt(n_i n_j n_k n_l)
    (reading its "n_k n_k" in B as n_k n_l), which factor into one weight per slot:
    sqrt(n) on hole slots and sqrt(1 - n) on particle slots.  Returns (orb, w): the MO index
    and the weight of every slot, holes first.  Integer occupations give
    ``active_orbitals`` with unit weights.
    """
    occ = np.asarray(occ, dtype=np.float64)
    if np.any(occ < 0) or np.any(occ > 1) or np.any(np.diff(occ) > 0):
        raise ValueError("occupations must lie in [0, 1] and be non-increasing")
    holes = np.flatnonzero(occ > 0)
    parts = np.flatnonzero(occ < 1)
    if not (0 <= nocc_act <= len(holes) and 0 <= nvir_act <= len(parts)):
        raise ValueError("active space larger than the orbital space")
    h = holes[len(holes) - nocc_act:]
    p = parts[:nvir_act]
    return np.concatenate([h, p]), np.concatenate([np.sqrt(occ[h]), np.sqrt(1.0 - occ[p])])


def fractional_integrals(ao3c, C, occ, eps, nocc_act, nvir_act):
    """Weighted integrals L~^P_st = w_s w_t L^P_{orb(s) orb(t)} and slot energies for the
    fractional-occupation matrix elements (see :func:`fractional_slots`); with them
    ``build_matrix`` gives the paper's fractional A, B and C."""
    orb, w = fractional_slots(occ, nocc_act, nvir_act)
    L = ao_to_mo(ao3c, C, orb) * w[None, :, None] * w[None, None, :]
    return L, np.asarray(eps, dtype=np.float64)[orb]


def ao_to_mo(ao3c, C, orb):
    """L^P_pq = sum_{mu,nu} C_{mu p} (P|mu nu) C_{nu q} for p, q in ``orb``.

    The paper's inputs are the MO-space density-fitting integrals, or
    equivalently MO coefficients and three-center integrals (Abstract;
    Sec. Implementation Details, input list).  The AO tensor is taken to be
    the metric-contracted fitting factor, so no (P|Q)^-1/2 is applied.
    """
    ca = np.asarray(C, dtype=np.float64)[:, orb]
    return np.einsum("Pmn,mp,nq->Ppq", ao3c, ca, ca, optimize=True)


def grad_ao(ao3c, C, orb, dL):
    """Adjoint of the AO->MO transform: from d f / d L^P_pq to d f / d (P|mu nu) and d f / d C.

    With L^P_pq = sum_{mu,nu} C_{mu p} (P|mu nu) C_{nu q} (the transform of
    :func:`ao_to_mo`; Abstract, inputs of Sec. Implementation Details) and every
    entry treated as independent, the chain rule gives
      d f / d (P|mu nu) = sum_pq C_{mu p} (d f / d L^P_pq) C_{nu q},
      d f / d C_{mu r}  = sum_P [ sum_q H^P_{mu q} (d f / d L^P_rq)
                                 + sum_p H'^P_{mu p} (d f / d L^P_pr) ],
    with H^P = (P|..) C_act and H'^P = (P|..)^T C_act (equal for the symmetric
    AO tensor).  Columns of C outside ``orb`` get zero.  Returns (dAO, dC) with
    the shapes of ``ao3c`` and ``C``.
    """
    ao = np.asarray(ao3c, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    ca = C[:, orb]
    dL = np.asarray(dL, dtype=np.float64)
    d_ao = np.einsum("mp,Ppq,nq->Pmn", ca, dL, ca, optimize=True)
    h = np.einsum("Pmn,nq->Pmq", ao, ca, optimize=True)
    ht = np.einsum("Pnm,nq->Pmq", ao, ca, optimize=True)
    d_ca = np.einsum("Pmq,Prq->mr", h, dL, optimize=True) + np.einsum("Pmp,Ppr->mr", ht, dL, optimize=True)
    d_c = np.zeros_like(C)
    np.add.at(d_c, (slice(None), np.asarray(orb)), d_ca)
    return d_ao, d_c


def ao_to_mo_rows(ao3c, C, orb, rows):
    """L^P_{p q} for p in ``rows`` (indices into ``orb``) and all q in ``orb``.

    The same transform as :func:`ao_to_mo`, restricted to a few rows, for
    checking sampled outputs of workloads whose full L does not fit.
    Returns an array (len(rows), naux, n).
    """
    ca = np.asarray(C, dtype=np.float64)[:, orb]
    half = np.einsum("Pmn,nq->Pmq", ao3c, ca, optimize=True) if len(rows) > 8 else None
    out = []
    for r in rows:
        cr = ca[:, r]
        if half is not None:
            out.append(np.einsum("m,Pmq->Pq", cr, half))
        else:
            out.append(np.einsum("Pmn,m->Pn", ao3c, cr) @ ca)
    return np.array(out)


def pair_list(n, mult):
    """Pair indices in row-major upper-triangle order.

    Singlet pairs have a <= b (Sec. ppRPA Equation, spin-adapted singlet
    elements); triplet pairs have a < b (spin-adapted triplet elements).
    """
    if mult == 1:
        return [(a, b) for a in range(n) for b in range(a, n)]
    if mult == 3:
        return [(a, b) for a in range(n) for b in range(a + 1, n)]
    raise ValueError("mult must be 1 (singlet) or 3 (triplet)")


def eri_phys(L):
    """Dense <pq|rs> = (pr|qs) = sum_P L^P_pr L^P_qs, indexed [p, q, r, s].

    Definition of <pq|rs> in Sec. Pairing Matrix (Dyson equation paragraph),
    with the density-fitting factorisation of (pr|qs).
    """
    chem = np.einsum("Ppr,Pqs->prqs", L, L, optimize=True)  # (pr|qs)
    return chem.transpose(0, 2, 1, 3)


def _block(V, eps, rows, cols, mult, sign):
    """One block of the spin-adapted ppRPA matrix, element by element.

    rows / cols are lists of orbital pairs (global active indices).
    Singlet: delta(eps_p + eps_q) + (<pq|rs> + <pq|sr>) / sqrt((1+d_pq)(1+d_rs)).
    Triplet: delta(eps_p + eps_q) + <pq|rs> - <pq|sr>.
    ``sign`` is +1 for the A block and -1 for the C block (whose diagonal
    carries -(eps_i + eps_j)); it is None for B (no diagonal term).
    """
    p = np.array([x[0] for x in rows], dtype=np.int64)[:, None]
    q = np.array([x[1] for x in rows], dtype=np.int64)[:, None]
    r = np.array([x[0] for x in cols], dtype=np.int64)[None, :]
    s = np.array([x[1] for x in cols], dtype=np.int64)[None, :]
    direct = V[p, q, r, s]
    exch = V[p, q, s, r]
    if mult == 1:
        fac = 1.0 / np.sqrt((1.0 + (p == q)) * (1.0 + (r == s)))
        out = fac * (direct + exch)
    else:
        out = direct - exch
    if sign is not None:
        same = (p == r) & (q == s)
        out = out + np.where(same, sign * (eps[p] + eps[q]), 0.0)
    return out


def matrix_blocks(eps_act, nocc_act, L_act, mult):
    """A, B, C blocks of the spin-adapted ppRPA matrix (Sec. ppRPA Equation).

    A_{ab,cd}: virtual pairs x virtual pairs, B_{ab,kl}: virtual x occupied
    pairs, C_{ij,kl}: occupied x occupied pairs.  Built element by element
    from a dense four-index <pq|rs>, so only small active spaces fit.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    n = eps.shape[0]
    no = nocc_act
    V = eri_phys(np.asarray(L_act, dtype=np.float64))
    vv = [(no + a, no + b) for (a, b) in pair_list(n - no, mult)]
    oo = pair_list(no, mult)
    A = _block(V, eps, vv, vv, mult, +1.0) if vv else np.zeros((0, 0))
    B = _block(V, eps, vv, oo, mult, None) if (vv and oo) else np.zeros((len(vv), len(oo)))
    C = _block(V, eps, oo, oo, mult, -1.0) if oo else np.zeros((0, 0))
    return A, B, C


def build_matrix(eps_act, nocc_act, L_act, mult):
    """Full ppRPA matrix M = [[A, B], [B^T, C]] (Sec. ppRPA Equation).

    Returns ``(M, nvv, noo)``.  The metric of the generalised eigenproblem
    is W = diag(I_nvv, -I_noo).
    """
    A, B, C = matrix_blocks(eps_act, nocc_act, L_act, mult)
    M = np.block([[A, B], [B.T, C]])
    return M, A.shape[0], C.shape[0]


def build_matrix_ab(eps_a, nocc_a, L_a, eps_b, nocc_b, L_b):
    """The (alpha alpha; beta beta) subspace of spin-unrestricted ppRPA (Sec. Implementation
    Details: the matrix is built and diagonalised in three subspaces).

    Pairs of one alpha and one beta orbital: (a, b) over every alpha-virtual x beta-virtual,
    (i, j) over every alpha-occupied x beta-occupied, row-major.  Opposite spins have no
    exchange, so with (pr|qs) = sum_P L^{alpha P}_pr L^{beta P}_qs:
      A_{ab,cd} = d_ac d_bd (eps_a + eps_b) + (ac|bd),  B_{ab,kl} = (ak|bl),
      C_{ij,kl} = -d_ik d_jl (eps_i + eps_j) + (ik|jl).
    The same-spin subspaces are ``build_matrix(eps, nocc, L, 3)`` of one spin (a < b,
    <ab|cd> - <ab|dc>).  Returns ``(M, nvv, noo)``.
    """
    ea = np.asarray(eps_a, dtype=np.float64)
    eb = np.asarray(eps_b, dtype=np.float64)
    La = np.asarray(L_a, dtype=np.float64)
    Lb = np.asarray(L_b, dtype=np.float64)
    na, nb = ea.shape[0], eb.shape[0]
    vv = [(a, b) for a in range(nocc_a, na) for b in range(nocc_b, nb)]
    oo = [(i, j) for i in range(nocc_a) for j in range(nocc_b)]
    V = np.einsum("Ppr,Pqs->pqrs", La, Lb, optimize=True)  # (pr|qs) for p, r alpha; q, s beta
    pairs = vv + oo
    nvv = len(vv)
    M = np.zeros((len(pairs), len(pairs)))
    for I, (p, q) in enumerate(pairs):
        for J, (r, t) in enumerate(pairs):
            M[I, J] = V[p, q, r, t]
        M[I, I] += (ea[p] + eb[q]) if I < nvv else -(ea[p] + eb[q])
    return M, nvv, len(oo)


def diag_of_matrix(eps_act, nocc_act, L_act, mult):
    """Diagonal of M, from the explicit matrix (for checking the GPU diagonal)."""
    M, _, _ = build_matrix(eps_act, nocc_act, L_act, mult)
    return np.diag(M).copy()


def _fix_phase(z):
    """Sign convention: the largest-magnitude component of each column is
    positive.  The paper does not fix the phase; this is a convention."""
    idx = np.argmax(np.abs(z), axis=0)
    sgn = np.sign(z[idx, np.arange(z.shape[1])])
    sgn[sgn == 0] = 1.0
    return z * sgn[None, :]


def solve_full(M, nvv, noo, imag_tol=1e-9):
    """All eigenpairs of M z = omega W z by dense non-symmetric diagonalisation.

    Solves W M z = omega z (W^2 = I), the generalised problem of
    Sec. ppRPA Equation.  Roots are classified by the sign of the norm
    z^T W z (positive: two-electron addition, N+2; negative: removal, N-2)
    and normalised to X^T X - Y^T Y = +-1 (Eq. xy_norm).

    Returns a dict with ascending ``omega_pp`` / ``z_pp`` (columns),
    ``omega_hh`` / ``z_hh`` and ``max_imag`` (largest |Im omega|; a value
    above ``imag_tol`` times the spectral scale marks an unstable problem).
    """
    n = nvv + noo
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    vals, vecs = sla.eig(w[:, None] * M)
    scale = max(1.0, float(np.max(np.abs(vals))))
    max_imag = float(np.max(np.abs(vals.imag))) if n else 0.0
    vals = vals.real
    vecs = vecs.real
    nrm = np.einsum("ik,i,ik->k", vecs, w, vecs)
    z = vecs / np.sqrt(np.abs(nrm))[None, :]
    pos = nrm > 0
    out = {"max_imag": max_imag, "unstable": max_imag > imag_tol * scale}
    for key, mask in (("pp", pos), ("hh", ~pos)):
        o = vals[mask]
        zz = z[:, mask]
        order = np.argsort(o)
        out["omega_" + key] = o[order]
        out["z_" + key] = _fix_phase(zz[:, order]) if zz.shape[1] else zz
    return out


def solve_full_shifted(M, nvv, noo, mu):
    """Same eigenpairs through a shifted symmetric reduction.

    If K = M - mu W is positive definite (K = R^T R), then
    R^-T W R^-1 y = kappa y with omega = mu + 1/kappa and z = R^-1 y; the
    sign of kappa is the sign of the norm z^T W z.  Raises
    ``numpy.linalg.LinAlgError`` when K is not positive definite.
    Independent second route to the eigenpairs of Sec. ppRPA Equation.
    """
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    K = M - mu * np.diag(w)
    R = np.linalg.cholesky(K).T  # K = R^T R
    Rinv = sla.solve_triangular(R, np.eye(R.shape[0]), lower=False)
    H = Rinv.T @ (w[:, None] * Rinv)
    H = 0.5 * (H + H.T)
    kap, Y = np.linalg.eigh(H)
    Z = Rinv @ Y
    omega = mu + 1.0 / kap
    Z = Z / np.sqrt(np.abs(kap))[None, :]
    pos = kap > 0
    out = {}
    for key, mask in (("pp", pos), ("hh", ~pos)):
        o = omega[mask]
        order = np.argsort(o)
        out["omega_" + key] = o[order]
        out["z_" + key] = _fix_phase(Z[:, mask][:, order])
    return out


def correlation_energy(M, nvv, noo, sol=None):
    """E_c from the N+2 roots and from the N-2 roots (Eq. correlation_energy).

    Returns ``(sum(Omega^+2e) - Tr A, -sum(Omega^-2e) - Tr C)``; the two are
    equal for a stable problem with all roots real.
    """
    if sol is None:
        sol = solve_full(M, nvv, noo)
    tr_a = float(np.trace(M[:nvv, :nvv]))
    tr_c = float(np.trace(M[nvv:, nvv:]))
    return float(np.sum(sol["omega_pp"])) - tr_a, -float(np.sum(sol["omega_hh"])) - tr_c


def grad_omega(eps_act, nocc_act, L_act, mult, z):
    """Hellmann-Feynman gradient of one root, d omega / d eps_p and d omega / d L^P_pq.

    Sec. Analytic Gradient: d Omega = [X^T Y^T] (dM) [X; Y] for the
    normalisation of Eq. xy_norm; with s = z^T W z = +-1 this reads
    d omega = s z^T (dM) z.  dM is formed element by element from the
    definitions of A, B, C (the same ones ``build_matrix`` uses), and
    the chain rule through <pq|rs> = sum_P L^P_pr L^P_qs gives the
    derivative with respect to every entry of L^P (entries treated as
    independent; the symmetric part is what a symmetric perturbation sees).

    Returns ``(d_eps (n,), d_L (naux, n, n))``.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    L = np.asarray(L_act, dtype=np.float64)
    n = eps.shape[0]
    no = nocc_act
    vv = [(no + a, no + b) for (a, b) in pair_list(n - no, mult)]
    oo = pair_list(no, mult)
    pairs = vv + oo
    nvv = len(vv)
    w = np.concatenate([np.ones(nvv), -np.ones(len(oo))])
    z = np.asarray(z, dtype=np.float64)
    s = float(np.sign(z @ (w * z)))
    gamma = s * np.outer(z, z)  # d omega / d M_IJ
    # eps part: diagonal of A carries +(eps_p + eps_q), diagonal of C -(eps_i + eps_j)
    d_eps = np.zeros(n)
    for I, (p, q) in enumerate(pairs):
        d_eps[p] += w[I] * gamma[I, I]
        d_eps[q] += w[I] * gamma[I, I]
    # two-electron part: M_IJ = f_IJ (V[p,q,r,s] + t V[p,q,s,r]), t = +1 singlet, -1 triplet
    P1 = np.array([x[0] for x in pairs])
    P2 = np.array([x[1] for x in pairs])
    if mult == 1:
        f = 1.0 / np.sqrt(np.outer(1.0 + (P1 == P2), 1.0 + (P1 == P2)))
        t = 1.0
    else:
        f = np.ones((len(pairs), len(pairs)))
        t = -1.0
    g4 = np.zeros((n, n, n, n))  # d omega / d V[p,q,r,s]
    gf = gamma * f
    np.add.at(g4, (P1[:, None], P2[:, None], P1[None, :], P2[None, :]), gf)
    np.add.at(g4, (P1[:, None], P2[:, None], P2[None, :], P1[None, :]), t * gf)
    # V[p,q,r,s] = sum_P L^P_pr L^P_qs  ->  dV/dL^P_xy = d_px d_ry L^P_qs + L^P_pr d_qx d_sy
    d_L = np.einsum("xqys,Pqs->Pxy", g4, L, optimize=True) + np.einsum(
        "pxry,Ppr->Pxy", g4, L, optimize=True
    )
    return d_eps, d_L


def grad_omega_ab(eps_a, nocc_a, L_a, eps_b, nocc_b, L_b, z):
    """Hellmann-Feynman gradient of one root of the (alpha alpha; beta beta) subspace.

    Sec. Analytic Gradient applied to the matrix of ``build_matrix_ab``: d omega =
    s z^T (dM) z with s = z^T W z = +-1.  dM is formed element by element from that
    matrix's definitions: the diagonal carries +(eps_a + eps_b) on virtual pairs and
    -(eps_i + eps_j) on occupied pairs, and every element carries
    (pr|qs) = sum_P L^{alpha P}_pr L^{beta P}_qs, whose chain rule gives the derivative
    with respect to every entry of L^alpha and L^beta (entries treated as independent).

    Returns ``(d_eps_a (na,), d_eps_b (nb,), d_La (naux, na, na), d_Lb (naux, nb, nb))``.
    """
    ea = np.asarray(eps_a, dtype=np.float64)
    eb = np.asarray(eps_b, dtype=np.float64)
    La = np.asarray(L_a, dtype=np.float64)
    Lb = np.asarray(L_b, dtype=np.float64)
    na, nb = ea.shape[0], eb.shape[0]
    vv = [(a, b) for a in range(nocc_a, na) for b in range(nocc_b, nb)]
    oo = [(i, j) for i in range(nocc_a) for j in range(nocc_b)]
    pairs = vv + oo
    nvv = len(vv)
    w = np.concatenate([np.ones(nvv), -np.ones(len(oo))])
    z = np.asarray(z, dtype=np.float64)
    s = float(np.sign(z @ (w * z)))
    gamma = s * np.outer(z, z)  # d omega / d M_IJ
    d_ea = np.zeros(na)
    d_eb = np.zeros(nb)
    for I, (p, q) in enumerate(pairs):
        d_ea[p] += w[I] * gamma[I, I]
        d_eb[q] += w[I] * gamma[I, I]
    # M_IJ = V[p_I, q_I, p_J, q_J] + diagonal, V[p, q, r, t] = sum_P La[P, p, r] Lb[P, q, t]
    P1 = np.array([x[0] for x in pairs])
    P2 = np.array([x[1] for x in pairs])
    g4 = np.zeros((na, nb, na, nb))  # d omega / d V[p, q, r, t]
    np.add.at(g4, (P1[:, None], P2[:, None], P1[None, :], P2[None, :]), gamma)
    d_La = np.einsum("pqrt,Pqt->Ppr", g4, Lb, optimize=True)
    d_Lb = np.einsum("pqrt,Ppr->Pqt", g4, La, optimize=True)
    return d_ea, d_eb, d_La, d_Lb


def _triangular(vec, n, mult):
    """Pair vector -> n x n upper-triangular matrix (Sec. Natural Transition
    Orbital: X and Y viewed as triangular matrices)."""
    T = np.zeros((n, n))
    for I, (p, q) in enumerate(pair_list(n, mult)):
        T[p, q] = vec[I]
    return T


def two_e_density_diag(z, nocc_act, nvir_act, mult):
    """Diagonal of the two-electron addition/removal density matrix.

    Sec. Density Matrix: D_ab = [X X^T + X^T X]_ab, D_ij = -[Y Y^T + Y^T Y]_ij,
    with X, Y the triangular matrices of the eigenvector.  Returned in
    active-orbital order (occupied first).
    """
    nvv = len(pair_list(nvir_act, mult))
    X = _triangular(z[:nvv], nvir_act, mult)
    Y = _triangular(z[nvv:], nocc_act, mult)
    dv = np.diag(X @ X.T + X.T @ X)
    do = -np.diag(Y @ Y.T + Y.T @ Y)
    return np.concatenate([do, dv])


def two_e_density(z, nocc_act, nvir_act, mult):
    """The two-electron addition/removal density matrix D^2e (Sec. Density Matrix), n x n in
    active-orbital order (occupied first): virtual block X X^T + X^T X, occupied block
    -(Y Y^T + Y^T Y), zero occupied-virtual blocks; X, Y the triangular matrices of z."""
    nvv = len(pair_list(nvir_act, mult))
    X = _triangular(z[:nvv], nvir_act, mult)
    Y = _triangular(z[nvv:], nocc_act, mult)
    n = nocc_act + nvir_act
    D = np.zeros((n, n))
    D[:nocc_act, :nocc_act] = -(Y @ Y.T + Y.T @ Y)
    D[nocc_act:, nocc_act:] = X @ X.T + X.T @ X
    return D


def nto(z, nocc_act, nvir_act, mult):
    """Natural transition orbitals (Eqs. nto_pp, nto_hh): X = C^p1 sqrt(lambda^p) C^p2^T and
    Y = C^h1 sqrt(lambda^h) C^h2^T, the singular value decompositions of the triangular X and
    Y, weights descending.  Phase convention: the largest-magnitude entry of each C^p1 / C^h1
    column is positive (C^p2 / C^h2 follow).  Returns (lam_p, Cp1, Cp2, lam_h, Ch1, Ch2)."""
    nvv = len(pair_list(nvir_act, mult))
    out = []
    for T in (_triangular(z[:nvv], nvir_act, mult), _triangular(z[nvv:], nocc_act, mult)):
        if T.shape[0] == 0:
            out += [np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0))]
            continue
        U, sv, Vt = np.linalg.svd(T)
        V = Vt.T
        for k in range(U.shape[1]):
            if U[np.argmax(np.abs(U[:, k])), k] < 0:
                U[:, k] *= -1
                V[:, k] *= -1
        out += [sv ** 2, U, V]
    return tuple(out)


def _rect_ab(z, nocc_a, nvir_a, nocc_b, nvir_b):
    """Alpha-beta pair vector -> X (nvir_a x nvir_b) and Y (nocc_a x nocc_b), the pair
    lists of ``build_matrix_ab`` (row-major) read as rectangles."""
    z = np.asarray(z, dtype=np.float64)
    nvv = nvir_a * nvir_b
    return z[:nvv].reshape(nvir_a, nvir_b), z[nvv:].reshape(nocc_a, nocc_b)


def two_e_density_ab(z, nocc_a, nvir_a, nocc_b, nvir_b):
    """Two-electron density of an alpha-beta root (Sec. Density Matrix with the two orbital
    slots of a pair resolved by spin): D^alpha has X X^T on its virtual block and -Y Y^T on
    its occupied block, D^beta has X^T X and -Y^T Y.  Returned as the block-diagonal
    (na + nb) x (na + nb) matrix diag(D^alpha, D^beta), each spin in active-orbital order
    (occupied first)."""
    X, Y = _rect_ab(z, nocc_a, nvir_a, nocc_b, nvir_b)
    na, nb = nocc_a + nvir_a, nocc_b + nvir_b
    D = np.zeros((na + nb, na + nb))
    D[:nocc_a, :nocc_a] = -(Y @ Y.T)
    D[nocc_a:na, nocc_a:na] = X @ X.T
    D[na:na + nocc_b, na:na + nocc_b] = -(Y.T @ Y)
    D[na + nocc_b:, na + nocc_b:] = X.T @ X
    return D


def nto_ab(z, nocc_a, nvir_a, nocc_b, nvir_b):
    """Natural transition orbitals of an alpha-beta root (Eqs. nto_pp, nto_hh with X and Y
    the rectangles of the pair vector): X = C^p1 sqrt(lambda^p) C^p2^T with C^p1 over alpha
    virtuals and C^p2 over beta virtuals (likewise Y).  lam has one entry per alpha orbital
    of the block (descending, zero beyond the rank); C1 is square (alpha), C2 is
    (beta x alpha) with zero columns where the weight is zero.  Phase: the largest-magnitude
    entry of each C1 column is positive.  Returns (lam_p, Cp1, Cp2, lam_h, Ch1, Ch2)."""
    out = []
    for T in _rect_ab(z, nocc_a, nvir_a, nocc_b, nvir_b):
        m1, m2 = T.shape
        if m1 == 0:
            out += [np.zeros(0), np.zeros((0, 0)), np.zeros((m2, 0))]
            continue
        U, sv, Vt = np.linalg.svd(T, full_matrices=True)
        lam = np.zeros(m1)
        lam[: sv.shape[0]] = sv ** 2
        C2 = np.zeros((m2, m1))
        r = min(m1, m2)
        C2[:, :r] = Vt[:r].T
        C2[:, lam <= 1e-28 * max(lam.max(), 1e-300)] = 0.0
        for k in range(m1):
            if U[np.argmax(np.abs(U[:, k])), k] < 0:
                U[:, k] *= -1
                C2[:, k] *= -1
        out += [lam, U, C2]
    return tuple(out)


def nto_weights(z, nocc_act, nvir_act, mult):
    """NTO weights lambda^p, lambda^h: squared singular values of the
    triangular X and Y (Eqs. nto_pp, nto_hh)."""
    nvv = len(pair_list(nvir_act, mult))
    X = _triangular(z[:nvv], nvir_act, mult)
    Y = _triangular(z[nvv:], nocc_act, mult)
    lp = np.linalg.svd(X, compute_uv=False) ** 2 if nvir_act else np.zeros(0)
    lh = np.linalg.svd(Y, compute_uv=False) ** 2 if nocc_act else np.zeros(0)
    return lp, lh
