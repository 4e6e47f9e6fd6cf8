"""Brute-force references that do not use the spin adaptation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``spinorb_matrix``: the ppRPA matrix over spin orbitals with the
  antisymmetrised interaction (Sec. ppRPA Equation, general A, B, C with
  a < b, i < j).  Its spectrum is the union of the singlet roots and three
  copies of the triplet roots.
* ``spinorb_matrix_fractional``: the same with the fractional-occupation weights of
  Sec. ppRPA for Fractional Charge Systems, over distinct orbitals (a fractionally
  occupied orbital gives both hole and particle spin orbitals).
* ``spinorb_matrix_unrestricted``: the spin-orbital matrix of a spin-unrestricted
  reference (different alpha and beta orbitals); its spectrum is the union of the three
  subspaces of spin-unrestricted ppRPA.
* ``two_electron_ci``: the Hamiltonian of two electrons in the virtual
  orbitals, in the basis of opposite-spin determinants, from the
  Slater-Condon rules.  With no occupied orbitals ppRPA is exact for two
  electrons (Sec. Total Energy results, the two-electron statement).
* ``mp2_pair_energy``: the second-order energy the ppRPA correlation energy
  reduces to for weak interaction (ladder-CCD equivalence, Introduction).
"""
from __future__ import annotations

import numpy as np

from .pprpa_ref import eri_phys


def _spin_eri(L):
    """Antisymmetrised <PQ||RS> over spin orbitals P = 2p + sigma."""
    V = eri_phys(np.asarray(L, dtype=np.float64))
    n = V.shape[0]
    spin = np.arange(2 * n) % 2
    sp = np.arange(2 * n) // 2
    Vso = V[np.ix_(sp, sp, sp, sp)]
    mask = (spin[:, None, None, None] == spin[None, None, :, None]) & (
        spin[None, :, None, None] == spin[None, None, None, :]
    )
    Vso = np.where(mask, Vso, 0.0)
    return Vso - Vso.transpose(0, 1, 3, 2)


def spinorb_matrix(eps_act, nocc_act, L_act):
    """Spin-orbital ppRPA matrix and its block sizes.

    A_{ab,cd} = d_ac d_bd (eps_a + eps_b) + <ab||cd>, B_{ab,kl} = <ab||kl>,
    C_{ij,kl} = -d_ik d_jl (eps_i + eps_j) + <ij||kl>, a < b, i < j over
    spin orbitals (Sec. ppRPA Equation).  Returns ``(M, nvv, noo)``.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    n = eps.shape[0]
    anti = _spin_eri(L_act)
    e_so = np.repeat(eps, 2)
    occ_so = [P for P in range(2 * n) if P // 2 < nocc_act]
    vir_so = [P for P in range(2 * n) if P // 2 >= nocc_act]
    vv = [(vir_so[x], vir_so[y]) for x in range(len(vir_so)) for y in range(x + 1, len(vir_so))]
    oo = [(occ_so[x], occ_so[y]) for x in range(len(occ_so)) for y in range(x + 1, len(occ_so))]
    allp = vv + oo
    nvv, noo = len(vv), len(oo)
    M = np.zeros((nvv + noo, nvv + noo))
    for I, (p, q) in enumerate(allp):
        for J, (r, s) in enumerate(allp):
            M[I, J] = anti[p, q, r, s]
        if I < nvv:
            M[I, I] += e_so[p] + e_so[q]
        else:
            M[I, I] -= e_so[p] + e_so[q]
    return M, nvv, noo


def spinorb_matrix_fractional(eps, occ, L, holes, parts):
    """Spin-orbital ppRPA matrix of a fractionally occupied system, element by element from
    the matrix elements of Sec. ppRPA for Fractional Charge Systems:
      A_{ab,cd} = d_ac d_bd (eps_a + eps_b) + sqrt((1-n_a)(1-n_b)(1-n_c)(1-n_d)) <ab||cd>,
      B_{ab,kl} = sqrt((1-n_a)(1-n_b) n_k n_l) <ab||kl>,
      C_{ij,kl} = -d_ik d_jl (eps_i + eps_j) + sqrt(n_i n_j n_k n_l) <ij||kl>,
    a < b over the spin orbitals of the particle orbitals ``parts``, i < j over those of the
    hole orbitals ``holes`` (indices into the distinct orbitals of ``eps``, ``occ`` and
    ``L``; an orbital may be in both lists).  Returns ``(M, nvv, noo)``."""
    eps = np.asarray(eps, dtype=np.float64)
    occ = np.asarray(occ, dtype=np.float64)
    anti = _spin_eri(L)
    so_h = [2 * p + sg for p in holes for sg in (0, 1)]
    so_p = [2 * p + sg for p in parts for sg in (0, 1)]
    vv = [(so_p[x], so_p[y]) for x in range(len(so_p)) for y in range(x + 1, len(so_p))]
    oo = [(so_h[x], so_h[y]) for x in range(len(so_h)) for y in range(x + 1, len(so_h))]
    wp = lambda P: np.sqrt(1.0 - occ[P // 2])
    wh = lambda P: np.sqrt(occ[P // 2])
    nvv, noo = len(vv), len(oo)
    M = np.zeros((nvv + noo, nvv + noo))
    for I, (a, b) in enumerate(vv + oo):
        fa = wp(a) * wp(b) if I < nvv else wh(a) * wh(b)
        for J, (c, d) in enumerate(vv + oo):
            fc = wp(c) * wp(d) if J < nvv else wh(c) * wh(d)
            M[I, J] = fa * fc * anti[a, b, c, d]
        e = eps[a // 2] + eps[b // 2]
        M[I, I] += e if I < nvv else -e
    return M, nvv, noo


def spinorb_matrix_unrestricted(eps_a, nocc_a, L_a, eps_b, nocc_b, L_b):
    """ppRPA matrix over spin orbitals with different alpha and beta spatial orbitals (a
    spin-unrestricted reference): spin orbitals are the alpha orbitals then the beta
    orbitals, <PQ||RS> = <PQ|RS> - <PQ|SR> with <PQ|RS> = (PR|QS) nonzero only for equal
    spins of P, R and of Q, S, and (pr|qs) from L^alpha / L^beta by the spins of the two
    charge distributions; pairs a < b over virtual and i < j over occupied spin orbitals.
    Returns ``(M, nvv, noo)``; its spectrum is the union of the alpha-alpha, beta-beta
    and alpha-beta subspaces."""
    ea = np.asarray(eps_a, dtype=np.float64)
    eb = np.asarray(eps_b, dtype=np.float64)
    La = np.asarray(L_a, dtype=np.float64)
    Lb = np.asarray(L_b, dtype=np.float64)
    na, nb = ea.shape[0], eb.shape[0]
    so = [(0, p) for p in range(na)] + [(1, p) for p in range(nb)]  # (spin, spatial index)
    e_so = np.concatenate([ea, eb])
    occ_so = [P for P, (sg, p) in enumerate(so) if p < (nocc_a if sg == 0 else nocc_b)]
    vir_so = [P for P in range(len(so)) if P not in occ_so]
    Ls = (La, Lb)

    def chem(P, R, Q, S):  # (PR|QS)
        (s1, p), (s2, r), (s3, q), (s4, t) = so[P], so[R], so[Q], so[S]
        if s1 != s2 or s3 != s4:
            return 0.0
        return float(np.dot(Ls[s1][:, p, r], Ls[s3][:, q, t]))

    def anti(P, Q, R, S):
        return chem(P, R, Q, S) - chem(P, S, Q, R)

    vv = [(vir_so[x], vir_so[y]) for x in range(len(vir_so)) for y in range(x + 1, len(vir_so))]
    oo = [(occ_so[x], occ_so[y]) for x in range(len(occ_so)) for y in range(x + 1, len(occ_so))]
    pairs = vv + oo
    nvv = len(vv)
    M = np.zeros((len(pairs), len(pairs)))
    for I, (P, Q) in enumerate(pairs):
        for J, (R, S) in enumerate(pairs):
            M[I, J] = anti(P, Q, R, S)
        M[I, I] += (e_so[P] + e_so[Q]) if I < nvv else -(e_so[P] + e_so[Q])
    return M, nvv, len(oo)


def two_electron_ci(eps_act, L_act):
    """Two electrons in all given orbitals: eigenvalues of the determinant CI.

    Basis: |p alpha, q beta> for all p, q (the M_s = 0 space, which holds
    every singlet and one component of every triplet).  Slater-Condon rules
    give <p q|H|r s> = d_pr d_qs (eps_p + eps_q) + <pq|rs>; the exchange
    integral vanishes between opposite spins.  Returns sorted eigenvalues.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    n = eps.shape[0]
    V = eri_phys(np.asarray(L_act, dtype=np.float64))
    H = V.reshape(n * n, n * n).copy()
    H[np.arange(n * n), np.arange(n * n)] += (eps[:, None] + eps[None, :]).reshape(-1)
    return np.sort(np.linalg.eigvalsh(0.5 * (H + H.T)))


def mp2_pair_energy(eps_act, nocc_act, L_act):
    """E2 = sum_{a<b, i<j} |<ab||ij>|^2 / (eps_i + eps_j - eps_a - eps_b), spin orbitals.

    The second-order energy that ppRPA (ladder CCD, exact to second order;
    Introduction) reproduces in the weak-interaction limit.
    """
    eps = np.asarray(eps_act, dtype=np.float64)
    n = eps.shape[0]
    anti = _spin_eri(L_act)
    e_so = np.repeat(eps, 2)
    occ = [P for P in range(2 * n) if P // 2 < nocc_act]
    vir = [P for P in range(2 * n) if P // 2 >= nocc_act]
    e2 = 0.0
    for x, a in enumerate(vir):
        for b in vir[x + 1:]:
            for y, i in enumerate(occ):
                for j in occ[y + 1:]:
                    e2 += anti[a, b, i, j] ** 2 / (e_so[i] + e_so[j] - e_so[a] - e_so[b])
    return e2
