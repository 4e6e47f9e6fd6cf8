"""Pins of the FP64 oracle against facts it does not compute itself.

Each test ties the oracle to the paper or to mathematics: a brute-force
spin-orbital build, a determinant CI, a closed form, a limit or an identity.
A plausible slip in the oracle (a dropped 1/sqrt(2), a wrong exchange sign,
a transposed index, a missing diagonal term) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(no, nv, naux, seed, nbasis_extra=3):
    """A small synthetic system (same generator as the workloads)."""
    nb = no + nv + nbasis_extra
    spec = synth.SystemSpec("t", nb, no + 1 if no else 0, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    return s["eps"][orb], L


def test_generator_chunked_stream_is_identical():
    spec = synth.SystemSpec("t", 12, 4, 10, 4, 8, 7)
    full = synth.make_system(spec)["ao3c"]
    parts = [blk for _, blk in synth.ao_slices(spec, 3)]
    assert np.array_equal(np.concatenate(parts), full)
    assert np.allclose(full, full.transpose(0, 2, 1))


def test_ao_to_mo_matches_two_step_transform():
    spec = synth.SystemSpec("t", 9, 3, 5, 2, 4, 3)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 2, 4)
    assert list(orb) == [1, 2, 3, 4, 5, 6]
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    C = s["C"][:, orb]
    for P in range(spec.naux):
        ref = C.T @ s["ao3c"][P] @ C
        assert np.allclose(L[P], ref, atol=1e-14)


@pytest.mark.parametrize("no,nv", [(2, 3), (3, 4), (1, 4)])
def test_spin_adapted_spectrum_equals_spin_orbital(no, nv):
    """Singlet roots + 3 x triplet roots = spin-orbital roots (general A, B, C)."""
    eps, L = small(no, nv, 7, 11 + no)
    Mso, nvv_so, noo_so = oracle.spinorb_matrix(eps, no, L)
    so = oracle.solve_full(Mso, nvv_so, noo_so)
    parts = {}
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
        parts[mult] = oracle.solve_full(M, nvv, noo)
        parts[mult]["Ec"] = oracle.correlation_energy(M, nvv, noo, parts[mult])[0]
    pp = np.sort(np.concatenate([parts[1]["omega_pp"]] + [parts[3]["omega_pp"]] * 3))
    hh = np.sort(np.concatenate([parts[1]["omega_hh"]] + [parts[3]["omega_hh"]] * 3))
    assert np.allclose(np.sort(so["omega_pp"]), pp, atol=1e-11)
    assert np.allclose(np.sort(so["omega_hh"]), hh, atol=1e-11)
    ec_so = oracle.correlation_energy(Mso, nvv_so, noo_so, so)[0]
    assert abs(ec_so - (parts[1]["Ec"] + 3 * parts[3]["Ec"])) < 1e-11


@pytest.mark.parametrize("frac", [0.6, 0.15, 0.97])
def test_fractional_occupation_folding_equals_spin_orbital_elements(frac):
    """Sec. ppRPA for Fractional Charge Systems: the weighted integrals over hole and particle
    slots (a fractional HOMO in both lists) give, through the spin adaptation, the spectrum
    of the spin-orbital matrix written element by element from the paper's fractional A, B
    and C: singlet roots + 3 x triplet roots, both root sets, and E_c."""
    spec = synth.SystemSpec("t", 10, 3, 8, 2, 4, 53)
    s = synth.make_system(spec)
    occ = np.zeros(spec.nmo)
    occ[:3] = [1.0, 1.0, frac]
    orb, w = oracle.fractional_slots(occ, 2, 4)
    assert list(orb) == [1, 2, 2, 3, 4, 5]
    assert np.allclose(w, [1.0, np.sqrt(frac), np.sqrt(1 - frac), 1.0, 1.0, 1.0])
    L, eps_s = oracle.fractional_integrals(s["ao3c"], s["C"], occ, s["eps"], 2, 4)
    uniq = np.array([1, 2, 3, 4, 5])
    Lu = oracle.ao_to_mo(s["ao3c"], s["C"], uniq)
    Mso, nvv_so, noo_so = oracle.spinorb_matrix_fractional(s["eps"][uniq], occ[uniq], Lu, [0, 1], [1, 2, 3, 4])
    so = oracle.solve_full(Mso, nvv_so, noo_so)
    parts, ec = {}, 0.0
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps_s, 2, L, mult)
        parts[mult] = oracle.solve_full(M, nvv, noo)
        ec += (1 if mult == 1 else 3) * oracle.correlation_energy(M, nvv, noo, parts[mult])[0]
    for key in ("pp", "hh"):
        ref = np.sort(np.concatenate([parts[1]["omega_" + key]] + [parts[3]["omega_" + key]] * 3))
        assert np.allclose(np.sort(so["omega_" + key]), ref, atol=1e-11)
    assert abs(oracle.correlation_energy(Mso, nvv_so, noo_so, so)[0] - ec) < 1e-11


def test_fractional_ao_adjoint_matches_finite_differences():
    """The AO adjoint of the fractional chain: slots with weights (a duplicated orbital) and
    d omega / d L~ scaled by w_s w_t, against central differences of a root in the AO
    integrals and in C."""
    spec = synth.SystemSpec("t", 10, 3, 7, 2, 4, 56)
    s = synth.make_system(spec)
    occ = np.zeros(spec.nmo)
    occ[:3] = [1.0, 1.0, 0.4]
    orb, w = oracle.fractional_slots(occ, 2, 4)

    def root(ao, C):
        L, e = oracle.fractional_integrals(ao, C, occ, s["eps"], 2, 4)
        M, nvv, noo = oracle.build_matrix(e, 2, L, 1)
        sol = oracle.solve_full(M, nvv, noo)
        return sol["omega_pp"][0], sol["z_pp"][:, 0], L, e

    _, z, L, e = root(s["ao3c"], s["C"])
    _, dL = oracle.grad_omega(e, 2, L, 1, z)
    d_ao, d_c = oracle.grad_ao(s["ao3c"], s["C"], orb, dL * w[None, :, None] * w[None, None, :])
    rng = np.random.default_rng(8)
    h = 1e-5
    E = rng.standard_normal(s["ao3c"].shape)
    E = (E + E.transpose(0, 2, 1)) / np.linalg.norm(E)
    fd = (root(s["ao3c"] + h * E, s["C"])[0] - root(s["ao3c"] - h * E, s["C"])[0]) / (2 * h)
    assert abs(fd - float(np.sum(d_ao * E))) < 1e-6 * max(1.0, abs(fd))
    D = rng.standard_normal(s["C"].shape)
    D /= np.linalg.norm(D)
    fd = (root(s["ao3c"], s["C"] + h * D)[0] - root(s["ao3c"], s["C"] - h * D)[0]) / (2 * h)
    assert abs(fd - float(np.sum(d_c * D))) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("frac", [0.2, 0.5, 0.9])
def test_fractional_single_orbital_closed_form(frac):
    """One orbital that is both the hole and the particle slot (occupation n): the singlet
    2 x 2 problem has A = 2 eps + (1-n)^2 g, B = n (1-n) g, C = -2 eps + n^2 g with
    g = (HH|HH), so its roots are 2 eps and 2 eps + ((1-n)^2 - n^2) g; at n = 1/2 they
    coincide (the pencil is defective there)."""
    spec = synth.SystemSpec("t", 6, 1, 5, 1, 1, 71)
    s = synth.make_system(spec)
    occ = np.zeros(spec.nmo)
    occ[0] = frac
    L, e = oracle.fractional_integrals(s["ao3c"], s["C"], occ, s["eps"], 1, 1)
    M, nvv, noo = oracle.build_matrix(e, 1, L, 1)
    g = float(np.sum(oracle.ao_to_mo(s["ao3c"], s["C"], [0])[:, 0, 0] ** 2))
    eps0 = s["eps"][0]
    want = np.sort([2 * eps0, 2 * eps0 + ((1 - frac) ** 2 - frac ** 2) * g])
    got = np.sort(np.linalg.eigvals(np.diag([1.0, -1.0]) @ M).real)
    assert np.allclose(got, want, atol=1e-7 if frac == 0.5 else 1e-12)


def test_fractional_path_reduces_to_integer_occupations():
    spec = synth.SystemSpec("t", 12, 4, 9, 3, 5, 54)
    s = synth.make_system(spec)
    L, e = oracle.fractional_integrals(s["ao3c"], s["C"], s["occ"], s["eps"], 3, 5)
    orb = oracle.active_orbitals(s["occ"], 3, 5)
    assert np.array_equal(L, oracle.ao_to_mo(s["ao3c"], s["C"], orb))
    assert np.array_equal(e, s["eps"][orb])


@pytest.mark.parametrize("no,nv", [(2, 3), (1, 4), (3, 3)])
def test_alpha_beta_subspace_restricted_limit(no, nv):
    """alpha = beta: the M_s = 0 pairs hold every singlet and one component of every
    triplet, so the alpha-beta spectrum is the singlet roots plus the triplet roots."""
    eps, L = small(no, nv, 6, 21 + no)
    M, nvv, noo = oracle.build_matrix_ab(eps, no, L, eps, no, L)
    ab = oracle.solve_full(M, nvv, noo)
    s1 = oracle.solve_full(*oracle.build_matrix(eps, no, L, 1))
    s3 = oracle.solve_full(*oracle.build_matrix(eps, no, L, 3))
    for key in ("pp", "hh"):
        ref = np.sort(np.concatenate([s1["omega_" + key], s3["omega_" + key]]))
        assert np.allclose(np.sort(ab["omega_" + key]), ref, atol=1e-11)


def test_unrestricted_three_subspaces_equal_spin_orbital_matrix():
    """Different alpha and beta orbitals (and occupied counts): the spin-orbital spectrum is
    alpha-alpha + beta-beta + alpha-beta (Sec. Implementation Details, three subspaces)."""
    spec = synth.SystemSpec("t", 9, 3, 6, 3, 6, 81)
    s = synth.make_system(spec)
    rng = np.random.default_rng(82)
    Q, _ = np.linalg.qr(rng.standard_normal((spec.nmo, spec.nmo)))
    Cb = s["C"] @ Q  # different beta orbitals
    ea = s["eps"]
    eb = np.sort(s["eps"] + 0.05 * rng.standard_normal(spec.nmo))
    oa, ob = 3, 2
    La = oracle.ao_to_mo(s["ao3c"], s["C"], np.arange(spec.nmo))
    Lb = oracle.ao_to_mo(s["ao3c"], Cb, np.arange(spec.nmo))
    Mso, nvv, noo = oracle.spinorb_matrix_unrestricted(ea, oa, La, eb, ob, Lb)
    so = oracle.solve_full(Mso, nvv, noo)
    parts = [oracle.solve_full(*oracle.build_matrix(ea, oa, La, 3)),
             oracle.solve_full(*oracle.build_matrix(eb, ob, Lb, 3)),
             oracle.solve_full(*oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb))]
    for key in ("pp", "hh"):
        ref = np.sort(np.concatenate([p["omega_" + key] for p in parts]))
        assert np.allclose(np.sort(so["omega_" + key]), ref, atol=1e-10)


def unrestricted_small(seed=83):
    """Different alpha and beta orbitals, energies and occupied counts (2 alpha, 1 beta)."""
    spec = synth.SystemSpec("t", 8, 3, 6, 3, 5, seed)
    s = synth.make_system(spec)
    rng = np.random.default_rng(seed + 1)
    Q, _ = np.linalg.qr(rng.standard_normal((spec.nmo, spec.nmo)))
    Cb = s["C"] @ (np.eye(spec.nmo) + 0.2 * (Q - np.eye(spec.nmo)))
    Cb, _ = np.linalg.qr(Cb)
    oa, va, ob, vb = 2, 4, 1, 4
    orb_a = np.arange(3 - oa, 3 + va)
    orb_b = np.arange(2 - ob, 2 + vb)
    eb_full = np.sort(s["eps"] + 0.04 * rng.standard_normal(spec.nmo))
    La = oracle.ao_to_mo(s["ao3c"], s["C"], orb_a)
    Lb = oracle.ao_to_mo(s["ao3c"], Cb, orb_b)
    return s["eps"][orb_a], oa, La, eb_full[orb_b], ob, Lb


def test_alpha_beta_gradient_matches_finite_differences():
    """grad_omega_ab: d omega / d eps (alpha, beta) and d omega / d L (alpha, beta) against
    central differences (h = 1e-4) of roots of the alpha-beta matrix, addition and removal."""
    ea, oa, La, eb, ob, Lb = unrestricted_small()
    M, nvv, noo = oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb)
    sol = oracle.solve_full(M, nvv, noo)
    assert sol["max_imag"] == 0.0
    h = 1e-4
    rng = np.random.default_rng(5)
    for key, r in (("pp", 0), ("pp", 3), ("hh", -1)):
        z = sol["z_" + key][:, r]
        dea, deb, dLa, dLb = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, z)

        def root(xa, Xa, xb, Xb):
            sx = oracle.solve_full(*oracle.build_matrix_ab(xa, oa, Xa, xb, ob, Xb))
            return sx["omega_" + key][r]

        for p in (0, 2, 4):
            for side in ("a", "b"):
                e = (ea if side == "a" else eb).copy()
                ep, em = e.copy(), e.copy()
                ep[p] += h
                em[p] -= h
                if side == "a":
                    fd = (root(ep, La, eb, Lb) - root(em, La, eb, Lb)) / (2 * h)
                    an = dea[p]
                else:
                    fd = (root(ea, La, ep, Lb) - root(ea, La, em, Lb)) / (2 * h)
                    an = deb[p]
                assert abs(fd - an) < 1e-5 * max(1.0, abs(an))
        for _ in range(2):
            for side in ("a", "b"):
                X = La if side == "a" else Lb
                D = rng.standard_normal(X.shape)
                D = D + D.transpose(0, 2, 1)
                D /= np.linalg.norm(D)
                if side == "a":
                    fd = (root(ea, La + h * D, eb, Lb) - root(ea, La - h * D, eb, Lb)) / (2 * h)
                    an = float(np.sum(dLa * D))
                else:
                    fd = (root(ea, La, eb, Lb + h * D) - root(ea, La, eb, Lb - h * D)) / (2 * h)
                    an = float(np.sum(dLb * D))
                assert abs(fd - an) < 1e-5 * max(1.0, abs(an))


def test_alpha_beta_gradient_uniform_shift_rule():
    """Shifting every alpha (or every beta) orbital energy by d adds d W to M, which moves
    every root by d: the alpha and the beta energy gradients of any root each sum to 1."""
    ea, oa, La, eb, ob, Lb = unrestricted_small(85)
    M, nvv, noo = oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb)
    sol = oracle.solve_full(M, nvv, noo)
    for key in ("pp", "hh"):
        for r in range(sol["z_" + key].shape[1]):
            dea, deb, _, _ = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, sol["z_" + key][:, r])
            assert abs(dea.sum() - 1.0) < 1e-10 and abs(deb.sum() - 1.0) < 1e-10


def test_alpha_beta_density_and_ntos():
    """two_e_density_ab / nto_ab: each spin's block traces to s = z^T W z, s times the
    diagonal of D^alpha (D^beta) is the alpha (beta) energy gradient of grad_omega_ab (pinned
    by finite differences), the NTOs rebuild X and Y, and sum(lam_p) - sum(lam_h) = s."""
    ea, oa, La, eb, ob, Lb = unrestricted_small(87)
    va, vb = len(ea) - oa, len(eb) - ob
    M, nvv, noo = oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb)
    sol = oracle.solve_full(M, nvv, noo)
    na = len(ea)
    for key, r, sgn in (("pp", 0, 1.0), ("pp", 2, 1.0), ("hh", -1, -1.0)):
        z = sol["z_" + key][:, r]
        D = oracle.two_e_density_ab(z, oa, va, ob, vb)
        assert abs(np.trace(D[:na, :na]) - sgn) < 1e-12 and abs(np.trace(D[na:, na:]) - sgn) < 1e-12
        assert np.abs(D[:na, na:]).max() == 0.0
        dea, deb, _, _ = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, z)
        assert np.abs(sgn * np.diag(D)[:na] - dea).max() < 1e-13
        assert np.abs(sgn * np.diag(D)[na:] - deb).max() < 1e-13
        lp, Cp1, Cp2, lh, Ch1, Ch2 = oracle.nto_ab(z, oa, va, ob, vb)
        X = z[:nvv].reshape(va, vb)
        Y = z[nvv:].reshape(oa, ob)
        assert np.abs(Cp1 @ np.diag(np.sqrt(lp)) @ Cp2.T - X).max() < 1e-12
        assert np.abs(Ch1 @ np.diag(np.sqrt(lh)) @ Ch2.T - Y).max() < 1e-12
        assert abs(lp.sum() - lh.sum() - sgn) < 1e-12
        assert np.all(np.diff(lp) <= 1e-15) and np.all(np.diff(lh) <= 1e-15)


@pytest.mark.parametrize("nv", [3, 5])
def test_two_electrons_are_exact(nv):
    """No occupied orbitals: ppRPA roots equal the two-electron determinant CI."""
    eps, L = small(0, nv, 6, 40 + nv, nbasis_extra=2)
    roots = []
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, 0, L, mult)
        assert noo == 0
        roots.append(oracle.solve_full(M, nvv, noo)["omega_pp"])
    ci = oracle.two_electron_ci(eps, L)
    assert np.allclose(np.sort(np.concatenate(roots)), ci, atol=1e-12)


def test_two_orbital_closed_form():
    """One occupied (i) and one virtual (a) orbital, one auxiliary function.

    Singlet pairs (a,a) and (i,i): A = 2 eps_a + L_aa^2, B = L_ai^2,
    C = -2 eps_i + L_ii^2, and det(W M - omega) = 0 gives
    omega = ((A - C) +- sqrt((A + C)^2 - 4 B^2)) / 2 (worked by hand).
    """
    eps = np.array([-0.7, 0.4])
    L = np.array([[[0.3, 0.2], [0.2, 0.5]]])
    A = 2 * 0.4 + 0.5 ** 2
    B = 0.2 ** 2
    C = -2 * (-0.7) + 0.3 ** 2
    disc = np.sqrt((A + C) ** 2 - 4 * B ** 2)
    M, nvv, noo = oracle.build_matrix(eps, 1, L, 1)
    assert np.allclose(M, [[A, B], [B, C]], atol=1e-15)
    sol = oracle.solve_full(M, nvv, noo)
    assert abs(sol["omega_pp"][0] - ((A - C) + disc) / 2) < 1e-14
    assert abs(sol["omega_hh"][0] - ((A - C) - disc) / 2) < 1e-14
    M3, nvv3, noo3 = oracle.build_matrix(eps, 1, L, 3)
    assert M3.shape == (0, 0)


@pytest.mark.parametrize("mult", [1, 3])
def test_b_zero_limit(mult):
    """With L^P_ai = 0 the coupling B vanishes: omega(N+2) = eig(A),
    omega(N-2) = -eig(C) (because C Y = -omega Y), and E_c = 0."""
    eps, L = small(3, 5, 8, 5)
    L = L.copy()
    L[:, :3, 3:] = 0.0
    L[:, 3:, :3] = 0.0
    M, nvv, noo = oracle.build_matrix(eps, 3, L, mult)
    assert np.abs(M[:nvv, nvv:]).max() == 0.0
    sol = oracle.solve_full(M, nvv, noo)
    assert np.allclose(sol["omega_pp"], np.linalg.eigvalsh(M[:nvv, :nvv]), atol=1e-12)
    assert np.allclose(sol["omega_hh"], np.sort(-np.linalg.eigvalsh(M[nvv:, nvv:])), atol=1e-12)
    e1, e2 = oracle.correlation_energy(M, nvv, noo, sol)
    assert abs(e1) < 1e-12 and abs(e2) < 1e-12


@pytest.mark.parametrize("mult", [1, 3])
def test_root_counting_normalisation_and_ec_identity(mult):
    """nvv roots of norm +1 and noo of norm -1 (Eq. xy_norm); the two forms
    of Eq. correlation_energy agree."""
    eps, L = small(4, 7, 10, 21)
    M, nvv, noo = oracle.build_matrix(eps, 4, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    assert not sol["unstable"]
    assert len(sol["omega_pp"]) == nvv and len(sol["omega_hh"]) == noo
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    assert np.allclose(np.einsum("ik,i,ik->k", sol["z_pp"], w, sol["z_pp"]), 1.0, atol=1e-12)
    assert np.allclose(np.einsum("ik,i,ik->k", sol["z_hh"], w, sol["z_hh"]), -1.0, atol=1e-12)
    assert sol["omega_pp"].min() > sol["omega_hh"].max()
    e1, e2 = oracle.correlation_energy(M, nvv, noo, sol)
    assert abs(e1 - e2) < 1e-12


@pytest.mark.parametrize("mult", [1, 3])
def test_shifted_reduction_equals_dense_eig(mult):
    eps, L = small(3, 6, 9, 8)
    M, nvv, noo = oracle.build_matrix(eps, 3, L, mult)
    a = oracle.solve_full(M, nvv, noo)
    mu = 0.5 * (a["omega_pp"][0] + a["omega_hh"][-1])
    b = oracle.solve_full_shifted(M, nvv, noo, mu)
    assert np.allclose(a["omega_pp"], b["omega_pp"], atol=1e-12)
    assert np.allclose(a["omega_hh"], b["omega_hh"], atol=1e-12)
    # non-degenerate roots: same eigenvectors under the phase convention
    assert np.allclose(a["z_pp"][:, :3], b["z_pp"][:, :3], atol=1e-9)


@pytest.mark.parametrize("mult", [1, 3])
def test_uniform_orbital_shift(mult):
    """eps_p -> eps_p + delta for all p moves every root by 2 delta; E_c fixed."""
    eps, L = small(3, 5, 6, 9)
    d = 0.37
    M0, nvv, noo = oracle.build_matrix(eps, 3, L, mult)
    M1, _, _ = oracle.build_matrix(eps + d, 3, L, mult)
    s0 = oracle.solve_full(M0, nvv, noo)
    s1 = oracle.solve_full(M1, nvv, noo)
    assert np.allclose(s1["omega_pp"], s0["omega_pp"] + 2 * d, atol=1e-12)
    assert np.allclose(s1["omega_hh"], s0["omega_hh"] + 2 * d, atol=1e-12)
    assert abs(oracle.correlation_energy(M1, nvv, noo, s1)[0]
               - oracle.correlation_energy(M0, nvv, noo, s0)[0]) < 1e-12


def test_second_order_limit_is_mp2():
    """Scaling L -> lam L, E_c(lam) / E2(lam) -> 1 (ladder CCD is exact to
    second order), with E_c = E_c(singlet) + 3 E_c(triplet)."""
    eps, L = small(3, 5, 8, 33)
    ratios = []
    for lam in (0.1, 0.01):
        ec = 0.0
        for mult, g in ((1, 1.0), (3, 3.0)):
            M, nvv, noo = oracle.build_matrix(eps, 3, lam * L, mult)
            ec += g * oracle.correlation_energy(M, nvv, noo)[0]
        e2 = oracle.mp2_pair_energy(eps, 3, lam * L)
        ratios.append(ec / e2)
    assert abs(ratios[0] - 1) < 2e-2
    assert abs(ratios[1] - 1) < 2e-4
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1) / 50


@pytest.mark.parametrize("mult", [1, 3])
def test_gradient_matches_finite_differences(mult):
    """Hellmann-Feynman d omega / d eps and d omega / d L against central FD (h = 1e-4)."""
    no, nv = 2, 4
    eps, L = small(no, nv, 5, 17)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    for key, r in (("pp", 0), ("pp", 2), ("hh", -1)):
        z = sol["z_" + key][:, r]
        de, dL = oracle.grad_omega(eps, no, L, mult, z)
        h = 1e-4

        def root(e, LL):
            Mx, a, b = oracle.build_matrix(e, no, LL, mult)
            sx = oracle.solve_full(Mx, a, b)
            return sx["omega_" + key][r]

        for p in (0, 3, 5):
            ep, em = eps.copy(), eps.copy()
            ep[p] += h
            em[p] -= h
            fd = (root(ep, L) - root(em, L)) / (2 * h)
            assert abs(fd - de[p]) < 1e-5 * max(1.0, abs(de[p]))
        rng = np.random.default_rng(3)
        for _ in range(3):
            D = rng.standard_normal(L.shape)
            D = D + D.transpose(0, 2, 1)
            D /= np.linalg.norm(D)
            fd = (root(eps, L + h * D) - root(eps, L - h * D)) / (2 * h)
            an = float(np.sum(dL * D))
            assert abs(fd - an) < 1e-5 * max(1.0, abs(an))


@pytest.mark.parametrize("mult", [1, 3])
def test_ao_side_adjoint_matches_finite_differences(mult):
    """d omega / d (P|mu nu) and d omega / d C through the AO->MO transform, against central
    differences of a root of the whole chain (AO integrals, C -> L -> M -> omega)."""
    spec = synth.SystemSpec("t", 10, 3, 7, 2, 5, 41)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 2, 5)
    eps = s["eps"][orb]

    def root(ao, C, key, r):
        L = oracle.ao_to_mo(ao, C, orb)
        M, nvv, noo = oracle.build_matrix(eps, 2, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        return sol["omega_" + key][r], sol["z_" + key][:, r], L

    rng = np.random.default_rng(5)
    h = 1e-5
    for key, r in (("pp", 0), ("hh", -1)):
        _, z, L = root(s["ao3c"], s["C"], key, r)
        _, dL = oracle.grad_omega(eps, 2, L, mult, z)
        d_ao, d_c = oracle.grad_ao(s["ao3c"], s["C"], orb, dL)
        for _ in range(2):
            E = rng.standard_normal(s["ao3c"].shape)
            E = (E + E.transpose(0, 2, 1)) / np.linalg.norm(E)
            fd = (root(s["ao3c"] + h * E, s["C"], key, r)[0] - root(s["ao3c"] - h * E, s["C"], key, r)[0]) / (2 * h)
            an = float(np.sum(d_ao * E))
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
            D = rng.standard_normal(s["C"].shape)
            D /= np.linalg.norm(D)
            fd = (root(s["ao3c"], s["C"] + h * D, key, r)[0] - root(s["ao3c"], s["C"] - h * D, key, r)[0]) / (2 * h)
            an = float(np.sum(d_c * D))
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
        # columns of C outside the active space do not enter L
        inactive = np.setdiff1d(np.arange(spec.nmo), orb)
        assert np.all(d_c[:, inactive] == 0.0)


def test_ao_side_adjoint_of_a_general_functional():
    """For f = sum_P,p,q G^P_pq L^P_pq with a non-symmetric G, f is linear in the AO tensor and
    quadratic in C, so central differences are exact up to rounding; a transposed operand or
    a dropped term in the adjoint changes the result."""
    spec = synth.SystemSpec("t", 9, 3, 5, 2, 4, 43)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 2, 4)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((5, 6, 6))

    def f(ao, C):
        return float(np.sum(G * oracle.ao_to_mo(ao, C, orb)))

    d_ao, d_c = oracle.grad_ao(s["ao3c"], s["C"], orb, G)
    h = 1e-3
    for _ in range(3):
        E = rng.standard_normal(s["ao3c"].shape)  # entries independent, as in the adjoint
        fd = (f(s["ao3c"] + h * E, s["C"]) - f(s["ao3c"] - h * E, s["C"])) / (2 * h)
        assert abs(fd - float(np.sum(d_ao * E))) < 1e-9 * max(1.0, abs(fd))
        D = rng.standard_normal(s["C"].shape)
        fd = (f(s["ao3c"], s["C"] + h * D) - f(s["ao3c"], s["C"] - h * D)) / (2 * h)
        assert abs(fd - float(np.sum(d_c * D))) < 1e-9 * max(1.0, abs(fd))


@pytest.mark.parametrize("mult", [1, 3])
def test_eps_gradient_is_density_diagonal_and_trace_rule(mult):
    """d omega / d eps_p = s D^2e_pp and Tr D^2e = +-2 (Sec. Density Matrix),
    so sum_p d omega / d eps_p = 2."""
    no, nv = 3, 5
    eps, L = small(no, nv, 6, 29)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    for key, s in (("pp", 1.0), ("hh", -1.0)):
        z = sol["z_" + key][:, 0]
        de, _ = oracle.grad_omega(eps, no, L, mult, z)
        D = oracle.two_e_density_diag(z, no, nv, mult)
        assert np.allclose(de, s * D, atol=1e-12)
        assert abs(D.sum() - 2 * s) < 1e-12
        assert abs(de.sum() - 2.0) < 1e-12


@pytest.mark.parametrize("mult", [1, 3])
def test_nto_weight_sum_rule(mult):
    no, nv = 3, 6
    eps, L = small(no, nv, 7, 5)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    for key, s in (("pp", 1.0), ("hh", -1.0)):
        lp, lh = oracle.nto_weights(sol["z_" + key][:, 1], no, nv, mult)
        assert abs(lp.sum() - lh.sum() - s) < 1e-12


@pytest.mark.parametrize("mult", [1, 3])
def test_density_matrix_and_ntos(mult):
    """Sec. Density Matrix and Eqs. nto_pp / nto_hh: the full D^2e has the epsilon gradient on
    its diagonal (d omega / d eps_p = s D^2e_pp), trace +-2, zero occupied-virtual blocks and a
    positive semidefinite virtual block; the NTOs rebuild X and Y, have orthonormal columns,
    obey the weight sum rule, and give back the density blocks."""
    no, nv = 3, 6
    eps, L = small(no, nv, 7, 6)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    for key, s in (("pp", 1.0), ("hh", -1.0)):
        z = sol["z_" + key][:, 1]
        D = oracle.two_e_density(z, no, nv, mult)
        de, _ = oracle.grad_omega(eps, no, L, mult, z)
        assert np.allclose(np.diag(D) * s, de, atol=1e-12)
        assert abs(np.trace(D) - 2 * s) < 1e-12
        assert np.all(D[:no, no:] == 0) and np.allclose(D, D.T, atol=1e-14)
        assert np.linalg.eigvalsh(D[no:, no:]).min() > -1e-12
        assert np.linalg.eigvalsh(-D[:no, :no]).min() > -1e-12
        lp, cp1, cp2, lh, ch1, ch2 = oracle.nto(z, no, nv, mult)
        X = np.zeros((nv, nv))
        Y = np.zeros((no, no))
        for I, (p, q) in enumerate(oracle.pair_list(nv, mult)):
            X[p, q] = z[I]
        for I, (p, q) in enumerate(oracle.pair_list(no, mult)):
            Y[p, q] = z[nvv + I]
        assert np.allclose(cp1 @ np.diag(np.sqrt(lp)) @ cp2.T, X, atol=1e-12)
        assert np.allclose(ch1 @ np.diag(np.sqrt(lh)) @ ch2.T, Y, atol=1e-12)
        for C in (cp1, cp2, ch1, ch2):
            assert np.allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-12)
        assert np.all(np.diff(lp) <= 1e-15) and np.all(np.diff(lh) <= 1e-15)
        assert abs(lp.sum() - lh.sum() - s) < 1e-12
        assert np.allclose(cp1 @ np.diag(lp) @ cp1.T + cp2 @ np.diag(lp) @ cp2.T, D[no:, no:], atol=1e-12)
        assert np.allclose(-(ch1 @ np.diag(lh) @ ch1.T + ch2 @ np.diag(lh) @ ch2.T), D[:no, :no], atol=1e-12)


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv", [(1, 2), (3, 7), (5, 9)])
def test_ri_sigma_equals_explicit_matrix(mult, no, nv):
    eps, L = small(no, nv, 11, 3 * no + nv)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    Z = synth.random_trial_vectors(nvv + noo, 4, 99)
    assert np.allclose(oracle.ri_sigma(eps, no, L, mult, Z), Z @ M.T, atol=1e-13)
    rows = [0, nvv - 1, nvv + noo - 1]
    got = oracle.ri_sigma_rows(eps, no, L, mult, Z[1], rows)
    assert np.allclose(got, (M @ Z[1])[rows], atol=1e-13)


@pytest.mark.parametrize("mult", [1, 3])
def test_davidson_matches_full_on_small_workload(mult):
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    full = oracle.solve_full(M, nvv, noo)
    res = oracle.davidson(lambda Z: oracle.ri_sigma(eps, spec.nocc_act, L, mult, Z),
                          np.diag(M), nvv, noo, 10, tol=1e-8)
    assert res["converged"]
    assert np.allclose(res["omega"], full["omega_pp"][:10], atol=1e-10)


def test_small_workload_matches_golden():
    """Regression of the small full-diagonalisation workload against values
    written by tests/golden/make_golden.py (oracle only)."""
    with open(os.path.join(GOLDEN, "c0_roots.json")) as f:
        g = json.load(f)
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        ref = g[str(mult)]
        assert np.allclose(sol["omega_pp"], ref["omega_pp"], atol=1e-10)
        assert np.allclose(sol["omega_hh"], ref["omega_hh"], atol=1e-10)
        assert abs(oracle.correlation_energy(M, nvv, noo, sol)[0] - ref["ec"]) < 1e-10


def test_ao_to_mo_rows_matches_full_transform():
    spec = synth.SystemSpec("t", 14, 4, 9, 3, 7, 4)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 3, 7)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    for rows in ([0, 4, 9], list(range(10))):
        got = oracle.ao_to_mo_rows(s["ao3c"], s["C"], orb, rows)
        assert np.allclose(got, L[:, rows, :].transpose(1, 0, 2), atol=1e-14)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, 3, L, 1)
    z = synth.random_trial_vectors(nvv + noo, 1, 2)[0]
    rows_cache = {}

    def Lrow(p):
        if p not in rows_cache:
            rows_cache[p] = oracle.ao_to_mo_rows(s["ao3c"], s["C"], orb, [p])[0]
        return rows_cache[p]

    got = oracle.ri_sigma_rows(eps, 3, None, 1, z, [0, 5, nvv + 1], Lrow=Lrow)
    assert np.allclose(got, (M @ z)[[0, 5, nvv + 1]], atol=1e-13)


def test_synthetic_generator_becomes_unstable_as_nv_over_sqrt_naux_grows():
    """The random part of <ab|cd> has variance ~0.0225/naux, so the A block spreads like
    a semicircle of radius ~0.3 nv / sqrt(naux).  The small full-diagonalisation workload
    (nv / sqrt(naux) = 1.8) is stable; analogues at 6.9 and 11.5 have complex roots, and at
    11.5 the lowest real addition roots lie below every complex pair."""
    def spectrum(no, nv, naux, nb, seed, mult=1):
        spec = synth.SystemSpec("u", nb, no + 2, naux, no, nv, seed)
        s = synth.make_system(spec)
        orb = oracle.active_orbitals(s["occ"], no, nv)
        L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
        M, nvv, noo = oracle.build_matrix(s["eps"][orb], no, L, mult)
        w = np.concatenate([np.ones(nvv), -np.ones(noo)])
        vals, vecs = np.linalg.eig(w[:, None] * M)
        nrm = np.einsum("ik,i,ik->k", vecs.real, w, vecs.real)
        return vals, nrm

    c0 = synth.CONFIGS["c0"]
    s = synth.make_system(c0)
    orb = oracle.active_orbitals(s["occ"], c0.nocc_act, c0.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    M, nvv, noo = oracle.build_matrix(s["eps"][orb], c0.nocc_act, L, 1)
    assert not oracle.solve_full(M, nvv, noo)["unstable"]
    vals, _ = spectrum(4, 24, 12, 32, 1)  # nv / sqrt(naux) = 6.9
    assert np.abs(vals.imag).max() > 1e-3
    vals, nrm = spectrum(4, 40, 12, 50, 1)  # nv / sqrt(naux) = 11.5
    real = np.abs(vals.imag) < 1e-9
    assert (~real).sum() >= 4
    pp_real = np.sort(vals.real[real & (nrm > 0)])
    assert pp_real[0] < vals.real[~real].min()
