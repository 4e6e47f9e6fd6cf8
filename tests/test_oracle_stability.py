"""Pins of the oracle's stability tools (oracle/stability.py) on small problems.

The explicit matrix built row by row from the density-fitted integrals must equal the
element-by-element build_matrix; the lowest eigenvalue of M - mu W must equal the dense
symmetric one (and be positive exactly for a definite shift); the shift-invert roots near a
point must be the dense eigenvalues of W M nearest it, with the norm sign of Eq. xy_norm.
"""
import numpy as np
import pytest

import oracle
import synth


def _case(no, nv, naux, seed, mult):
    spec = synth.SystemSpec("t", no + nv + 3, no + 1, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    return eps, L


@pytest.mark.parametrize("mult", [1, 3])
def test_rows_equal_the_element_by_element_matrix(mult):
    eps, L = _case(4, 13, 21, 51, mult)
    M, nvv, noo = oracle.build_matrix(eps, 4, L, mult)
    M2, a, b = oracle.explicit_matrix_ri(eps, 4, L, mult)
    assert (a, b) == (nvv, noo)
    assert np.abs(M - M2).max() <= 1e-13 * np.abs(M).max()


@pytest.mark.parametrize("mult", [1, 3])
def test_shifted_lambda_min_is_the_dense_value(mult):
    eps, L = _case(4, 13, 21, 52, mult)
    M, nvv, noo = oracle.build_matrix(eps, 4, L, mult)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    sol = oracle.solve_full(M, nvv, noo)
    for mu in (sol["omega_pp"][0] - 0.3, 0.5 * (sol["omega_pp"][0] + sol["omega_hh"][-1]), 0.0):
        ref = np.linalg.eigvalsh(M - mu * np.diag(w))[0]
        assert abs(oracle.shifted_lambda_min(M, nvv, noo, mu) - ref) <= 1e-9
    # a shift between the highest removal and the lowest addition root is definite
    mid = 0.5 * (sol["omega_pp"][0] + sol["omega_hh"][-1])
    if sol["max_imag"] == 0.0 and sol["omega_hh"][-1] < sol["omega_pp"][0]:
        assert oracle.shifted_lambda_min(M, nvv, noo, mid) > 0.0


def test_roots_near_a_point_are_the_dense_roots():
    # an unstable problem (complex pairs): nv large against sqrt(naux)
    eps, L = _case(6, 30, 12, 53, 3)
    M, nvv, noo = oracle.build_matrix(eps, 6, L, 3)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    vals, vecs = np.linalg.eig(w[:, None] * M)
    sigma = -0.3
    k = 12
    near = vals[np.argsort(np.abs(vals - sigma))[:k]]
    got, metric = oracle.roots_near(M, nvv, noo, sigma, k=k)
    # compared up to conjugation: at the cut-off k may hold one member of a conjugate pair
    def key(v):
        return np.sort_complex(v.real + 1j * np.abs(v.imag))

    assert np.abs(key(got) - key(near)).max() <= 1e-8
    # norm signs: real roots carry +-1 after normalisation by z^H z only when X or Y
    # dominates; complex roots have z^H W z = 0 exactly
    for v, m in zip(got, metric):
        if abs(v.imag) > 1e-6:
            assert abs(m) <= 1e-8


@pytest.mark.parametrize("mult", [1, 3])
def test_block_shift_window_bounds_the_dense_blocks(mult):
    eps, L = _case(4, 13, 21, 54, mult)
    M, nvv, noo = oracle.build_matrix(eps, 4, L, mult)
    lam_a = np.linalg.eigvalsh(M[:nvv, :nvv])[0]
    lam_c = np.linalg.eigvalsh(M[nvv:, nvv:])[0]
    r = oracle.block_shift_window(eps, 4, L, mult, steps=nvv)
    assert abs(r["lambda_min_C"] - lam_c) <= 1e-12
    # a full Lanczos run reaches lambda_min(A); fewer steps bound it from above
    assert abs(r["theta_A"] - lam_a) <= 1e-9
    r5 = oracle.block_shift_window(eps, 4, L, mult, steps=5)
    assert r5["theta_A"] >= lam_a - 1e-12
    # proven indefinite means no shift makes M - mu W positive definite (dense check on a grid)
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    if r["proven_indefinite"]:
        for mu in np.linspace(-3, 3, 121):
            assert np.linalg.eigvalsh(M - mu * np.diag(w))[0] <= 1e-12


def test_block_shift_window_proves_an_unstable_case():
    eps, L = _case(6, 30, 12, 53, 3)
    r = oracle.block_shift_window(eps, 6, L, 3, steps=60)
    assert r["proven_indefinite"]


@pytest.mark.parametrize("mult", [1, 3])
def test_classified_spectrum_of_a_stable_problem_is_solve_full(mult):
    eps, L = _case(4, 13, 21, 55, mult)
    M, nvv, noo = oracle.build_matrix(eps, 4, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    if sol["unstable"]:
        pytest.skip("this draw is unstable")
    add, rem, c = oracle.classified_spectrum(M, nvv, noo)
    assert len(c) == 0 and len(add) == nvv and len(rem) == noo
    assert np.abs(add - sol["omega_pp"]).max() <= 1e-10
    assert np.abs(rem - sol["omega_hh"]).max() <= 1e-10


def test_classified_spectrum_counts_conjugate_pairs():
    eps, L = _case(6, 30, 12, 53, 3)
    M, nvv, noo = oracle.build_matrix(eps, 6, L, 3)
    add, rem, c = oracle.classified_spectrum(M, nvv, noo)
    assert len(c) > 0 and len(c) % 2 == 0
    assert len(add) + len(rem) + len(c) == nvv + noo
    # conjugate pairs: the imaginary parts cancel in pairs
    assert abs(np.sum(c.imag)) <= 1e-8 * np.abs(c.imag).max()
    # every complex pair removes one addition and one removal root from the count
    assert len(add) == nvv - len(c) // 2 and len(rem) == noo - len(c) // 2
