"""The pins are not vacuous: plausible mistakes planted in the oracle (on the CPU, in copies
made here) make them fail, while the oracle as written passes.

Each planted mistake is the effect of one wrong line in the oracle's arithmetic: a dropped
singlet normalisation, a wrong sign of the occupied-pair energies, a missing coupling block,
a gradient that ignores the metric or the root's norm sign, a density with a wrong sign."""
import numpy as np
import pytest

import oracle
from test_oracle_pins import small, unrestricted_small

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---- restricted matrix: the spin-orbital brute-force pin -----------------------------------

def _energy_diag(eps, no, mult):
    n = len(eps)
    vv = [(no + a, no + b) for (a, b) in oracle.pair_list(n - no, mult)]
    oo = oracle.pair_list(no, mult)
    return np.array([eps[p] + eps[q] for p, q in vv] + [-(eps[i] + eps[j]) for i, j in oo]), len(vv)


def _spin_orbital_pin_holds(build):
    """Singlet + 3 x triplet roots of `build` equal the spin-orbital roots."""
    eps, L = small(2, 3, 7, 13)
    Mso, a, b = oracle.spinorb_matrix(eps, 2, L)
    so = oracle.solve_full(Mso, a, b)
    pp, hh = [], []
    for mult in (1, 3):
        M, nvv, noo = build(eps, 2, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        reps = 1 if mult == 1 else 3
        pp += [sol["omega_pp"]] * reps
        hh += [sol["omega_hh"]] * reps
    pp, hh = np.sort(np.concatenate(pp)), np.sort(np.concatenate(hh))
    if pp.shape != so["omega_pp"].shape or hh.shape != so["omega_hh"].shape:
        return False
    return bool(np.allclose(np.sort(so["omega_pp"]), pp, atol=1e-9)
                and np.allclose(np.sort(so["omega_hh"]), hh, atol=1e-9))


def _dropped_singlet_normalisation(eps, no, L, mult):
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    if mult != 1:
        return M, nvv, noo
    E, _ = _energy_diag(eps, no, mult)
    n = len(eps)
    pairs = [(no + a, no + b) for (a, b) in oracle.pair_list(n - no, 1)] + oracle.pair_list(no, 1)
    S = np.diag([np.sqrt(2.0) if p == q else 1.0 for p, q in pairs])
    V = M - np.diag(E)
    return np.diag(E) + S @ V @ S, nvv, noo


def _wrong_occupied_energy_sign(eps, no, L, mult):
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    E, _ = _energy_diag(eps, no, mult)
    M = M.copy()
    idx = np.arange(nvv, nvv + noo)
    M[idx, idx] -= 2.0 * E[idx]  # -(eps_i + eps_j) became +(eps_i + eps_j)
    return M, nvv, noo


def _missing_b_block(eps, no, L, mult):
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    M = M.copy()
    M[:nvv, nvv:] = 0.0
    M[nvv:, :nvv] = 0.0
    return M, nvv, noo


def test_spin_orbital_pin_accepts_the_oracle():
    assert _spin_orbital_pin_holds(oracle.build_matrix)


@pytest.mark.parametrize("mutant", [_dropped_singlet_normalisation, _wrong_occupied_energy_sign,
                                    _missing_b_block])
def test_spin_orbital_pin_rejects_planted_mistakes(mutant):
    assert not _spin_orbital_pin_holds(mutant)


# ---- alpha-beta gradient: the finite-difference and uniform-shift pins ---------------------

def _ab_gradient_pins_hold(grad):
    ea, oa, La, eb, ob, Lb = unrestricted_small()
    M, nvv, noo = oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb)
    sol = oracle.solve_full(M, nvv, noo)
    h = 1e-4
    rng = np.random.default_rng(9)
    for key, r in (("pp", 0), ("hh", -1)):
        z = sol["z_" + key][:, r]
        dea, deb, dLa, dLb = grad(ea, oa, La, eb, ob, Lb, z)
        if abs(dea.sum() - 1.0) > 1e-10 or abs(deb.sum() - 1.0) > 1e-10:
            return False

        def root(xa, Xa, xb, Xb):
            return oracle.solve_full(*oracle.build_matrix_ab(xa, oa, Xa, xb, ob, Xb))["omega_" + key][r]

        for p in (0, 3):
            ep, em = ea.copy(), ea.copy()
            ep[p] += h
            em[p] -= h
            if abs((root(ep, La, eb, Lb) - root(em, La, eb, Lb)) / (2 * h) - dea[p]) > 1e-5 * max(1.0, abs(dea[p])):
                return False
        D = rng.standard_normal(Lb.shape)
        D = (D + D.transpose(0, 2, 1)) / np.linalg.norm(D + D.transpose(0, 2, 1))
        fd = (root(ea, La, eb, Lb + h * D) - root(ea, La, eb, Lb - h * D)) / (2 * h)
        an = float(np.sum(dLb * D))
        if abs(fd - an) > 1e-5 * max(1.0, abs(an)):
            return False
    return True


def _gradient_without_metric_sign(ea, oa, La, eb, ob, Lb, z):
    dea, deb, dLa, dLb = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, z)
    X, Y = z[: (len(ea) - oa) * (len(eb) - ob)], z[(len(ea) - oa) * (len(eb) - ob):]
    s = np.sign(X @ X - Y @ Y)
    corr = np.zeros(len(ea))
    corr[:oa] = 2.0 * s * (Y.reshape(oa, ob) ** 2).sum(axis=1)
    # the occupied pairs contributed +s z^2 instead of -s z^2 to the alpha energies
    return dea + corr, deb, dLa, dLb


def _gradient_without_root_sign(ea, oa, La, eb, ob, Lb, z):
    dea, deb, dLa, dLb = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, z)
    nvv = (len(ea) - oa) * (len(eb) - ob)
    s = np.sign(z[:nvv] @ z[:nvv] - z[nvv:] @ z[nvv:])
    return s * dea, s * deb, s * dLa, s * dLb  # gamma = z z^T without the factor s


def test_ab_gradient_pins_accept_the_oracle():
    assert _ab_gradient_pins_hold(oracle.grad_omega_ab)


@pytest.mark.parametrize("mutant", [_gradient_without_metric_sign, _gradient_without_root_sign])
def test_ab_gradient_pins_reject_planted_mistakes(mutant):
    assert not _ab_gradient_pins_hold(mutant)


# ---- alpha-beta density: the trace and gradient-diagonal pins ------------------------------

def _ab_density_pins_hold(density):
    ea, oa, La, eb, ob, Lb = unrestricted_small(87)
    va, vb = len(ea) - oa, len(eb) - ob
    M, nvv, noo = oracle.build_matrix_ab(ea, oa, La, eb, ob, Lb)
    sol = oracle.solve_full(M, nvv, noo)
    na = len(ea)
    for key, r, sgn in (("pp", 0, 1.0), ("hh", -1, -1.0)):
        z = sol["z_" + key][:, r]
        D = density(z, oa, va, ob, vb)
        if abs(np.trace(D[:na, :na]) - sgn) > 1e-12 or abs(np.trace(D[na:, na:]) - sgn) > 1e-12:
            return False
        dea, deb, _, _ = oracle.grad_omega_ab(ea, oa, La, eb, ob, Lb, z)
        if np.abs(sgn * np.diag(D) - np.concatenate([dea, deb])).max() > 1e-13:
            return False
    return True


def _density_with_positive_occupied_blocks(z, oa, va, ob, vb):
    D = oracle.two_e_density_ab(z, oa, va, ob, vb)
    na = oa + va
    D = D.copy()
    D[:oa, :oa] *= -1.0
    D[na:na + ob, na:na + ob] *= -1.0
    return D


def _density_with_spins_summed(z, oa, va, ob, vb):
    # the restricted form X X^T + X^T X on the alpha block only, beta block left empty
    D = oracle.two_e_density_ab(z, oa, va, ob, vb)
    na = oa + va
    D = D.copy()
    D[:na, :na] *= 2.0
    D[na:, na:] = 0.0
    return D


def test_ab_density_pins_accept_the_oracle():
    assert _ab_density_pins_hold(oracle.two_e_density_ab)


@pytest.mark.parametrize("mutant", [_density_with_positive_occupied_blocks, _density_with_spins_summed])
def test_ab_density_pins_reject_planted_mistakes(mutant):
    assert not _ab_density_pins_hold(mutant)


# ---- restricted RI sigma, correlation energy and gradient ----------------------------------

def _ri_pin_holds(ri):
    eps, L = small(2, 4, 6, 31)
    rng = np.random.default_rng(4)
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, 2, L, mult)
        Z = rng.standard_normal((3, nvv + noo))
        if not np.allclose(ri(eps, 2, L, mult, Z), Z @ M.T, atol=1e-12):
            return False
    return True


def _ri_sigma_without_sqrt2(eps, no, L, mult, Z):
    # Zt_cc = X_cc instead of sqrt(2) X_cc on the singlet diagonal pairs
    if mult != 1:
        return oracle.ri_sigma(eps, no, L, mult, Z)
    n = len(eps)
    pairs = [(no + a, no + b) for (a, b) in oracle.pair_list(n - no, 1)] + oracle.pair_list(no, 1)
    d = np.array([1.0 / np.sqrt(2.0) if p == q else 1.0 for p, q in pairs])
    S = oracle.ri_sigma(eps, no, L, mult, Z * d)
    E, _ = _energy_diag(eps, no, 1)
    return S + (Z - Z * d) * E  # the orbital-energy term keeps the unscaled vector


def _ec_identity_holds(ce):
    eps, L = small(2, 3, 6, 33)
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, 2, L, mult)
        e1, e2 = ce(M, nvv, noo)
        if abs(e1 - e2) > 1e-10:
            return False
    return True


def _ec_with_wrong_trace_sign(M, nvv, noo, sol=None):
    e1, e2 = oracle.correlation_energy(M, nvv, noo, sol)
    return e1, e2 + 2.0 * float(np.trace(M[nvv:, nvv:]))  # -sum(omega) + Tr C


def _restricted_gradient_pin_holds(grad):
    eps, L = small(2, 4, 5, 17)
    h = 1e-4
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, 2, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        for key, r in (("pp", 0), ("hh", -1)):
            de, _ = grad(eps, 2, L, mult, sol["z_" + key][:, r])
            for p in (0, 1, 4):
                ep, em = eps.copy(), eps.copy()
                ep[p] += h
                em[p] -= h
                fd = (oracle.solve_full(*oracle.build_matrix(ep, 2, L, mult))["omega_" + key][r]
                      - oracle.solve_full(*oracle.build_matrix(em, 2, L, mult))["omega_" + key][r]) / (2 * h)
                if abs(fd - de[p]) > 1e-5 * max(1.0, abs(de[p])):
                    return False
    return True


def _restricted_gradient_without_metric_sign(eps, no, L, mult, z):
    de, dL = oracle.grad_omega(eps, no, L, mult, z)
    n = len(eps)
    nvv = len(oracle.pair_list(n - no, mult))
    s = np.sign(z[:nvv] @ z[:nvv] - z[nvv:] @ z[nvv:])
    corr = np.zeros(n)
    for I, (i, j) in enumerate(oracle.pair_list(no, mult)):
        corr[i] += 2.0 * s * z[nvv + I] ** 2  # +s z^2 instead of -s z^2 on occupied pairs
        corr[j] += 2.0 * s * z[nvv + I] ** 2
    return de + corr, dL


def test_restricted_pins_accept_the_oracle():
    assert _ri_pin_holds(oracle.ri_sigma)
    assert _ec_identity_holds(oracle.correlation_energy)
    assert _restricted_gradient_pin_holds(oracle.grad_omega)


def test_restricted_pins_reject_planted_mistakes():
    assert not _ri_pin_holds(_ri_sigma_without_sqrt2)
    assert not _ec_identity_holds(_ec_with_wrong_trace_sign)
    assert not _restricted_gradient_pin_holds(_restricted_gradient_without_metric_sign)
