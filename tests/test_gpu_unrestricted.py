"""Spin-unrestricted ppRPA through the C ABI: the alpha-beta subspace (pprpa_set_beta,
mult = AB) and the three-subspace correlation energy, against the oracle
(oracle.build_matrix_ab, pinned by its restricted limit and by the spin-orbital matrix of
a spin-unrestricted reference)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as m

    return m


def unrestricted_system(nbasis, nocc, naux, oa, va, ob, vb, seed):
    """alpha: the synthetic orbitals; beta: rotated orbitals with shifted energies."""
    spec = synth.SystemSpec("t", nbasis, nocc, naux, oa, va, seed)
    s = synth.make_system(spec)
    rng = np.random.default_rng(seed + 1)
    Q, _ = np.linalg.qr(rng.standard_normal((spec.nmo, spec.nmo)))
    Cb = s["C"] @ (np.eye(spec.nmo) + 0.15 * (Q - np.eye(spec.nmo)))
    Cb, _ = np.linalg.qr(Cb)
    eb = np.sort(s["eps"] + 0.03 * rng.standard_normal(spec.nmo))
    orb_a = oracle.active_orbitals(s["occ"], oa, va)
    La = oracle.ao_to_mo(s["ao3c"], s["C"], orb_a)
    nocc_b = nocc - 1  # one fewer beta electron
    orb_b = np.concatenate([np.arange(nocc_b - ob, nocc_b), np.arange(nocc_b, nocc_b + vb)])
    Lb = oracle.ao_to_mo(s["ao3c"], Cb, orb_b)
    return spec, s, La, s["eps"][orb_a], Lb, eb[orb_b]


def ab_ctx(pp, spec, s, oa, va, ob, Lb, eb):
    c = pp.Context(0)
    c.set_orbitals(s["occ"], s["eps"])
    c.set_active(oa, va)
    c.set_ao(s["C"], s["ao3c"])
    c.set_beta(ob, len(eb) - ob, np.ascontiguousarray(eb), np.ascontiguousarray(Lb))
    return c


def test_alpha_beta_matrix_sigma_and_roots(pp):
    spec, s, La, ea, Lb, eb = unrestricted_system(16, 4, 14, 3, 6, 2, 7, 91)
    M, nvv, noo = oracle.build_matrix_ab(ea, 3, La, eb, 2, Lb)
    ref = oracle.solve_full(M, nvv, noo)
    assert ref["max_imag"] == 0.0
    ec_pp, ec_hh = oracle.correlation_energy(M, nvv, noo, ref)
    Z = synth.random_trial_vectors(nvv + noo, 4, 5)
    with ab_ctx(pp, spec, s, 3, 6, 2, Lb, eb) as c:
        n, naux, a_nvv, a_noo = c.dims(pp.AB)
        assert (a_nvv, a_noo) == (nvv, noo)
        assert np.abs(c.build_matrix(pp.AB) - M).max() <= 1e-12 * np.abs(M).max()
        assert np.abs(c.diag(pp.AB) - np.diag(M)).max() <= 1e-12 * np.abs(M).max()
        sig = c.sigma(pp.AB, Z, pp.PREC_FP64)
        full = c.solve(mult=pp.AB, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)
        hh = c.solve(mult=pp.AB, nroots=noo, method=pp.METHOD_FULL, want_ec=True, channel=pp.CHANNEL_HH)
        dav = c.solve(mult=pp.AB, nroots=4, conv_tol=1e-8)
        with pytest.raises(pp.PprpaError):
            c.sigma(pp.AB, Z, pp.PREC_BF16)
        with pytest.raises(pp.PprpaError):
            c.grad(0)
    assert np.abs(sig - Z @ M.T).max() <= 1e-11 * np.abs(Z @ M.T).max()
    assert np.abs(full["omega"] - ref["omega_pp"]).max() <= 1e-8
    assert np.abs(hh["omega"] - ref["omega_hh"][::-1]).max() <= 1e-8
    assert abs(full["ec"] - ec_pp) <= 1e-8 and abs(hh["ec"] - ec_hh) <= 1e-8
    assert dav["info"]["converged"] == 1
    assert np.abs(dav["omega"] - ref["omega_pp"][:4]).max() <= 1e-8


def test_restricted_limit_on_the_gpu(pp):
    """beta = alpha: the alpha-beta roots are the singlet roots plus the triplet roots."""
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 3, 8)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    e = s["eps"][orb]
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(3, 8)
        c.set_ao(s["C"], s["ao3c"])
        c.set_beta(3, 8, np.ascontiguousarray(e), np.ascontiguousarray(L))
        _, _, nvv, noo = c.dims(pp.AB)
        ab = c.solve(mult=pp.AB, nroots=nvv, method=pp.METHOD_FULL)
        _, _, n1, _ = c.dims(1)
        _, _, n3, _ = c.dims(3)
        s1 = c.solve(mult=1, nroots=n1, method=pp.METHOD_FULL)
        s3 = c.solve(mult=3, nroots=n3, method=pp.METHOD_FULL)
    assert np.abs(ab["omega"] - np.sort(np.concatenate([s1["omega"], s3["omega"]]))).max() <= 1e-8


def test_three_subspace_correlation_energy(pp):
    """E_c of a spin-unrestricted reference = alpha-alpha + beta-beta + alpha-beta, each from
    its own FULL solve on the GPU, against the spin-orbital matrix of the oracle."""
    spec, s, La, ea, Lb, eb = unrestricted_system(12, 3, 9, 2, 5, 1, 6, 93)
    Mso, nvv, noo = oracle.spinorb_matrix_unrestricted(ea, 2, La, eb, 1, Lb)
    so = oracle.solve_full(Mso, nvv, noo)
    ec_ref = oracle.correlation_energy(Mso, nvv, noo, so)[0]
    ec = 0.0
    with ab_ctx(pp, spec, s, 2, 5, 1, Lb, eb) as c:
        _, _, nvv_ab, _ = c.dims(pp.AB)
        ec += c.solve(mult=pp.AB, nroots=nvv_ab, method=pp.METHOD_FULL, want_ec=True)["ec"]
        _, _, nvv_a, _ = c.dims(3)
        ec += c.solve(mult=3, nroots=nvv_a, method=pp.METHOD_FULL, want_ec=True)["ec"]
    occ_b = np.zeros(len(eb))
    occ_b[:1] = 1.0
    with pp.Context(0) as cb:  # beta-beta: the triplet problem of the beta orbitals
        cb.set_orbitals(occ_b, np.ascontiguousarray(eb))
        cb.set_mo(np.ascontiguousarray(Lb))
        _, _, nvv_b, _ = cb.dims(3)
        ec += cb.solve(mult=3, nroots=nvv_b, method=pp.METHOD_FULL, want_ec=True)["ec"]
    assert abs(ec - ec_ref) <= 1e-8


def test_alpha_beta_gradient(pp):
    """pprpa_grad_ab of addition and removal roots against oracle.grad_omega_ab (pinned by
    finite differences and the uniform-shift rule)."""
    spec, s, La, ea, Lb, eb = unrestricted_system(16, 4, 14, 3, 6, 2, 7, 91)
    M, nvv, noo = oracle.build_matrix_ab(ea, 3, La, eb, 2, Lb)
    ref = oracle.solve_full(M, nvv, noo)
    cases = []
    with ab_ctx(pp, spec, s, 3, 6, 2, Lb, eb) as c:
        c.solve(mult=pp.AB, nroots=nvv, method=pp.METHOD_FULL)
        for r in (0, 3):
            cases.append((c.grad_ab(r), ref["z_pp"][:, r], ref["omega_pp"], r))
        c.solve(mult=pp.AB, nroots=noo, method=pp.METHOD_FULL, channel=pp.CHANNEL_HH)
        cases.append((c.grad_ab(0), ref["z_hh"][:, -1], ref["omega_hh"], len(ref["omega_hh"]) - 1))
        with pytest.raises(pp.PprpaError):
            c.grad_ab(noo)
    for (dLa, dLb, dea, deb), z, omegas, r in cases:
        gaps = np.abs(np.delete(omegas, r) - omegas[r])
        assert gaps.min() > 1e-4  # a non-degenerate root: z and its gradient are unique
        rea, reb, ra, rb = oracle.grad_omega_ab(ea, 3, La, eb, 2, Lb, z)
        for got, want in ((dLa, ra), (dLb, rb), (dea, rea), (deb, reb)):
            assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max())
        assert abs(dea.sum() - 1.0) <= 1e-10 and abs(deb.sum() - 1.0) <= 1e-10


def test_alpha_beta_analysis(pp):
    """pprpa_analyze of alpha-beta roots (addition and removal) against the pinned oracle:
    spin-resolved density blocks and the NTOs of the rectangular X and Y."""
    spec, s, La, ea, Lb, eb = unrestricted_system(16, 4, 14, 3, 6, 2, 7, 91)
    M, nvv, noo = oracle.build_matrix_ab(ea, 3, La, eb, 2, Lb)
    ref = oracle.solve_full(M, nvv, noo)
    got = []
    with ab_ctx(pp, spec, s, 3, 6, 2, Lb, eb) as c:
        c.solve(mult=pp.AB, nroots=nvv, method=pp.METHOD_FULL)
        got.append((c.analyze(1, ab=True), ref["z_pp"][:, 1]))
        c.solve(mult=pp.AB, nroots=noo, method=pp.METHOD_FULL, channel=pp.CHANNEL_HH)
        got.append((c.analyze(0, ab=True), ref["z_hh"][:, -1]))
    for a, z in got:
        D = oracle.two_e_density_ab(z, 3, 6, 2, 7)
        assert a["D2e"].shape == D.shape
        assert np.abs(a["D2e"] - D).max() <= 1e-12 * max(1.0, np.abs(D).max())
        lp, Cp1, Cp2, lh, Ch1, Ch2 = oracle.nto_ab(z, 3, 6, 2, 7)
        for lam_g, lam_r, C1g, C1r, C2g, C2r in ((a["lam_p"], lp, a["Cp1"], Cp1, a["Cp2"], Cp2),
                                                 (a["lam_h"], lh, a["Ch1"], Ch1, a["Ch2"], Ch2)):
            assert np.abs(lam_g - lam_r).max() <= 1e-11
            big = lam_r > 1e-8 * lam_r.max()
            gaps = np.abs(lam_r[:, None] - lam_r[None, :]) + np.eye(len(lam_r))
            uniq = big & (gaps.min(axis=1) > 1e-6)
            assert np.abs(C1g[:, uniq] - C1r[:, uniq]).max() <= 1e-8
            assert np.abs(C2g[:, uniq] - C2r[:, uniq]).max() <= 1e-8


def test_new_beta_space_invalidates_the_alpha_beta_solve(pp):
    """A new beta space changes the alpha-beta pair table: the stored solve is dropped and its
    gradient and analysis are refused (no read of vectors of the old pair space)."""
    spec, s, La, ea, Lb, eb = unrestricted_system(16, 4, 14, 3, 6, 2, 7, 91)
    with ab_ctx(pp, spec, s, 3, 6, 2, Lb, eb) as c:
        c.solve(mult=pp.AB, nroots=4, method=pp.METHOD_FULL)
        c.grad_ab(0)
        c.set_beta(3, 6, np.ascontiguousarray(eb), np.ascontiguousarray(Lb))  # 3 occupied now
        with pytest.raises(pp.PprpaError) as e:
            c.grad_ab(0)
        assert e.value.code == -7
        with pytest.raises(pp.PprpaError):
            c.analyze(0)
