"""GPU path against the FP64 oracle, element by element, through the C ABI.

Tolerances:
* FP64 kernels (AO->MO, diagonal, explicit matrix, FP64 sigma): 1e-11
  relative to the largest entry; only the summation order differs.
* Eigenvalues, FP64 (full diagonalisation and Davidson): 1e-8 Ha.
* BF16 sigma: operands rounded to 8 significant bits, so a few 1e-3 of
  the two-electron magnitude; BF16x3 split sigma: a few 1e-6.
* Mixed-precision Davidson (BF16, then BF16x3 split): |d omega| <= 1e-5 Ha.
"""
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


def make(no, nv, naux, seed, extra=4):
    nb = no + nv + extra
    spec = synth.SystemSpec("t", nb, no + 2, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    return spec, s, L, s["eps"][orb]


def gpu_ctx(pp, spec, s):
    c = pp.Context(0)
    c.set_orbitals(s["occ"], s["eps"])
    c.set_active(spec.nocc_act, spec.nvir_act)
    c.set_ao(s["C"], s["ao3c"])
    return c


CASES = [(5, 20, 120, 1), (1, 7, 9, 2), (3, 33, 50, 3), (13, 70, 97, 4)]

# BF16 keeps 8 significant bits: unit roundoff u = 2^-8.  Each product of the sandwich
# carries four roundings (L^P twice, Zt, and T = L^P Zt rounded to BF16 before the second
# product); FP32 accumulation adds nothing comparable.  The roundings are incoherent over
# the long sums, and a CPU emulation of the same arithmetic (torch bfloat16 casts of L, Zt
# and T, FP32/FP64 sums) gives max|err| / max|two-electron part| = 0.0022-0.0042 and a
# relative Frobenius error of 0.0027-0.0034 on these cases and on an nv = 600 orbital space,
# i.e. about u.  The bounds allow 2u (max) and 1.5u (Frobenius).
BF16_U = 2.0 ** -8


def check_bf16(err, two_e):
    assert np.abs(err).max() <= 2.0 * BF16_U * np.abs(two_e).max()
    assert np.linalg.norm(err) <= 1.5 * BF16_U * np.linalg.norm(two_e)


@pytest.mark.parametrize("no,nv,naux,seed", CASES)
def test_ao_to_mo(pp, no, nv, naux, seed):
    spec, s, L, eps = make(no, nv, naux, seed)
    with gpu_ctx(pp, spec, s) as c:
        got = c.get_L()
    assert np.abs(got - L).max() <= 1e-12 * np.abs(L).max()


def test_set_mo_matches_set_ao(pp):
    spec, s, L, eps = make(4, 11, 30, 5)
    Lfull = oracle.ao_to_mo(s["ao3c"], s["C"], np.arange(spec.nmo))
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(4, 11)
        c.set_mo(np.ascontiguousarray(Lfull))
        got = c.get_L()
    assert np.abs(got - L).max() <= 1e-13


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv,naux,seed", CASES[:3])
def test_diag_and_explicit_matrix(pp, mult, no, nv, naux, seed):
    spec, s, L, eps = make(no, nv, naux, seed)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    with gpu_ctx(pp, spec, s) as c:
        D = c.diag(mult)
        Mg = c.build_matrix(mult)
    scale = np.abs(M).max()
    assert np.abs(D - np.diag(M)).max() <= 1e-12 * scale
    assert np.abs(Mg - M).max() <= 1e-12 * scale


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv,naux,seed", CASES)
def test_sigma_all_precisions(pp, mult, no, nv, naux, seed):
    spec, s, L, eps = make(no, nv, naux, seed)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    Z = synth.random_trial_vectors(nvv + noo, 5, 7 + seed)
    ref = Z @ M.T
    two_e = Z @ (M - np.diag(np.diag(M))).T
    scale = np.abs(two_e).max()
    with gpu_ctx(pp, spec, s) as c:
        s64 = c.sigma(mult, Z, pp.PREC_FP64)
        s16 = c.sigma(mult, Z, pp.PREC_BF16)
        s48 = c.sigma(mult, Z, pp.PREC_BF16_SPLIT)
    assert np.abs(s64 - ref).max() <= 1e-11 * np.abs(ref).max()
    check_bf16(s16 - ref, two_e)
    assert np.abs(s48 - ref).max() <= 2e-5 * scale


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv,naux,seed", CASES)
def test_sigma_fp8(pp, mult, no, nv, naux, seed):
    """E4M3 first stage (per-P and per-vector scales), BF16 second stage.

    E4M3 keeps 3 mantissa bits (unit roundoff 2^-4); with both stage-1 operands rounded the
    two-electron part carries a relative error of about 4 % in the Frobenius norm (a CPU
    emulation with torch's float8_e4m3fn cast gives 0.033-0.038 on these cases, max/scale
    up to 0.041).  The bounds leave 1.5-2x headroom for accumulation order.
    """
    spec, s, L, eps = make(no, nv, naux, seed)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    Z = synth.random_trial_vectors(nvv + noo, 5, 7 + seed)
    ref = Z @ M.T
    two_e = Z @ (M - np.diag(np.diag(M))).T
    with gpu_ctx(pp, spec, s) as c:
        s8 = c.sigma(mult, Z, pp.PREC_FP8)
        s8b = c.sigma(mult, Z, pp.PREC_FP8)
    err = s8 - ref
    assert np.array_equal(s8, s8b) or np.abs(s8 - s8b).max() <= 1e-6 * np.abs(two_e).max()
    assert np.linalg.norm(err) <= 0.06 * np.linalg.norm(two_e)
    assert np.abs(err).max() <= 0.08 * np.abs(two_e).max()


@pytest.mark.parametrize("k", [1, 3, 17])
def test_sigma_batch_sizes_and_device_pointers(pp, k):
    import torch

    spec, s, L, eps = make(6, 40, 64, 8)
    M, nvv, noo = oracle.build_matrix(eps, 6, L, 1)
    Z = synth.random_trial_vectors(nvv + noo, k, 3)
    with gpu_ctx(pp, spec, s) as c:
        zd = torch.as_tensor(Z, device="cuda")
        out = c.sigma(1, zd, pp.PREC_BF16_SPLIT)
        got = out.cpu().numpy()
    two_e = Z @ (M - np.diag(np.diag(M))).T
    assert np.abs(got - Z @ M.T).max() <= 2e-5 * np.abs(two_e).max()


@pytest.mark.parametrize("mult", [1, 3])
def test_full_diagonalisation_small_workload(pp, mult):
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    ref = oracle.solve_full(M, nvv, noo)
    ec_ref = oracle.correlation_energy(M, nvv, noo, ref)[0]
    with gpu_ctx(pp, spec, s) as c:
        res = c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)
    assert np.abs(res["omega"] - ref["omega_pp"]).max() <= 1e-8
    assert abs(res["ec"] - ec_ref) <= 1e-8
    Z = np.hstack([res["X"], res["Y"]]).T
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    assert np.allclose(np.einsum("ik,i,ik->k", Z, w, Z), 1.0, atol=1e-10)
    # eigenvectors of the non-degenerate lowest roots, under the phase convention
    gap = np.diff(ref["omega_pp"][:6])
    for r in range(5):
        if gap[r] > 1e-4 and (r == 0 or gap[r - 1] > 1e-4):
            assert np.abs(Z[:, r] - ref["z_pp"][:, r]).max() < 1e-7


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("prec,tol", [("PREC_FP64", 1e-8), ("PREC_BF16", 1e-5), ("PREC_FP8", 1e-5)])
def test_davidson_small_workload(pp, mult, prec, tol):
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    ref = oracle.solve_full(M, nvv, noo)["omega_pp"][:10]
    with gpu_ctx(pp, spec, s) as c:
        res = c.solve(mult=mult, nroots=10, precision=getattr(pp, prec),
                      conv_tol=1e-7 if prec == "PREC_FP64" else 1e-5)
    assert res["info"]["converged"] == 1
    assert np.abs(res["omega"] - ref).max() <= tol


@pytest.mark.parametrize("mult", [1, 3])
def test_gradient_matches_oracle(pp, mult):
    spec, s, L, eps = make(3, 9, 14, 12)
    M, nvv, noo = oracle.build_matrix(eps, 3, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    with gpu_ctx(pp, spec, s) as c:
        c.solve(mult=mult, nroots=3, method=pp.METHOD_FULL)
        for r in range(3):
            dL, de = c.grad(r)
            de_ref, dL_ref = oracle.grad_omega(eps, 3, L, mult, sol["z_pp"][:, r])
            assert np.abs(de - de_ref).max() <= 1e-9
            assert np.abs(dL - dL_ref).max() <= 1e-9 * max(1.0, np.abs(dL_ref).max())


def test_error_paths(pp):
    spec, s, L, eps = make(2, 5, 8, 1)
    with pp.Context(0) as c:
        with pytest.raises(pp.PprpaError) as e:
            c.solve(mult=1, nroots=2)
        assert e.value.code == -7  # no integrals yet
        c.set_orbitals(s["occ"], s["eps"])
        with pytest.raises(pp.PprpaError):
            c.set_active(100, 2)
        c.set_active(2, 5)
        c.set_ao(s["C"], s["ao3c"])
        with pytest.raises(pp.PprpaError):
            c.solve(mult=2, nroots=1)
        with pytest.raises(pp.PprpaError):
            c.solve(mult=1, nroots=1000)
        with pytest.raises(pp.PprpaError):
            c.grad(0)
        r = c.solve(mult=1, nroots=2, max_iter=1, conv_tol=1e-14, raise_noconv=False)
        assert r["rc"] == -4


UNSTABLE = [(4, 40, 12, 50, 1), (4, 48, 18, 56, 2)]


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv,naux,nb,seed", UNSTABLE)
@pytest.mark.parametrize("prec,tol", [("PREC_FP64", 1e-8), ("PREC_BF16", 1e-5)])
def test_davidson_unstable_problem(pp, mult, no, nv, naux, nb, seed, prec, tol):
    """Synthetic problems whose removal roots have become complex: no shift makes
    the pencil definite, the general subspace solver takes over, and the lowest
    real roots of positive norm (here below every complex pair) are found."""
    spec = synth.SystemSpec("u", nb, no + 2, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    ref = oracle.solve_full(M, nvv, noo, imag_tol=1e-9)
    assert ref["unstable"]
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    vals, vecs = np.linalg.eig(w[:, None] * M)
    real = np.abs(vals.imag) < 1e-9
    nrm = np.einsum("ik,i,ik->k", vecs.real, w, vecs.real)
    pp_real = np.sort(vals.real[real & (nrm > 0)])
    # targets: up to 5 lowest real addition roots lying below every complex pair
    nr = int(min(5, np.count_nonzero(pp_real < vals.real[~real].min())))
    assert nr >= 3
    lowest = pp_real[:nr]
    with gpu_ctx(pp, spec, s) as c:
        res = c.solve(mult=mult, nroots=nr, precision=getattr(pp, prec),
                      conv_tol=1e-7 if prec == "PREC_FP64" else 1e-5)
        with pytest.raises(pp.PprpaError) as e:
            c.solve(mult=mult, nroots=nr, method=pp.METHOD_FULL)
        # no definite shift (unstable) or, beyond 1024 pairs, outside the full-diagonalisation range
        assert e.value.code == (-5 if nvv + noo <= 1024 else -1)
    assert res["info"]["converged"] == 1
    assert res["info"]["max_imag"] == 0.0
    assert np.abs(res["omega"] - lowest).max() <= tol
    Z = np.hstack([res["X"], res["Y"]])
    resid = Z @ M.T - res["omega"][:, None] * (w[None, :] * Z)
    assert np.linalg.norm(resid, axis=1).max() <= (1e-6 if prec == "PREC_FP64" else 1e-4)


@pytest.mark.parametrize("mult", [1, 3])
def test_correlation_energy_gradient(pp, mult):
    """dE_c/dL and dE_c/d eps (all addition roots of a full solve, minus d Tr A) against
    the oracle's central difference of E_c (Eq. correlation_energy), h = 1e-4."""
    spec, s, L, eps = make(3, 8, 12, 13)
    no = 3
    with gpu_ctx(pp, spec, s) as c:
        _, _, nvv, noo = c.dims(mult)
        c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)
        dL, de = c.grad_ec()

    def ec(e, LL):
        M, a, b = oracle.build_matrix(e, no, LL, mult)
        return oracle.correlation_energy(M, a, b)[0]

    h = 1e-4
    for p in (0, 2, 5, 9):
        ep, em = eps.copy(), eps.copy()
        ep[p] += h
        em[p] -= h
        fd = (ec(ep, L) - ec(em, L)) / (2 * h)
        assert abs(fd - de[p]) < 1e-6 * max(1.0, abs(fd))
    rng = np.random.default_rng(4)
    for _ in range(3):
        D = rng.standard_normal(L.shape)
        D = D + D.transpose(0, 2, 1)
        D /= np.linalg.norm(D)
        fd = (ec(eps, L + h * D) - ec(eps, L - h * D)) / (2 * h)
        assert abs(fd - float(np.sum(dL * D))) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("env", [{"PPRPA_PAIR1": "1", "PPRPA_PAIR2": "1"}, {"PPRPA_TSTORE": "1"},
                                 {"PPRPA_TSTORE": "0", "PPRPA_CLUSTER": "1", "PPRPA_CLUSTER2": "1"}])
@pytest.mark.parametrize("mult", [1, 3])
def test_sigma_alternative_tensor_core_forms(pp, monkeypatch, env, mult):
    """The non-default launch forms of the sandwich give the same sigma: tcgen05 CTA pairs
    (M = 256 tiles, each CTA holding half of B), bulk tensor stores of T, and single-CTA
    launches without clusters."""
    for k_, v in env.items():
        monkeypatch.setenv(k_, v)
    spec, s, L, eps = make(13, 70, 97, 4)
    M, nvv, noo = oracle.build_matrix(eps, 13, L, mult)
    Z = synth.random_trial_vectors(nvv + noo, 5, 9)
    ref = Z @ M.T
    two_e = Z @ (M - np.diag(np.diag(M))).T
    scale = np.abs(two_e).max()
    with gpu_ctx(pp, spec, s) as c:
        s16 = c.sigma(mult, Z, pp.PREC_BF16)
        s48 = c.sigma(mult, Z, pp.PREC_BF16_SPLIT)
        s8 = c.sigma(mult, Z, pp.PREC_FP8)
    check_bf16(s16 - ref, two_e)
    assert np.abs(s48 - ref).max() <= 2e-5 * scale
    assert np.linalg.norm(s8 - ref) <= 0.06 * np.linalg.norm(two_e)
