"""The hh channel: the highest two-electron removal roots (N-2) through the C ABI.

The removal roots are the eigenpairs of M z = omega W z with z^T W z = -1 (Sec. "ppRPA
Equation", lower sign of Eq. xy_norm).  The library finds them as the lowest positive-norm
roots of the pencil (M, -W); the oracle takes them from a dense non-symmetric
diagonalisation (oracle.solve_full, "omega_hh"), pinned by the spin-orbital brute force.
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


def small_workload():
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    return spec, s, L, eps


def ctx(pp, spec, s):
    c = pp.Context(0)
    c.set_orbitals(s["occ"], s["eps"])
    c.set_active(spec.nocc_act, spec.nvir_act)
    c.set_ao(s["C"], s["ao3c"])
    return c


@pytest.mark.parametrize("mult", [1, 3])
def test_full_hh_every_root_and_correlation_energy(pp, mult):
    spec, s, L, eps = small_workload()
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    ref = oracle.solve_full(M, nvv, noo)
    ec_pp_ref, ec_hh_ref = oracle.correlation_energy(M, nvv, noo, ref)
    want = ref["omega_hh"][::-1]  # highest first
    with ctx(pp, spec, s) as c:
        hh = c.solve(mult=mult, nroots=noo, method=pp.METHOD_FULL, want_ec=True,
                     channel=pp.CHANNEL_HH)
        ppc = c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)
    assert np.abs(hh["omega"] - want).max() <= 1e-8
    # Eq. correlation_energy from either channel
    assert abs(hh["ec"] - ec_hh_ref) <= 1e-8
    assert abs(hh["ec"] - ppc["ec"]) <= 1e-8
    assert abs(ec_pp_ref - ec_hh_ref) <= 1e-9
    Z = np.hstack([hh["X"], hh["Y"]]).T
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    assert np.allclose(np.einsum("ik,i,ik->k", Z, w, Z), -1.0, atol=1e-10)
    zref = ref["z_hh"][:, ::-1]
    gap = np.abs(np.diff(want))
    for r in range(min(5, noo - 1)):
        if gap[r] > 1e-4 and (r == 0 or gap[r - 1] > 1e-4):
            assert np.abs(Z[:, r] - zref[:, r]).max() < 1e-7


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("prec,tol", [("PREC_FP64", 1e-8), ("PREC_BF16", 1e-5)])
def test_davidson_hh(pp, mult, prec, tol):
    spec, s, L, eps = small_workload()
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    want = oracle.solve_full(M, nvv, noo)["omega_hh"][::-1][:4]
    with ctx(pp, spec, s) as c:
        res = c.solve(mult=mult, nroots=4, precision=getattr(pp, prec), channel=pp.CHANNEL_HH,
                      conv_tol=1e-7 if prec == "PREC_FP64" else 1e-5)
    assert res["info"]["converged"] == 1
    assert np.abs(res["omega"] - want).max() <= tol
    Z = np.hstack([res["X"], res["Y"]])
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    assert np.allclose(np.einsum("ki,i,ki->k", Z, w, Z), -1.0, atol=1e-8)
    # residual of the returned pairs against the explicit matrix
    resid = Z @ M.T - res["omega"][:, None] * (Z * w[None, :])
    assert np.linalg.norm(resid, axis=1).max() <= (1e-6 if prec == "PREC_FP64" else 1e-4)


@pytest.mark.parametrize("mult", [1, 3])
def test_gradient_of_removal_roots(pp, mult):
    """d omega / d L and d omega / d eps of removal roots carry s = z^T W z = -1."""
    no, nv, naux = 3, 9, 14
    spec = synth.SystemSpec("t", no + nv + 4, no + 1, naux, no, nv, 12)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        c.solve(mult=mult, nroots=2, method=pp.METHOD_FULL, channel=pp.CHANNEL_HH)
        for r in range(2):
            dL, de = c.grad(r)
            z = sol["z_hh"][:, noo - 1 - r]
            de_ref, dL_ref = oracle.grad_omega(eps, no, L, mult, z)
            assert np.abs(de - de_ref).max() <= 1e-9
            assert np.abs(dL - dL_ref).max() <= 1e-9 * max(1.0, np.abs(dL_ref).max())


def test_hh_argument_checks(pp):
    spec, s, L, eps = small_workload()
    with ctx(pp, spec, s) as c:
        _, _, nvv, noo = c.dims(1)
        with pytest.raises(pp.PprpaError):
            c.solve(mult=1, nroots=noo + 1, channel=pp.CHANNEL_HH)
        with pytest.raises(pp.PprpaError):
            c.solve(mult=1, nroots=2, channel=7)
        c.solve(mult=1, nroots=noo - 1, method=pp.METHOD_FULL, channel=pp.CHANNEL_HH)
        with pytest.raises(pp.PprpaError):
            c.grad_ec()  # the correlation-energy gradient needs every root of the channel
