"""Fractional occupations (Sec. ppRPA for Fractional Charge Systems) through the C ABI:
weighted integrals from AO and MO inputs, roots of both channels, E_c and the AO adjoint,
against the oracle (oracle.fractional_integrals, pinned by the element-by-element
spin-orbital matrix of the paper's fractional A, B and C)."""
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


def fractional_system(nbasis, nfull, frac, naux, no, nv, seed):
    spec = synth.SystemSpec("t", nbasis, nfull + 1, naux, no, nv, seed)
    s = synth.make_system(spec)
    occ = np.zeros(spec.nmo)
    occ[:nfull] = 1.0
    occ[nfull] = frac
    return spec, s, occ


@pytest.mark.parametrize("frac", [0.35, 0.8])
@pytest.mark.parametrize("mult", [1, 3])
def test_fractional_full_solve_and_integrals(pp, frac, mult):
    spec, s, occ = fractional_system(14, 3, frac, 12, 3, 6, 63)  # stable, separated roots
    L, e = oracle.fractional_integrals(s["ao3c"], s["C"], occ, s["eps"], 3, 6)
    M, nvv, noo = oracle.build_matrix(e, 3, L, mult)
    ref = oracle.solve_full(M, nvv, noo)
    ec_pp, ec_hh = oracle.correlation_energy(M, nvv, noo, ref)
    Lfull = oracle.ao_to_mo(s["ao3c"], s["C"], np.arange(spec.nmo))
    with pp.Context(0) as c:
        c.set_orbitals(occ, s["eps"])
        c.set_active(3, 6)
        c.set_ao(s["C"], s["ao3c"])
        assert np.abs(c.get_L() - L).max() <= 1e-13
        res = c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)
        hh = c.solve(mult=mult, nroots=noo, method=pp.METHOD_FULL, want_ec=True, channel=pp.CHANNEL_HH)
        c.set_mo(np.ascontiguousarray(Lfull))
        assert np.abs(c.get_L() - L).max() <= 1e-13
    assert np.abs(res["omega"] - ref["omega_pp"]).max() <= 1e-8
    assert np.abs(hh["omega"] - ref["omega_hh"][::-1]).max() <= 1e-8
    assert abs(res["ec"] - ec_pp) <= 1e-8 and abs(hh["ec"] - ec_hh) <= 1e-8


@pytest.mark.parametrize("prec,tol", [("PREC_FP64", 1e-8), ("PREC_BF16", 1e-5)])
def test_fractional_davidson(pp, prec, tol):
    # n = 0.7: at n = 1/2 the lowest addition and the highest removal root of the fractional
    # orbital coincide at 2 eps (a defective pencil), which no shift separates
    spec, s, occ = fractional_system(40, 4, 0.7, 120, 5, 20, 12515001)
    L, e = oracle.fractional_integrals(s["ao3c"], s["C"], occ, s["eps"], 5, 20)
    M, nvv, noo = oracle.build_matrix(e, 5, L, 1)
    want = oracle.solve_full(M, nvv, noo)["omega_pp"][:6]
    with pp.Context(0) as c:
        c.set_orbitals(occ, s["eps"])
        c.set_active(5, 20)
        c.set_ao(s["C"], s["ao3c"])
        res = c.solve(mult=1, nroots=6, precision=getattr(pp, prec),
                      conv_tol=1e-7 if prec == "PREC_FP64" else 1e-5)
    assert res["info"]["converged"] == 1
    assert np.abs(res["omega"] - want).max() <= tol


def test_fractional_ao_adjoint(pp):
    spec, s, occ = fractional_system(12, 2, 0.6, 9, 2, 5, 62)
    orb, w = oracle.fractional_slots(occ, 2, 5)
    with pp.Context(0) as c:
        c.set_orbitals(occ, s["eps"])
        c.set_active(2, 5)
        c.set_ao(s["C"], s["ao3c"])
        c.solve(mult=1, nroots=2, method=pp.METHOD_FULL)
        dL, _ = c.grad(0)
        d_ao, d_c = c.grad_ao(s["C"], dL, s["ao3c"])
    ref_ao, ref_c = oracle.grad_ao(s["ao3c"], s["C"], orb, dL * w[None, :, None] * w[None, None, :])
    assert np.abs(d_ao - ref_ao).max() <= 1e-12 * max(1.0, np.abs(ref_ao).max())
    assert np.abs(d_c - ref_c).max() <= 1e-12 * max(1.0, np.abs(ref_c).max())


def test_occupation_checks(pp):
    spec, s, occ = fractional_system(10, 2, 0.5, 6, 2, 3, 63)
    with pp.Context(0) as c:
        bad = occ.copy()
        bad[5] = 0.3  # increases after zeros
        with pytest.raises(pp.PprpaError):
            c.set_orbitals(bad, s["eps"])
        bad = occ.copy()
        bad[0] = 1.5
        with pytest.raises(pp.PprpaError):
            c.set_orbitals(bad, s["eps"])
        c.set_orbitals(occ, s["eps"])
        n, _, nvv, noo = c.dims(1)
        assert n == 3 + spec.nmo - 2  # the fractional orbital is a hole and a particle slot
