"""The clustered Rayleigh-Ritz kernel (subspaces up to 72, eight CTAs of a thread-block
cluster sharing the FP64 products through distributed shared memory) against the one-CTA
kernel and against the oracle.

Full diagonalisation (Sec. ppRPA Equation: the whole pencil M z = omega W z, Eq. xy_norm
splitting the roots by the sign of their norm) runs the Rayleigh-Ritz kernel on the whole
matrix, so problems with N <= 72 pairs reach the clustered kernel with every size parity;
PPRPA_RR_CLUSTER=0 sends the same call to the one-CTA kernel.  With PPRPA_RR_PROF=1 each
kernel prints its phase clocks under its own tag, which shows which one ran.
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


def make(no, nv, naux, seed):
    spec = synth.SystemSpec("t", no + nv + 3, no + 2, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    return spec, s, L, s["eps"][orb]


def full_solve(pp, spec, s, mult, nvv):
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(spec.nocc_act, spec.nvir_act)
        c.set_ao(s["C"], s["ao3c"])
        return c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL, want_ec=True)


# (nocc, nvir, naux, seed): singlet / triplet pair counts N = 7 / 3, 42 / 31, 58 / 46, 65 / 51
CASES = [(1, 3, 6, 21), (3, 8, 30, 22), (2, 10, 40, 23), (4, 10, 40, 24)]


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("no,nv,naux,seed", CASES)
def test_full_diagonalisation_on_the_cluster(pp, monkeypatch, capfd, mult, no, nv, naux, seed):
    spec, s, L, eps = make(no, nv, naux, seed)
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    ref = oracle.solve_full(M, nvv, noo)
    if len(ref["omega_pp"]) != nvv or len(ref["omega_hh"]) != noo:
        pytest.skip("the pencil has complex roots")  # the full path needs a definite shift
    ec_ref = oracle.correlation_energy(M, nvv, noo, ref)[0]
    monkeypatch.setenv("PPRPA_RR_PROF", "1")
    out = {}
    for cl in ("1", "0"):
        monkeypatch.setenv("PPRPA_RR_CLUSTER", cl)
        capfd.readouterr()
        out[cl] = full_solve(pp, spec, s, mult, nvv)
        text = capfd.readouterr().out
        # the clustered kernel takes every N <= 72 unless it is switched off
        assert ("[rr-cl]" in text) == (cl == "1"), text[-400:]
    for r in out.values():
        assert np.abs(r["omega"] - ref["omega_pp"]).max() <= 1e-8
        assert abs(r["ec"] - ec_ref) <= 1e-8
        Z = np.hstack([r["X"], r["Y"]]).T
        w = np.concatenate([np.ones(nvv), -np.ones(noo)])
        assert np.allclose(np.einsum("ik,i,ik->k", Z, w, Z), 1.0, atol=1e-10)
    # the two kernels reach the same FP64 eigenpairs (up to rounding)
    assert np.abs(out["1"]["omega"] - out["0"]["omega"]).max() <= 1e-10


@pytest.mark.parametrize("mult", [1, 3])
def test_davidson_small_workload_on_the_cluster(pp, monkeypatch, mult):
    """The c0 lowest-10 FP64 Davidson solve (subspaces 20..72, odd sizes among them) with the
    clustered and with the one-CTA Rayleigh-Ritz kernel, both against the oracle."""
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    M, nvv, noo = oracle.build_matrix(s["eps"][orb], spec.nocc_act, L, mult)
    ref = oracle.solve_full(M, nvv, noo)["omega_pp"][:10]
    got = {}
    for cl in ("1", "0"):
        monkeypatch.setenv("PPRPA_RR_CLUSTER", cl)
        with pp.Context(0) as c:
            c.set_orbitals(s["occ"], s["eps"])
            c.set_active(spec.nocc_act, spec.nvir_act)
            c.set_ao(s["C"], s["ao3c"])
            r = c.solve(mult=mult, nroots=10, precision=pp.PREC_FP64, conv_tol=1e-7)
        assert r["info"]["converged"] == 1
        assert np.abs(r["omega"] - ref).max() <= 1e-8
        got[cl] = r["omega"]
    assert np.abs(got["1"] - got["0"]).max() <= 1e-9
