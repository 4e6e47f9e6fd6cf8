"""pprpa_analyze: two-electron density matrix and natural transition orbitals of a root,
against the oracle (oracle.two_e_density, oracle.nto) on the same eigenvector."""
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


def check_against_oracle(res, a, no, nv, mult, s):
    z = np.concatenate([res["X"][1], res["Y"][1]])
    D = oracle.two_e_density(z, no, nv, mult)
    assert np.abs(a["D2e"] - D).max() <= 1e-12 * max(1.0, np.abs(D).max())
    assert abs(np.trace(a["D2e"]) - 2 * s) <= 1e-10
    lp, cp1, cp2, lh, ch1, ch2 = oracle.nto(z, no, nv, mult)
    assert np.abs(a["lam_p"] - lp).max() <= 1e-11
    assert np.abs(a["lam_h"] - lh).max() <= 1e-11
    assert abs(a["lam_p"].sum() - a["lam_h"].sum() - s) <= 1e-10
    for lam, c1, c2, r1, r2 in ((lp, a["Cp1"], a["Cp2"], cp1, cp2), (lh, a["Ch1"], a["Ch2"], ch1, ch2)):
        m = len(lam)
        if m == 0:
            continue
        # rebuild the triangular matrix from the NTOs (zero-weight columns drop out)
        T = c1 @ np.diag(np.sqrt(lam)) @ c2.T
        Tref = r1 @ np.diag(np.sqrt(lam)) @ r2.T
        assert np.abs(T - Tref).max() <= 1e-9
        assert np.allclose(c1.T @ c1, np.eye(m), atol=1e-9)
        # vectors of well-separated, non-negligible weights agree column by column
        for k in range(min(m, 6)):
            gaps = np.abs(lam - lam[k])
            gaps[k] = np.inf
            if lam[k] > 1e-6 * lam[0] and gaps.min() > 1e-6 * lam[0]:
                assert np.abs(c1[:, k] - r1[:, k]).max() <= 1e-7
                assert np.abs(c2[:, k] - r2[:, k]).max() <= 1e-7


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("channel,s", [("CHANNEL_PP", 1.0), ("CHANNEL_HH", -1.0)])
def test_analysis_small_workload(pp, mult, channel, s):
    spec = synth.CONFIGS["c0"]
    st = synth.make_system(spec)
    no, nv = spec.nocc_act, spec.nvir_act
    with pp.Context(0) as c:
        c.set_orbitals(st["occ"], st["eps"])
        c.set_active(no, nv)
        c.set_ao(st["C"], st["ao3c"])
        res = c.solve(mult=mult, nroots=3, method=pp.METHOD_FULL, channel=getattr(pp, channel))
        a = c.analyze(1)
        _, de = c.grad(1)
    check_against_oracle(res, a, no, nv, mult, s)
    # Sec. Density Matrix: d omega / d eps_p = s D^2e_pp
    assert np.abs(de - s * np.diag(a["D2e"])).max() <= 1e-10


def test_analysis_larger_block(pp):
    """nv = 61: the one-CTA Jacobi on a 61 x 61 X X^T (the vector is the solver's last
    iterate, whether converged or not; the oracle analyses the same vector)."""
    no, nv, naux = 8, 61, 97
    spec = synth.SystemSpec("t", no + nv + 4, no + 1, naux, no, nv, 2)
    st = synth.make_system(spec)
    with pp.Context(0) as c:
        c.set_orbitals(st["occ"], st["eps"])
        c.set_active(no, nv)
        c.set_ao(st["C"], st["ao3c"])
        res = c.solve(mult=1, nroots=2, max_iter=40, conv_tol=1e-8, raise_noconv=False)
        a = c.analyze(1)
    w = np.concatenate([np.ones(res["X"].shape[1]), -np.ones(res["Y"].shape[1])])
    z = np.concatenate([res["X"][1], res["Y"][1]])
    s = float(np.sign(z @ (w * z)))
    check_against_oracle(res, a, no, nv, 1, s)
