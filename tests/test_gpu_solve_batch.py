"""pprpa_solve_batch: Davidson solves of several molecules at once, their BF16 / BF16x3
sigma products gathered into one batched tensor-core launch per round.

Each molecule's roots (mixed singlet / triplet, different sizes) are compared with the
oracle's full diagonalisation of its explicit matrix (Sec. ppRPA Equation) at the mixed
tolerance 1e-5 Ha, and with the same molecule solved alone.  A molecule that fails
(too many roots requested) reports its own code without stopping the others.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# (nocc_act, nvir_act, naux, mult, nroots): stable problems (nv small against sqrt(naux))
MOLS = [(5, 20, 120, 1, 8), (6, 24, 220, 3, 6), (4, 30, 300, 1, 8), (8, 16, 100, 3, 5),
        (3, 12, 60, 1, 4), (7, 28, 400, 1, 8)]


@pytest.fixture(scope="module")
def pp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as m

    return m


def build(pp):
    ctxs, refs = [], []
    for i, (no, nv, naux, mult, nr) in enumerate(MOLS):
        spec = synth.SystemSpec("b", no + nv + 3, no + 1, naux, no, nv, 700 + i)
        s = synth.make_system(spec)
        orb = oracle.active_orbitals(s["occ"], no, nv)
        L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
        M, nvv, noo = oracle.build_matrix(s["eps"][orb], no, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        assert sol["max_imag"] == 0.0
        refs.append(sol["omega_pp"][:nr])
        c = pp.Context(0)
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        ctxs.append(c)
    return ctxs, refs


@pytest.mark.parametrize("prec", ["PREC_BF16", "PREC_FP64"])
def test_solve_batch_matches_oracle_and_single_solves(pp, prec):
    ctxs, refs = build(pp)
    mults = [m[3] for m in MOLS]
    nroots = [m[4] for m in MOLS]
    p = getattr(pp, prec)
    tol = 1e-5 if prec == "PREC_BF16" else 1e-8
    ctol = 1e-5 if prec == "PREC_BF16" else 1e-7
    try:
        out = pp._lib.solve_batch(ctxs, mults, nroots, precision=p, conv_tol=ctol, max_iter=300)
        for r, ref, c, mult, nr in zip(out, refs, ctxs, mults, nroots):
            assert r["rc"] == 0
            assert r["info"]["converged"] == 1
            assert np.abs(r["omega"] - ref).max() <= tol
            alone = c.solve(mult=mult, nroots=nr, precision=p, conv_tol=ctol, max_iter=300)
            assert np.abs(alone["omega"] - r["omega"]).max() <= tol
        # a second batch on the same contexts (plans and graphs rebuilt or replayed)
        again = pp._lib.solve_batch(ctxs, mults, nroots, precision=p, conv_tol=ctol, max_iter=300)
        for r, ref in zip(again, refs):
            assert r["rc"] == 0 and np.abs(r["omega"] - ref).max() <= tol
    finally:
        for c in ctxs:
            c.close()


def test_solve_batch_one_molecule_fails_alone(pp):
    ctxs, refs = build(pp)
    try:
        nvv_last = ctxs[-1].dims(1)[2]
        nroots = [m[4] for m in MOLS[:-1]] + [nvv_last + 5]  # the last asks for too many roots
        out = pp._lib.solve_batch(ctxs, [m[3] for m in MOLS], nroots, precision=pp.PREC_BF16,
                                  conv_tol=1e-5, max_iter=300)
        assert out[-1]["rc"] == pp._lib.ERR_ARG
        for r, ref in zip(out[:-1], refs[:-1]):
            assert r["rc"] == 0 and np.abs(r["omega"] - ref).max() <= 1e-5
    finally:
        for c in ctxs:
            c.close()
