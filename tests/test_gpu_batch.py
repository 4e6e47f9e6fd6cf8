"""Batched sigma over molecules of uneven size (one persistent launch per stage,
captured in a CUDA graph and replayed) and the tile autotuner, against the
per-molecule sigma and the explicit matrix of the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MOLS = [(5, 50, 165, 1), (12, 70, 250, 3), (3, 31, 100, 1), (20, 90, 330, 3)]


@pytest.fixture(scope="module")
def pp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as m

    return m


def molecule(no, nv, naux, seed):
    spec = synth.SystemSpec("b", no + nv + 2, no + 1, naux, no, nv, 100 + seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    return spec, s, orb


@pytest.mark.parametrize("seq_tiles", [None, "0", "500", "1000000"])
# BF16: 2u with u = 2^-8 (see check_bf16 in test_gpu_parity.py); BF16x3 drops lo*lo (2^-16)
@pytest.mark.parametrize("prec_name,tol", [("PREC_BF16", 2.0 * 2.0 ** -8), ("PREC_BF16_SPLIT", 2e-5)])
def test_sigma_batch_matches_per_molecule(pp, monkeypatch, prec_name, tol, seq_tiles):
    """seq_tiles: the first-stage tile count at which a molecule runs on its own launches
    ("0": all of them; "500": the two largest here; default and huge: none, one persistent
    launch)."""
    import torch

    if seq_tiles is not None:
        monkeypatch.setenv("PPRPA_BATCH_SEQ_TILES", seq_tiles)

    prec = getattr(pp, prec_name)
    ctxs, zs, outs, refs, scales, mults = [], [], [], [], [], []
    for i, (no, nv, naux, mult) in enumerate(MOLS):
        spec, s, orb = molecule(no, nv, naux, i)
        L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
        M, nvv, noo = oracle.build_matrix(s["eps"][orb], no, L, mult)
        c = pp.Context(0)
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        Z = synth.random_trial_vectors(nvv + noo, 8, 7 + i)
        ctxs.append(c)
        mults.append(mult)
        zs.append(torch.as_tensor(Z, device="cuda"))
        outs.append(torch.zeros_like(zs[-1]))
        refs.append(Z @ M.T)
        scales.append(np.abs(Z @ (M - np.diag(np.diag(M))).T).max())
    for call in range(2):  # capture, then replay
        for o in outs:
            o.zero_()
        pp._lib.sigma_batch(ctxs, mults, zs, outs, prec, graph=True)
        for o, r, sc in zip(outs, refs, scales):
            assert np.abs(o.cpu().numpy() - r).max() <= tol * sc
    single = [c.sigma(m, z, prec).cpu().numpy() for c, m, z in zip(ctxs, mults, zs)]
    for o, s1, sc in zip(outs, single, scales):
        assert np.abs(o.cpu().numpy() - s1).max() <= 1e-5 * sc  # same products, other atomics order
    for c in ctxs:
        c.close()


def test_autotune_keeps_results(pp):
    no, nv, naux, mult = 12, 70, 250, 1
    spec, s, orb = molecule(no, nv, naux, 9)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    M, nvv, noo = oracle.build_matrix(s["eps"][orb], no, L, mult)
    Z = synth.random_trial_vectors(nvv + noo, 8, 2)
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        tiles = c.autotune(mult, 8, pp.PREC_BF16)
        assert all(t % 16 == 0 and 16 <= t <= 256 for t in tiles)
        got = c.sigma(mult, Z, pp.PREC_BF16_SPLIT)
    scale = np.abs(Z @ (M - np.diag(np.diag(M))).T).max()
    assert np.abs(got - Z @ M.T).max() <= 2e-5 * scale
