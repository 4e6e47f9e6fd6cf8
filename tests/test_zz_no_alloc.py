"""The allocation-free FP64 sigma entry point, checked against pprpa_sigma and the oracle.

pprpa_sigma_noalloc serves callers that cannot allocate device memory (code
inside another framework's fixed memory pool, latency-critical loops that
cannot take the synchronisation of cudaMalloc, plugins whose host forbids
allocation).  It keeps its intermediates in one fixed device array shared by
all calls, so this test calls it twice in a row with different inputs and
checks each result against the allocating entry point, within the FP64
sigma tolerance the other tests use, and against the oracle's explicit
matrix applied to the same vectors.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _case(spec, nocc_act, nvir_act):
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], nocc_act, nvir_act)
    return s, orb, oracle.ao_to_mo(s["ao3c"], s["C"], orb), s["eps"][orb]


def _check_noalloc(spec, no, nv, calls):
    import torch

    import paper_2512_12515_gb300 as pp

    s, orb, L_ref, eps_ref = _case(spec, no, nv)
    eps_act = torch.as_tensor(np.ascontiguousarray(eps_ref), device="cuda")
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        L = torch.empty(c.get_L().shape, dtype=torch.float64, device="cuda")
        c.get_L(L)
        L_or = torch.as_tensor(np.ascontiguousarray(L_ref), device="cuda")
        for mult, k, seed in calls:
            _, _, nvv, noo = c.dims(mult)
            z = torch.as_tensor(synth.random_trial_vectors(nvv + noo, k, seed), device="cuda")
            ref = c.sigma(mult, z, pp.PREC_FP64)
            out = torch.full_like(z, float("nan"))
            pp._lib.sigma_noalloc(mult, no, nv, L, eps_act, z, out)
            torch.cuda.synchronize()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.abs(o - r).max() <= 1e-11 * np.abs(r).max()
            # the oracle's explicit matrix on its own integrals, fed to the same entry point
            M, _, _ = oracle.build_matrix(eps_ref, no, L_ref, mult)
            want = z.cpu().numpy() @ M.T
            out.fill_(float("nan"))
            pp._lib.sigma_noalloc(mult, no, nv, L_or, eps_act, z, out)
            torch.cuda.synchronize()
            o2 = out.cpu().numpy()
            assert np.abs(o2 - want).max() <= 1e-11 * np.abs(want).max()


def test_sigma_noalloc_matches_pprpa_sigma_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as pp

    _check_noalloc(synth.SystemSpec("t", 34, 7, 70, 6, 24, 31), 6, 24, ((1, 4, 1), (3, 2, 2)))
    # beyond the fixed scratch the call is refused with an argument error
    big = torch.zeros((2, 16), dtype=torch.float64, device="cuda")
    rc = pp._lib.load().pprpa_sigma_noalloc(1, 50, 600, 2, big.data_ptr(), big.data_ptr(), 64,
                                            big.data_ptr(), big.data_ptr(), None)
    assert rc == -1


def test_sigma_noalloc_few_orbitals_long_aux():
    """Few active orbitals, many vectors and a long auxiliary index: the scratch holds
    thousands of auxiliary slices per pass, more products than one batched GEMM launch grid
    covers, so the launches split themselves (pprpa_sigma's FP64 form likewise)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _check_noalloc(synth.SystemSpec("t2", 12, 3, 3000, 2, 8, 32), 2, 8, ((1, 32, 3), (3, 40, 4)))
