"""The allocation-free FP64 sigma entry point, checked against pprpa_sigma.

pprpa_sigma_noalloc serves callers that cannot allocate device memory (code
inside another framework's fixed memory pool, latency-critical loops that
cannot take the synchronisation of cudaMalloc, plugins whose host forbids
allocation).  It keeps its intermediates in one fixed device array shared by
all calls, so this test calls it twice in a row with different inputs and
checks each result against the allocating entry point, within the FP64
sigma tolerance the other tests use.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_sigma_noalloc_matches_pprpa_sigma_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as pp

    spec = synth.SystemSpec("t", 34, 7, 70, 6, 24, 31)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 6, 24)
    eps_act = torch.as_tensor(s["eps"][orb], device="cuda")
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(6, 24)
        c.set_ao(s["C"], s["ao3c"])
        L = torch.empty(c.get_L().shape, dtype=torch.float64, device="cuda")
        c.get_L(L)
        for mult, k, seed in ((1, 4, 1), (3, 2, 2)):
            _, _, nvv, noo = c.dims(mult)
            z = torch.as_tensor(synth.random_trial_vectors(nvv + noo, k, seed), device="cuda")
            ref = c.sigma(mult, z, pp.PREC_FP64)
            out = torch.full_like(z, float("nan"))
            pp._lib.sigma_noalloc(mult, 6, 24, L, eps_act, z, out)
            torch.cuda.synchronize()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.abs(o - r).max() <= 1e-11 * np.abs(r).max()
    # beyond the fixed scratch the call is refused with an argument error
    big = torch.zeros((2, 16), dtype=torch.float64, device="cuda")
    rc = pp._lib.load().pprpa_sigma_noalloc(1, 50, 600, 2, big.data_ptr(), big.data_ptr(), 64,
                                            big.data_ptr(), big.data_ptr(), None)
    assert rc == -1
