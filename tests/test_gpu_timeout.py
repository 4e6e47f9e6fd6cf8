"""The tensor-core GEMM's bounded waits: a wait that runs out ends the kernel with an error
status, the call returns PPRPA_ERR_TIMEOUT, and the context stays usable.

Every mbarrier wait of the sigma kernels has a time limit (4 s by default).  With
PPRPA_TC_WAIT_NS set to 1 us, the waits of an ordinary launch (the epilogue waiting for a
tile's whole reduction, tens of microseconds here) run out: the kernel raises DEV_TIMEOUT,
lets its own copies and MMAs land, frees its tensor memory and returns.  Nothing is left
waiting: the next call with the default limit gives the right sigma on the same context.
The launches are forced onto single CTAs (no clusters), where every copy a CTA waits for is
its own.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12515_gb300 as m

    return m


def test_expired_wait_returns_timeout_and_context_recovers(pp, monkeypatch):
    import torch

    rng = np.random.default_rng(41)
    no, nv, naux = 16, 240, 400
    n = no + nv
    G = rng.normal(0.0, np.sqrt(0.3 / naux), (naux, n, n))
    L = torch.as_tensor(0.5 * (G + G.transpose(0, 2, 1)), device="cuda")
    eps = np.concatenate([np.sort(rng.uniform(-1.0, -0.3, no)), np.sort(rng.uniform(0.05, 3.0, nv))])
    occ = np.concatenate([np.ones(no), np.zeros(nv)])
    for k_, v in {"PPRPA_CLUSTER": "1", "PPRPA_CLUSTER2": "1", "PPRPA_TSTORE": "0"}.items():
        monkeypatch.setenv(k_, v)
    with pp.Context(0) as c:
        c.set_orbitals(occ, eps)
        c.set_mo(L)
        _, _, nvv, noo = c.dims(1)
        z = torch.as_tensor(rng.standard_normal((4, nvv + noo)), device="cuda")
        ref = c.sigma(1, z, pp.PREC_FP64).cpu().numpy()
        monkeypatch.setenv("PPRPA_TC_WAIT_NS", "1000")
        with pytest.raises(pp.PprpaError) as e:
            c.sigma(1, z, pp.PREC_BF16)
        assert e.value.code == pp._lib.ERR_TIMEOUT
        monkeypatch.delenv("PPRPA_TC_WAIT_NS")
        out = c.sigma(1, z, pp.PREC_BF16).cpu().numpy()
    # the recovered call is an ordinary BF16 sigma (BF16 operands, FP32 accumulation)
    two_e = np.abs(ref - out).max() / np.abs(ref).max()
    assert two_e < 1e-2
