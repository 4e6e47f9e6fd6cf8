"""pprpa_grad_ao: the adjoint of the AO->MO transform through the C ABI, against the oracle.

The oracle's adjoint (oracle.grad_ao) is pinned by finite differences of the whole chain
(AO integrals, C -> L -> M -> omega) and of a general linear functional of L.
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


def system(no=3, nv=7, naux=11, seed=31):
    spec = synth.SystemSpec("t", no + nv + 5, no + 1, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    return spec, s, orb


@pytest.mark.parametrize("mult,channel", [(1, "CHANNEL_PP"), (3, "CHANNEL_PP"), (1, "CHANNEL_HH")])
def test_root_gradient_back_to_ao_inputs(pp, mult, channel):
    spec, s, orb = system()
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(spec.nocc_act, spec.nvir_act)
        c.set_ao(s["C"], s["ao3c"])
        c.solve(mult=mult, nroots=2, method=pp.METHOD_FULL, channel=getattr(pp, channel))
        dL, _ = c.grad(1)
        d_ao, d_c = c.grad_ao(s["C"], dL, s["ao3c"])
    ref_ao, ref_c = oracle.grad_ao(s["ao3c"], s["C"], orb, dL)
    assert np.abs(d_ao - ref_ao).max() <= 1e-12 * max(1.0, np.abs(ref_ao).max())
    assert np.abs(d_c - ref_c).max() <= 1e-12 * max(1.0, np.abs(ref_c).max())


@pytest.mark.parametrize("device", [False, True])
def test_general_adjoint_host_and_device(pp, device):
    import torch

    spec, s, orb = system(4, 9, 17, 32)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((spec.naux, len(orb), len(orb)))  # not symmetric
    ref_ao, ref_c = oracle.grad_ao(s["ao3c"], s["C"], orb, G)
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(spec.nocc_act, spec.nvir_act)
        if device:
            args = [torch.from_numpy(a).cuda() for a in (s["C"], G, s["ao3c"])]
            d_ao, d_c = c.grad_ao(*args)
            d_ao, d_c = d_ao.cpu().numpy(), d_c.cpu().numpy()
        else:
            d_ao, d_c = c.grad_ao(s["C"], G, s["ao3c"])
        only_ao, none_c = c.grad_ao(s["C"], G, None, want_dao=True, want_dc=False)
    assert np.abs(d_ao - ref_ao).max() <= 1e-12 * np.abs(ref_ao).max()
    assert np.abs(d_c - ref_c).max() <= 1e-12 * np.abs(ref_c).max()
    assert none_c is None
    assert np.abs(only_ao - ref_ao).max() <= 1e-12 * np.abs(ref_ao).max()
    inactive = np.setdiff1d(np.arange(spec.nmo), orb)
    assert np.all(d_c[:, inactive] == 0.0)
