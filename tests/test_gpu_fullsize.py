"""Full-size checks at the benchmark's launch configuration, on sampled outputs.

The oracle cannot hold the explicit matrix at these sizes, so it computes
selected components sigma_I = sum_J M_IJ z_J one row at a time from the
definition, with the needed rows of L^P transformed from the AO integrals
(oracle.ao_to_mo_rows).  The GPU computes the whole 10-vector block through
the C ABI exactly as bench.py does.
"""
import os

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


def sampled_rows(spec, mult):
    nv, no = spec.nvir_act, spec.nocc_act
    vv = oracle.pair_list(nv, mult)
    oo = oracle.pair_list(no, mult)
    pick_v = [(0, 0 if mult == 1 else 1), (0, 1 if mult == 1 else 2), (5, nv // 2), (nv // 3, nv - 1),
              (nv - 2, nv - 1)]
    pick_o = [(0, 1), (no // 2, no - 1)]
    rows = [vv.index(p) for p in pick_v] + [len(vv) + oo.index(p) for p in pick_o]
    return rows, len(vv), len(oo)


@pytest.mark.parametrize("name,mult", [("c2", 1), ("c1", 1), ("c1", 3)])
def test_sigma_sampled_rows_full_size(pp, name, mult):
    import torch

    spec = synth.CONFIGS[name]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    eps = s["eps"][orb]
    rows, nvv, noo = sampled_rows(spec, mult)
    # oracle: the rows of L^P the sampled pairs touch
    p1, p2, _, _ = __import__("oracle.davidson_ref", fromlist=["_pairs_all"])._pairs_all(
        len(orb), spec.nocc_act, mult)
    need = sorted({int(p1[i]) for i in rows} | {int(p2[i]) for i in rows})
    Lr = dict(zip(need, oracle.ao_to_mo_rows(s["ao3c"], s["C"], orb, need)))
    k = 10
    Z = synth.random_trial_vectors(nvv + noo, k, 21)
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    ref = np.array([oracle.ri_sigma_rows(eps, spec.nocc_act, None, mult, Z[j], rows,
                                         Lrow=lambda p: Lr[p]) for j in range(k)])
    diag_part = np.array([[(1.0 if I < nvv else -1.0) * (eps[p1[I]] + eps[p2[I]]) * Z[j, I]
                           for I in rows] for j in range(k)])
    scale = np.abs(ref - diag_part).max()
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(spec.nocc_act, spec.nvir_act)
        c.set_ao(s["C"], s["ao3c"])
        del s["ao3c"]
        zd = torch.from_numpy(Z).cuda()
        out = {}
        for key, prec in (("bf16", pp.PREC_BF16), ("split", pp.PREC_BF16_SPLIT), ("fp8", pp.PREC_FP8)):
            out[key] = c.sigma(mult, zd, prec).cpu().numpy()[:, rows]
        out["fp64"] = c.sigma(mult, zd[:1].contiguous(), pp.PREC_FP64).cpu().numpy()[:, rows]
    err64 = np.abs(out["fp64"][0] - ref[0]).max()
    err16 = np.abs(out["bf16"] - ref).max()
    err48 = np.abs(out["split"] - ref).max()
    print(f"{name} mult {mult}: scale {scale:.3e} err fp64 {err64:.3e} bf16 {err16:.3e} split {err48:.3e}")
    assert err64 <= 1e-10 * max(1.0, scale)
    # BF16: unit roundoff u = 2^-8, about u of the two-electron scale in a CPU emulation of
    # the same arithmetic; bound 2u (the reasoning beside check_bf16 in test_gpu_parity.py)
    assert err16 <= 2.0 * 2.0 ** -8 * scale
    # BF16x3 drops the lo*lo product (2^-16 ~ 1.5e-5 relative) and accumulates at most
    # two auxiliary slices per tensor-memory accumulator before the FP32 partial sums
    assert err48 <= 3e-5 * scale
    # E4M3 operands in the first stage: about 4 % relative error (unit roundoff 2^-4)
    two = ref - diag_part
    e8 = out["fp8"] - ref
    print(f"  fp8 max/scale {np.abs(e8).max() / scale:.4f} fro {np.linalg.norm(e8) / np.linalg.norm(two):.4f}")
    assert np.linalg.norm(e8) <= 0.08 * np.linalg.norm(two)
    assert np.abs(e8).max() <= 0.1 * scale


def test_fp64_sigma_chunking_over_aux_index(pp, monkeypatch):
    """The FP64 sigma processes the auxiliary index in chunks; a forced small
    chunk must reproduce the single-chunk result and the explicit matrix."""
    spec = synth.SystemSpec("t", 30, 6, 90, 5, 20, 5)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], 5, 20)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    M, nvv, noo = oracle.build_matrix(s["eps"][orb], 5, L, 1)
    Z = synth.random_trial_vectors(nvv + noo, 3, 4)
    results = []
    for chunk in ("4096", "1"):
        monkeypatch.setenv("PPRPA_F64_CHUNK_MB", chunk)
        with pp.Context(0) as c:
            c.set_orbitals(s["occ"], s["eps"])
            c.set_active(5, 20)
            c.set_ao(s["C"], s["ao3c"])
            results.append(c.sigma(1, Z, pp.PREC_FP64))
    ref = Z @ M.T
    assert np.abs(results[0] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(results[1] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mult", [1, 3])
def test_adjoint_gradient_full_size(pp, mult):
    """FP64 adjoint at the 1500-function gradient workload: for a fixed pair vector z
    (z^T W z = 1), d(z^T M z)/dL along random symmetric directions against the
    oracle's central difference of the Rayleigh quotient (quadratic in L, so the
    central difference is exact up to rounding), and d/d eps against its closed form
    (the two-electron density diagonal, Sec. Density Matrix)."""
    spec = synth.CONFIGS["c4"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    eps = s["eps"][orb]
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    no, nv = spec.nocc_act, spec.nvir_act
    nvv = len(oracle.pair_list(nv, mult))
    noo = len(oracle.pair_list(no, mult))
    w = np.concatenate([np.ones(nvv), -np.ones(noo)])
    z = synth.random_trial_vectors(nvv + noo, 1, 5)[0]
    z[nvv:] *= 0.1
    z /= np.sqrt(z @ (w * z))
    with pp.Context(0) as c:
        c.set_orbitals(s["occ"], s["eps"])
        c.set_active(no, nv)
        c.set_ao(s["C"], s["ao3c"])
        dL, de = c.grad_vector(mult, z)
    de_ref = oracle.two_e_density_diag(z, no, nv, mult)
    assert np.abs(de - de_ref).max() <= 1e-12 * max(1.0, np.abs(de_ref).max())
    rng = np.random.default_rng(9)
    h = 1e-3
    for _ in range(2):
        D = rng.standard_normal(L.shape)
        D = D + D.transpose(0, 2, 1)
        D /= np.linalg.norm(D)
        qp = z @ oracle.ri_sigma(eps, no, L + h * D, mult, z[None])[0]
        qm = z @ oracle.ri_sigma(eps, no, L - h * D, mult, z[None])[0]
        fd = (qp - qm) / (2 * h)
        an = float(np.sum(dL * D))
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))
