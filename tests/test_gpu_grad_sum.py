"""Gradients of several roots in one call, the torch.autograd wrapper, and the correlation
energy of the removal channel from a Davidson solve (Sec. "Analytic Gradient", Eq.
correlation_energy).

pprpa_grad_sum returns sum_r w_r d omega_r; it is compared with the oracle's Hellmann-Feynman
gradient (oracle.grad_omega, pinned by finite differences) of the oracle's own eigenvectors
and with pprpa_grad root by root.  PPRPARoots (forward pprpa_solve, backward pprpa_grad_sum)
is checked against the same oracle gradient and against central finite differences of the
oracle's roots.  A Davidson solve of the hh channel asked for every removal root returns
E_c = -sum Omega^{N-2} - Tr C, compared with the oracle's two forms of Eq.
correlation_energy, and pprpa_grad_ec after it with finite differences of the oracle's E_c.
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


def make(no, nv, naux, seed, extra=4):
    nb = no + nv + extra
    spec = synth.SystemSpec("t", nb, no + 2, naux, no, nv, seed)
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], no, nv)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    return spec, s, L, s["eps"][orb]


def gpu_ctx(pp, spec, s):
    c = pp.Context(0)
    c.set_orbitals(s["occ"], s["eps"])
    c.set_active(spec.nocc_act, spec.nvir_act)
    c.set_ao(s["C"], s["ao3c"])
    return c


def oracle_weighted_grad(eps, no, L, mult, Z, w):
    de = np.zeros_like(eps)
    dL = np.zeros_like(L)
    for r, wr in enumerate(w):
        a, b = oracle.grad_omega(eps, no, L, mult, Z[:, r])
        de += wr * a
        dL += wr * b
    return de, dL


@pytest.mark.parametrize("mult", [1, 3])
def test_grad_sum_matches_oracle_and_single_roots(pp, mult):
    spec, s, L, eps = make(4, 14, 30, 21)
    no = 4
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    w = np.array([0.7, -1.3, 0.25, 2.0])
    de_ref, dL_ref = oracle_weighted_grad(eps, no, L, mult, sol["z_pp"], w)
    with gpu_ctx(pp, spec, s) as c:
        c.solve(mult=mult, nroots=4, method=pp.METHOD_FULL)
        dL, de = c.grad_sum(w)
        dL1 = np.zeros_like(dL)
        de1 = np.zeros_like(de)
        for r in range(4):
            a, b = c.grad(r)
            dL1 += w[r] * a
            de1 += w[r] * b
        with pytest.raises(pp.PprpaError):
            c.grad_sum(np.ones(5))  # more weights than roots
        with pytest.raises(pp.PprpaError):
            c.grad_sum(np.array([np.nan]))
    scale = np.abs(dL_ref).max()
    assert np.abs(de - de_ref).max() <= 1e-9
    assert np.abs(dL - dL_ref).max() <= 1e-9 * max(1.0, scale)
    assert np.abs(dL - dL1).max() <= 1e-12 * max(1.0, scale)
    assert np.abs(de - de1).max() <= 1e-12


def test_autograd_roots_match_oracle_and_finite_differences(pp):
    import torch

    spec, s, L, eps = make(3, 11, 24, 22)
    no, mult = 3, 1
    M, nvv, noo = oracle.build_matrix(eps, no, L, mult)
    sol = oracle.solve_full(M, nvv, noo)
    w = np.array([1.0, -0.5, 0.3])
    de_ref, dL_ref = oracle_weighted_grad(eps, no, L, mult, sol["z_pp"], w)
    Lt = torch.tensor(L, device="cuda", requires_grad=True)
    et = torch.tensor(eps, device="cuda", requires_grad=True)
    om = pp.PPRPARoots.apply(Lt, et, no, mult, 3, pp.METHOD_DAVIDSON, pp.PREC_FP64, 1e-10)
    assert np.abs(om.detach().cpu().numpy() - sol["omega_pp"][:3]).max() <= 1e-8
    loss = (om * torch.tensor(w, device="cuda")).sum()
    loss.backward(retain_graph=True)
    gL, ge = Lt.grad.cpu().numpy().copy(), et.grad.cpu().numpy().copy()
    assert np.abs(ge - de_ref).max() <= 1e-8
    assert np.abs(gL - dL_ref).max() <= 1e-8 * max(1.0, np.abs(dL_ref).max())
    # central finite differences of the oracle's roots along symmetric directions
    h = 1e-4

    def f(e, LL):
        Mx, a, b = oracle.build_matrix(e, no, LL, mult)
        return float(w @ oracle.solve_full(Mx, a, b)["omega_pp"][:3])

    rng = np.random.default_rng(5)
    for _ in range(2):
        D = rng.standard_normal(L.shape)
        D = D + D.transpose(0, 2, 1)
        D /= np.linalg.norm(D)
        fd = (f(eps, L + h * D) - f(eps, L - h * D)) / (2 * h)
        assert abs(fd - float(np.sum(gL * D))) <= 1e-6 * max(1.0, abs(fd))
    # the context lives with the graph: a second backward adds the same gradient again
    loss.backward()
    assert np.abs(Lt.grad.cpu().numpy() - 2 * gL).max() <= 1e-12 * max(1.0, np.abs(gL).max())
    assert np.abs(et.grad.cpu().numpy() - 2 * ge).max() <= 1e-12


@pytest.mark.parametrize("mult", [1, 3])
@pytest.mark.parametrize("prec", ["PREC_FP64", "PREC_BF16"])
def test_davidson_hh_every_root_gives_correlation_energy(pp, mult, prec):
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
    ec_pp, ec_hh = oracle.correlation_energy(M, nvv, noo)
    fp64 = prec == "PREC_FP64"
    with gpu_ctx(pp, spec, s) as c:
        res = c.solve(mult=mult, nroots=noo, precision=getattr(pp, prec), channel=pp.CHANNEL_HH,
                      conv_tol=1e-8 if fp64 else 1e-5, want_ec=True, max_iter=300)
        part = c.solve(mult=mult, nroots=noo - 1, channel=pp.CHANNEL_HH, conv_tol=1e-8, want_ec=True)
    assert res["info"]["converged"] == 1
    # every root within its tolerance, so E_c within noo times it
    tol = 1e-8 if fp64 else noo * 1e-5
    assert abs(res["ec"] - ec_hh) <= tol
    assert abs(res["ec"] - ec_pp) <= tol
    assert np.isnan(part["ec"])  # not every removal root: no correlation energy


@pytest.mark.parametrize("mult", [1, 3])
def test_grad_ec_after_davidson_hh(pp, mult):
    spec, s, L, eps = make(3, 9, 16, 23)
    no = 3
    with gpu_ctx(pp, spec, s) as c:
        _, _, nvv, noo = c.dims(mult)
        res = c.solve(mult=mult, nroots=noo, channel=pp.CHANNEL_HH, conv_tol=1e-10, want_ec=True)
        assert res["info"]["converged"] == 1
        dL, de = c.grad_ec()
        c.solve(mult=mult, nroots=nvv, method=pp.METHOD_FULL)
        dL_pp, de_pp = c.grad_ec()
        c.solve(mult=mult, nroots=2, channel=pp.CHANNEL_HH, conv_tol=1e-8)
        with pytest.raises(pp.PprpaError):
            c.grad_ec()  # needs every root of the channel

    def ec(e, LL):
        Mx, a, b = oracle.build_matrix(e, no, LL, mult)
        return oracle.correlation_energy(Mx, a, b)[1]

    # both channels give the same gradient of the same energy
    assert np.abs(de - de_pp).max() <= 1e-8
    assert np.abs(dL - dL_pp).max() <= 1e-8 * max(1.0, np.abs(dL_pp).max())
    h = 1e-4
    for p in (0, 2, 5, 9):
        ep, em = eps.copy(), eps.copy()
        ep[p] += h
        em[p] -= h
        fd = (ec(ep, L) - ec(em, L)) / (2 * h)
        assert abs(fd - de[p]) < 1e-6 * max(1.0, abs(fd))
    rng = np.random.default_rng(6)
    for _ in range(3):
        D = rng.standard_normal(L.shape)
        D = D + D.transpose(0, 2, 1)
        D /= np.linalg.norm(D)
        fd = (ec(eps, L + h * D) - ec(eps, L - h * D)) / (2 * h)
        assert abs(fd - float(np.sum(dL * D))) < 1e-6 * max(1.0, abs(fd))
