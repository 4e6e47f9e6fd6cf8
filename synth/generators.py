"""Synthetic closed-shell mean-field data for ppRPA (inputs only, no method arithmetic).

Recipe (one PCG64 stream per system, drawn in this order):

1. occupied orbital energies ~ U(-1.0, -0.3) Ha, sorted ascending;
2. virtual orbital energies  ~ U(0.05, 3.0) Ha, sorted ascending;
3. MO coefficients C = Q * sign(diag(R)) from the QR factorisation of an
   nbasis x nbasis N(0, 1) matrix (orthogonal, unique signs);
4. the AO three-center tensor (P|mu nu), one slice per auxiliary index P:
   G ~ N(0, sigma^2) with sigma = sqrt(0.3 / naux), slice = (G + G^T) / 2.

The same stream order is reproduced whether the AO slices are drawn one at a
time or in chunks, so very large tensors can be streamed to the device.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Iterator, Tuple

import numpy as np


@dataclass(frozen=True)
class SystemSpec:
    """Sizes and seed of one synthetic system.

    nbasis = number of AO basis functions = number of MOs (nocc + nvir).
    nocc_act / nvir_act select the active space: the highest nocc_act
    occupied and the lowest nvir_act virtual orbitals.
    """

    name: str
    nbasis: int
    nocc: int
    naux: int
    nocc_act: int
    nvir_act: int
    seed: object

    @property
    def nvir(self) -> int:
        return self.nbasis - self.nocc

    @property
    def nmo(self) -> int:
        return self.nbasis

    @property
    def n_act(self) -> int:
        return self.nocc_act + self.nvir_act


# Workloads of the synthetic benchmark suite (sizes and seeds).
CONFIGS = {
    # small full-diagonalisation case
    "c0": SystemSpec("c0", 40, 5, 120, 5, 20, 12515000),
    # FP64 Davidson case
    "c1": SystemSpec("c1", 400, 20, 1200, 20, 200, 12515001),
    # mixed-precision case
    "c2": SystemSpec("c2", 900, 50, 2700, 50, 600, 12515002),
    # gradient case
    "c4": SystemSpec("c4", 500, 30, 1500, 30, 300, 12515004),
}


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.default_rng(seed)


def _draw_head(rng: np.random.Generator, nbasis: int, nocc: int):
    nvir = nbasis - nocc
    eocc = np.sort(rng.uniform(-1.0, -0.3, nocc))
    evir = np.sort(rng.uniform(0.05, 3.0, nvir))
    g = rng.standard_normal((nbasis, nbasis))
    q, r = np.linalg.qr(g)
    c = q * np.sign(np.diag(r))[None, :]
    eps = np.concatenate([eocc, evir])
    occ = np.concatenate([np.ones(nocc), np.zeros(nvir)])
    return occ, eps, np.ascontiguousarray(c)


def _draw_ao(rng: np.random.Generator, count: int, nbasis: int, sigma: float) -> np.ndarray:
    g = rng.normal(0.0, sigma, (count, nbasis, nbasis))
    return 0.5 * (g + g.transpose(0, 2, 1))


def make_system(spec: SystemSpec, rng=None, with_ao: bool = True) -> dict:
    """Draw the whole input set of ``spec``.

    Returns a dict with ``occ`` (nmo,), ``eps`` (nmo,), ``C`` (nbasis, nmo) and,
    when ``with_ao``, ``ao3c`` (naux, nbasis, nbasis), all float64 C-contiguous.
    ``rng`` overrides the spec's seed (used by the batched-molecule draws).
    """
    g = _rng(spec.seed if rng is None else rng)
    occ, eps, c = _draw_head(g, spec.nbasis, spec.nocc)
    out = {"occ": occ, "eps": eps, "C": c, "spec": spec}
    if with_ao:
        sigma = np.sqrt(0.3 / spec.naux)
        out["ao3c"] = np.ascontiguousarray(_draw_ao(g, spec.naux, spec.nbasis, sigma))
    return out


def ao_slices(spec: SystemSpec, chunk: int, rng=None) -> Iterator[Tuple[int, np.ndarray]]:
    """Yield ``(p0, ao[p0:p0+chunk])`` in stream order, after the head draws.

    Produces exactly the tensor ``make_system(spec)['ao3c']`` would hold,
    without ever materialising all of it on the host.
    """
    g = _rng(spec.seed if rng is None else rng)
    _draw_head(g, spec.nbasis, spec.nocc)
    sigma = np.sqrt(0.3 / spec.naux)
    p0 = 0
    while p0 < spec.naux:
        cnt = min(chunk, spec.naux - p0)
        yield p0, np.ascontiguousarray(_draw_ao(g, cnt, spec.nbasis, sigma))
        p0 += cnt


def batch_molecule_spec(m: int, redraw: int = 0):
    """Spec and generator of molecule ``m`` of the 64-molecule batch workload.

    nocc ~ U{5..40}, nvir ~ U{50..400}, nbasis = nocc + nvir (all orbitals
    active), naux = 3 * nbasis; even m is a singlet, odd m a triplet.
    ``redraw`` > 0 selects the replacement stream [12515, 3, m, redraw].
    Returns ``(spec, rng, mult)``; pass ``rng`` to :func:`make_system`.
    """
    key = [12515, 3, m] + ([redraw] if redraw else [])
    rng = np.random.default_rng(key)
    nocc = int(rng.integers(5, 41))
    nvir = int(rng.integers(50, 401))
    nb = nocc + nvir
    spec = SystemSpec(f"mol{m}", nb, nocc, 3 * nb, nocc, nvir, tuple(key))
    mult = 1 if m % 2 == 0 else 3
    return spec, rng, mult


def random_trial_vectors(dim: int, k: int, seed: int) -> np.ndarray:
    """k random unit-free test vectors of length ``dim`` (k, dim), float64."""
    g = np.random.default_rng(seed)
    return g.standard_normal((k, dim))
