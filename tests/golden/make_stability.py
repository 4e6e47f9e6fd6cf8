"""Write tests/golden/stability_<workload>_<mult>.json from the FP64 oracle alone.

Run from the repository root:
    python tests/golden/make_stability.py c1 1      (or c1 3, c4 1)
    python tests/golden/make_stability.py c2 1 --window

For one workload of the synthetic suite and one multiplicity it records whether the ppRPA
pencil M z = omega W z (Sec. ppRPA Equation) has a definite shift, and what its spectrum
looks like around the two-electron addition / removal gap:

* lambda_min(M - mu W) on a grid of shifts mu (Lanczos on the explicit matrix); a positive
  value means mu is a definite shift and every root is real (Eq. xy_norm splits them);
* the diagonal-block test of ``oracle.block_shift_window`` (a definite shift must lie
  between -lambda_min(C) and lambda_min(A));
* every real eigenvalue of W M in an interval of the real axis from below the spectrum up
  past the 12th real addition root, and the complex ones inside the disks that cover it
  (shift-invert Arnoldi, dense LU, on disks that overlap: each centred on the upper edge of
  the previous one, radius = the distance to the farthest eigenvalue returned there), with
  the norm sign of each eigenvector: real addition roots (z^T W z > 0), real removal roots
  (< 0) and complex pairs.  Skipped above 30 000 pairs, where each factorisation takes
  minutes.

The explicit matrix is built row by row from the density-fitted integrals (tens of
thousands of pairs: a few GB to tens of GB of host memory).  Where it does not fit (the
nbasis-900 workload, 181 575 pairs), ``--window`` records only the diagonal-block test of
``oracle.block_shift_window``: a definite shift must lie between -lambda_min(C) and
lambda_min(A), and a Lanczos upper bound on lambda_min(A) below -lambda_min(C) proves that
none exists.  Nothing here comes from the GPU path.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def integrals(spec):
    head = synth.make_system(spec, with_ao=False)
    orb = oracle.active_orbitals(head["occ"], spec.nocc_act, spec.nvir_act)
    L = np.empty((spec.naux, spec.n_act, spec.n_act))
    for p0, blk in synth.ao_slices(spec, 64):
        L[p0:p0 + blk.shape[0]] = oracle.ao_to_mo(blk, head["C"], orb)
    return head["eps"][orb], L


def main(name, mult, start=-2.6, k=40, want_add=12, max_steps=60, roots_max_pairs=30000):
    spec = synth.CONFIGS[name]
    t0 = time.time()
    eps, L = integrals(spec)
    M, nvv, noo = oracle.explicit_matrix_ri(eps, spec.nocc_act, L, mult)
    t_build = time.time() - t0
    homo_lumo = float(eps[spec.nocc_act - 1] + eps[spec.nocc_act])
    mus = sorted(set([round(x, 2) for x in np.arange(-1.2, 0.45, 0.1)] + [homo_lumo]))
    lam = {f"{mu:.4f}": oracle.shifted_lambda_min(M, nvv, noo, mu) for mu in mus}
    window = oracle.block_shift_window(eps, spec.nocc_act, L, mult, steps=60)
    del L
    out = {
        "workload": f"{name}: nbasis={spec.nbasis} nocc={spec.nocc} nocc_act={spec.nocc_act} "
                    f"nvir_act={spec.nvir_act} naux={spec.naux} seed={spec.seed}",
        "mult": mult, "nvv": nvv, "noo": noo, "eps_homo_plus_lumo": homo_lumo,
        "lambda_min_shifted": lam,
        "definite_shift_found": any(v > 0 for v in lam.values()),
        "block_shift_window": window,
    }
    if nvv + noo <= roots_max_pairs:
        # disks of shift-invert Arnoldi walked upward from `start`, each centred on the upper
        # edge of the previous one, so that the covered interval of the real axis has no gap;
        # stop once it reaches past the want_add-th real addition root
        found, disks = [], []
        c = start
        for _ in range(max_steps):
            vals, metric = oracle.roots_near(M, nvv, noo, c, k=k)
            r = float(np.abs(vals - c).max())
            disks.append({"center": c, "radius": r})
            for v, m in zip(vals, metric):
                if not any(abs(v - f[0]) < 1e-9 * max(1.0, abs(v)) for f in found):
                    found.append((v, float(m)))
            adds = sorted(v.real for v, m in found if abs(v.imag) <= 1e-9 and m > 0)
            hi = c + r
            if len(adds) >= want_add and hi > adds[want_add - 1] + 1e-3:
                break
            c = hi
        found.sort(key=lambda t: (t[0].real, abs(t[0].imag)))
        rows = []
        for v, m in found:
            kind = "complex" if abs(v.imag) > 1e-9 else ("addition" if m > 0 else "removal")
            rows.append({"re": float(v.real), "im": float(v.imag), "metric": m, "kind": kind})
        add = [r_["re"] for r_ in rows if r_["kind"] == "addition"]
        rem = [r_["re"] for r_ in rows if r_["kind"] == "removal"]
        cplx = [r_ for r_ in rows if r_["kind"] == "complex"]
        out.update({
            "covered_interval": [disks[0]["center"] - disks[0]["radius"], disks[-1]["center"] + disks[-1]["radius"]],
            "disks": disks,
            "eigenvalues_found": rows,
            "lowest_real_addition_roots": add[:20],
            "highest_real_removal_roots": rem[-10:],
            "complex_pairs_with_re_below_10th_addition_root":
                sum(1 for r_ in cplx if len(add) >= 10 and r_["re"] < add[9] and r_["im"] > 0),
            "max_abs_imag": max([abs(r_["im"]) for r_ in cplx], default=0.0),
        })
    out["seconds"] = {"build": t_build, "total": time.time() - t0}
    path = os.path.join(os.path.dirname(__file__), f"stability_{name}_{mult}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, json.dumps({k_: out.get(k_) for k_ in ("definite_shift_found", "max_abs_imag",
                                                      "complex_pairs_with_re_below_10th_addition_root")}))


def main_window(name, mult, steps=40):
    spec = synth.CONFIGS[name]
    t0 = time.time()
    eps, L = integrals(spec)
    r = oracle.block_shift_window(eps, spec.nocc_act, L, mult, steps=steps)
    out = {
        "workload": f"{name}: nbasis={spec.nbasis} nocc={spec.nocc} nocc_act={spec.nocc_act} "
                    f"nvir_act={spec.nvir_act} naux={spec.naux} seed={spec.seed}",
        "mult": mult, "eps_homo_plus_lumo": float(eps[spec.nocc_act - 1] + eps[spec.nocc_act]),
        "block_shift_window": r, "definite_shift_found": False if r["proven_indefinite"] else None,
        "seconds": {"total": time.time() - t0},
    }
    path = os.path.join(os.path.dirname(__file__), f"stability_{name}_{mult}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, json.dumps(r))


if __name__ == "__main__":
    if "--window" in sys.argv:
        main_window(sys.argv[1], int(sys.argv[2]))
    else:
        main(sys.argv[1], int(sys.argv[2]))
