"""Write tests/golden/stability_<workload>_<mult>.json from the FP64 oracle alone.

Run from the repository root:
    python tests/golden/make_stability.py c1 1      (or c1 3, c4 1)

For one workload of the synthetic suite and one multiplicity it records whether the ppRPA
pencil M z = omega W z (Sec. ppRPA Equation) has a definite shift, and what its spectrum
looks like around the two-electron addition / removal gap:

* lambda_min(M - mu W) on a grid of shifts mu (Lanczos on the explicit matrix); a positive
  value means mu is a definite shift and every root is real (Eq. xy_norm splits them);
* the eigenvalues of W M near a set of points (shift-invert Arnoldi, dense LU), merged,
  with the norm sign of each eigenvector: real addition roots (z^T W z > 0), real removal
  roots (< 0) and complex pairs.  Every eigenvalue inside each point's disk (radius = the
  distance to the farthest one returned there) is found.

The explicit matrix is built row by row from the density-fitted integrals (tens of
thousands of pairs: a few GB to tens of GB of host memory).  Nothing here comes from the
GPU path.
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


def main(name, mult, points=(-1.2, -0.9, -0.6, -0.3, 0.0, 0.3), k=40):
    spec = synth.CONFIGS[name]
    t0 = time.time()
    eps, L = integrals(spec)
    M, nvv, noo = oracle.explicit_matrix_ri(eps, spec.nocc_act, L, mult)
    del L
    t_build = time.time() - t0
    homo_lumo = float(eps[spec.nocc_act - 1] + eps[spec.nocc_act])
    mus = sorted(set([round(x, 2) for x in np.arange(-1.2, 0.45, 0.1)] + [homo_lumo]))
    lam = {f"{mu:.4f}": oracle.shifted_lambda_min(M, nvv, noo, mu) for mu in mus}
    found = []
    disks = []
    for s in points:
        vals, metric = oracle.roots_near(M, nvv, noo, s, k=k)
        disks.append({"center": s, "radius": float(np.abs(vals - s).max())})
        for v, m in zip(vals, metric):
            if not any(abs(v - f[0]) < 1e-9 * max(1.0, abs(v)) for f in found):
                found.append((v, float(m)))
    found.sort(key=lambda t: (t[0].real, abs(t[0].imag)))
    rows = []
    for v, m in found:
        kind = "complex" if abs(v.imag) > 1e-9 else ("addition" if m > 0 else "removal")
        rows.append({"re": float(v.real), "im": float(v.imag), "metric": m, "kind": kind})
    add = [r["re"] for r in rows if r["kind"] == "addition"]
    rem = [r["re"] for r in rows if r["kind"] == "removal"]
    cplx = [r for r in rows if r["kind"] == "complex"]
    out = {
        "workload": f"{name}: nbasis={spec.nbasis} nocc={spec.nocc} nocc_act={spec.nocc_act} "
                    f"nvir_act={spec.nvir_act} naux={spec.naux} seed={spec.seed}",
        "mult": mult, "nvv": nvv, "noo": noo, "eps_homo_plus_lumo": homo_lumo,
        "lambda_min_shifted": lam,
        "definite_shift_found": any(v > 0 for v in lam.values()),
        "disks": disks,
        "eigenvalues_near_gap": rows,
        "lowest_real_addition_roots": add[:20],
        "highest_real_removal_roots": rem[-10:],
        "complex_pairs_with_re_below_10th_addition_root":
            sum(1 for r in cplx if len(add) >= 10 and r["re"] < add[9] and r["im"] > 0),
        "max_abs_imag": max([abs(r["im"]) for r in cplx], default=0.0),
        "seconds": {"build": t_build, "total": time.time() - t0},
    }
    path = os.path.join(os.path.dirname(__file__), f"stability_{name}_{mult}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, json.dumps({k_: out[k_] for k_ in ("definite_shift_found", "max_abs_imag",
                                                  "complex_pairs_with_re_below_10th_addition_root")}))


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]))
