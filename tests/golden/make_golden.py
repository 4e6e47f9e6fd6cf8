"""Write tests/golden/c0_roots.json from the FP64 oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
The stored values are the oracle's roots and correlation energy of the small
full-diagonalisation workload (nbasis 40, 5 occupied + 20 virtual active,
naux 120, seed 12515000).  The file serves as a cross-machine regression of
the oracle; the GPU tests compare against the oracle directly.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    spec = synth.CONFIGS["c0"]
    s = synth.make_system(spec)
    orb = oracle.active_orbitals(s["occ"], spec.nocc_act, spec.nvir_act)
    L = oracle.ao_to_mo(s["ao3c"], s["C"], orb)
    eps = s["eps"][orb]
    out = {"workload": "nbasis=40 nocc=5 nvir_act=20 naux=120 seed=12515000"}
    for mult in (1, 3):
        M, nvv, noo = oracle.build_matrix(eps, spec.nocc_act, L, mult)
        sol = oracle.solve_full(M, nvv, noo)
        ec = oracle.correlation_energy(M, nvv, noo, sol)[0]
        out[str(mult)] = {"omega_pp": [float(x) for x in sol["omega_pp"]],
                          "omega_hh": [float(x) for x in sol["omega_hh"]],
                          "ec": ec}
    with open(os.path.join(os.path.dirname(__file__), "c0_roots.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
