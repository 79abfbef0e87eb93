"""Write rocksalt222_ground_state.txt: the exhaustive ground state of the
rocksalt 2x2x2 cation problem (a = 4.2 A, 32 anions fixed at -2, 32 cation
positions holding 16 x +1 and 16 x +3: C(32, 16) = 601,080,390 configurations),
computed by the oracle alone (orc_enumerate_two_species, about 20 s).

    python tests/golden/make_rocksalt222_ground_state.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import goac_synth as synth  # noqa: E402
import oracle  # noqa: E402


def main():
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    r = oracle.enumerate_two_species(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, tol=1e-9,
                                     max_argmin=4096)
    lines = ["# Exhaustive ground state of the rocksalt 2x2x2 cation problem (goac_synth.rocksalt_problem((2, 2, 2), 4.2)):",
             "# 32 anions fixed at -2, 32 cation positions with 16 x +1 (species 0) and 16 x +3 (species 1).",
             "# Written by tests/golden/make_rocksalt222_ground_state.py from the oracle's enumeration of all",
             "# C(32, 16) placements (orc_enumerate_two_species); minimisers within 1e-9 eV of the minimum.",
             f"n_configs {r['n_configs']}",
             f"E_min_eV {r['Emin']!r}",
             f"n_argmin {r['n_argmin']}",
             "# one line per minimiser: species of the 32 variable sites in site order"]
    lines += ["argmin " + "".join(str(int(x)) for x in a) for a in r["argmin"]]
    with open(os.path.join(HERE, "rocksalt222_ground_state.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
