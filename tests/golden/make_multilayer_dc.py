"""Writes tests/golden/multilayer_dc.json: the k = 0 finite part of the coating
stacks that the GPU tests build, computed by the oracle
(``oracle.kernel.khat_multilayer_dc``, mpmath arithmetic).  The GPU machine has no
mpmath, so the GPU tests read the stored values; ``tests/test_oracle_kernel.py``
recomputes them on the CPU and checks that the file is current.

Run from the repository root: python tests/golden/make_multilayer_dc.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import kernel  # noqa: E402

# name -> (layers from the surface down as (h, E, nu), substrate E, substrate nu)
STACKS = {
    "two_on_substrate": ([(0.2, 3.0, 0.3), (0.5, 0.5, 0.4)], 1.0, 0.45),
    "three_on_rigid": ([(0.1, 0.8, 0.25), (0.15, 4.0, 0.35), (0.3, 1.5, 0.3)], math.inf, 0.3),
    "stiff_over_soft": ([(0.3, 10.0, 0.3), (0.2, 0.2, 0.45)], 1.0, 0.3),
}


def compute():
    out = {"_about": "k = 0 finite part lim_{k->0}[K(k) - 2/(E_sub* k)] of coating stacks, by "
                     "oracle.kernel.khat_multilayer_dc; written by tests/golden/make_multilayer_dc.py"}
    for name, (layers, Es, nus) in STACKS.items():
        out[name] = {"layers": layers, "E_sub": "inf" if math.isinf(Es) else Es, "nu_sub": nus,
                     "dc": kernel.khat_multilayer_dc(layers, Es, nus)}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "multilayer_dc.json"), "w") as fh:
        json.dump(compute(), fh, indent=1)
        fh.write("\n")
