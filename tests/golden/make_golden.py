"""Writes tests/golden/config0_oracle.json from the FP64 oracle alone.

The stored values are the oracle's energy, per-atom energies and forces for
the 24-atom workload (seed 0) with the seed-1234 random-init weights. They
pin the oracle against later edits: a change to its arithmetic must name the
passage or reading that justifies it. Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402


def main():
    c = gen.make_config(0)
    W = oracle.Weights(gen.make_weights(1234))
    E, F, e = oracle.energy_forces(c.species, c.coords, c.cell, W, per_atom=True)
    out = {
        "what": "FP64 oracle on the 24-atom workload (seed 0), weights seed 1234",
        "cites": "paper: section 'OpenMM-ML' (ANI-2x), 'Optimization Through NNPOps' (symmetry functions), "
                 "'PyTorch Model Support' (forces by backpropagation)",
        "energy": E,
        "atom_energies": e.tolist(),
        "forces": F.tolist(),
    }
    with open(os.path.join(HERE, "config0_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
