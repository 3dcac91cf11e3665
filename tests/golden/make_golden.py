"""Writes the golden files of this directory from the FP64 oracle alone (run from the repository
root: ``python tests/golden/make_golden.py``).  Inputs come from the seeded generators of
``paper_2210_13069_gb300/synth.py`` (inputs only, no arithmetic of the method).

Each file holds entries B^lr(mu, nu, ka, la) of the long-range two-electron integrals tensor as
the oracle computes them by Algorithm 1 (the Hadamard form of Theorem 1, with the prefactor
omega / sqrt(pi) of eq. approx33), for a few corner quadruples and seeded random ones, printed
with 17 significant digits.  The paper prints no worked example with values, so these are
regression anchors of the oracle (pinned itself by closed forms and brute force in
``tests/test_oracle_pins.py``) and expected values for the GPU entries.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def cases():
    from paper_2210_13069_gb300 import synth
    return {
        "nb20_s": (synth.workload_small_s(), 11),
        "spd2": (synth.random_molecule(2001, natoms=2, cube=4.0, nprim=3, alpha_range=(0.1, 50.0), omega=0.4,
                                       n=12, P=12, name="spd2"), 12),
    }


def quadruples(nbf, seed, count=48):
    rng = np.random.default_rng(seed)
    corners = [[0, 0, 0, 0], [nbf - 1] * 4, [0, nbf - 1, nbf - 1, 0], [1 % nbf, 0, 0, 1 % nbf]]
    return np.vstack([np.array(corners), rng.integers(0, nbf, size=(count, 4))]).astype(np.int32)


def path(name):
    return os.path.join(HERE, f"{name}_entries.txt")


def read(name):
    """(mol parameters dict, idx4 int array, values) from a golden file."""
    idx, vals, params = [], [], {}
    for line in open(path(name)):
        if line.startswith("# param "):
            k, v = line[len("# param "):].split("=", 1)
            params[k.strip()] = v.strip()
        elif line.strip() and not line.startswith("#"):
            a, b, c, d, v = line.split()
            idx.append((int(a), int(b), int(c), int(d)))
            vals.append(float(v))
    return params, np.array(idx, dtype=np.int32), np.array(vals)


def main():
    import oracle
    for name, (mol, seed) in cases().items():
        o = oracle.Oracle.from_molecule(mol)
        idx = quadruples(o.nbf, seed)
        vals = o.entries(idx)
        with open(path(name), "w") as f:
            f.write(f"# {name}: entries B^lr(mu, nu, ka, la) of the long-range TEI tensor by Algorithm 1\n")
            f.write("# (Hadamard form of Theorem 1, prefactor omega / sqrt(pi) of eq. approx33), FP64 oracle.\n")
            f.write("# Written by tests/golden/make_golden.py from oracle/ only; do not edit by hand.\n")
            f.write(f"# param nbf = {o.nbf}\n# param omega = {o.omega!r}\n# param n = {o.n}\n# param P = {o.P}\n")
            f.write("# mu nu ka la value\n")
            for (a, b, c, d), v in zip(idx, vals):
                f.write(f"{a} {b} {c} {d} {v:.17g}\n")
        print(f"wrote {path(name)}: {len(vals)} entries")


if __name__ == "__main__":
    main()
