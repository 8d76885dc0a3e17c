"""Writes tests/golden/oracle_frozen.txt: per-event results of the FP64
oracle on small samples of the slab, calorimeter and calorimeter-in-2-T
workloads, so that tests/test_oracle_frozen.py can tell when the oracle's
arithmetic changes.  Calls only oracle/ (and the seeded input generators).

The oracle's arithmetic is frozen: kernel changes must agree with it as it
stands.  A deliberate change to the oracle rewrites this file with this
script, in a commit that names the passage of the paper, or the reading of
it, that justifies the change.

Run: python tests/golden/make_oracle_frozen.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2203_09467_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_frozen.txt")

# (name, setup, primaries, events)
SAMPLES = (
    ("slab", lambda: W.slab_setup(), lambda n: W.slab_primaries(n), 200),
    ("calo", lambda: W.calo_setup(), lambda n: W.calo_primaries(n), 12),
    ("calo_field", lambda: W.calo_field_setup(), lambda n: W.calo_field_primaries(n), 8),
)


def results(name):
    for nm, setup, prim, n in SAMPLES:
        if nm != name:
            continue
        s = setup()
        p = prim(n)
        orc = oracle.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
        _, summ = orc.run(p, n, np.arange(n), n_threads=1)
        orc.close()
        return summ
    raise KeyError(name)


def main():
    oracle.build()
    lines = ["# workload event edep escaped killed e_in steps tracks (energies as C99 hex floats)"]
    for name, _, _, _ in SAMPLES:
        summ = results(name)
        for e, row in enumerate(summ):
            vals = " ".join(float(v).hex() for v in row[:4])
            lines.append(f"{name} {e} {vals} {int(row[4])} {int(row[5])}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    return OUT


if __name__ == "__main__":
    print(main())
