"""Readers for the cited golden fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_param_table(name):
    """Returns {K: (radii list, constants list)} from a 'K | p.. | c..' fixture."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, p, c = [s.strip() for s in line.split("|")]
            out[int(k)] = ([int(v) for v in p.split()], [float(v) for v in c.split()])
    return out
