"""Writes `schechter15.txt`, the per-subsample tables of the paper's fifteen-bin
artificial survey (Sec. 5), from the printed constants in `sec5_setup.txt` and
the FP64 oracle only (`oracle.mock`: the Schechter integral of App. D and the
luminosity bias law of Eq. rel_bias).

  * Magnitude bins: n_sub equal bins from M_max to M_min, brightest first.
  * Nbar^l = Phi_* int Phi dM over bin l (Sec. 5).  The paper prints no Phi_*;
    it is read here as the value that gives the faintest bin Nbar = 8.
  * b^l = b(M^l) of Eq. rel_bias at the bin centre M^l.

Run from the repository root:  python -m tests.golden.schechter15
Test infrastructure: imported by tests only.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SETUP = os.path.join(HERE, "sec5_setup.txt")
TABLE = os.path.join(HERE, "schechter15.txt")
NBAR_FAINTEST = 8.0


def read_setup(path=SETUP):
    """{name: (float value, citation)} of a `name = value | citation` file."""
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, cite = line.split("|", 1)
            name, value = lhs.split("=", 1)
            out[name.strip()] = (float(value), cite.strip())
    return out


def compute(setup):
    """phi_star and rows (l, M_lo, M_hi, Nbar, b), all FP64, from the oracle."""
    from oracle import mock

    v = {k: x[0] for k, x in setup.items()}
    n = int(v["n_sub"])
    edges = np.array([v["M_max"] + (v["M_min"] - v["M_max"]) * i / n for i in range(n + 1)])
    sch = dict(M_star=v["schechter_M_star"], alpha=v["schechter_alpha"])
    phi_star = NBAR_FAINTEST / float(mock.schechter_integral(edges[-2], edges[-1], **sch))
    nbar = mock.nbar_per_bin(edges, phi_star, **sch)
    b = mock.bias_law(0.5 * (edges[:-1] + edges[1:]), b_star=v["bias_b_star"], M_star=v["bias_M_star"],
                      a=v["bias_a"], b=v["bias_b"], c=v["bias_c"])
    rows = [(l, float(edges[l]), float(edges[l + 1]), float(nbar[l]), float(b[l])) for l in range(n)]
    return phi_star, rows


def read_table(path=TABLE):
    """(phi_star, rows) as written by `write`."""
    phi_star, rows = None, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("phi_star"):
                phi_star = float(line.split("=", 1)[1])
                continue
            t = line.split()
            rows.append((int(t[0]), float(t[1]), float(t[2]), float(t[3]), float(t[4])))
    return phi_star, rows


def write(path=TABLE):
    phi_star, rows = compute(read_setup())
    with open(path, "w") as f:
        f.write("# Fifteen-subsample survey of Sec. 5: per magnitude bin l, its edges\n")
        f.write("# [M_lo, M_hi), Nbar^l = Phi_* int Phi dM (App. D) and b^l of Eq. rel_bias\n")
        f.write("# at the bin centre.  Written by tests/golden/schechter15.py from the\n")
        f.write("# constants of sec5_setup.txt and the FP64 oracle; floats are repr() values.\n")
        f.write(f"phi_star = {phi_star!r}\n")
        f.write("# l  M_lo  M_hi  Nbar  b\n")
        for l, lo, hi, nb, b in rows:
            f.write(f"{l} {lo!r} {hi!r} {nb!r} {b!r}\n")


if __name__ == "__main__":
    write()
