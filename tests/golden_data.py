"""Readers of the stored expected values under ``tests/golden/`` (each file
cites where its values come from in its header)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def philox_kat():
    """[(key, [c0..c3], [r0..r3])] for Philox4x32-10."""
    out = []
    for line in _rows("philox4x32_10_kat.txt"):
        key, ctr, res = (part.split() for part in line.split("|"))
        out.append((int(key[0], 16), [int(x, 16) for x in ctr], [int(x, 16) for x in res]))
    return out


def weight_table():
    """[(p, eta, scale, W_X, W_Y, Wt)] of Eqs. coeff_in_energy / coeff_in_distance."""
    out = []
    for line in _rows("weights_eq_coeff.txt"):
        p, eta, scale, wx, wy, wt = line.split()
        out.append((float(p), float(eta), int(scale), int(wx), int(wy), int(wt)))
    return out
