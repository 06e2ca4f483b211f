"""Test helper: the oracle's generators read back from its syndrome map."""
import numpy as np

import oracle as O


def generators_from_syndromes(d):
    """Rebuild each G_f from which single-qubit Paulis it anticommutes with."""
    nq, ns, _ = O.code_sizes(d)
    G = np.zeros((ns, nq), np.uint8)
    for q in range(nq):
        for lab, bit in ((2, 1), (1, 2)):  # X_q flags a Z part, Z_q flags an X part
            cfg = np.zeros(nq, np.uint8)
            cfg[q] = lab
            s = O.syndrome(d, cfg)
            G[s == 1, q] |= bit
    return G
