"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the decoding method: it only draws random
bits and random Pauli labels with numpy so that both sides can be fed the same
inputs.  Noise-model errors and their syndromes are produced by each side's own
sampler, not here.
"""
import numpy as np


def random_syndromes(n_faces, n_shots, density, seed):
    """Independent Bernoulli(density) syndrome bits, one row per shot."""
    rng = np.random.default_rng(seed)
    return (rng.random((n_shots, n_faces)) < density).astype(np.uint8)


def random_paulis(n_qubits, n, seed, p_nontrivial=0.5):
    """Random single-qubit Pauli labels (0..3) per qubit, one row per sample."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(1, 4, size=(n, n_qubits), dtype=np.uint8)
    keep = rng.random((n, n_qubits)) < p_nontrivial
    return (lab * keep).astype(np.uint8)
