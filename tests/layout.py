"""Test helpers: convert between the C-ABI word layouts and the oracle's
one-byte-per-qubit / one-byte-per-generator arrays.  Pure bit bookkeeping; no
arithmetic of the decoding method."""
import numpy as np


def words_to_labels(words, n_qubits):
    """(..., 2w) uint32 planar words -> (..., n) uint8 labels (x<<1 | z)."""
    words = np.ascontiguousarray(words).view(np.uint32)
    w = words.shape[-1] // 2
    bits = np.unpackbits(words.view(np.uint8), axis=-1, bitorder="little")
    x = bits[..., : 32 * w][..., :n_qubits]
    z = bits[..., 32 * w:][..., :n_qubits]
    return ((x << 1) | z).astype(np.uint8)


def labels_to_words(labels):
    """(..., n) uint8 labels -> (..., 2w) uint32 planar words."""
    labels = np.asarray(labels, np.uint8)
    n = labels.shape[-1]
    w = (n + 31) // 32
    pad = [(0, 0)] * (labels.ndim - 1) + [(0, 32 * w - n)]
    x = np.pad((labels >> 1) & 1, pad)
    z = np.pad(labels & 1, pad)
    px = np.packbits(x, axis=-1, bitorder="little").view(np.uint32)
    pz = np.packbits(z, axis=-1, bitorder="little").view(np.uint32)
    return np.concatenate([px, pz], axis=-1)


def syn_words_to_bits(words, n_stab):
    words = np.ascontiguousarray(words).view(np.uint32)
    bits = np.unpackbits(words.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :n_stab].astype(np.uint8)


def syn_bits_to_words(bits):
    bits = np.asarray(bits, np.uint8)
    n = bits.shape[-1]
    sw = (n + 31) // 32
    pad = [(0, 0)] * (bits.ndim - 1) + [(0, 32 * sw - n)]
    return np.packbits(np.pad(bits, pad), axis=-1, bitorder="little").view(np.uint32)
