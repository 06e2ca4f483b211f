"""GB300 (sm_103a) simulated-annealing decoder for the XZZX code.

Hot path of arXiv:2509.17837 (Algs. 2, 3, 6, 7) as hand-written CUDA behind
the C ABI of ``include/xzzx.h`` (``libxzzx.so``); this package is the thin
Python binding.  There is no CPU fallback: importing the binding without the
built library raises.
"""
from . import _lib
from ._lib import XzzxError
from .api import (CONVENTION_Y_OVER_XZ, CONVENTION_PAPER, EMIN_PER_ATTEMPT, EMIN_PER_PHASE, LAYOUT_PLANAR,
                  LAYOUT_ROTATED, LINEAR, ORDER_COLOUR, ORDER_RANDOM_SITE, PAPER_LOG, Batch, Code, Schedule, Server, anneal,
                  decode_batch, decode_reduce, decode_workspace_size, greedy_init, make_noise, noise_from_eta,
                  sample_errors, version)

__all__ = ["Batch", "Code", "Server", "Schedule", "XzzxError", "anneal", "decode_batch", "decode_reduce", "decode_workspace_size",
           "greedy_init", "make_noise", "noise_from_eta", "sample_errors", "version", "LINEAR", "PAPER_LOG",
           "CONVENTION_Y_OVER_XZ", "CONVENTION_PAPER", "ORDER_COLOUR", "ORDER_RANDOM_SITE", "EMIN_PER_PHASE",
           "EMIN_PER_ATTEMPT", "LAYOUT_ROTATED", "LAYOUT_PLANAR"]
