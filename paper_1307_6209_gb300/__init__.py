"""SELL-C-sigma sparse matrix-vector multiply for GB300 (sm_103a).

The compute path is the C-ABI library built from ``csrc/`` (declared in
``include/sell.h``); ``sell`` is its thin ctypes binding.  Importing this
package does not load the library; ``sell`` does, and raises if it is missing.
"""
__all__ = ["sell", "synth"]
