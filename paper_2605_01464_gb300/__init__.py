"""GB300-native quaternion Moore-Penrose pseudoinverse by hyperpower iterations
(QRAPID, QSAI, QHPI19 and Newton-Schulz).

The compute path is the C-ABI library ``libqpinv.so`` built from ``csrc/``;
``paper_2605_01464_gb300.qpinv`` is its thin ctypes binding.  Importing this
package does not load the library; the first call into ``qpinv`` does, and
fails loudly if it is missing.
"""
__all__ = ["inputs", "qpinv"]
