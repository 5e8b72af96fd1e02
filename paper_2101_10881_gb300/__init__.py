"""pes: polynomial evaluation and differentiation at power series in multiple
double precision, on GB300 (sm_103a).

The compute path is the CUDA library libpes.so behind the C-ABI declared in
include/pes.h; `paper_2101_10881_gb300.pes` is its thin Python binding.  Importing
this package does not load the library; the first call into the binding does,
and fails loudly when the library is missing.
"""
__all__ = ["pes", "synth"]
