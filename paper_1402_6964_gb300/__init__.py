"""GB300-native single-pass TSQR reduction for near-separable NMF of
tall-and-skinny matrices (Benson, Lee, Rajwa, Gleich, arXiv 1402.6964).

The compute path is the C-ABI library ``libmrnmf.so`` built from ``csrc/``;
``paper_1402_6964_gb300.mrnmf`` is its thin ctypes binding.  Importing this
package does not load the library; the binding loads it on first use and
raises if it is missing.
"""
__all__ = ["mrnmf", "synth"]
