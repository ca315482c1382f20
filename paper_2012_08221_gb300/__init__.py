"""GB300-native batched PDF and alpha_s interpolation (PDFFlow's hot path).

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_2012_08221_gb300.pdf`` (and fails loudly if it is missing).
"""
__all__ = ["synth"]
