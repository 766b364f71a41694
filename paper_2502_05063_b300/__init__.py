"""Vietoris-Rips persistence barcodes over Z/2 on NVIDIA B300 (sm_103a).

Importing the package loads nothing; ``paper_2502_05063_b300.vr`` loads the
CUDA library (and raises if it is missing), ``paper_2502_05063_b300.synth``
draws seeded inputs.
"""
