"""GB300-native local-FFT PSATD Maxwell push (arXiv:1707.08500, Sec. 3).

The solver lives in the C-ABI library ``libpsatd.so`` (built from ``csrc/``);
``paper_1707_08500_gb300.psatd`` is the thin ctypes binding.  Nothing is
loaded at import time: the binding loads the library on first use and raises
if it is missing.
"""
