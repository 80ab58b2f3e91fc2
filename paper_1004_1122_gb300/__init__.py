"""GB300-native FFT/CG solver for periodic homogenization (trigonometric
collocation Lippmann-Schwinger system, conjugate-gradient accelerated).

The compute path is the CUDA library ``libfh.so`` (C ABI in ``include/fh.h``);
``paper_1004_1122_gb300.fh`` is a thin ctypes binding over it.  Importing this
package does not load the library; ``microstructure`` (synthetic inputs) is
usable without a GPU.
"""
__version__ = "0.1.0"
