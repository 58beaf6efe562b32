"""GB300-native hot path of the PGET Levenberg-Marquardt reconstruction (arXiv 2604.26745).

``pget`` is the thin ctypes binding of the C-ABI library ``libpget.so`` (CUDA kernels
for sm_103a); ``synth`` draws seeded synthetic inputs.  Importing the package loads
nothing; ``pget.load()`` loads the library and raises if it is missing.
"""
