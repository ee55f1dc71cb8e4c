"""GB300-native periodic FM-BEM for acoustic transmission through 2D periodic fiber media.

The compute path is the CUDA library ``libpfmbem.so`` (built by ``build.build()``);
``pfmbem`` is a thin ctypes binding with the C-ABI names.
"""
