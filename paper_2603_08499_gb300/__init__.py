"""GB300-native VBGS coordinate-ascent update (Variational Bayes Gaussian Splatting).

The CUDA library (``libvbgs.so``, built by ``build.py``) implements the hot
path; ``vbgs`` is its ctypes binding and ``synth`` the seeded input
generators.
"""
