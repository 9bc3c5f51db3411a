"""GB300-native even-odd clover-Wilson operator and solvers (arXiv:1711.03836, BQCD).

The compute path is the CUDA shared library ``libbqcd_gb300.so`` built from
``csrc/``; ``bqcd`` is its thin ctypes binding.  ``synth`` draws the seeded
synthetic inputs.
"""
