"""GB300-native staggered phase-field fracture load step (arXiv:2203.16467).

The compute path is the CUDA library ``libpff.so`` (sources in ``csrc/``,
public C ABI in ``include/pff.h``); ``pff`` is its thin ctypes binding and
loads the library on import, failing loudly when it is missing.
``inputs`` draws the seeded synthetic modulus fields.
"""
