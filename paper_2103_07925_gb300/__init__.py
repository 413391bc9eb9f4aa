"""GB300-native SPH interaction sweep (fluid, rigid bodies, heat, phase transitions).

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI, built into
``libsph.so``); ``sph.py`` is the ctypes binding; ``scenes.py`` builds seeded
synthetic inputs.
"""
