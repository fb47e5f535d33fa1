"""GB300-native ACAT (Adaptive Compact Approximate Taylor) time step.

The compute path is the CUDA library ``libacat.so`` (built from ``csrc/``);
``acat`` is its thin ctypes binding. Importing the package does not load the
library; the first call into ``acat`` does, and raises if it is missing.
"""
