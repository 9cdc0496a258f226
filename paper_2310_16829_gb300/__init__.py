"""GB300-native Lattice Multislice Algorithm (LMA) hot path.

The compute path lives in the CUDA library ``csrc/`` (built by
``__graft_entry__.build``) behind the C-ABI declared in ``include/lma.h``;
``lma.py`` is the ctypes binding. ``workloads.py`` holds the seeded synthetic
inputs. Importing this package loads nothing native.
"""
