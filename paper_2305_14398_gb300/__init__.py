"""GB300-native (sm_103a) unitary-matrix quantum circuit simulation.

The product is the C-ABI library libtqs.so (include/tqs.h) built from csrc/;
``binding`` is its ctypes marshalling layer and ``workloads`` draws the seeded
synthetic circuits.  Importing this package loads nothing; ``binding.lib()``
loads the library and raises if it has not been built.
"""
