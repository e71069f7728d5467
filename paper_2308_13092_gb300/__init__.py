"""GB300-native (sm_103a) EC-PIC for 1D3V RF capacitively coupled discharges.

The compute path is the CUDA library ``libecpic.so`` built from ``csrc/``;
``ecpic`` is its ctypes binding.  ``inputs`` holds seeded workload recipes.
"""
