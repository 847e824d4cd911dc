"""GB300-native NUFFT dipole-dipole interaction (DDI) solver for dipolar BECs.

The compute path is the CUDA library ``lib/libddi_gb300.so`` (sources in ``csrc/``,
C-ABI declared in ``include/ddi.h``); ``ddi`` is its thin ctypes binding.  Importing
this package does not load the library; ``paper_1504_02897_gb300.ddi`` does, and
raises if it is missing.
"""
