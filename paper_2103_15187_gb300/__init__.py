"""GB300-native fractional-step Navier-Stokes step (FSEI fluid hot path,
arXiv 2103.15187, Sec. 2.1 and Sec. 3.1).

``fsei``    -- ctypes binding of the C-ABI library ``libfsei.so`` (hand-written
               CUDA for sm_103a); loading fails loudly if the library is absent.
``build``   -- nvcc build of the library, in-tree.
``inputs``  -- seeded synthetic workloads (numpy, no solver arithmetic).
"""
