"""GB300-native hybrid PIC ion loop (kinetic ions, massless fluid electrons).

The compute path lives in the CUDA library ``libhv`` (``csrc/``) behind the
C ABI declared in ``include/hv.h``; ``hv`` is its thin ctypes binding."""
