"""Bit-sliced PCPD Monte Carlo sweep on GB300 (sm_103a): a C-ABI CUDA library
(libpcpd.so, declared in include/pcpd.h) with a thin ctypes binding (``pcpd``)."""
