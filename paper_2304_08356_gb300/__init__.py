"""GB300 (sm_103a) implementation of MANTRA's per-sample temporal path
sampling and progressive c-MCERA estimation (arXiv 2304.08356).

``mantra``  ctypes binding of libmantra.so (the C ABI of include/mantra.h)
``synth``   seeded synthetic temporal graphs (inputs only)
``build``   nvcc build of libmantra.so for sm_103a
"""
