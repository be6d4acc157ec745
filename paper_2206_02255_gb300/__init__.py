"""GB300 (sm_103a) Mandelbrot dwell maps by Mariani-Silver subdivision,
scheduled as Adaptive Serial Kernels (ASK), with an exhaustive kernel and a
CUDA Dynamic Parallelism (CDP2 tail launch) variant beside it.

The compute lives in ``libask.so`` (C ABI: ``include/ask.h``); ``ask`` is
its Python binding.  Importing this package loads nothing; the library is
loaded on first use and a missing build raises.
"""
__all__ = ["ask", "build", "inputs"]
