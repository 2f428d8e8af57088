"""GB300-native localised-order-parameter Kuramoto integrator (arXiv 2102.07167).

The compute path is the C-ABI library ``libkura.so`` (hand-written CUDA for
sm_103a, declared in ``include/kura.h``); ``paper_2102_07167_gb300.kura`` is
its thin ctypes binding.  Importing this package loads nothing: the binding
loads the library on first use and raises if it is missing.
"""
__all__ = ["kura", "gen"]
