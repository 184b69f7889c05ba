"""GB300-native (sm_103a) q-LSKUM flux-residual solver.

The solver is the native library ``_build/liblskum.so`` (C ABI:
``include/lskum.h``, ``include/lskum_mlp.h``), built by ``build.py`` from the
CUDA and C++ sources in ``csrc/``. The Python modules marshal arguments:

- ``lskum``: ctypes binding of the solver (``Solver``, options, errors);
- ``surrogate``: the warm-start MLP binding and its training loop;
- ``cloud``: seeded synthetic NACA 0012 point clouds and condition sets;
- ``precision_study``, ``warmstart_study``: measurement scripts.
"""
