"""CPU oracle of the stage residual and Runge-Kutta update (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package; the CUDA library never does.
"""
