"""GB300-native MGRIT/Parareal for periodic linear advection with
least-squares optimised coarse-grid operators.

The solver is the shared library ``libmgrit_gb300.so`` (CUDA kernels for
sm_103a plus a C++ host driver) behind the C ABI in ``include/mgrit.h``;
``paper_1910_03726_gb300.capi`` is its ctypes binding.  Build the library with
``python -m paper_1910_03726_gb300.build``.
"""

__all__ = ["capi", "build"]
