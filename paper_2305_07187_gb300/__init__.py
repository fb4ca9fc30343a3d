"""GB300-native hot path of the Spring-Ising Algorithm (arXiv 2305.07187).

The coupling force F = J q, the spring integrator of Eq. 8 with the walls of
Eq. 6, the sign readout and the exact energy of Eq. 1 run in hand-written
sm_103a CUDA kernels behind the C ABI of include/spring_ising.h.  This package
is the Python binding of that library (``Context``) plus the seeded input
generators (``inputs``).
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    # The binding is imported lazily so that the input generators work on
    # machines without the compiled library.
    if name in ("Context", "SpringIsingError", "default_params", "load", "SiParams"):
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
