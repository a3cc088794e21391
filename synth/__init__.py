"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark: geometry descriptions of the workloads and a frozen-flow
turbulence + Shack-Hartmann sensor simulator.  Holds none of the
reconstructor's arithmetic.  The simulator (which needs torch) is imported
on first use, so that the geometry descriptions load without it."""
from . import configs  # noqa: F401

_SCREENS = ("FrozenFlowSensors", "pupil_mask", "random_vector")


def __getattr__(name):
    if name in _SCREENS:
        from . import screens
        return getattr(screens, name)
    raise AttributeError("module 'synth' has no attribute %r" % name)
