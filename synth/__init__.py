"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark: geometry descriptions of the workloads and a frozen-flow
turbulence + Shack-Hartmann sensor simulator.  Holds none of the
reconstructor's arithmetic."""
from . import configs  # noqa: F401
from .screens import FrozenFlowSensors, pupil_mask, random_vector  # noqa: F401
