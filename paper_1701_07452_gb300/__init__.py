"""GB300-native (sm_103a) FP64 implementation of the WOMBAT per-patch ideal-MHD
step (Mendygral et al. 2017, arXiv:1701.07452): the App. A MHDTVD flux inside
the 3D CTU+CT integrator, behind the C ABI of include/wombat.h.

``binding`` is the ctypes layer over ``libwombat_gb300.so``;
``initial_conditions`` holds the seeded synthetic inputs."""
from . import _build  # noqa: F401

__all__ = ["binding", "initial_conditions"]
