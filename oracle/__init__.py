"""FP64 CPU oracle for the time-frequency semi-coherent statistic (arXiv:2510.19047).

TEST INFRASTRUCTURE. This package is the slow, plain reference that the CUDA library
is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path never does. It shares no code
with the CUDA library (``paper_2510_19047_b300``) and imports nothing from it.

The arithmetic lives in ``tfs_oracle.cpp`` (C++17, FP64, OpenMP over templates); this
module compiles it on first use and wraps its ``extern "C"`` entry points with numpy.
Every function cites, in the C++ source, the passage of the paper it follows.

Functions whose exact numeric form the paper does not fix, and what pins them: the
long-wavelength A/E detector tensors (the closed-form antenna power of two 90-degree
Michelsons 45 degrees apart pins the constellation's tilt and normal, the polarisation
tensors and the amplitude factors; the in-plane orientation at t = 0 is a convention
of the detector model and stays "parity unpinned"), and the 1PN TaylorT3 coefficients
(pinned through f = (1/2pi) dPhi/dt, the Newtonian limit and the paper's printed table
of the injections' coalescence times).
"""
from .build import load_library, build  # noqa: F401
from .api import (  # noqa: F401
    statistic, gradient, segments, fresnel, tranche_ft, source_constants, track, response,
    detector_tensors, polarisation, max_threads, response_tdi, spacecraft_offsets,
    statistic_harm, segments_harm, gradient_scale,
)
