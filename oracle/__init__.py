"""FP64 CPU oracle of the lattice Boltzmann model for resistive relativistic MHD.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package. The product
library (``paper_1508_03452_gb300``) never imports it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
