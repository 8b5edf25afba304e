"""FP64 CPU oracle of the ODGS ERP rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference legs may
import this package. It shares no code with the CUDA path (``paper_2410_20686_gb300``) and
never imports it; both sides read the same seeded inputs from the scene generator.
"""
from .oracle import *  # noqa: F401,F403
