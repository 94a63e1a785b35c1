"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Nothing in this package computes any part of the enumeration method; it only
builds labelled edge lists from seeds (see ``configs`` for the workloads).
"""
from .graphs import Graph  # noqa: F401
from .rng import Stream, sub_seed  # noqa: F401
from . import configs  # noqa: F401
