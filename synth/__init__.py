"""Seeded synthetic inputs shared by the CPU checker, the tests and the bench.

Holds graph/matrix generators and counter-based random numbers only; none of
the sparsification method's arithmetic lives here.
"""
from . import rng, graphs  # noqa: F401
from .graphs import Graph  # noqa: F401
