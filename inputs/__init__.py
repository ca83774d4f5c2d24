"""Seeded synthetic input generators shared by the oracle tests, the GPU
tests and the benchmark.  No sampler arithmetic lives here."""
from . import philox, configs  # noqa: F401
