"""Seeded synthetic input generators shared by the oracle, tests and bench."""
from . import generators  # noqa: F401
