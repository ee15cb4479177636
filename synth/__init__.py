"""Seeded synthetic input series, shared by the tests, the benchmark and the
oracle checks.  This package holds input recipes only -- no embedding,
distance, line or measure arithmetic of the method lives here."""
from .generators import *  # noqa: F401,F403
