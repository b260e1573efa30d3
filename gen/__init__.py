"""Seeded synthetic input generators (no hashing arithmetic)."""
from .inputs import *  # noqa: F401,F403
