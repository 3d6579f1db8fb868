"""Seeded synthetic input generators shared by the oracle tests and the CUDA path."""
from .generators import *  # noqa: F401,F403
