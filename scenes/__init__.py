"""Seeded synthetic scene generator shared by the oracle tests and the CUDA path."""
from .generator import *  # noqa: F401,F403
