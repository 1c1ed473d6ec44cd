"""Seeded synthetic inputs (grid, Gaussian-well potential, ground-state orbitals, trial vectors)."""
from .systems import *  # noqa: F401,F403
