"""Seeded synthetic inputs for the SFT step (maps, parameters, observations).

This package is shared by the tests, the benchmark and the smoke check.  It
holds none of the method's arithmetic: it only draws seeded random numbers
and evaluates closed-form fields on the grid's coordinates.
"""
from .generators import *  # noqa: F401,F403
