"""Seeded synthetic inputs for the batched tridiagonal solver and its oracle.

This package only draws random numbers and lays out test problems; it holds
none of the solver's arithmetic. Both the CUDA path's tests/bench and the CPU
oracle take their inputs from here, which is the one module the two share.
"""
from .inputs import *  # noqa: F401,F403
