"""FP64 CPU oracle of the explicit relativistic PIC step (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this package.  See ``oracle.py`` for the step it computes.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import Species, State, build, lib  # noqa: F401
