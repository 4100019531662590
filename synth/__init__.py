"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

Nothing here computes any step of the factorisation method: it only draws the
input matrices and start points (see ``synth.rng`` for the generator's
definition and ``synth.workloads`` for the recipes).
"""

from . import rng, workloads  # noqa: F401
