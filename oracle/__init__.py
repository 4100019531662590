"""FP64 CPU oracle of the DID sweep (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the GPU library never does.
"""

from . import did_oracle  # noqa: F401
