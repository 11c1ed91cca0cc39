"""FP64 CPU oracle of the Omni-Seg slide-wise path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline arm
may import this package; the product path never does.
"""
from . import omniseg_oracle  # noqa: F401
