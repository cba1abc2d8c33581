"""Test infrastructure: the FP64 CPU oracle of the QTAM transform pair.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package; the library never does.
"""
from . import qtam_oracle  # noqa: F401
