"""FP64 CPU oracle for the ms2 molecular-dynamics hot path — TEST INFRASTRUCTURE.

Only tests/, the smoke check and the CPU-baseline leg of bench.py may import
this package.  The GPU library never imports it.  See ms2_oracle.c for the
definitions it implements and the paper passages they restate.
"""
from .binding import Oracle, build, units  # noqa: F401
