"""FP64 CPU oracle for the spectrum-reweighting likelihood (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the CUDA library never imports it and shares no code with it.
"""
from .srw_oracle import *  # noqa: F401,F403
from . import srw_oracle  # noqa: F401
