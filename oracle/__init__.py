"""FP64 CPU oracle (test infrastructure only; see sma_oracle's header)."""
from . import sma_oracle  # noqa: F401
