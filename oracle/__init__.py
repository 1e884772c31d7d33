"""FP64 CPU oracle (test infrastructure only; see sg_oracle's header)."""
from .sg_oracle import *  # noqa: F401,F403
from .sg_oracle import Options, SolveInfo  # noqa: F401
