"""CPU oracle package (test infrastructure only; see hs_oracle's docstring)."""
from .hs_oracle import *  # noqa: F401,F403
from . import hs_oracle  # noqa: F401
