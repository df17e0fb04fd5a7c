"""FP64 CPU oracle (test infrastructure only; see fr3d_oracle's header)."""
from .fr3d_oracle import *  # noqa: F401,F403
from .learned_oracle import *  # noqa: F401,F403
from . import unet_oracle  # noqa: F401  (the U-Net post-corrector, used as oracle.unet_oracle)
