"""Method parameters of the WR3L pipeline (Sec. 2.1, Eq. 2; Sec. 2.3, Eq. 9-11)."""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class Params:
    K: float = 0.006          # Wiener noise weight (Eq. 2)
    alpha: float = 0.003      # regularisation weight (Eq. 9)
    eps_phi: float = 1.0      # robust data penaliser: phi'(z) = eps/sqrt(z + eps^2)
    eps_psi: float = 10.0     # TV diffusivity: psi'(z) = 1/sqrt(z + eps^2), grey levels
    pos_floor: float = 0.1    # positivity floor delta for f and the Wiener output
    phi_robust: int = 1       # 1: robust phi', 0: phi' == 1 (plain RL data term)
    psi_tv: int = 1           # 1: TV psi', 0: psi' == 1 (linear diffusion)
    conv: str = "clamp"       # "clamp" (spatial) or "periodic" (Fourier)
    rf_eval: str = "log1p"    # r_f by log1p ("log1p") or by the lookup table of Sec. 4.1 ("lut")
