"""FP64 CPU oracle for the Wiener + robust regularised Richardson-Lucy (WR3L)
deblurring pipeline of Welk et al., "Fast and Robust Linear Motion Deblurring".

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check of the package entry point and the CPU
baseline leg of the benchmark may use it.  It shares no code with the CUDA
library; the one module both sides use is the seeded input generator.

Every function follows one equation or paragraph of the paper, in float64,
with no blocking or fusion: see `oracle.ops` for the citations and the
readings taken where the paper is silent or its formulas are garbled.
"""
from .ops import (  # noqa: F401
    conv_clamp, corr_clamp, conv_clamp_T, corr_clamp_T, conv_periodic, corr_periodic, conv, corr,
    box_running_sum_rows, box_running_sum_cols, box_ends_running_sum_rows, box_ends_running_sum_cols,
    psf_transfer, wiener, wiener_rows, wiener_cols,
    info_divergence, info_divergence_lut, r1, r1_lut, r1_lut_table, RF_LUT_N, RF_LUT_SMAX,
    phi_prime, psi_prime, diffusion,
    rrrl_step, rrrl, wr3l, condition_input, positivity_floor,
    wr3l_loss, snr_db,
)
