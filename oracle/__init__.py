"""CPU FP64 oracle (test infrastructure only; see stokes_oracle)."""
from .stokes_oracle import (  # noqa: F401
    INV_PI, INV_4PI, dlp_kernel, self_blocks, stokeslet, rotlet, operator_blocks,
    assemble, moments, apply_rows, matvec, velocity, BlockDiagonal, gmres,
    solve_dense, solve_gmres, trig_interpolation, coarse_geometry, TwoGrid, fgmres,
)
from . import learned_coarse  # noqa: F401,E402
