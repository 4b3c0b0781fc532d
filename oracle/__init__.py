"""Plain FP64 CPU oracle of the weakly-compressible SPH hot path and of reaction-diffusion
on its particles.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or run
this package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it. It shares no code, constant table or helper with the CUDA
library; both are fed from the seeded input generators alone.

Every function follows the paper's equations in the paper's order (cited per
function). Parity status per function is listed in each module's header (`wcsph`,
`mpnn`, `diffusion`, `reaction`).
"""
from . import diffusion, mpnn, reaction, wcsph  # noqa: F401
