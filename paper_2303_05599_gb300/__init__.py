"""GB300-native colored particle-in-cell (CPIC) Glasma + Wong solver
(arXiv:2303.05599): CUDA kernels for sm_103a behind a C ABI
(include/glasma.h), with a thin ctypes binding."""
from ._binding import (Event, GlasmaError, lib, gl_workspace_bytes, GL_FP64, GL_FP32_2ROW,  # noqa: F401
                       GL_BUF_LINKS, GL_BUF_PHI, GL_BUF_E, GL_BUF_PI, GL_BUF_SITE, GL_BUF_PARTICLES)
from . import workloads  # noqa: F401
