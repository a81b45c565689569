"""GB300 (sm_103a) IMEX Runge-Kutta / SDC solver for incompressible flow on a DG
spectral-element mesh.  The compute path is the CUDA library built from
``csrc/`` (see ``build.py``) and reached through the C ABI of ``include/imex.h``;
``imex`` is its ctypes binding."""
from . import imex  # noqa: F401
from .imex import Context, ImexError  # noqa: F401
