"""Diffusion Restore hot path for GB300 (sm_103a).

The compute lives in the C-ABI CUDA library ``libdiffrestore.so`` (declared in
``include/diffrestore.h``); ``_lib`` is its ctypes binding and ``renderer``
the torch-facing wrapper (device tensors and streams only).  ``scenes``
generates the seeded synthetic inputs."""
from . import scenes  # noqa: F401

__all__ = ["scenes", "load_renderer"]


def load_renderer():
    """Imports the torch-facing wrapper (requires torch; the library is
    built in-tree on first use)."""
    from . import renderer
    return renderer
