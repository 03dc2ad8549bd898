"""GB300-native layered unified tomographic reconstruction (arXiv 2206.09151).

The computation lives in ``librecon.so`` (CUDA kernels for sm_103a behind the C-ABI
of ``include/recon.h``); this package holds its ctypes binding (``_abi``), a
PyTorch-facing wrapper (``recon.Reconstructor``), the build step (``build``) and the
seeded synthetic inputs (``phantoms``)."""
from . import _abi  # noqa: F401
from ._abi import (  # noqa: F401
    ReconError, recon_backproject, recon_default_options, recon_destroy, recon_error_string, recon_filter_stage,
    recon_last_error, recon_plan, recon_plan_info, recon_profile_enable, recon_profile_read, recon_run, recon_sync, recon_workspace_size,
)


def __getattr__(name):
    if name == "Reconstructor":
        from .recon import Reconstructor
        return Reconstructor
    raise AttributeError(name)
