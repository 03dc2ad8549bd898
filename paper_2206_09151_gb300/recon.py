"""PyTorch-facing wrapper of the C-ABI: device memory and streams come from PyTorch;
the computation is ``librecon.so``'s kernels (``recon_run`` and the stage entry points)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

_FILTERS = {"off": _abi.RECON_FILTER_OFF, "tikhonov": _abi.RECON_FILTER_TIKHONOV, "mlp": _abi.RECON_FILTER_MLP,
            "pair": _abi.RECON_FILTER_PAIR}
_INPUTS = {"intensity": _abi.RECON_INPUT_INTENSITY, "contrast": _abi.RECON_INPUT_CONTRAST}
_STACKS = {"f32": _abi.RECON_STACK_F32, "bf16": _abi.RECON_STACK_BF16}
_RAMPS = {"single_axis": _abi.RECON_RAMP_SINGLE_AXIS, "density": _abi.RECON_RAMP_DENSITY}
_BP_KERNELS = {"auto": _abi.RECON_BP_AUTO, "direct": _abi.RECON_BP_DIRECT, "staged": _abi.RECON_BP_STAGED,
               "tma": _abi.RECON_BP_TMA}
_LAYER_INTERP = {"nearest": _abi.RECON_LAYER_NEAREST, "linear": _abi.RECON_LAYER_LINEAR}


class Reconstructor:
    """One plan plus its workspace on the current CUDA device.

    ``rot`` (D, 3, 3) volume->beam rotations, ``nu``/``nv`` image size, ``grid`` =
    (nx, ny, nz), ``lam`` wavelength, ``delta`` pitch, ``defocus`` (D,) R_n,
    ``nz_layers`` depth layers (0: as many as the depth of field asks for); options as in
    ``recon_options``."""

    def __init__(self, rot, nu: int, nv: int, grid, *, lam: float, delta: float, defocus, nz_layers: int,
                 sigma: float = 0.0, eps: float = 0.1, cs: float = 0.0, filter: str = "tikhonov",
                 input_mode: str = "intensity", stack_dtype: str = "f32", accumulate: bool = False,
                 dir_block: int = 0, ramp: str = "single_axis", mlp_weights=None, nsr: float = 0.0,
                 stage_block: int = 0, bp_kernel: str = "auto", check_finite: bool = False,
                 layer_interp: str = "nearest", mlp_views: float = 0.0, bp_warp: int = 0, bp_tile_z: int = 0,
                 device=None,
                 allocate: bool = True):
        o = _abi.recon_default_options()
        o.sigma, o.eps, o.cs = float(sigma), float(eps), float(cs)
        o.filter, o.input_mode, o.stack_dtype = _FILTERS[filter], _INPUTS[input_mode], _STACKS[stack_dtype]
        o.accumulate, o.dir_block = int(bool(accumulate)), int(dir_block)
        o.ramp_mode = _RAMPS[ramp]
        o.nsr = float(nsr)
        o.stage_block = int(stage_block)
        o.bp_kernel = _BP_KERNELS[bp_kernel]
        o.check_finite = int(bool(check_finite))
        o.layer_interp = _LAYER_INTERP[layer_interp]
        o.mlp_views = float(mlp_views)
        o.bp_tile_z = int(bp_tile_z)
        o.bp_warp = int(bp_warp)
        self._weights = None
        if mlp_weights is not None:
            self._weights = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            o.mlp_weights = self._weights.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        self.rot = np.ascontiguousarray(rot, np.float64).reshape(-1, 3, 3)
        self.D = self.rot.shape[0]
        self.nu, self.nv, self.grid = nu, nv, tuple(grid)
        self.stack_dtype = torch.bfloat16 if stack_dtype == "bf16" else torch.float32
        self.plan = _abi.recon_plan(self.rot, nu, nv, lam, delta, defocus, nz_layers, self.grid, o)
        self.nz_layers = _abi.recon_plan_layers(self.plan)
        # the backprojection kernel the plan runs ("direct", "staged" or "tma")
        self.bp_kernel_used = {v: k for k, v in _BP_KERNELS.items()}[_abi.recon_plan_bp_kernel(self.plan)]
        self.ws_bytes = _abi.recon_workspace_size(self.plan)
        # recon_run_host's workspace: the same head plus two direction blocks of images
        self.ws_bytes_host = _abi.recon_run_host_workspace_size(self.plan)
        self.padded, self.dir_block, self.n_blocks, self.stage_block = _abi.recon_plan_info(self.plan)
        self.device = torch.device(device) if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None)
        self.workspace = None
        if allocate:
            self.workspace = torch.empty(max(self.ws_bytes_host, 256), dtype=torch.uint8, device=self.device)

    # -------------------------------------------------------------- helpers
    @staticmethod
    def _stream(stream) -> int:
        s = stream if stream is not None else torch.cuda.current_stream()
        return int(s.cuda_stream)

    def _check_images(self, images: torch.Tensor):
        if images.dtype != torch.float32 or not images.is_cuda or not images.is_contiguous():
            raise ValueError("images must be a contiguous float32 CUDA tensor")
        if tuple(images.shape) != (self.D, self.nv, self.nu):
            raise ValueError(f"images shape {tuple(images.shape)} != {(self.D, self.nv, self.nu)}")

    def new_volume(self) -> torch.Tensor:
        nx, ny, nz = self.grid
        return torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)

    # -------------------------------------------------------------- entry points
    def run(self, images: torch.Tensor, volume: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """``recon_run``: the whole operator into ``volume`` (allocated if None)."""
        self._check_images(images)
        if volume is None:
            volume = self.new_volume()
        nx, ny, nz = self.grid
        if volume.dtype != torch.float32 or not volume.is_contiguous() or tuple(volume.shape) != (nz, ny, nx):
            raise ValueError("volume must be a contiguous float32 tensor of shape (nz, ny, nx)")
        _abi.recon_run(self.plan, images.data_ptr(), volume.data_ptr(), self.workspace.data_ptr(), self.ws_bytes,
                       self._stream(stream))
        return volume

    @property
    def stack_row_stride(self) -> int:
        """Entries per stack row: the nu + 1 tap pairs rounded up to a multiple of 4 (every
        row starts on a 16-byte boundary); the entries past nu are padding, never read."""
        return (self.nu + 4) // 4 * 4

    def run_host(self, host_images: torch.Tensor, volume: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """``recon_run_host``: the whole operator with the images in host memory (a CPU
        tensor, pinned for the copies to overlap the compute); they must stay untouched until
        the stream's work has finished."""
        if host_images.dtype != torch.float32 or host_images.is_cuda or not host_images.is_contiguous():
            raise ValueError("host_images must be a contiguous float32 CPU tensor")
        if tuple(host_images.shape) != (self.D, self.nv, self.nu):
            raise ValueError(f"images shape {tuple(host_images.shape)} != {(self.D, self.nv, self.nu)}")
        if volume is None:
            volume = self.new_volume()
        nx, ny, nz = self.grid
        if volume.dtype != torch.float32 or not volume.is_contiguous() or tuple(volume.shape) != (nz, ny, nx):
            raise ValueError("volume must be a contiguous float32 tensor of shape (nz, ny, nx)")
        if self.workspace.numel() < self.ws_bytes_host:
            raise ValueError("the workspace is smaller than recon_run_host_workspace_size")
        _abi.recon_run_host(self.plan, host_images.data_ptr(), volume.data_ptr(), self.workspace.data_ptr(),
                            self.workspace.numel(), self._stream(stream))
        return volume

    def filter_stage(self, images: torch.Tensor, dir_begin: int, dir_count: int, stream=None) -> torch.Tensor:
        """``recon_filter_stage``: a view of the workspace holding the layer stacks as
        horizontal tap pairs, shape (dir_count, Nz, nv + 2, nu + 1, 2) (rows
        :attr:`stack_row_stride` entries apart): entry [n, k, v + 1, c] = (Y[v][c - 1],
        Y[v][c]), zero outside the image."""
        self._check_images(images)
        ptr = _abi.recon_filter_stage(self.plan, images.data_ptr(), dir_begin, dir_count,
                                      self.workspace.data_ptr(), self.ws_bytes, self._stream(stream))
        off = ptr - self.workspace.data_ptr()
        esz = 2 if self.stack_dtype == torch.bfloat16 else 4
        su = self.stack_row_stride
        n = dir_count * self.nz_layers * (self.nv + 2) * su * 2
        return self.workspace[off:off + n * esz].view(self.stack_dtype).view(
            dir_count, self.nz_layers, self.nv + 2, su, 2)[:, :, :, :self.nu + 1, :]

    def backproject(self, stack: torch.Tensor, dir_begin: int, dir_count: int, volume: torch.Tensor,
                    accumulate: bool, stream=None) -> torch.Tensor:
        """``recon_backproject``: layered backprojection of ``stack`` (tap-pair layout of
        :meth:`filter_stage`: its views are passed as they are; a contiguous
        (dir_count, Nz, nv + 2, nu + 1, 2) tensor is first copied into the plan's row
        stride) into ``volume``."""
        su = self.stack_row_stride
        shape = (dir_count, self.nz_layers, self.nv + 2, self.nu + 1, 2)
        strides = (self.nz_layers * (self.nv + 2) * su * 2, (self.nv + 2) * su * 2, su * 2, 2, 1)
        if stack.dtype != self.stack_dtype or tuple(stack.shape) != shape:
            raise ValueError("stack dtype/shape does not match the plan")
        if tuple(stack.stride()) != strides:
            if not stack.is_contiguous():
                raise ValueError("stack layout does not match the plan")
            padded = torch.zeros((dir_count, self.nz_layers, self.nv + 2, su, 2), dtype=stack.dtype,
                                 device=stack.device)
            padded[:, :, :, :self.nu + 1, :] = stack
            stack = padded
        _abi.recon_backproject(self.plan, stack.data_ptr(), dir_begin, dir_count, volume.data_ptr(),
                               int(bool(accumulate)), self.workspace.data_ptr(), self.ws_bytes, self._stream(stream))
        return volume

    def swap_ct(self, images: torch.Tensor, stream=None) -> torch.Tensor:
        """``recon_swap_ct`` (Eq. 12's CT step) into a workspace of its own, which is returned
        and which :meth:`swap_phase` takes."""
        self._check_images(images)
        n = _abi.recon_swap_workspace_size(self.plan)
        ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        _abi.recon_swap_ct(self.plan, images.data_ptr(), ws.data_ptr(), n, self._stream(stream))
        return ws

    def swap_phase(self, ws: torch.Tensor, sigma: float, eps: float, volume: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """``recon_swap_phase``: Eq. 12's 3D CTF inversion with (sigma, eps) of the spectrum
        that :meth:`swap_ct` left in ``ws``."""
        if volume is None:
            volume = self.new_volume()
        _abi.recon_swap_phase(self.plan, float(sigma), float(eps), volume.data_ptr(), ws.data_ptr(), ws.numel(),
                              self._stream(stream))
        return volume

    def grid_run(self, images: torch.Tensor, nsr: float = 0.0, volume: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
        """``recon_grid_run``: the Fourier-gridding UTR (with the NSR noise filter when nsr > 0)."""
        self._check_images(images)
        if volume is None:
            volume = self.new_volume()
        n = _abi.recon_grid_workspace_size(self.plan)
        ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        _abi.recon_grid_run(self.plan, images.data_ptr(), volume.data_ptr(), float(nsr), ws.data_ptr(), n,
                            self._stream(stream))
        return volume

    def close(self):
        if getattr(self, "plan", None) is not None:
            _abi.recon_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def train_mlp(weights, images: torch.Tensor, targets: torch.Tensor, rot, defocus, grid, *, nz_layers: int,
              lam: float, delta: float, sigma: float, nsr: float, cs: float = 0.0, input_mode: str = "intensity",
              steps: int = 200, lr: float = 1e-3, want_grad: bool = False, stream=None, adam_state=None,
              adam_step: int = 0):
    """``recon_mlp_train``: fits the regulariser network on the GPU.  ``images`` (N, nv, nu)
    and ``targets`` (N, Nz, nv, nu) are contiguous float32 CUDA tensors.  Returns
    (weights, loss history, gradient at the input weights when steps == 0 and want_grad).
    ``adam_state`` (float32 numpy [2 RECON_MLP_PARAMS], updated in place) and ``adam_step``
    continue one Adam optimisation over mini-batches passed in successive calls."""
    N, nv, nu = images.shape
    if tuple(targets.shape) != (N, nz_layers, nv, nu):
        raise ValueError("targets must be (N, nz_layers, nv, nu)")
    cfg, keep = _abi.make_train_cfg(rot, defocus, nu, nv, nz_layers, grid, lam, delta, sigma, cs, nsr,
                                    _INPUTS[input_mode], images.data_ptr(), targets.data_ptr(), steps, lr,
                                    adam_state, adam_step)
    ws_bytes = _abi.recon_mlp_train_workspace_size(cfg)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=images.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    out = _abi.recon_mlp_train(cfg, weights, ws.data_ptr(), ws_bytes, int(s.cuda_stream), want_grad)
    del keep
    return out


class Batch:
    """``recon_batch_*``: several :class:`Reconstructor` plans (uneven sizes) run together,
    stage A per tomogram and one persistent backprojection per round of ``dir_block``
    directions; ``run(..., graph=True)`` captures the launches once as a CUDA graph and
    replays it."""

    def __init__(self, recons, dir_block: int = 0, device=None):
        self.recons = list(recons)
        self.batch = _abi.recon_batch_create([r.plan for r in self.recons], dir_block)
        self.ws_bytes = _abi.recon_batch_workspace_size(self.batch)
        # recon_batch_run_host's workspace: the same plus two round slots of images
        self.ws_bytes_host = _abi.recon_batch_run_host_workspace_size(self.batch)
        dev = device if device is not None else self.recons[0].device if self.recons else None
        self.workspace = torch.empty(max(self.ws_bytes_host, 256), dtype=torch.uint8, device=dev)
        self.stream = None

    def run(self, images, volumes=None, graph: bool = False, stream=None):
        if volumes is None:
            volumes = [r.new_volume() for r in self.recons]
        for r, im in zip(self.recons, images):
            r._check_images(im)
        if graph:
            if stream is None:
                if self.stream is None:
                    self.stream = torch.cuda.Stream()
                stream = self.stream
            stream.wait_stream(torch.cuda.current_stream())
        s = stream if stream is not None else torch.cuda.current_stream()
        _abi.recon_batch_run(self.batch, [im.data_ptr() for im in images], [v.data_ptr() for v in volumes],
                             self.workspace.data_ptr(), self.ws_bytes, int(s.cuda_stream), graph)
        if graph:
            torch.cuda.current_stream().wait_stream(stream)
        return volumes

    def run_host(self, host_images, volumes=None, stream=None):
        """``recon_batch_run_host``: the images as contiguous float32 CPU tensors (pinned for the
        uploads to overlap the rounds); they must stay untouched until the stream's work has
        finished."""
        if volumes is None:
            volumes = [r.new_volume() for r in self.recons]
        for r, im in zip(self.recons, host_images):
            if im.dtype != torch.float32 or im.is_cuda or not im.is_contiguous():
                raise ValueError("host images must be contiguous float32 CPU tensors")
            if tuple(im.shape) != (r.D, r.nv, r.nu):
                raise ValueError(f"images shape {tuple(im.shape)} != {(r.D, r.nv, r.nu)}")
        s = stream if stream is not None else torch.cuda.current_stream()
        _abi.recon_batch_run_host(self.batch, [im.data_ptr() for im in host_images], [v.data_ptr() for v in volumes],
                                  self.workspace.data_ptr(), self.workspace.numel(), int(s.cuda_stream))
        return volumes

    def close(self):
        if getattr(self, "batch", None) is not None:
            _abi.recon_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
