"""ctypes binding of ``include/recon.h``: the same entry points, argument marshalling
only.  Every step of the reconstruction runs in ``librecon.so``'s CUDA kernels;
there is no Python or CPU fallback -- a missing library raises."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librecon.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "recon.h")

RECON_OK = 0
RECON_E_INVALID_ARG = -1
RECON_E_UNSUPPORTED_SIZE = -2
RECON_E_CUDA = -3
RECON_E_WORKSPACE = -4
RECON_E_NO_MEMORY = -5
RECON_E_NONFINITE = -6
RECON_E_NO_WEIGHTS = -7
RECON_E_DEVICE_CHECK = -8

RECON_FILTER_OFF = 0
RECON_FILTER_TIKHONOV = 1
RECON_FILTER_MLP = 2
RECON_FILTER_PAIR = 3
RECON_MLP_PARAMS = 4481
RECON_INPUT_INTENSITY = 0
RECON_INPUT_CONTRAST = 1
RECON_STACK_F32 = 0
RECON_STACK_BF16 = 1
RECON_RAMP_SINGLE_AXIS = 0
RECON_RAMP_DENSITY = 1
RECON_BP_AUTO, RECON_BP_DIRECT, RECON_BP_STAGED, RECON_BP_TMA = 0, 1, 2, 3
RECON_LAYER_NEAREST, RECON_LAYER_LINEAR = 0, 1
RECON_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
RECON_MAX_LAYERS = 96


class ReconGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class ReconGeometry(ctypes.Structure):
    _fields_ = [("n_dir", ctypes.c_int), ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("rot", ctypes.POINTER(ctypes.c_double))]


class ReconOptions(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("eps", ctypes.c_double), ("cs", ctypes.c_double),
                ("filter", ctypes.c_int), ("input_mode", ctypes.c_int), ("stack_dtype", ctypes.c_int),
                ("ramp_mode", ctypes.c_int), ("accumulate", ctypes.c_int), ("dir_block", ctypes.c_int),
                ("mlp_weights", ctypes.POINTER(ctypes.c_float)), ("nsr", ctypes.c_double),
                ("stage_block", ctypes.c_int), ("bp_kernel", ctypes.c_int), ("check_finite", ctypes.c_int),
                ("layer_interp", ctypes.c_int), ("bp_warp", ctypes.c_int), ("mlp_views", ctypes.c_double),
                ("bp_tile_z", ctypes.c_int)]


class ReconTrainCfg(ctypes.Structure):
    _fields_ = [("n_img", ctypes.c_int), ("nu", ctypes.c_int), ("nv", ctypes.c_int), ("nz_layers", ctypes.c_int),
                ("rot", ctypes.POINTER(ctypes.c_double)), ("defocus", ctypes.POINTER(ctypes.c_double)),
                ("grid_nx", ctypes.c_int), ("grid_ny", ctypes.c_int), ("grid_nz", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("delta", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cs", ctypes.c_double), ("nsr", ctypes.c_double), ("input_mode", ctypes.c_int),
                ("images", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("steps", ctypes.c_int),
                ("lr", ctypes.c_float), ("adam_state", ctypes.POINTER(ctypes.c_float)), ("adam_step", ctypes.c_int)]


class ReconError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {message} [{code}]")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads ``librecon.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2206_09151_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, sz, ip = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    L.recon_default_options.argtypes = [ctypes.POINTER(ReconOptions)]
    L.recon_default_options.restype = None
    L.recon_plan.argtypes = [ctypes.POINTER(ReconGeometry), ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double), ip, ctypes.POINTER(ReconGrid),
                             ctypes.POINTER(ReconOptions), ctypes.POINTER(vp)]
    L.recon_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_run.argtypes = [vp, vp, vp, vp, sz, vp]
    L.recon_run_host.argtypes = [vp, vp, vp, vp, sz, vp]
    L.recon_run_host_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_filter_stage.argtypes = [vp, vp, ip, ip, vp, sz, vp, ctypes.POINTER(vp)]
    L.recon_backproject.argtypes = [vp, vp, ip, ip, vp, ip, vp, sz, vp]
    L.recon_plan_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.recon_run_noalloc.argtypes = [vp, vp, vp, vp]
    L.recon_plan_dof.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.recon_plan_layers.argtypes = [vp, ctypes.POINTER(ip)]
    L.recon_plan_bp_kernel.argtypes = [vp, ctypes.POINTER(ip)]
    L.recon_swap_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_swap_ct.argtypes = [vp, vp, vp, sz, vp]
    L.recon_swap_phase.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp, sz, vp]
    L.recon_grid_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_grid_run.argtypes = [vp, vp, vp, ctypes.c_double, vp, sz, vp]
    L.recon_plan_warning.argtypes = [vp]
    L.recon_plan_warning.restype = ctypes.c_char_p
    L.recon_layers_for_dof.argtypes = [ctypes.POINTER(ReconGeometry), ctypes.POINTER(ReconGrid), ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(ip)]
    L.recon_mlp_train_workspace_size.argtypes = [ctypes.POINTER(ReconTrainCfg), ctypes.POINTER(sz)]
    L.recon_mlp_train.argtypes = [ctypes.POINTER(ReconTrainCfg), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), vp, sz, vp]
    pp = ctypes.POINTER(vp)
    L.recon_batch_create.argtypes = [ip, pp, ip, pp]
    L.recon_batch_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_batch_run.argtypes = [vp, pp, pp, vp, sz, vp]
    L.recon_batch_run_graph.argtypes = [vp, pp, pp, vp, sz, vp]
    L.recon_batch_run_host.argtypes = [vp, pp, pp, vp, sz, vp]
    L.recon_batch_run_host_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.recon_batch_destroy.argtypes = [vp]
    L.recon_run_batch_workspace_size.argtypes = [ip, pp, ctypes.POINTER(sz)]
    L.recon_run_batch.argtypes = [ip, pp, pp, pp, vp, sz, vp]
    L.recon_profile_enable.argtypes = [vp, ip]
    L.recon_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ip)]
    L.recon_sync.argtypes = [vp]
    L.recon_selftest_wait_limit.argtypes = [vp]
    L.recon_destroy.argtypes = [vp]
    L.recon_error_string.argtypes = [ip]
    L.recon_error_string.restype = ctypes.c_char_p
    L.recon_last_error.argtypes = []
    L.recon_last_error.restype = ctypes.c_char_p
    for name in ("recon_plan", "recon_workspace_size", "recon_run", "recon_filter_stage", "recon_backproject",
                 "recon_plan_info", "recon_sync", "recon_destroy", "recon_profile_enable", "recon_profile_read",
                 "recon_run_noalloc", "recon_mlp_train_workspace_size", "recon_mlp_train", "recon_batch_create",
                 "recon_batch_workspace_size", "recon_batch_run", "recon_batch_run_graph", "recon_batch_destroy",
                 "recon_run_batch_workspace_size", "recon_run_batch", "recon_plan_dof", "recon_layers_for_dof",
                 "recon_plan_layers", "recon_swap_workspace_size", "recon_swap_ct", "recon_swap_phase",
                 "recon_grid_workspace_size", "recon_grid_run", "recon_selftest_wait_limit", "recon_plan_bp_kernel",
                 "recon_run_host", "recon_run_host_workspace_size", "recon_batch_run_host",
                 "recon_batch_run_host_workspace_size"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def header_entry_points(path: str = HEADER) -> list[str]:
    """Names of the functions ``include/recon.h`` declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z_0-9]+)\s*\(", text)))


def _check(rc: int, where: str):
    if rc != RECON_OK:
        L = load_library()
        raise ReconError(rc, where, L.recon_last_error().decode() or L.recon_error_string(rc).decode())


def recon_default_options() -> ReconOptions:
    o = ReconOptions()
    load_library().recon_default_options(ctypes.byref(o))
    return o


def recon_plan(rot: np.ndarray, nu: int, nv: int, lam: float, delta: float, defocus, nz_layers: int, grid,
               opts: ReconOptions | None = None) -> ctypes.c_void_p:
    """Marshals the arguments of ``recon_plan``; returns the plan handle."""
    L = load_library()
    rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 3, 3)
    defocus = np.ascontiguousarray(defocus, dtype=np.float64).reshape(-1)
    geom = ReconGeometry(rot.shape[0], nu, nv, rot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    g = ReconGrid(*grid)
    out = ctypes.c_void_p()
    rc = L.recon_plan(ctypes.byref(geom), lam, delta, defocus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      nz_layers, ctypes.byref(g), ctypes.byref(opts) if opts is not None else None, ctypes.byref(out))
    _check(rc, "recon_plan")
    return out


def make_train_cfg(rot, defocus, nu, nv, nz_layers, grid, lam, delta, sigma, cs, nsr, input_mode, images_ptr,
                   targets_ptr, steps, lr, adam_state=None, adam_step=0):
    """A recon_train_cfg; returns it with the host arrays it points to (keep both alive).
    ``adam_state`` (float32 [2 RECON_MLP_PARAMS], updated in place) carries Adam's moments
    from one call to the next."""
    rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 3, 3)
    defocus = np.ascontiguousarray(defocus, dtype=np.float64).reshape(-1)
    fp = ctypes.POINTER(ctypes.c_float)
    if adam_state is not None and (adam_state.dtype != np.float32 or adam_state.size != 2 * RECON_MLP_PARAMS
                                   or not adam_state.flags["C_CONTIGUOUS"]):
        raise ValueError("adam_state must be a contiguous float32 array of 2 * RECON_MLP_PARAMS values")
    cfg = ReconTrainCfg(rot.shape[0], nu, nv, nz_layers, rot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        defocus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), grid[0], grid[1], grid[2], lam,
                        delta, sigma, cs, nsr, input_mode, images_ptr, targets_ptr, steps, lr,
                        adam_state.ctypes.data_as(fp) if adam_state is not None else None, int(adam_step))
    return cfg, (rot, defocus, adam_state)


def recon_mlp_train_workspace_size(cfg: ReconTrainCfg) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_mlp_train_workspace_size(ctypes.byref(cfg), ctypes.byref(n)),
           "recon_mlp_train_workspace_size")
    return n.value


def recon_mlp_train(cfg: ReconTrainCfg, weights: np.ndarray, ws_ptr: int, ws_bytes: int, stream: int,
                    want_grad: bool = False):
    """Runs the training; returns (weights, loss history, gradient or None)."""
    w = np.ascontiguousarray(weights, dtype=np.float32).copy()
    if w.size != RECON_MLP_PARAMS:
        raise ValueError("weights must hold RECON_MLP_PARAMS values")
    loss = np.zeros(max(cfg.steps, 1), np.float32)
    grad = np.zeros(RECON_MLP_PARAMS, np.float32) if want_grad else None
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load_library().recon_mlp_train(ctypes.byref(cfg), w.ctypes.data_as(fp), loss.ctypes.data_as(fp),
                                          grad.ctypes.data_as(fp) if grad is not None else None, ws_ptr, ws_bytes,
                                          stream), "recon_mlp_train")
    return w, loss, grad


def recon_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_workspace_size(plan, ctypes.byref(n)), "recon_workspace_size")
    return n.value


def recon_plan_info(plan) -> tuple[int, int, int, int]:
    """(padded FFT size, directions per block, blocks, directions per FFT/filter sub-block)"""
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().recon_plan_info(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "recon_plan_info")
    return a.value, b.value, c.value, d.value


def recon_plan_dof(plan) -> tuple[float, float]:
    """(largest layer pitch over the directions, depth of field Delta^2 / (2 lambda)), metres."""
    h, d = ctypes.c_double(), ctypes.c_double()
    _check(load_library().recon_plan_dof(plan, ctypes.byref(h), ctypes.byref(d)), "recon_plan_dof")
    return h.value, d.value


def recon_plan_layers(plan) -> int:
    n = ctypes.c_int()
    _check(load_library().recon_plan_layers(plan, ctypes.byref(n)), "recon_plan_layers")
    return n.value


def recon_plan_bp_kernel(plan) -> int:
    k = ctypes.c_int()
    _check(load_library().recon_plan_bp_kernel(plan, ctypes.byref(k)), "recon_plan_bp_kernel")
    return k.value


def recon_plan_warning(plan) -> str:
    return load_library().recon_plan_warning(plan).decode()


def recon_layers_for_dof(rot: np.ndarray, grid, lam: float, delta: float) -> int:
    """Smallest Nz whose layers are no thicker than the depth of field for every direction."""
    rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 3, 3)
    geom = ReconGeometry(rot.shape[0], 1, 1, rot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    g = ReconGrid(*grid)
    nz = ctypes.c_int()
    _check(load_library().recon_layers_for_dof(ctypes.byref(geom), ctypes.byref(g), lam, delta, ctypes.byref(nz)),
           "recon_layers_for_dof")
    return nz.value


def recon_run(plan, images_ptr: int, volume_ptr: int, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_run(plan, images_ptr, volume_ptr, ws_ptr, ws_bytes, stream), "recon_run")


def recon_run_host_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_run_host_workspace_size(plan, ctypes.byref(n)), "recon_run_host_workspace_size")
    return n.value


def recon_run_host(plan, host_images_ptr: int, volume_ptr: int, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_run_host(plan, host_images_ptr, volume_ptr, ws_ptr, ws_bytes, stream),
           "recon_run_host")


def recon_swap_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_swap_workspace_size(plan, ctypes.byref(n)), "recon_swap_workspace_size")
    return n.value


def recon_swap_ct(plan, images_ptr: int, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_swap_ct(plan, images_ptr, ws_ptr, ws_bytes, stream), "recon_swap_ct")


def recon_swap_phase(plan, sigma: float, eps: float, volume_ptr: int, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_swap_phase(plan, sigma, eps, volume_ptr, ws_ptr, ws_bytes, stream), "recon_swap_phase")


def recon_grid_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_grid_workspace_size(plan, ctypes.byref(n)), "recon_grid_workspace_size")
    return n.value


def recon_grid_run(plan, images_ptr: int, volume_ptr: int, nsr: float, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_grid_run(plan, images_ptr, volume_ptr, nsr, ws_ptr, ws_bytes, stream), "recon_grid_run")


def recon_run_noalloc(plan, images_ptr: int, volume_ptr: int, stream: int):
    """``recon_run`` in the library's static device scratch (no allocation anywhere)."""
    _check(load_library().recon_run_noalloc(plan, images_ptr, volume_ptr, stream), "recon_run_noalloc")


def recon_filter_stage(plan, images_ptr: int, dir_begin: int, dir_count: int, ws_ptr: int, ws_bytes: int,
                       stream: int) -> int:
    out = ctypes.c_void_p()
    _check(load_library().recon_filter_stage(plan, images_ptr, dir_begin, dir_count, ws_ptr, ws_bytes, stream,
                                             ctypes.byref(out)), "recon_filter_stage")
    return out.value


def recon_backproject(plan, stack_ptr: int, dir_begin: int, dir_count: int, volume_ptr: int, accumulate: int,
                      ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_backproject(plan, stack_ptr, dir_begin, dir_count, volume_ptr, accumulate, ws_ptr,
                                            ws_bytes, stream), "recon_backproject")


def recon_profile_enable(plan, enable: bool):
    _check(load_library().recon_profile_enable(plan, int(bool(enable))), "recon_profile_enable")


def recon_profile_read(plan) -> tuple[list[float], list[int]]:
    """Summed milliseconds and launch counts of (row FFT, column filter/iFFT, row iFFT,
    backprojection) over the plan's last profiled run."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int * 4)()
    _check(load_library().recon_profile_read(plan, ms, n), "recon_profile_read")
    return list(ms), list(n)


def _ptrs(values):
    arr = (ctypes.c_void_p * max(len(values), 1))()
    for i, v in enumerate(values):
        arr[i] = v
    return arr


def recon_batch_create(plans, dir_block: int = 0):
    out = ctypes.c_void_p()
    _check(load_library().recon_batch_create(len(plans), _ptrs([p.value for p in plans]), dir_block,
                                             ctypes.byref(out)), "recon_batch_create")
    return out


def recon_batch_workspace_size(batch) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_batch_workspace_size(batch, ctypes.byref(n)), "recon_batch_workspace_size")
    return n.value


def recon_batch_run_host_workspace_size(batch) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_batch_run_host_workspace_size(batch, ctypes.byref(n)),
           "recon_batch_run_host_workspace_size")
    return n.value


def recon_batch_run_host(batch, host_image_ptrs, volume_ptrs, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_batch_run_host(batch, _ptrs(host_image_ptrs), _ptrs(volume_ptrs), ws_ptr, ws_bytes,
                                               stream), "recon_batch_run_host")


def recon_batch_run(batch, image_ptrs, volume_ptrs, ws_ptr: int, ws_bytes: int, stream: int, graph: bool = False):
    L = load_library()
    fn = L.recon_batch_run_graph if graph else L.recon_batch_run
    _check(fn(batch, _ptrs(image_ptrs), _ptrs(volume_ptrs), ws_ptr, ws_bytes, stream),
           "recon_batch_run_graph" if graph else "recon_batch_run")


def recon_batch_destroy(batch):
    load_library().recon_batch_destroy(batch)


def recon_run_batch_workspace_size(plans) -> int:
    n = ctypes.c_size_t()
    _check(load_library().recon_run_batch_workspace_size(len(plans), _ptrs([p.value for p in plans]),
                                                         ctypes.byref(n)), "recon_run_batch_workspace_size")
    return n.value


def recon_run_batch(plans, image_ptrs, volume_ptrs, ws_ptr: int, ws_bytes: int, stream: int):
    _check(load_library().recon_run_batch(len(plans), _ptrs([p.value for p in plans]), _ptrs(image_ptrs),
                                          _ptrs(volume_ptrs), ws_ptr, ws_bytes, stream), "recon_run_batch")


def recon_sync(stream: int):
    _check(load_library().recon_sync(stream), "recon_sync")


def recon_selftest_wait_limit(stream: int) -> int:
    """The status of the TMA-staged backprojection's wait-limit self-test (RECON_OK when its
    waits ran out after their limit and the kernel reported it)."""
    return int(load_library().recon_selftest_wait_limit(stream))


def recon_destroy(plan):
    load_library().recon_destroy(plan)


def recon_error_string(code: int) -> str:
    return load_library().recon_error_string(code).decode()


def recon_last_error() -> str:
    return load_library().recon_last_error().decode()
