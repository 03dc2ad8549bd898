"""recon_run_noalloc: the entry point for callers that may not allocate device memory
(components of a host application that owns the device memory, real-time loops in
which cudaMalloc/cudaFree are banned because they can synchronise the device, plugins
in processes whose allocator owns every byte).  It works in the library's static
device scratch; here it is called twice in a row through the C-ABI and each result is
checked against recon_run with a caller-provided workspace, within the float32 parity
tolerance of the other tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2206_09151_gb300 import _abi, phantoms as ph

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 3e-3


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()
    torch.cuda.init()


def rel_l2(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("n,D,nzl", [(64, 90, 8), (256, 12, 4)])
def test_noalloc_run_matches_recon_run_twice(n, D, nzl):
    cfg = ph.config_workload("small", scale_dirs=D)
    cfg["nu"] = cfg["nv"] = n
    cfg["grid"] = (n, n, n // 4)
    rng = np.random.default_rng(n + D)
    img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((D, n, n))).astype(np.float32)).cuda()
    opts = _abi.recon_default_options()
    opts.sigma, opts.eps = cfg["sigma"], cfg["eps"]
    plan = _abi.recon_plan(cfg["rot"], n, n, cfg["lam"], cfg["delta"], cfg["defocus"], nzl, cfg["grid"], opts)
    ws_bytes = _abi.recon_workspace_size(plan)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, nz = cfg["grid"]
    ref = torch.empty((nz, ny, nx), device="cuda")
    _abi.recon_run(plan, img.data_ptr(), ref.data_ptr(), ws.data_ptr(), ws_bytes, stream)
    for _ in range(2):
        vol = torch.full((nz, ny, nx), float("nan"), device="cuda")
        _abi.recon_run_noalloc(plan, img.data_ptr(), vol.data_ptr(), stream)
        _abi.recon_sync(stream)
        assert torch.isfinite(vol).all()
        assert rel_l2(vol, ref) <= TOL_F32
    _abi.recon_destroy(plan)


def test_noalloc_learned_filter_bf16_density_matches_recon_run_twice():
    """The learned regulariser keeps its power spectra and eps table in the static scratch
    (after the stacks), the bfloat16 stack and the sampling-density grid too: 64^2 images,
    Nz = 4, 24 directions of a 60-degree cone, against recon_run with its own workspace.
    The learned regulariser's radial power spectrum is summed with float atomics, so two
    runs differ in the last bits of eps and a few stack values round to the other
    bfloat16 neighbour: the bfloat16-stack tolerance of the other tests applies."""
    n, D, nzl = 64, 24, 4
    rot = ph.cone_rotations(D, 60.0, seed=11)
    rng = np.random.default_rng(5)
    img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((D, n, n))).astype(np.float32)).cuda()
    w = ph.mlp_init(17).astype(np.float32)
    opts = _abi.recon_default_options()
    opts.sigma, opts.filter, opts.nsr = 0.07, _abi.RECON_FILTER_MLP, 0.1
    opts.stack_dtype, opts.ramp_mode = _abi.RECON_STACK_BF16, _abi.RECON_RAMP_DENSITY
    opts.dir_block = 5  # several blocks on the caller-owned path
    opts.mlp_weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    grid = (n, n, 32)
    plan = _abi.recon_plan(rot, n, n, 1.97e-12, 1e-10, np.full(D, 1e-6), nzl, grid, opts)
    ws_bytes = _abi.recon_workspace_size(plan)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty((grid[2], grid[1], grid[0]), device="cuda")
    _abi.recon_run(plan, img.data_ptr(), ref.data_ptr(), ws.data_ptr(), ws_bytes, stream)
    for _ in range(2):
        vol = torch.full_like(ref, float("nan"))
        _abi.recon_run_noalloc(plan, img.data_ptr(), vol.data_ptr(), stream)
        _abi.recon_sync(stream)
        assert torch.isfinite(vol).all()
        assert rel_l2(vol, ref) <= TOL_BF16
    _abi.recon_destroy(plan)


def test_noalloc_refuses_a_plan_beyond_its_scratch():
    """1024x1024 images with 4 layers need ~59 MB of scratch per direction: refused
    before anything is launched."""
    rot = ph.single_axis_rotations(2)
    plan = _abi.recon_plan(rot, 1024, 1024, 1e-10, 1e-9, np.zeros(2), 4, (8, 8, 8))
    vol = torch.zeros((8, 8, 8), device="cuda")
    img = torch.ones((2, 1024, 1024), device="cuda")
    with pytest.raises(_abi.ReconError) as e:
        _abi.recon_run_noalloc(plan, img.data_ptr(), vol.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == _abi.RECON_E_UNSUPPORTED_SIZE
    assert "scratch" in str(e.value)
    _abi.recon_destroy(plan)
