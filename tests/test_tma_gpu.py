"""The TMA-staged backprojection (``bp_kernel="tma"``): every (16 x 16 x 8 voxel tile,
direction) footprint box of the layer stack is copied into a shared-memory ring by one
``cp.async.bulk.tensor`` load.  Its volumes must match the FP64 oracle at the stated
tolerances and the direct general kernel to rounding, for float32 and bfloat16 stacks,
nearest layer and the layer blend, tiles partly outside the volume, footprints partly
outside the detector and several direction blocks; its bounded waits must report a
run-out wait through the status word and leave the context usable."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2206_09151_gb300 import _abi
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 3e-3


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cone_case(n=40, nu=36, D=23, nz=16, seed=5):
    """A single-axis scan about a tilted axis over 360 degrees (every in-plane orientation
    of the footprints, and deterministic single-axis ramp weights): the detector (nu^2) is
    smaller than the volume's projection, so footprints leave the detector; the grid is not
    a multiple of the 16 x 16 x 8 tile."""
    rng = np.random.default_rng(seed)
    rot = ph.single_axis_rotations(D, span=2 * np.pi, start=0.3, axis=(0.2, 0.9, 0.4))
    grid = (n, n + 5, nz + 3)
    img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((D, nu, nu))).astype(np.float32)).cuda()
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 80e-9, D), sigma=0.05, eps=0.02)
    return rot, nu, grid, img, kw


def _run(rot, nu, grid, img, kw, **extra):
    from paper_2206_09151_gb300.recon import Reconstructor
    r = Reconstructor(rot, nu, nu, grid, **kw, **extra)
    v = r.run(img).cpu().numpy()
    r.close()
    return v


_ORACLE = {}


def _oracle(interp):
    """The FP64 oracle's volume of the tilted-axis case (cached per layer mode)."""
    if interp not in _ORACLE:
        rot, nu, grid, img, kw = _cone_case()
        _ORACLE[interp] = O.recon(img.cpu().numpy(), rot, grid=grid, nz_layers=7,
                                  layer_interp=O.LAYER_LINEAR if interp == "linear" else O.LAYER_NEAREST, **kw)
    return _ORACLE[interp]


@pytest.mark.parametrize("stack_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("interp", ["nearest", "linear"])
@pytest.mark.parametrize("dir_block", [0, 6])
def test_tma_matches_oracle_and_the_direct_general_kernel(stack_dtype, interp, dir_block):
    rot, nu, grid, img, kw = _cone_case()
    common = dict(nz_layers=7, stack_dtype=stack_dtype, layer_interp=interp, dir_block=dir_block)
    a = _run(rot, nu, grid, img, kw, bp_kernel="direct", **common)
    b = _run(rot, nu, grid, img, kw, bp_kernel="tma", **common)
    ref = _oracle(interp)
    tol = TOL_F32 if stack_dtype == "f32" else TOL_BF16
    assert rel_l2(b, ref) <= tol, rel_l2(b, ref)
    # the same stack, taps and weights: only the FP32 rounding of the in-tile coordinates
    # (box-local instead of tile-local origins) differs from the direct kernel
    assert rel_l2(b, a) <= TOL_F32, rel_l2(b, a)
    assert np.max(np.abs(b - a)) <= 1e-4 * np.max(np.abs(a))


def test_tma_whole_run_matches_oracle():
    """Cone geometry with sampling-density weighting: the whole operator through the
    TMA-staged kernel against the oracle (float32 and bfloat16 stacks)."""
    n, D, nzl = 32, 30, 4
    grid = (n, n, 16)
    rng = np.random.default_rng(78)
    rot = ph.cone_rotations(D, 60.0, seed=13)
    defocus = rng.uniform(40e-9, 60e-9, D)
    phan = ph.blob_phantom(grid, 12, seed=4, s_vox=1.5, amp_unit=3e-6)
    img = ph.multislice_images(phan, rot, n, n, 1e-9, 2e-10, defocus, 0.05, n_slabs=8, photons=1e5, seed=5).numpy()
    kw = dict(lam=2e-10, delta=1e-9, defocus=defocus, nz_layers=nzl, sigma=0.05, eps=1e-2)
    ref = O.recon(img, rot, grid=grid, density=True, **kw)
    dimg = torch.from_numpy(img).cuda()
    got = _run(rot, n, grid, dimg, kw, ramp="density", bp_kernel="tma")
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)
    got16 = _run(rot, n, grid, dimg, kw, ramp="density", bp_kernel="tma", stack_dtype="bf16")
    assert rel_l2(got16, ref) <= TOL_BF16, rel_l2(got16, ref)


def test_tma_single_axis_scan_and_accumulate():
    """A single-axis scan through the TMA-staged kernel equals the single-axis kernel to
    rounding, and accumulate adds onto the volume."""
    from paper_2206_09151_gb300.recon import Reconstructor
    cfg = ph.config_workload("small", scale_dirs=24)
    rng = np.random.default_rng(3)
    img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((24, cfg["nv"], cfg["nu"]))).astype(np.float32)).cuda()
    kw = dict(lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"], nz_layers=cfg["nz_layers"],
              sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"])
    vols = {}
    for k in ("direct", "tma"):
        r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], bp_kernel=k, **kw)
        vols[k] = r.run(img).cpu().numpy()
        r.close()
    assert rel_l2(vols["tma"], vols["direct"]) <= TOL_F32
    # accumulating onto the run's own volume doubles it exactly (the kernel is deterministic)
    r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], bp_kernel="tma", accumulate=True, **kw)
    v = torch.from_numpy(vols["tma"]).cuda()
    r.run(img, v)
    r.close()
    assert np.array_equal(v.cpu().numpy(), 2 * vols["tma"])


def test_tma_wait_limit_reports_and_leaves_the_context_usable():
    """The self-test launches the kernel with a producer that issues nothing: every
    consumer wait runs out after its limit, the kernel sets its status bit and returns,
    and the call reports it; a normal run afterwards still matches the direct kernel."""
    s = torch.cuda.current_stream()
    assert _abi.recon_selftest_wait_limit(int(s.cuda_stream)) == _abi.RECON_OK, _abi.recon_last_error()
    rot, nu, grid, img, kw = _cone_case(n=24, nu=24, D=5, nz=8, seed=9)
    a = _run(rot, nu, grid, img, kw, nz_layers=3, bp_kernel="direct")
    b = _run(rot, nu, grid, img, kw, nz_layers=3, bp_kernel="tma")
    assert rel_l2(b, a) <= TOL_F32


def test_tile_depths_agree_and_the_tuner_picks_one():
    """16 x 16 x 8 and 16 x 16 x 16 tiles: both match the oracle and each other to rounding
    (the box-local origins differ), and the autotuner returns one of the timed depths."""
    from paper_2206_09151_gb300.autotune import tune_bp_tile
    rot, nu, grid, img, kw = _cone_case()
    ref = _oracle("nearest")
    vols = {}
    for tz in (8, 16):
        vols[tz] = _run(rot, nu, grid, img, kw, nz_layers=7, bp_kernel="tma", bp_tile_z=tz)
        assert rel_l2(vols[tz], ref) <= TOL_F32, (tz, rel_l2(vols[tz], ref))
    assert rel_l2(vols[8], vols[16]) <= TOL_F32
    out = tune_bp_tile(rot, nu, nu, grid, img, nz_layers=7, candidates=(8, 16), repeats=2, **kw)
    assert out["bp_tile_z"] in (8, 16) and set(out["ms"]) == {"8", "16"}
