"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle, element by element
on the same seeded inputs.  Tolerances: relative L2 <= 1e-5 with a float32 layer
stack and <= 3e-3 with a bfloat16 stack (the stated accuracy targets); layer
decisions are exact, so the worst voxel is also bounded."""
import math

import numpy as np
import pytest
import torch

import oracle as O
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
    torch.cuda.init()
    yield


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(rot, nu, nv, grid, **kw):
    from paper_2206_09151_gb300.recon import Reconstructor
    return Reconstructor(rot, nu, nv, grid, **kw)


# ---------------------------------------------------------------- stage A
STAGE_A_CASES = [
    # nu, nv, Nz, filter, input, cs, sigma, eps, lam, delta, R
    (64, 64, 8, "tikhonov", "intensity", 0.0, 0.01, 1e-2, 1e-10, 1e-9, 110e-9),
    (50, 37, 3, "tikhonov", "contrast", 2e-6, 0.2, 1e-3, 1e-10, 1e-9, 60e-9),
    (33, 200, 5, "off", "intensity", 0.0, 0.0, 0.1, 1e-10, 1e-9, 60e-9),
    (256, 256, 4, "tikhonov", "intensity", 2.7e-3, 0.07, 0.1, 1.97e-12, 1e-10, 1e-6),
    (1024, 1024, 2, "tikhonov", "intensity", 2.7e-3, 0.07, 0.1, 1.97e-12, 5e-11, 1e-6),
    (512, 400, 3, "tikhonov", "intensity", 2.7e-3, 0.07, 0.1, 1.97e-12, 1e-10, 1e-6),   # P = 1024, ragged rows
    (1000, 777, 3, "off", "contrast", 0.0, 0.0, 0.1, 1.97e-12, 5e-11, 1e-6),           # P = 2048, ragged both
    (1, 1, 1, "tikhonov", "intensity", 0.0, 0.1, 0.1, 1e-10, 1e-9, 1e-7),
    # the opposite-pair filter (Eq. 10 / 11): radix-2 path, 8-value and 16-value FFTs
    (3, 4, 2, "pair", "intensity", 0.0, 0.1, 0.05, 1e-10, 1e-9, 1e-7),
    (64, 50, 6, "pair", "intensity", 2e-6, 0.2, 1e-2, 1e-10, 1e-9, 60e-9),
    (256, 256, 4, "pair", "contrast", 2.7e-3, 0.07, 0.1, 1.97e-12, 1e-10, 1e-6),
    (700, 1000, 3, "pair", "intensity", 2.7e-3, 0.07, 0.1, 1.97e-12, 5e-11, 1e-6),
]


@pytest.mark.parametrize("case", STAGE_A_CASES, ids=lambda c: f"{c[0]}x{c[1]}_nz{c[2]}_{c[3]}_{c[4]}")
def test_stage_a_layer_stack_matches_oracle(case):
    nu, nv, nzl, filt, inp, cs, sigma, eps, lam, delta, R = case
    D = 3
    rng = np.random.default_rng(nu * 1000 + nv)
    rot = ph.single_axis_rotations(D, start=0.3)
    defocus = R * (1 + 0.1 * rng.random(D))
    grid = (max(nu, 8), max(nv, 8), max(nu // 2, 4))
    img = (1.0 + 1e-2 * rng.standard_normal((D, nv, nu))).astype(np.float32)
    if inp == "contrast":
        img = np.log(img).astype(np.float32)
    r = make(rot, nu, nv, grid, lam=lam, delta=delta, defocus=defocus, nz_layers=nzl, sigma=sigma, eps=eps,
             cs=cs, filter=filt, input_mode=inp, dir_block=D)
    dimg = torch.from_numpy(img).cuda()
    st = r.filter_stage(dimg, 0, D).float().cpu().numpy()
    torch.cuda.synchronize()
    zc = O.layer_centres(rot, grid, nzl, delta)
    for n in range(D):
        ref = O.layer_stack(img[n], delta=delta, lam=lam, r_n=defocus[n], z_layers=zc[n], n_dir=D, sigma=sigma,
                            eps=eps, cs=cs, filt={"tikhonov": O.FILTER_TIKHONOV, "pair": O.FILTER_PAIR,
                                                  "off": O.FILTER_OFF}[filt],
                            input_mode=O.INPUT_INTENSITY if inp == "intensity" else O.INPUT_CONTRAST)
        got = st[n, :, 1:-1, 1:, 0]  # pair (Y[u], Y[u+1]) at column u + 1
        for k in range(nzl):
            assert rel_l2(got[k], ref[k]) <= TOL_F32, (n, k, rel_l2(got[k], ref[k]))
        # pairs are consistent, and the border (rows 0 and nv+1, columns -1 and nu) is zero
        assert np.array_equal(st[n, :, :, :-1, 1], st[n, :, :, 1:, 0])
        assert not st[n, :, 0].any() and not st[n, :, -1].any()
        assert not st[n, :, :, 0, 0].any() and not st[n, :, :, -1, 1].any()
    r.close()


# ---------------------------------------------------------------- stage B
def _stage_b_case(grid, nu, nv, nzl, D, seed, start=0.1, span=math.pi, axis=None, bp_kernel="auto",
                  interp="nearest", rot=None):
    rng = np.random.default_rng(seed)
    if rot is None:
        rot = ph.single_axis_rotations(D, span=span, start=start, axis=axis)
    r = make(rot, nu, nv, grid, lam=1e-10, delta=1e-9, defocus=np.zeros(D), nz_layers=nzl, dir_block=D,
             bp_kernel=bp_kernel, layer_interp=interp)
    stacks = rng.standard_normal((D, nzl, nv, nu)).astype(np.float32)
    padded = np.zeros((D, nzl, nv + 2, nu + 2), np.float32)
    padded[:, :, 1:-1, 1:-1] = stacks
    pairs = np.stack([padded[..., :-1], padded[..., 1:]], axis=-1).copy()  # (Y[c-1], Y[c])
    vol = torch.full((grid[2], grid[1], grid[0]), 7.0, device="cuda")
    r.backproject(torch.from_numpy(pairs).cuda(), 0, D, vol, accumulate=False)
    got = vol.cpu().numpy()
    A, B = O.pixel_coefficients(rot, grid, nu, nv)
    T = O.layer_constants(rot, grid, nzl)
    kk, jj, ii = np.meshgrid(*(np.arange(g) for g in grid[::-1]), indexing="ij")
    i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
    ref = np.zeros(i.size)
    mode = O.LAYER_LINEAR if interp == "linear" else O.LAYER_NEAREST
    for n in range(D):
        ref += O.backproject_direction(stacks[n].astype(np.float64), A[n], B[n], T[n], i, j, k, mode)
    r.close()
    return got.ravel(), ref


@pytest.mark.parametrize("grid,nu,nv,nzl,D,axis", [
    ((37, 20, 9), 41, 23, 5, 7, None),          # half-integer row offset (two detector rows)
    ((64, 64, 64), 64, 64, 8, 90, None),
    ((33, 70, 130), 160, 72, 16, 11, None),
    ((20, 50, 10), 30, 24, 3, 5, None),         # volume taller than the detector
    ((20, 51, 10), 30, 24, 3, 5, None),         # ... with a half-integer offset
    ((1, 1, 1), 1, 1, 1, 2, None),
    ((37, 20, 9), 41, 23, 5, 7, (0.3, 1.0, -0.2)),   # tilted axis: general kernel
    ((48, 40, 56), 64, 64, 6, 30, (0.0, 1.0, 0.5)),
    ((64, 64, 64), 64, 64, 96, 12, None),       # thin layers: staged boxes overflow to direct loads
], ids=["y-half", "y-64", "y-tall", "y-rows-outside", "y-rows-outside-half", "y-1", "tilted", "tilted-2",
        "y-thin-layers"])
@pytest.mark.parametrize("bp_kernel", ["direct", "staged", "tma"])
def test_stage_b_backprojection_matches_oracle(grid, nu, nv, nzl, D, axis, bp_kernel):
    got, ref = _stage_b_case(grid, nu, nv, nzl, D, seed=sum(grid) + D, axis=axis, bp_kernel=bp_kernel)
    assert rel_l2(got, ref) <= TOL_F32
    # any layer or tap decided differently would show as an O(1) error at that voxel
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1.0)


@pytest.mark.parametrize("grid,nu,nv,nzl,D,axis", [
    ((37, 20, 9), 41, 23, 5, 7, None),          # single axis (runs in the general kernel)
    ((33, 70, 130), 160, 72, 16, 11, None),
    ((37, 20, 9), 41, 23, 5, 7, (0.3, 1.0, -0.2)),
    ((48, 40, 56), 64, 64, 6, 30, (0.0, 1.0, 0.5)),
    ((20, 20, 20), 24, 24, 1, 4, (0.2, 1.0, 0.1)),   # one layer: the blend is that layer
    ((64, 64, 64), 64, 64, 96, 12, (0.1, 1.0, 0.3)),
], ids=["y", "y-tall", "tilted", "tilted-2", "one-layer", "thin-layers"])
@pytest.mark.parametrize("bp_kernel", ["auto", "tma"])
def test_stage_b_layer_blend_matches_oracle(grid, nu, nv, nzl, D, axis, bp_kernel):
    """The blend of the two layers whose centres bracket each voxel's depth (exact 2^-24
    weights on both sides), voxel by voxel, in the general kernel and the TMA-staged one."""
    got, ref = _stage_b_case(grid, nu, nv, nzl, D, seed=sum(grid) + 3 * D, axis=axis, interp="linear",
                             bp_kernel=bp_kernel)
    assert rel_l2(got, ref) <= TOL_F32
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1.0)


# ---------------------------------------------------------------- whole operator
def _small_workload(n_dir=None):
    cfg = ph.config_workload("small", scale_dirs=n_dir)
    phan = ph.make_phantom(cfg)
    img = ph.multislice_images(phan, cfg["rot"], cfg["nu"], cfg["nv"], cfg["delta"], cfg["lam"], cfg["defocus"],
                               cfg["sigma"], photons=cfg["photons"], seed=cfg["seed"]).numpy()
    return cfg, img


@pytest.fixture(scope="module")
def small():
    cfg, img = _small_workload()
    ref = O.recon(img, cfg["rot"], lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"],
                  nz_layers=cfg["nz_layers"], grid=cfg["grid"], sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"])
    return cfg, img, ref


def _gpu_recon(cfg, img, **kw):
    r = make(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
             defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"],
             **kw)
    vol = r.run(torch.from_numpy(img).cuda())
    out = vol.cpu().numpy()
    r.close()
    return out


def test_small_workload_f32_matches_oracle(small):
    cfg, img, ref = small
    got = _gpu_recon(cfg, img)
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)


def test_small_workload_ragged_direction_blocks(small):
    cfg, img, ref = small
    got = _gpu_recon(cfg, img, dir_block=7)  # 90 = 12 * 7 + 6
    assert rel_l2(got, ref) <= TOL_F32


def test_small_workload_layer_blend_matches_oracle(small):
    """The whole operator with the layer blend (float32 stack) against the oracle's."""
    cfg, img, _ = small
    ref = O.recon(img, cfg["rot"], lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"],
                  nz_layers=cfg["nz_layers"], grid=cfg["grid"], sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"],
                  layer_interp=O.LAYER_LINEAR)
    got = _gpu_recon(cfg, img, layer_interp="linear")
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)
    got16 = _gpu_recon(cfg, img, layer_interp="linear", stack_dtype="bf16")
    assert rel_l2(got16, ref) <= TOL_BF16, rel_l2(got16, ref)


def test_pair_filter_whole_run_over_360_degrees_matches_oracle():
    """The opposite-pair filter on a 360-degree single-axis scan (every view has its
    opposite): 64^3, 60 views, Nz 8, the small workload's physics, against the oracle."""
    cfg = ph.config_workload("small", scale_dirs=60)
    cfg["rot"] = ph.single_axis_rotations(60, span=2 * math.pi)
    phan = ph.make_phantom(cfg)
    img = ph.multislice_images(phan, cfg["rot"], cfg["nu"], cfg["nv"], cfg["delta"], cfg["lam"], cfg["defocus"],
                               cfg["sigma"], photons=cfg["photons"], seed=cfg["seed"]).numpy()
    ref = O.recon(img, cfg["rot"], lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"],
                  nz_layers=cfg["nz_layers"], grid=cfg["grid"], sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"],
                  filt=O.FILTER_PAIR)
    got = _gpu_recon(cfg, img, filter="pair")
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)
    got16 = _gpu_recon(cfg, img, filter="pair", stack_dtype="bf16", layer_interp="nearest")
    assert rel_l2(got16, ref) <= TOL_BF16, rel_l2(got16, ref)


def test_small_workload_bf16_stack(small):
    cfg, img, ref = small
    got = _gpu_recon(cfg, img, stack_dtype="bf16")
    assert rel_l2(got, ref) <= TOL_BF16, rel_l2(got, ref)


@pytest.mark.parametrize("stack_dtype", ["f32", "bf16"])
def test_small_workload_staged_backprojection_equals_direct(small, stack_dtype):
    """Both single-axis kernels gather the same taps and add in the same order: the
    staged one (footprints copied to shared memory) gives the direct one's bits."""
    cfg, img, ref = small
    a = _gpu_recon(cfg, img, stack_dtype=stack_dtype, bp_kernel="direct")
    b = _gpu_recon(cfg, img, stack_dtype=stack_dtype, bp_kernel="staged")
    assert np.array_equal(a, b)


def test_accumulate_adds_and_empty_scan_clears():
    cfg, img = _small_workload(n_dir=6)
    r = make(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
             defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"])
    one = r.run(torch.from_numpy(img).cuda()).clone()
    r.close()
    ra = make(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
              defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
              accumulate=True)
    vol = one.clone()
    ra.run(torch.from_numpy(img).cuda(), vol)
    assert torch.allclose(vol, 2 * one, rtol=1e-6, atol=1e-6 * one.abs().max().item())
    ra.close()
    e = make(np.zeros((0, 3, 3)), 8, 8, (5, 6, 7), lam=1e-10, delta=1e-9, defocus=np.zeros(0), nz_layers=2)
    v = torch.full((7, 6, 5), 3.0, device="cuda")
    e.run(torch.zeros((0, 8, 8), device="cuda"), v)
    assert not v.any()
    e.close()


def test_check_finite_refuses_nan_and_inf_images():
    """check_finite: a NaN or an Inf anywhere in the images is reported as
    RECON_E_NONFINITE before anything is written; clean images run as usual."""
    from paper_2206_09151_gb300 import _abi
    cfg, img = _small_workload(n_dir=6)
    r = make(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
             defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
             check_finite=True)
    good = r.run(torch.from_numpy(img).cuda()).clone()
    assert torch.isfinite(good).all()
    for bad_value, where in ((float("nan"), (5, 63, 0)), (float("inf"), (0, 0, 17))):
        bad = img.copy()
        bad[where] = bad_value
        vol = torch.full_like(good, 7.0)
        with pytest.raises(_abi.ReconError) as e:
            r.run(torch.from_numpy(bad).cuda(), vol)
        assert e.value.code == _abi.RECON_E_NONFINITE
        assert bool((vol == 7.0).all())
    r.close()


def test_filter_off_is_independent_of_layer_count():
    """Filter off: every layer is the same ramp-filtered image, so Nz = 4 and Nz = 1 give
    bitwise the same volume (conventional FBP, Eq. 15)."""
    cfg, img = _small_workload(n_dir=10)
    kw = dict(lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"], filter="off")
    vols = []
    for nzl in (4, 1):
        r = make(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], nz_layers=nzl, **kw)
        vols.append(r.run(torch.from_numpy(img).cuda()).cpu())
        r.close()
    assert torch.equal(vols[0], vols[1])


# ---------------------------------------------------------------- arbitrary geometry (density weighting)
@pytest.mark.parametrize("nu,nv,nzl,D", [(40, 36, 3, 9), (64, 64, 4, 30), (200, 190, 2, 5)])
def test_stage_a_density_weighting_matches_oracle(nu, nv, nzl, D):
    rng = np.random.default_rng(nu + D)
    rot = ph.cone_rotations(D, 60.0, seed=nu)
    defocus = rng.uniform(50e-9, 80e-9, D)
    grid = (nu, nv, 24)
    lam, delta, sigma, eps = 1e-10, 1e-9, 0.1, 1e-2
    img = (1.0 + 1e-2 * rng.standard_normal((D, nv, nu))).astype(np.float32)
    r = make(rot, nu, nv, grid, lam=lam, delta=delta, defocus=defocus, nz_layers=nzl, sigma=sigma, eps=eps,
             ramp="density", dir_block=D)
    st = r.filter_stage(torch.from_numpy(img).cuda(), 0, D).float().cpu().numpy()
    r.close()
    W = O.density_weights(rot, O.padded_size(max(nu, nv)), delta)
    zc = O.layer_centres(rot, grid, nzl, delta)
    for n in range(D):
        ref = O.layer_stack(img[n], delta=delta, lam=lam, r_n=defocus[n], z_layers=zc[n], n_dir=D, sigma=sigma,
                            eps=eps, cs=0.0, filt=O.FILTER_TIKHONOV, input_mode=O.INPUT_INTENSITY, weight=W[n])
        for k in range(nzl):
            assert rel_l2(st[n, k, 1:-1, 1:, 0], ref[k]) <= TOL_F32


def test_arbitrary_geometry_whole_run_matches_oracle():
    """Haar-random directions in a 60-degree cone (a tilted-slab scan), density weighting,
    layered Tikhonov filter: the whole operator against the oracle."""
    n, D, nzl = 32, 40, 4
    grid = (n, n, 16)
    rng = np.random.default_rng(77)
    rot = ph.cone_rotations(D, 60.0, seed=12)
    defocus = rng.uniform(40e-9, 60e-9, D)
    phan = ph.blob_phantom((n, n, 16), 12, seed=3, s_vox=1.5, amp_unit=3e-6)
    img = ph.multislice_images(phan, rot, n, n, 1e-9, 2e-10, defocus, 0.05, n_slabs=8, photons=1e5, seed=4).numpy()
    kw = dict(lam=2e-10, delta=1e-9, defocus=defocus, nz_layers=nzl, sigma=0.05, eps=1e-2)
    ref = O.recon(img, rot, grid=grid, density=True, **kw)
    r = make(rot, n, n, grid, ramp="density", **kw)
    got = r.run(torch.from_numpy(img).cuda()).cpu().numpy()
    r.close()
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)
