"""Batches of uneven tomograms: one persistent backprojection per round over all
tomograms' voxel tiles, optionally replayed as a CUDA graph.  Each volume must match the
same plan run alone (and the FP64 oracle for one of them)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _tomograms():
    """Seeded uneven tomograms: grids 24..64, images 24..72, 7..70 directions, 1..8
    layers; single-axis and cone geometries (density weighting), float32 and bfloat16
    stacks, a learned-filter one, an accumulating one and two with the layer blend."""
    rng = np.random.default_rng(41)
    specs = [
        dict(n=64, nu=64, D=70, nz=8, ramp="single_axis", stack="f32"),
        dict(n=40, nu=48, D=33, nz=4, ramp="single_axis", stack="bf16"),
        dict(n=24, nu=24, D=7, nz=1, ramp="single_axis", stack="f32", filter="off"),
        dict(n=48, nu=56, D=40, nz=3, ramp="density", stack="f32"),
        dict(n=32, nu=72, D=35, nz=5, ramp="single_axis", stack="f32", filter="mlp"),
        dict(n=36, nu=40, D=12, nz=2, ramp="single_axis", stack="f32", accumulate=True),
        dict(n=30, nu=30, D=0, nz=2, ramp="single_axis", stack="f32"),
        dict(n=40, nu=40, D=25, nz=6, ramp="single_axis", stack="f32", interp="linear"),
        dict(n=32, nu=36, D=20, nz=4, ramp="density", stack="bf16", interp="linear"),
    ]
    out = []
    for q, sp in enumerate(specs):
        n, nu, D = sp["n"], sp["nu"], sp["D"]
        grid = (n, n + 3 * q, max(8, n // 2))
        if sp["ramp"] == "density":
            rot = ph.cone_rotations(D, 60.0, seed=q)
        else:
            rot = ph.single_axis_rotations(D, start=0.1 * q)
        R = rng.uniform(50e-9, 80e-9, D)
        img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((D, nu, nu))).astype(np.float32)).cuda()
        kw = dict(lam=1e-10, delta=1e-9, defocus=R, nz_layers=sp["nz"], sigma=0.05, eps=0.02, ramp=sp["ramp"],
                  stack_dtype=sp["stack"], filter=sp.get("filter", "tikhonov"),
                  accumulate=sp.get("accumulate", False), layer_interp=sp.get("interp", "nearest"))
        if kw["filter"] == "mlp":
            kw.update(mlp_weights=ph.mlp_init(q).astype(np.float32), nsr=1e-2)
        out.append((rot, nu, grid, kw, img))
    return out


def _single_runs(toms):
    from paper_2206_09151_gb300.recon import Reconstructor
    recons, refs = [], []
    for rot, nu, grid, kw, img in toms:
        r = Reconstructor(rot, nu, nu, grid, **kw)
        v = torch.full((grid[2], grid[1], grid[0]), 0.5, device="cuda")
        r.run(img, v)
        refs.append(v.cpu().numpy())
        recons.append(r)
    return recons, refs


@pytest.mark.parametrize("dir_block", [0, 16])
def test_batch_matches_single_runs(dir_block):
    from paper_2206_09151_gb300.recon import Batch
    toms = _tomograms()
    recons, refs = _single_runs(toms)
    b = Batch(recons, dir_block=dir_block)
    vols = [torch.full((g[2], g[1], g[0]), 0.5, device="cuda") for _, _, g, _, _ in toms]
    b.run([t[4] for t in toms], vols)
    for q, (v, ref) in enumerate(zip(vols, refs)):
        got = v.cpu().numpy()
        if toms[q][3]["stack_dtype"] == "bf16":
            assert rel_l2(got, ref) <= 1e-3, q
        elif toms[q][1] and toms[q][0].shape[0] == 0:
            assert not got.any()
        else:
            assert rel_l2(got, ref) <= 1e-5, (q, rel_l2(got, ref))
    b.close()
    for r in recons:
        r.close()


def _same(q, toms, a, c):
    """Bitwise for the deterministic tomograms; the density splat and the learned path's
    power spectrum sum with float atomics, whose order varies from run to run (with a
    bfloat16 stack a few values then round to the other neighbour: the bfloat16
    tolerance applies)."""
    kw = toms[q][3]
    if kw["ramp"] == "density" or kw["filter"] == "mlp":
        if kw["stack_dtype"] == "bf16":
            return rel_l2(a.cpu().numpy(), c.cpu().numpy()) <= 3e-3
        return torch.allclose(a, c, rtol=1e-6, atol=1e-6 * float(c.abs().max()))
    return torch.equal(a, c)


def test_batch_graph_replays_are_identical_to_the_run():
    from paper_2206_09151_gb300.recon import Batch
    toms = _tomograms()
    recons, _ = _single_runs(toms)
    b = Batch(recons)
    imgs = [t[4] for t in toms]
    v1 = [r.new_volume().fill_(0.5) for r in recons]
    b.run(imgs, v1)
    torch.cuda.synchronize()
    for _ in range(2):
        v2 = [r.new_volume().fill_(0.5) for r in recons]
        b.run(imgs, v2, graph=True)  # pointers change: captured again, then replayed below
        torch.cuda.synchronize()
        for q, (a, c) in enumerate(zip(v1, v2)):
            assert _same(q, toms, a, c), q
    v3 = [r.new_volume().fill_(0.5) for r in recons]
    b.run(imgs, v3, graph=True)
    for _ in range(3):
        for v in v3:
            v.fill_(0.5)
        b.run(imgs, v3, graph=True)  # same pointers: a replay of the captured graph
        torch.cuda.synchronize()
        for q, (a, c) in enumerate(zip(v1, v3)):
            assert _same(q, toms, a, c), q
    b.close()
    for r in recons:
        r.close()


def test_batch_member_matches_oracle():
    from paper_2206_09151_gb300.recon import Batch
    toms = _tomograms()
    recons, _ = _single_runs(toms)
    b = Batch(recons)
    vols = b.run([t[4] for t in toms])
    rot, nu, grid, kw, img = toms[0]
    ref = O.recon(img.cpu().numpy(), rot, lam=kw["lam"], delta=kw["delta"], defocus=kw["defocus"],
                  nz_layers=kw["nz_layers"], grid=grid, sigma=kw["sigma"], eps=kw["eps"])
    assert rel_l2(vols[0].cpu().numpy(), ref) <= 1e-5
    q = next(q for q, t in enumerate(toms) if t[3]["layer_interp"] == "linear" and t[3]["stack_dtype"] == "f32")
    rot, nu, grid, kw, img = toms[q]
    ref = O.recon(img.cpu().numpy(), rot, lam=kw["lam"], delta=kw["delta"], defocus=kw["defocus"],
                  nz_layers=kw["nz_layers"], grid=grid, sigma=kw["sigma"], eps=kw["eps"], layer_interp=O.LAYER_LINEAR)
    assert rel_l2(vols[q].cpu().numpy(), ref) <= 1e-5
    b.close()
    for r in recons:
        r.close()


def test_autotuner_picks_a_measured_candidate():
    from paper_2206_09151_gb300.autotune import tune_batch_round, tune_dir_block
    from paper_2206_09151_gb300.recon import Reconstructor
    toms = _tomograms()
    rot, nu, grid, kw, img = toms[0]
    kw = dict(kw)
    out = tune_dir_block(rot, nu, nu, grid, img, candidates=[10, 35, 70], repeats=2, **kw)
    assert out["dir_block"] in (10, 35, 70) and set(out["ms"]) == {"10", "35", "70"}
    recons = [Reconstructor(t[0], t[1], t[1], t[2], **t[3]) for t in toms[:3]]
    out = tune_batch_round(recons, [t[4] for t in toms[:3]], candidates=(8, 32), repeats=2)
    assert out["dir_block"] in (8, 32)
    for r in recons:
        r.close()


@pytest.mark.parametrize("interp", ["nearest", "linear"])
def test_bp_warp_shapes_are_bitwise_equal_and_the_tuner_picks_one(interp):
    """The general backprojection's warp patch (8 x 4, 16 x 2, 32 x 1 voxel columns) only
    moves voxels between threads: the volumes are identical bit for bit, and the autotuner
    returns one of the timed shapes.  The scan is a single-axis series about a tilted axis
    (not the volume y axis), so the general kernel runs and the
    single-axis ramp keeps the weights deterministic (the density weights come from float
    atomics and may differ in the last bit from run to run)."""
    from paper_2206_09151_gb300.autotune import tune_bp_warp
    from paper_2206_09151_gb300.recon import Reconstructor
    rng = np.random.default_rng(43)
    rot = ph.single_axis_rotations(40, start=0.2, axis=(0.0, 0.94, 0.34))
    nu, grid = 56, (48, 52, 24)
    img = torch.from_numpy((1.0 + 1e-2 * rng.standard_normal((40, nu, nu))).astype(np.float32)).cuda()
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 80e-9, 40), sigma=0.05, eps=0.02,
              ramp="single_axis", stack_dtype="f32", layer_interp=interp)
    vols = []
    for wc in (8, 16, 32):
        r = Reconstructor(rot, nu, nu, grid, nz_layers=3, bp_warp=wc, **kw)
        vols.append(r.run(img).clone())
        r.close()
    assert float(vols[0].abs().max()) > 0
    assert torch.equal(vols[0], vols[1]) and torch.equal(vols[0], vols[2])
    out = tune_bp_warp(rot, nu, nu, grid, img, nz_layers=3, candidates=(8, 16, 32), repeats=2, **kw)
    assert out["bp_warp"] in (8, 16, 32) and set(out["ms"]) == {"8", "16", "32"}


def test_batch_with_host_images_matches_the_device_image_run():
    """recon_batch_run_host (round r + 1's images uploaded while round r runs) gives the
    volumes of recon_batch_run, over several rounds, from pinned host memory, twice in a row."""
    from paper_2206_09151_gb300.recon import Batch
    toms = _tomograms()
    recons, _ = _single_runs(toms)
    b = Batch(recons, dir_block=16)
    ref = b.run([t[4] for t in toms], [torch.full((g[2], g[1], g[0]), 0.5, device="cuda") for _, _, g, _, _ in toms])
    host = [t[4].cpu().pin_memory() for t in toms]
    for _ in range(2):
        got = b.run_host(host, [torch.full((g[2], g[1], g[0]), 0.5, device="cuda") for _, _, g, _, _ in toms])
        torch.cuda.synchronize()
        for q, (a, c) in enumerate(zip(got, ref)):
            assert _same(q, toms, a, c), q
    b.close()
    for r in recons:
        r.close()
