"""Parity at the full sizes of the other workloads: 512^3 voxels with 512 x 512 images and
Nz = 64 (Tikhonov and learned filters), the 1024 x 1024 x 256 slab under Haar-random
views with 1024 x 1024 images, Nz = 64 and the sampling-density weighting (both filters),
all with bfloat16 stacks; and 48 uneven tomograms in one batched, graph-captured run.

The FP64 oracle cannot afford every view of the two large scans, so both sides run the
first 48 views as a scan of their own (same images, same geometry), and the oracle
computes sampled voxels one by one over a spawned process pool."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import learned as L
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu

TOL_BF16 = 3e-3
WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _voxels(grid, seed, n_rand=384):
    """Random voxels, a full x line through the centre and the eight corners."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid
    i = np.concatenate([rng.integers(0, nx, n_rand), np.arange(nx), [0, nx - 1] * 4])
    j = np.concatenate([rng.integers(0, ny, n_rand), np.full(nx, ny // 2), [0, 0, ny - 1, ny - 1] * 2])
    k = np.concatenate([rng.integers(0, nz, n_rand), np.full(nx, nz // 3), [0] * 4 + [nz - 1] * 4])
    return i, j, k


def _network(seed):
    w = ph.mlp_init(seed)
    w[-65:-1] *= 50.0  # an eps that varies visibly over the features
    return w.astype(np.float32)


@pytest.mark.parametrize("filt", ["tikhonov", "mlp"])
@pytest.mark.parametrize("name", ["learned", "slab"])
def test_large_scan_first_48_views_match_oracle(name, filt):
    from paper_2206_09151_gb300.recon import Reconstructor
    cfg = ph.config_workload(name, scale_dirs=48)
    img = ph.make_images(cfg, device="cuda")
    density = cfg["ramp"] == "density"
    kw = dict(lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"], nz_layers=cfg["nz_layers"],
              sigma=cfg["sigma"], cs=cfg["cs"])
    nsr = float(cfg["photons"]) ** -0.5
    if filt == "mlp":
        w = _network(31)
        fkw = dict(filter="mlp", mlp_weights=w, nsr=nsr)
    else:
        fkw = dict(eps=cfg["eps"])
    r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], stack_dtype="bf16", ramp=cfg["ramp"],
                      **fkw, **kw)
    vol = r.run(img)
    i, j, k = _voxels(cfg["grid"], seed=len(name) + len(filt))
    got = vol[torch.as_tensor(k, device="cuda"), torch.as_tensor(j, device="cuda"),
              torch.as_tensor(i, device="cuda")].cpu().numpy()
    r.close()
    del vol
    torch.cuda.empty_cache()
    images = img.cpu().numpy()
    if filt == "mlp":
        ref = L.recon_learned(images, cfg["rot"], w.astype(np.float64), grid=cfg["grid"], nsr=nsr, voxels=(i, j, k),
                              workers=WORKERS, density=density, **kw)
    else:
        ref = O.recon(images, cfg["rot"], grid=cfg["grid"], eps=cfg["eps"], voxels=(i, j, k), workers=WORKERS,
                      density=density, **kw)
    err = rel_l2(got, ref)
    assert err <= TOL_BF16, err


def test_48_uneven_tomograms_in_one_graph_match_single_runs_and_oracle():
    """48 tomograms (grids 64^3-256^3, 60-360 views, Nz 4-32, balls and blobs, soft X-ray
    and electron physics), bfloat16 stacks, one persistent backprojection per round,
    captured as a CUDA graph and replayed: each member equals its own single run up to the
    order of the float sums, and three members match the FP64 oracle."""
    from paper_2206_09151_gb300.recon import Batch, Reconstructor
    cfgs = ph.batch_workloads()
    imgs = [ph.make_images(c, device="cuda") for c in cfgs]

    def plan(c, allocate):
        return Reconstructor(c["rot"], c["nu"], c["nv"], c["grid"], lam=c["lam"], delta=c["delta"],
                             defocus=c["defocus"], nz_layers=c["nz_layers"], sigma=c["sigma"], eps=c["eps"],
                             cs=c["cs"], stack_dtype="bf16", allocate=allocate)

    singles = []
    for c, im in zip(cfgs, imgs):
        r = plan(c, True)
        singles.append(r.run(im))
        r.close()
        del r
        torch.cuda.empty_cache()
    recons = [plan(c, False) for c in cfgs]
    b = Batch(recons)
    vols = [r.new_volume() for r in recons]
    b.run(imgs, vols, graph=True)  # capture
    for v in vols:
        v.fill_(-1.0)
    b.run(imgs, vols, graph=True)  # replay (same pointers); the run overwrites the volumes
    torch.cuda.synchronize()
    for q, (a, s) in enumerate(zip(vols, singles)):
        err = float(torch.linalg.vector_norm((a - s).double()) / torch.linalg.vector_norm(s.double()))
        assert err <= 1e-6, (q, err)
    size = [c["n_dir"] * int(np.prod(c["grid"])) for c in cfgs]
    order = np.argsort(size)
    for q in (int(order[0]), int(order[1])):  # the two smallest, every voxel
        c = cfgs[q]
        ref = O.recon(imgs[q].cpu().numpy(), c["rot"], lam=c["lam"], delta=c["delta"], defocus=c["defocus"],
                      nz_layers=c["nz_layers"], grid=c["grid"], sigma=c["sigma"], eps=c["eps"], cs=c["cs"],
                      workers=WORKERS)
        err = rel_l2(vols[q].cpu().numpy(), ref)
        assert err <= TOL_BF16, (q, err)
    big = max(range(len(cfgs)), key=lambda q: (cfgs[q]["grid"][0], cfgs[q]["n_dir"]))
    c = cfgs[big]
    i, j, k = _voxels(c["grid"], seed=48)
    ref = O.recon(imgs[big].cpu().numpy(), c["rot"], lam=c["lam"], delta=c["delta"], defocus=c["defocus"],
                  nz_layers=c["nz_layers"], grid=c["grid"], sigma=c["sigma"], eps=c["eps"], cs=c["cs"],
                  voxels=(i, j, k), workers=WORKERS)
    err = rel_l2(vols[big].cpu().numpy()[k, j, i], ref)
    assert err <= TOL_BF16, (big, err)
    b.close()
    for r in recons:
        r.close()
