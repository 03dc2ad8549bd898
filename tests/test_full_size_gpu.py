"""Parity at the full size of the benchmarked workload (256^3 voxels, 360 single-axis
views of 256 x 256 pixels, Nz = 32 layers, Cs = 2.7 mm), in the launch configuration that
bench.py times (default direction blocks), on sampled voxels that the FP64 oracle
computes one by one (all 360 views, spread over a spawned process pool)."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()
    cfg = ph.config_workload("mid")
    phan = ph.make_phantom(cfg)
    img = ph.multislice_images(phan, cfg["rot"], cfg["nu"], cfg["nv"], cfg["delta"], cfg["lam"], cfg["defocus"],
                               cfg["sigma"], cs=cfg["cs"], photons=cfg["photons"], seed=cfg["seed"], device="cuda")
    rng = np.random.default_rng(5)
    nx, ny, nz = cfg["grid"]
    # 384 random voxels, plus a full x line through the centre and the eight corners
    i = np.concatenate([rng.integers(0, nx, 384), np.arange(nx), [0, nx - 1] * 4])
    j = np.concatenate([rng.integers(0, ny, 384), np.full(nx, ny // 2), [0, 0, ny - 1, ny - 1] * 2])
    k = np.concatenate([rng.integers(0, nz, 384), np.full(nx, nz // 3), [0] * 4 + [nz - 1] * 4])
    workers = max(1, min(16, (os.cpu_count() or 1)))
    ref = O.recon(img.cpu().numpy(), cfg["rot"], lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"],
                  nz_layers=cfg["nz_layers"], grid=cfg["grid"], sigma=cfg["sigma"], eps=cfg["eps"], cs=cfg["cs"],
                  voxels=(i, j, k), workers=workers)
    return cfg, img, (i, j, k), ref


@pytest.mark.parametrize("stack,tol", [("f32", 1e-5), ("bf16", 3e-3)])
def test_full_size_sampled_voxels_match_oracle(workload, stack, tol):
    from paper_2206_09151_gb300.recon import Reconstructor
    cfg, img, (i, j, k), ref = workload
    r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                      defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
                      cs=cfg["cs"], stack_dtype=stack)
    vol = r.run(img).cpu().numpy()
    r.close()
    got = vol[k, j, i]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err
