"""The learned regulariser on the GPU: the reconstruction with a given network against the
FP64 oracle, the training loss and gradient against the oracle's backpropagation, and
what training gains over the fixed Tikhonov eps on held-out phantoms."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import learned as L
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _weights(seed):
    w = ph.mlp_init(seed)
    w[-65:-1] *= 50.0  # a network whose eps varies visibly over the features
    return w


PHYS = dict(lam=1e-10, delta=1e-9, sigma=0.05)


@pytest.mark.parametrize("views", [0.0, 20.0])
def test_learned_filter_reconstruction_matches_oracle(views):
    """The learned regulariser, with the network's per-view eps as it is and divided by the
    20 views the scan averages (mlp_views), against the oracle voxel by voxel."""
    from paper_2206_09151_gb300.recon import Reconstructor
    n, D, nzl = 32, 20, 4
    grid = (n, n, n)
    rng = np.random.default_rng(3)
    rot = ph.single_axis_rotations(D)
    R = rng.uniform(60e-9, 70e-9, D)
    phan = ph.blob_phantom(grid, 15, seed=4, s_vox=1.5, amp_unit=4e-6)
    img = ph.multislice_images(phan, rot, n, n, PHYS["delta"], PHYS["lam"], R, PHYS["sigma"], n_slabs=8,
                               photons=1e4, seed=5).numpy()
    w = _weights(6)
    r = Reconstructor(rot, n, n, grid, defocus=R, nz_layers=nzl, filter="mlp", mlp_weights=w.astype(np.float32),
                      nsr=1e-2, mlp_views=views, **PHYS)
    got = r.run(torch.from_numpy(img).cuda()).cpu().numpy()
    r.close()
    ref = L.recon_learned(img, rot, w.astype(np.float32).astype(np.float64), defocus=R, nz_layers=nzl, grid=grid,
                          nsr=1e-2, views=max(1.0, views), **PHYS)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


def _train_set(n_phantoms, dirs_each, n, nzl, seed, photons=1e4, amp=1e-4, s_vox=2.0):
    grid = (n, n, n)
    imgs, tgts, rots, Rs = [], [], [], []
    for p in range(n_phantoms):
        phan = ph.blob_phantom(grid, 10, seed=seed + p, s_vox=s_vox, amp_unit=amp)
        rot = ph.single_axis_rotations(dirs_each, start=0.37 * p)
        R = np.random.default_rng(seed + 100 + p).uniform(40e-9, 60e-9, dirs_each)
        imgs.append(ph.multislice_images(phan, rot, n, n, PHYS["delta"], PHYS["lam"], R, PHYS["sigma"], n_slabs=8,
                                         photons=photons, seed=seed + 200 + p).numpy())
        tgts.append(ph.layer_projections(phan, rot, n, n, grid, nzl, PHYS["delta"]))
        rots.append(rot)
        Rs.append(R)
    return (np.concatenate(imgs), np.concatenate(tgts).astype(np.float32), np.concatenate(rots), np.concatenate(Rs),
            grid)


def test_training_loss_and_gradient_match_oracle():
    from paper_2206_09151_gb300.recon import train_mlp
    n, nzl = 32, 2
    img, tgt, rot, R, grid = _train_set(2, 2, n, nzl, seed=11, photons=1e4)
    w = _weights(12)
    nsr = 1e-2
    _, loss, grad = train_mlp(w.astype(np.float32), torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), rot, R,
                              grid, nz_layers=nzl, nsr=nsr, steps=0, want_grad=True, **PHYS)
    zc = O.layer_centres(rot, grid, nzl, PHYS["delta"])
    r_eff = R[:, None] - zc
    ref_loss, ref_grad = L.train_loss_grad(w.astype(np.float32).astype(np.float64), img.astype(np.float64),
                                           tgt.astype(np.float64), r_eff=r_eff, nsr=nsr, **PHYS)
    assert abs(loss[0] - ref_loss) <= 1e-5 * ref_loss, (loss[0], ref_loss)
    assert rel_l2(grad, ref_grad) <= 1e-4, rel_l2(grad, ref_grad)


def test_training_gains_over_the_fixed_tikhonov_eps():
    """Train on 48 noisy images (24 phantoms x 2 views, 1e4 photons/pixel), then
    reconstruct 3 held-out phantoms from 60 views each: the trained network is closer to
    the phantoms than the Tikhonov eps = 0.1 that Sec. 3 used."""
    from paper_2206_09151_gb300.recon import Reconstructor, train_mlp
    n, nzl, photons = 32, 4, 1e4
    nsr = photons ** -0.5
    img, tgt, rot, R, grid = _train_set(24, 2, n, nzl, seed=100, photons=photons)
    w0 = ph.mlp_init(7).astype(np.float32)
    w, loss, _ = train_mlp(w0, torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), rot, R, grid,
                           nz_layers=nzl, nsr=nsr, steps=400, lr=3e-3, **PHYS)
    assert loss[-1] < 0.9 * loss[0], (loss[0], loss[-1])
    errs = {"learned": [], "eps=0.1": [], "eps=0.01": []}
    for p in range(3):
        phan = ph.blob_phantom(grid, 10, seed=900 + p, s_vox=2.0, amp_unit=1e-4)
        rot_t = ph.single_axis_rotations(60)
        R_t = np.full(60, 50e-9)
        im = ph.multislice_images(phan, rot_t, n, n, PHYS["delta"], PHYS["lam"], R_t, PHYS["sigma"], n_slabs=8,
                                  photons=photons, seed=950 + p).cuda()
        kk, jj, ii = np.meshgrid(*(np.arange(n) - (n - 1) / 2,) * 3, indexing="ij")
        truth = np.zeros(grid)
        for c, s, a in zip(phan.centre, phan.size, phan.amp):
            truth += a * np.exp(-((ii - c[0]) ** 2 + (jj - c[1]) ** 2 + (kk - c[2]) ** 2) / (2 * s * s))
        for name, kw in (("learned", dict(filter="mlp", mlp_weights=w, nsr=nsr)), ("eps=0.1", dict(eps=0.1)),
                         ("eps=0.01", dict(eps=0.01))):
            r = Reconstructor(rot_t, n, n, grid, defocus=R_t, nz_layers=nzl, **kw, **PHYS)
            errs[name].append(rel_l2(r.run(im).cpu().numpy(), truth))
            r.close()
    mean = {k: float(np.mean(v)) for k, v in errs.items()}
    print("held-out rel-L2 to the phantoms:", mean, "training loss", float(loss[0]), "->", float(loss[-1]))
    assert mean["learned"] < 0.95 * mean["eps=0.1"]


def test_training_does_not_depend_on_the_workspace_contents():
    """Adam's moments and the gradient accumulators start from zero whatever the workspace
    held: a few steps on a workspace that held NaN bytes give the losses of one that held
    zeros (up to the order of the float atomics)."""
    from paper_2206_09151_gb300.recon import train_mlp
    n, nzl = 32, 2
    img, tgt, rot, R, grid = _train_set(2, 2, n, nzl, seed=21, photons=1e4)
    w = _weights(22).astype(np.float32)
    out = {}
    for fill in (0x00, 0xFF):  # 0xFF bytes are NaNs in float32
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        junk = torch.full((64 << 20,), fill, dtype=torch.uint8, device="cuda")
        del junk  # the caching allocator hands these bytes to the training workspace
        _, loss, _ = train_mlp(w, torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), rot, R, grid,
                               nz_layers=nzl, nsr=1e-2, steps=5, lr=1e-3, **PHYS)
        out[fill] = np.asarray(loss, np.float64)
    assert np.all(np.isfinite(out[0xFF])), out[0xFF]
    np.testing.assert_allclose(out[0xFF], out[0x00], rtol=1e-5)


def test_adam_state_carries_over_between_calls():
    """Six Adam steps in one call equal three plus three in two calls that pass Adam's
    moments and step count along (the mini-batch training of the regulariser relies on it)."""
    from paper_2206_09151_gb300.recon import train_mlp
    n, nzl = 32, 2
    img, tgt, rot, R, grid = _train_set(2, 2, n, nzl, seed=31, photons=1e4)
    w = _weights(32).astype(np.float32)
    dimg, dtgt = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
    kw = dict(nz_layers=nzl, nsr=1e-2, lr=1e-3, **PHYS)
    w6, loss6, _ = train_mlp(w, dimg, dtgt, rot, R, grid, steps=6, **kw)
    state = np.zeros(2 * w.size, np.float32)
    wa, la, _ = train_mlp(w, dimg, dtgt, rot, R, grid, steps=3, adam_state=state, adam_step=0, **kw)
    assert np.any(state != 0)
    wb, lb, _ = train_mlp(wa, dimg, dtgt, rot, R, grid, steps=3, adam_state=state, adam_step=3, **kw)
    np.testing.assert_allclose(np.concatenate([la, lb]), loss6, rtol=1e-5)
    np.testing.assert_allclose(wb, w6, rtol=1e-4, atol=1e-6)


def _held_out_tomogram(seed, D=180, n=128):
    """A held-out 128^3 pseudo-atom phantom at the 512^3 scan's physics (0.1 nm voxels,
    lambda 1.97 pm, R ~ U[0.5, 1.5] um, Cs 2.7 mm, sigma 0.07, 100 e/px), seen from D
    single-axis views; returns (config, images on the GPU, phantom volume)."""
    from paper_2206_09151_gb300.layer_study import phantom_volume
    cfg = ph.config_workload("learned", scale_dirs=D)
    cfg.update(grid=(n, n, n), nu=n, nv=n, count=2500, seed=seed)
    cfg["rot"] = ph.single_axis_rotations(D)
    cfg["defocus"] = np.random.default_rng(seed + 7).uniform(0.5e-6, 1.5e-6, D)
    phan = ph.make_phantom(cfg)
    img = ph.make_images(cfg, device="cuda")
    return cfg, img, phantom_volume(phan, cfg["grid"], "cuda")


def test_trained_regulariser_beats_the_fixed_eps_on_held_out_128cubed_tomograms():
    """The committed network (``train_regulariser``: 5000 + 1000 seeded 128^3 phantoms, four
    views each) against the eps = 0.1 that Sec. 3 chose ad hoc, and against eps = 0.3 (the
    best fixed eps of a sweep on these tomograms), on two held-out 128^3 phantoms of 180
    views at 100 e/px, Nz = 16.  The network's eps is a per-view noise-to-signal power; the
    reconstruction averages the 180 views, so it is divided by 180 (mlp_views).  The
    learned regulariser is closer to the phantom inside the field of view than both."""
    from paper_2206_09151_gb300.recon import Reconstructor
    from paper_2206_09151_gb300.train_regulariser import load_weights
    w = load_weights()
    errs = {"learned": [], "eps=0.1": [], "eps=0.3": []}
    for seed in (2_000_001, 2_000_003):
        cfg, img, truth = _held_out_tomogram(seed)
        n = cfg["grid"][0]
        xx = torch.arange(n, device="cuda") - (n - 1) / 2
        fov = ((xx[None, :] ** 2 + xx[:, None] ** 2) <= (n / 2 - 2) ** 2)[:, None, :].expand(n, n, n)
        learned = dict(filter="mlp", mlp_weights=w, nsr=cfg["photons"] ** -0.5, mlp_views=cfg["n_dir"])
        for name, kw in (("learned", learned), ("eps=0.1", dict(eps=0.1)), ("eps=0.3", dict(eps=0.3))):
            r = Reconstructor(cfg["rot"], n, n, cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                              defocus=cfg["defocus"], nz_layers=16, sigma=cfg["sigma"], cs=cfg["cs"], **kw)
            v = r.run(img).double()
            r.close()
            errs[name].append(float(torch.linalg.norm((v - truth)[fov]) / torch.linalg.norm(truth[fov])))
    mean = {k: float(np.mean(v)) for k, v in errs.items()}
    print("held-out 128^3 rel-L2 to the phantoms:", mean)
    assert mean["learned"] < 0.95 * mean["eps=0.3"] < mean["eps=0.1"], mean
