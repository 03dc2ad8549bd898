"""Parity of the CUDA 3D-Fourier forms (through the C-ABI) with the FP64 oracle: Eq. 12
(CT step, then the 3D CTF inversion, rerun for a second sigma) and the Fourier-gridding
UTR (with and without the NSR noise filter).  Float32 tolerance 1e-5 relative L2, except
where the noise filter decides per coefficient whether to keep it: those decisions are
taken in float32 on the GPU and in float64 by the oracle, so coefficients at the
threshold may go either way (1e-3 there)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import fourier as F
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _scan(grid, nu, nv, D, span, lam, R, photons=None, cone=False, seed=8):
    phan = ph.blob_phantom(grid, 12, seed=seed, s_vox=1.5, amp_unit=2e-6)
    rot = ph.cone_rotations(D, 60.0, seed=seed) if cone else ph.single_axis_rotations(D, span=span)
    Rs = np.full(D, R) if np.isscalar(R) else np.asarray(R)
    img = ph.multislice_images(phan, rot, nu, nv, 1e-9, lam, Rs, 0.3, n_slabs=16, photons=photons, seed=3).numpy()
    return img, rot, Rs


@pytest.mark.parametrize("grid,nu,nv", [((32, 32, 32), 32, 32), ((24, 20, 12), 30, 22)])
def test_swapped_order_matches_oracle_and_reruns_for_another_sigma(grid, nu, nv):
    from paper_2206_09151_gb300.recon import Reconstructor
    D, lam, R = 60, 4e-10, 20e-9
    img, rot, Rs = _scan(grid, nu, nv, D, 2 * math.pi, lam, R)
    r = Reconstructor(rot, nu, nv, grid, lam=lam, delta=1e-9, defocus=Rs, nz_layers=8, sigma=0.3, eps=1e-2,
                      filter="pair")
    ws = r.swap_ct(torch.from_numpy(img).cuda())
    vc, vs = F.swap_ct(img, rot, lam=lam, delta=1e-9, defocus=Rs, nz_layers=8, grid=grid)
    for sig, eps in ((0.3, 1e-2), (0.05, 0.1)):
        got = r.swap_phase(ws, sig, eps).cpu().numpy()
        ref = F.swap_phase(vc, vs, lam=lam, delta=1e-9, defocus=R, sigma=sig, eps=eps)
        assert rel_l2(got, ref) <= TOL_F32, (sig, rel_l2(got, ref))
    r.close()


@pytest.mark.parametrize("grid,nu,nv,cone", [((32, 32, 32), 32, 32, False), ((24, 20, 12), 30, 22, True)])
def test_gridding_matches_oracle(grid, nu, nv, cone):
    from paper_2206_09151_gb300.recon import Reconstructor
    D, lam = 60, 4e-10
    Rs = np.random.default_rng(4).uniform(15e-9, 25e-9, D)
    img, rot, Rs = _scan(grid, nu, nv, D, 2 * math.pi, lam, Rs, cone=cone)
    r = Reconstructor(rot, nu, nv, grid, lam=lam, delta=1e-9, defocus=Rs, nz_layers=4, sigma=0.3, eps=1e-2,
                      ramp="density" if cone else "single_axis")
    got = r.grid_run(torch.from_numpy(img).cuda()).cpu().numpy()
    r.close()
    ref = F.recon_gridding(img, rot, lam=lam, delta=1e-9, defocus=Rs, grid=grid, sigma=0.3, eps=1e-2)
    assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)


def test_gridding_noise_filter_matches_oracle():
    from paper_2206_09151_gb300.recon import Reconstructor
    grid, D, lam = (32, 32, 32), 60, 1e-10
    img, rot, Rs = _scan(grid, 32, 32, D, 2 * math.pi, lam, 30e-9, photons=1e4)
    r = Reconstructor(rot, 32, 32, grid, lam=lam, delta=1e-9, defocus=Rs, nz_layers=4, sigma=0.3, eps=1e-2)
    got = r.grid_run(torch.from_numpy(img).cuda(), nsr=1e-2).cpu().numpy()
    r.close()
    ref = F.recon_gridding(img, rot, lam=lam, delta=1e-9, defocus=Rs, grid=grid, sigma=0.3, eps=1e-2, nsr=1e-2)
    assert rel_l2(got, ref) <= 1e-3, rel_l2(got, ref)
