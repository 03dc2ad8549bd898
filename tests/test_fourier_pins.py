"""Pins of the FP64 oracle's two 3D-Fourier-space forms (``oracle.fourier``): Eq. 12 (the
CT step first, one 3D CTF inversion after it) and the paper's own Fourier-gridding UTR (Sec.
2 after Eq. 11) with the NSR noise filter of Sec. 3.  CPU only."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import fourier as F
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _blobs(n, D, span, lam, amp, R, photons=None, sigma=0.3, delta=1e-9, seed=8):
    grid = (n, n, n)
    phan = ph.blob_phantom(grid, 12, seed=seed, s_vox=1.5, amp_unit=amp)
    rot = ph.single_axis_rotations(D, span=span)
    img = ph.multislice_images(phan, rot, n, n, delta, lam, np.full(D, R), sigma, n_slabs=32, photons=photons,
                               seed=3, dtype=torch.float64).numpy()
    kk, jj, ii = np.meshgrid(*(np.arange(n) - (n - 1) / 2,) * 3, indexing="ij")
    truth = np.zeros(grid)
    for c, s, a in zip(phan.centre, phan.size, phan.amp):
        truth += a * np.exp(-((ii - c[0]) ** 2 + (jj - c[1]) ** 2 + (kk - c[2]) ** 2) / (2 * s * s))
    return img, rot, grid, truth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- Eq. 12 (swapped order)
def test_swapped_order_with_one_layer_is_the_per_view_inverse():
    """One layer (no depth phase, so V_s = 0): Eq. 12's 3D filter after the CT step equals
    Eq. 13's filter applied to every view before it, up to the 3D vs 2D discretisation (a
    radial filter commutes with the backprojection for a single-axis scan)."""
    img, rot, grid, _ = _blobs(32, 90, math.pi, 1e-10, 5e-6, 30e-9)
    kw = dict(lam=1e-10, delta=1e-9, grid=grid, sigma=0.3, eps=1e-2)
    a = O.recon(img, rot, defocus=np.full(90, 30e-9), nz_layers=1, **kw)
    b = F.recon_swapped(img, rot, defocus=30e-9, nz_layers=1, **kw)
    assert rel(b, a) < 0.04


def test_swapped_order_matches_the_pair_form_under_ewald_curvature():
    """A 360-degree scan with one R and a DOF (1.25 nm) far below the object (32-45 nm):
    Eq. 12 (CT of the Ewald-placed contrasts, then the complex bracket in 3D) and Eq. 11 in
    the opposite-pair form (the bracket per view, then the layered backprojection) are the
    same sum in two orders; they agree to the discretisation (6 % here; dropping or
    flipping the imaginary part of the CT step gives 9.5 %)."""
    img, rot, grid, _ = _blobs(32, 120, 2 * math.pi, 4e-10, 2e-6, 20e-9)
    kw = dict(lam=4e-10, delta=1e-9, grid=grid, sigma=0.3, eps=1e-2)
    p = O.recon(img, rot, defocus=np.full(120, 20e-9), nz_layers=16, filt=O.FILTER_PAIR, **kw)
    b = F.recon_swapped(img, rot, defocus=20e-9, nz_layers=16, **kw)
    assert rel(b, p) < 0.075


def test_phase_step_reruns_for_another_omega_without_the_ct_step():
    """The CT step does not depend on sigma (omega) or eps: one CT step serves every phase
    retrieval (the use Sec. 2 gives for Eq. 12), and omega = 0 differs from sigma = 0.3."""
    img, rot, grid, _ = _blobs(24, 60, 2 * math.pi, 1e-10, 5e-6, 30e-9)
    vc, vs = F.swap_ct(img, rot, lam=1e-10, delta=1e-9, defocus=np.full(60, 30e-9), nz_layers=4, grid=grid)
    for sig in (0.0, 0.3):
        a = F.swap_phase(vc, vs, lam=1e-10, delta=1e-9, defocus=30e-9, sigma=sig, eps=1e-2)
        b = F.recon_swapped(img, rot, lam=1e-10, delta=1e-9, defocus=30e-9, nz_layers=4, grid=grid, sigma=sig,
                            eps=1e-2)
        assert np.array_equal(a, b)
    assert rel(F.swap_phase(vc, vs, lam=1e-10, delta=1e-9, defocus=30e-9, sigma=0.0, eps=1e-2), b) > 0.05


# ---------------------------------------------------------------- Fourier gridding UTR
@pytest.mark.parametrize("span", [math.pi, 2 * math.pi])
def test_gridding_recovers_the_closed_form_ball(span):
    """Closed-form Radon projections of a uniform ball (delta0 = 1), as the contrast of a
    pure absorber at R = 0 (Eq. 15: ln I = -(4 pi sigma / lambda) integral delta): the
    8-neighbour gridding onto the Ewald paraboloids with the sampling-matrix inverse
    S_eps^-1 returns delta0 inside the ball and zero outside."""
    nb, D = 32, 120
    ball = ph.Phantom("ball", np.array([[2.0, -1.0, 1.5]]), np.array([8.0]), np.array([1.0]))
    rot = ph.single_axis_rotations(D, span=span)
    lam, sig, dl = 1e-10, 1.0, 1e-9
    g = -(4 * math.pi / lam) * sig * ph.ball_projections(ball, rot, nb, nb) * dl
    v = F.recon_gridding(g, rot, lam=lam, delta=dl, defocus=np.zeros(D), grid=(nb, nb, nb), sigma=sig, eps=1e-6,
                         input_mode=O.INPUT_CONTRAST)
    kk, jj, ii = np.meshgrid(*(np.arange(nb) - (nb - 1) / 2,) * 3, indexing="ij")
    r = np.sqrt((ii - 2.0) ** 2 + (jj + 1.0) ** 2 + (kk - 1.5) ** 2)
    inner = v[r < 0.8 * 8]
    assert abs(inner.mean() - 1.0) < 0.02 and inner.std() < 0.08
    assert abs(v[r > 10].mean()) < 1e-3


def test_gridding_agrees_with_the_layered_pair_form():
    """Noise-free blobs, 360 degrees: the paper's gridding form and the layered pair form
    of the same Eq. 11 agree to the gridding's interpolation error (5 % here) and are
    equally close to the phantom."""
    img, rot, grid, truth = _blobs(32, 120, 2 * math.pi, 1e-10, 5e-6, 30e-9)
    kw = dict(lam=1e-10, delta=1e-9, defocus=np.full(120, 30e-9), grid=grid, sigma=0.3, eps=1e-2)
    p = O.recon(img, rot, filt=O.FILTER_PAIR, nz_layers=8, **kw)
    g = F.recon_gridding(img, rot, **kw)
    assert rel(g, p) < 0.08
    assert abs(rel(g, truth) - rel(p, truth)) < 0.03


def test_gridding_places_samples_on_the_ewald_paraboloid():
    """Strong curvature (DOF 1.25 nm, object 32-45 nm, 360 degrees, R = 60 nm): each sample
    sits at (q, -lambda q^2 / 2) (Eq. 8), and the gridding then matches the layered pair
    form to 7.4 %; placed on the mirror paraboloid (+lambda q^2 / 2) it is 9.2 % off."""
    img, rot, grid, _ = _blobs(32, 120, 2 * math.pi, 4e-10, 2e-6, 60e-9)
    kw = dict(lam=4e-10, delta=1e-9, defocus=np.full(120, 60e-9), grid=grid, sigma=0.3, eps=1e-2)
    p = O.recon(img, rot, filt=O.FILTER_PAIR, nz_layers=16, **kw)
    g = F.recon_gridding(img, rot, **kw)
    assert rel(g, p) < 0.083


def test_noise_filter_at_the_true_nsr_lowers_the_error():
    """Sec. 3's Fourier noise filter: with Poisson noise (1e4 photons per pixel, NSR 0.01)
    zeroing the coefficients whose gridded contrast lies below NSR M / sqrt(S) brings the
    reconstruction closer to the phantom than no filter."""
    img, rot, grid, truth = _blobs(32, 120, 2 * math.pi, 1e-10, 5e-6, 30e-9, photons=1e4)
    kw = dict(lam=1e-10, delta=1e-9, defocus=np.full(120, 30e-9), grid=grid, sigma=0.3, eps=1e-2)
    plain = F.recon_gridding(img, rot, **kw)
    filtered = F.recon_gridding(img, rot, nsr=1e-2, **kw)
    assert rel(filtered, truth) < 0.7 * rel(plain, truth)
