"""Pins of the FP64 oracle of the learned regulariser: backpropagation against central
differences, the training loss gradient against finite differences, the constant-eps
network against the Tikhonov filter, and the Parseval noise floor."""
import math

import numpy as np

import oracle as O
from oracle import learned as L
from paper_2206_09151_gb300 import phantoms as ph


def _theta(seed):
    return ph.mlp_init(seed)


def test_parameter_count():
    assert L.N_PARAMS == 4481 and _theta(0).size == 4481


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = _theta(2) + 0.1 * rng.standard_normal(L.N_PARAMS)
    X = rng.uniform(-1, 1, (40, 3))
    d = rng.standard_normal(40)
    _, cache = L.mlp_forward(theta, X)
    g = L.mlp_backward(theta, cache, d)
    for _ in range(5):
        v = rng.standard_normal(L.N_PARAMS)
        h = 1e-6
        fp = np.sum(d * L.mlp_forward(theta + h * v, X)[0])
        fm = np.sum(d * L.mlp_forward(theta - h * v, X)[0])
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g @ v) <= 1e-6 * max(1.0, abs(fd))


def _train_case(seed=3, N=2, n=16, nzl=2):
    rng = np.random.default_rng(seed)
    img = 1.0 + 1e-2 * rng.standard_normal((N, n, n))
    tgt = 1e-11 * rng.standard_normal((N, nzl, n, n))
    r_eff = rng.uniform(50e-9, 90e-9, (N, nzl))
    kw = dict(r_eff=r_eff, lam=1e-10, delta=1e-9, sigma=0.1, nsr=1e-2)
    return img, tgt, kw


def test_training_gradient_matches_finite_differences():
    img, tgt, kw = _train_case()
    theta = _theta(4)
    loss, g = L.train_loss_grad(theta, img, tgt, **kw)
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(L.N_PARAMS)
        h = 1e-5
        fd = (L.train_loss_grad(theta + h * v, img, tgt, **kw)[0] - L.train_loss_grad(theta - h * v, img, tgt, **kw)[0]) / (2 * h)
        assert abs(fd - g @ v) <= 1e-5 * max(abs(fd), 1e-3 * abs(loss))


def test_constant_eps_network_is_the_tikhonov_filter():
    """W1 = W2 = w3 = 0 gives eps = softplus(b3) everywhere: the learned path must then be
    the Tikhonov reconstruction of Eq. 11 with that eps."""
    eps0 = 0.05
    theta = np.zeros(L.N_PARAMS)
    theta[-1] = math.log(math.expm1(eps0))
    rng = np.random.default_rng(6)
    D, n = 6, 12
    rot = ph.single_axis_rotations(D)
    img = 1.0 + 1e-3 * rng.standard_normal((D, n, n))
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 60e-9, D), nz_layers=3, grid=(n, n, 8), sigma=0.05)
    a = L.recon_learned(img, rot, theta, nsr=1e-2, **kw)
    b = O.recon(img, rot, eps=eps0, **kw)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_constant_eps_network_is_the_tikhonov_filter_with_density_weights():
    """The same reduction for an arbitrary scan (sampling-density weighting): a constant
    network is the Tikhonov path, and the spawned process pool sums the same terms."""
    eps0 = 0.08
    theta = np.zeros(L.N_PARAMS)
    theta[-1] = math.log(math.expm1(eps0))
    rng = np.random.default_rng(16)
    D, n = 7, 12
    rot = ph.cone_rotations(D, 60.0, seed=3)
    img = 1.0 + 1e-3 * rng.standard_normal((D, n, n))
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 60e-9, D), nz_layers=3, grid=(n, 10, 8), sigma=0.05)
    a = L.recon_learned(img, rot, theta, nsr=1e-2, density=True, **kw)
    b = O.recon(img, rot, eps=eps0, density=True, **kw)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    c = L.recon_learned(img, rot, theta, nsr=1e-2, density=True, workers=2, **kw)
    assert np.max(np.abs(c - a)) <= 1e-12 * np.max(np.abs(a))


def test_white_noise_sits_on_the_parseval_floor():
    """A noise image of variance nsr^2 per pixel has radial power ~ nsr^2 * n_pix per DFT
    coefficient (Parseval), so its estimated SNR is at the floor."""
    rng = np.random.default_rng(7)
    n, nsr = 128, 0.03
    P = O.padded_size(n)
    g = np.zeros((P, P))
    g[:n, :n] = nsr * rng.standard_normal((n, n))
    G = np.fft.fft2(g)
    b = L.radial_bin(P).ravel()
    pw = np.bincount(b, weights=np.abs(G.ravel()) ** 2) / np.maximum(np.bincount(b), 1)
    N0 = nsr * nsr * n * n
    mid = slice(5, L.n_bins(P) // 2)
    assert abs(np.mean(pw[mid]) / N0 - 1.0) < 0.05
    assert np.median(L.radial_snr(G, nsr, n * n)[mid]) < 0.2


def test_radial_bins_are_integer_radii():
    P = 256
    b = L.radial_bin(P)
    m = O.signed_freq(P)
    for (v, u) in [(0, 0), (3, 4), (100, 0), (127, 127), (-128, -128), (12, -35)]:
        r = math.isqrt(v * v + u * u)
        assert b[v % P, u % P] == min(r // L.bin_width(P), L.n_bins(P) - 1)
    assert b.max() == L.n_bins(P) - 1
    del m
