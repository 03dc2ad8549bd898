"""FP64 oracle of the learned CTF-inverse regulariser (test infrastructure only).

The Tikhonov parameter eps of Eq. 11 (chosen "ad hoc" in Sec. 3) is replaced by
eps_theta = softplus(MLP(x)), evaluated per (direction n, layer k, radial bin b) from
three features: the signal-to-noise ratio of the image's radial power spectrum (the
noise floor per DFT coefficient is (NSR M)^2 by Parseval, as in the noise filter of
Sec. 3), the normalised radius of the bin, and the layer's effective defocus
lambda (R_n - z_k) / delta^2.  The per-layer filter becomes
    H(q) = lambda / (4 pi sqrt(1+sigma^2)) * sin chi / (sin^2 chi + eps_theta(b(q))).
Training minimises the normalised spectral L2 error of H G against the DFT T of the true
projection of the layer's slab, summed over images and layers.

Every definition here is shared, in meaning, with the CUDA path; the code is not.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import recon_fp64 as R

N_HIDDEN = 64
N_PARAMS = 3 * N_HIDDEN + N_HIDDEN + N_HIDDEN * N_HIDDEN + N_HIDDEN + N_HIDDEN + 1  # 4481
SNR_FLOOR = 1e-3


# ----------------------------------------------------------------------------- bins and SNR
def bin_width(P: int) -> int:
    return max(1, P // 128)


def n_bins(P: int) -> int:
    return math.isqrt(P * P // 2) // bin_width(P) + 1


@functools.lru_cache(maxsize=8)
def radial_bin(P: int) -> np.ndarray:
    """Bin of every frequency of the P x P DFT grid: floor(isqrt(m_u^2 + m_v^2) / w),
    exact integer arithmetic (so every implementation bins identically).  Cached per P;
    the array is read-only."""
    m = R.signed_freq(P).astype(np.int64)
    msq = m[:, None] ** 2 + m[None, :] ** 2
    r = np.array([math.isqrt(int(x)) for x in msq.ravel()]).reshape(msq.shape)
    out = np.minimum(r // bin_width(P), n_bins(P) - 1)
    out.setflags(write=False)
    return out


def radial_snr(G: np.ndarray, nsr: float, n_pix: int) -> np.ndarray:
    """SNR per radial bin of one image spectrum G (P x P): mean |G|^2 over the bin minus the
    noise floor N0 = nsr^2 * n_pix (Parseval: white noise of variance nsr^2 per pixel), over
    N0, floored at 1e-3."""
    P = G.shape[0]
    b = radial_bin(P).ravel()
    nb = n_bins(P)
    pw = np.bincount(b, weights=np.abs(G.ravel()) ** 2, minlength=nb)
    cnt = np.bincount(b, minlength=nb)
    N0 = nsr * nsr * n_pix
    return np.maximum(pw / np.maximum(cnt, 1) - N0, SNR_FLOOR * N0) / N0


def features(snr: np.ndarray, P: int, r_eff: np.ndarray, lam: float, delta: float) -> np.ndarray:
    """Rows (k, b) of the three inputs: log10 SNR_b / 3 (clamped to [-1, 2]), bin-centre
    radius / (P/2), lambda r_eff_k / delta^2 / 100."""
    nb = n_bins(P)
    w = bin_width(P)
    x0 = np.clip(np.log10(snr), -3.0, 6.0) / 3.0
    x1 = (np.arange(nb) + 0.5) * w / (P / 2)
    x2 = lam * np.asarray(r_eff) / (delta * delta) / 100.0
    K = len(x2)
    X = np.empty((K, nb, 3))
    X[:, :, 0] = x0[None, :]
    X[:, :, 1] = x1[None, :]
    X[:, :, 2] = x2[:, None]
    return X


# ----------------------------------------------------------------------------- MLP
def unpack(theta: np.ndarray):
    h = N_HIDDEN
    o = 0
    W1 = theta[o:o + 3 * h].reshape(h, 3); o += 3 * h
    b1 = theta[o:o + h]; o += h
    W2 = theta[o:o + h * h].reshape(h, h); o += h * h
    b2 = theta[o:o + h]; o += h
    w3 = theta[o:o + h]; o += h
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def softplus(o):
    return np.where(o > 20.0, o, np.log1p(np.exp(np.minimum(o, 20.0))))


def mlp_forward(theta: np.ndarray, X: np.ndarray):
    """eps = softplus(w3 . relu(W2 relu(W1 x + b1) + b2) + b3) for rows X (..., 3)."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(theta, np.float64))
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    o = h2 @ w3 + b3
    return softplus(o), (X, a1, h1, a2, h2, o)


def mlp_backward(theta: np.ndarray, cache, d_eps: np.ndarray) -> np.ndarray:
    """Gradient of sum(d_eps * eps) with respect to the flat parameters (backpropagation)."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(theta, np.float64))
    X, a1, h1, a2, h2, o = cache
    X = X.reshape(-1, 3); a1 = a1.reshape(-1, N_HIDDEN); h1 = h1.reshape(-1, N_HIDDEN)
    a2 = a2.reshape(-1, N_HIDDEN); h2 = h2.reshape(-1, N_HIDDEN); o = o.reshape(-1)
    d_o = d_eps.reshape(-1) / (1.0 + np.exp(-o))  # softplus' = sigmoid
    g_w3 = h2.T @ d_o
    g_b3 = d_o.sum()
    d_a2 = np.outer(d_o, w3) * (a2 > 0)
    g_W2 = d_a2.T @ h1
    g_b2 = d_a2.sum(0)
    d_a1 = (d_a2 @ W2) * (a1 > 0)
    g_W1 = d_a1.T @ X
    g_b1 = d_a1.sum(0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


# ----------------------------------------------------------------------------- filter and loss
def eps_table(theta, image, *, r_eff, lam, delta, nsr, input_mode=R.INPUT_INTENSITY):
    """eps_theta[k, b] of one image (layers at effective defocus r_eff[k])."""
    nv, nu = image.shape
    P = R.padded_size(max(nu, nv))
    g = np.zeros((P, P))
    g[:nv, :nu] = R.contrast(image, input_mode)
    G = np.fft.fft2(g)
    snr = radial_snr(G, nsr, nu * nv)
    eps, _ = mlp_forward(theta, features(snr, P, r_eff, lam, delta))
    return eps


def learned_filter(P, delta, lam, r_eff, sigma, eps_bins, cs=0.0):
    """H(q) with eps taken from the radial-bin table ``eps_bins`` (Eq. 11's real bracket)."""
    m = R.signed_freq(P).astype(np.float64)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    chi = math.pi * lam * r_eff * q2 + 0.5 * math.pi * cs * lam ** 3 * q2 * q2 - math.atan(sigma)
    s = np.sin(chi)
    eps = eps_bins[radial_bin(P)]
    return lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma)) * s / (s * s + eps), s


def _partial_learned(args):
    """Sum over directions ``dirs`` of their learned-filter contributions to voxels (i, j, k)."""
    (images, rot, dirs, theta, lam, delta, defocus, nz_layers, grid, sigma, nsr, cs, input_mode, i, j, k,
     density, interp, views) = args
    D, nv, nu = images.shape
    P = R.padded_size(max(nu, nv))
    A, B = R.pixel_coefficients(rot, grid, nu, nv)
    T = R.layer_constants(rot, grid, nz_layers)
    zc = R.layer_centres(rot, grid, nz_layers, delta)
    dens = R.density_weights(rot, P, delta, dirs) if density else None
    ramp = R.ramp_weights(P, delta, D)[None, :]
    ou, ov = (P - nu) // 2, (P - nv) // 2
    acc = np.zeros(i.shape)
    for o, n in enumerate(dirs):
        r_eff = float(defocus[n]) - zc[n]
        eps = eps_table(theta, images[n], r_eff=r_eff, lam=lam, delta=delta, nsr=nsr, input_mode=input_mode)
        eps = eps / views
        g = np.zeros((P, P))
        g[ov:ov + nv, ou:ou + nu] = R.contrast(images[n], input_mode)
        G = np.fft.fft2(g)
        W = ramp if dens is None else dens[o]
        st = np.empty((nz_layers, nv, nu))
        for kk_ in range(nz_layers):
            H, _ = learned_filter(P, delta, lam, r_eff[kk_], sigma, eps[kk_], cs)
            st[kk_] = np.fft.ifft2(G * H * W).real[ov:ov + nv, ou:ou + nu]
        acc += R.backproject_direction(st, A[n], B[n], T[n], i, j, k, interp)
    return acc


def recon_learned(images, rot, theta, *, lam, delta, defocus, nz_layers, grid, sigma, nsr, cs=0.0,
                  input_mode=R.INPUT_INTENSITY, voxels=None, workers: int = 1, density: bool = False,
                  layer_interp: int = R.LAYER_NEAREST, views: float = 1.0):
    """The whole operator with the learned regulariser: the single-axis ramp, or the
    sampling-density weighting of an arbitrary scan (``density``).  ``voxels`` = (i, j, k)
    returns those voxels only; ``workers`` > 1 splits the directions over a spawned
    process pool (the same arithmetic, summed in another order).  ``views`` > 1 divides the
    network's eps (a per-view noise-to-signal power, the Wiener reading) by the number of
    independent views the reconstruction averages."""
    images = np.asarray(images)
    rot = np.asarray(rot, np.float64)
    theta = np.asarray(theta, np.float64)
    D = images.shape[0]
    nx, ny, nz = grid
    if voxels is None:
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
    else:
        i, j, k = (np.asarray(x, np.int64) for x in voxels)
    common = (theta, lam, delta, np.asarray(defocus, np.float64), nz_layers, tuple(grid), sigma, nsr, cs, input_mode,
              i, j, k, density, layer_interp, max(1.0, float(views)))
    dirs = list(range(D))
    if workers <= 1 or D < 2:
        acc = _partial_learned((images, rot, dirs) + common)
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        groups = [dirs[w::workers] for w in range(workers) if dirs[w::workers]]
        with ProcessPoolExecutor(max_workers=len(groups), mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_partial_learned, [(images, rot, g) + common for g in groups]))
        acc = np.sum(parts, axis=0)
    return acc.reshape(nz, ny, nx) if voxels is None else acc


def train_loss_grad(theta, images, targets, *, r_eff, lam, delta, sigma, nsr, cs=0.0,
                    input_mode=R.INPUT_INTENSITY):
    """Normalised loss sum_{n,k,q} |H G_n - T_nk|^2 / sum |T_nk|^2 over the full DFT grid,
    and its gradient with respect to theta.  ``images`` (N, nv, nu), ``targets``
    (N, Nz, nv, nu) true layer projections (length units), ``r_eff`` (N, Nz)."""
    images = np.asarray(images, np.float64)
    N, nv, nu = images.shape
    P = R.padded_size(max(nu, nv))
    nb = n_bins(P)
    bins = radial_bin(P).ravel()
    pref = lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma))
    num = 0.0
    den = 0.0
    d_eps_all = []
    caches = []
    for n in range(N):
        g = np.zeros((P, P))
        g[:nv, :nu] = R.contrast(images[n], input_mode)
        G = np.fft.fft2(g)
        snr = radial_snr(G, nsr, nu * nv)
        X = features(snr, P, r_eff[n], lam, delta)
        eps, cache = mlp_forward(theta, X)
        caches.append(cache)
        d_eps = np.zeros_like(eps)
        for k in range(len(r_eff[n])):
            t = np.zeros((P, P))
            t[:nv, :nu] = targets[n][k]
            Tq = np.fft.fft2(t)
            H, s = learned_filter(P, delta, lam, r_eff[n][k], sigma, eps[k], cs)
            res = H * G - Tq
            num += np.sum(np.abs(res) ** 2)
            den += np.sum(np.abs(Tq) ** 2)
            dH = -pref * s / (s * s + eps[k][radial_bin(P)]) ** 2
            contrib = 2.0 * (res.real * G.real + res.imag * G.imag) * dH
            d_eps[k] = np.bincount(bins, weights=contrib.ravel(), minlength=nb)
        d_eps_all.append(d_eps)
    loss = num / den
    grad = np.zeros(N_PARAMS)
    for n in range(N):
        grad += mlp_backward(theta, caches[n], d_eps_all[n] / den)
    return loss, grad
