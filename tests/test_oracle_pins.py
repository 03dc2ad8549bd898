"""Pins of the FP64 oracle to things other than itself (closed forms, brute force,
invariants, limits the paper derives).  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- DFT convention (Eq. 3)
def test_library_fft_is_the_papers_forward_transform():
    """F2 f(q) = sum f(r) exp(-i 2 pi r.q): brute-force DFT on a 6x8 grid."""
    rng = np.random.default_rng(0)
    f = rng.standard_normal((6, 8))
    v, u = np.meshgrid(np.arange(6), np.arange(8), indexing="ij")
    F = np.zeros((6, 8), complex)
    for mv in range(6):
        for mu in range(8):
            F[mv, mu] = np.sum(f * np.exp(-2j * np.pi * (mu * u / 8 + mv * v / 6)))
    assert np.allclose(np.fft.fft2(f), F, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- ramp (Sec. 2, |q_x|)
@pytest.mark.parametrize("P", [16, 128, 1024])
def test_ramp_approximates_pi_abs_q_over_D(P):
    delta, D = 1e-9, 90
    W = O.ramp_weights(P, delta, D)
    m = O.signed_freq(P)
    ideal = (math.pi / D) * np.abs(m) / (P * delta)
    band = (np.abs(m) >= 1) & (np.abs(m) <= P // 4)
    # band-limited Ram-Lak truncated to P taps: |q| up to an offset below 3% of the
    # first bin (the truncated tail of the kernel), in the whole lower half band
    assert np.max(np.abs(W[band] - ideal[band])) < 0.03 * ideal[1]
    # even in m, real, DC small and positive (no "dishing" offset)
    assert np.allclose(W, W[(-m) % P])
    assert 0 < W[0] < ideal[1]


def test_ramp_is_the_dft_of_its_spatial_kernel():
    """Direct evaluation of the P-tap kernel's DFT, sum over n of h[n] cos(2 pi m n / P)."""
    P, delta, D = 32, 2e-9, 7
    n = np.arange(-P // 2, P // 2)
    h = np.where(n == 0, 1 / (4 * delta ** 2), np.where(n % 2 != 0, -1 / (n ** 2 * np.pi ** 2 * delta ** 2), 0.0))
    for mm in range(P):
        direct = (np.pi / D) * delta * np.sum(h * np.cos(2 * np.pi * mm * n / P))
        assert abs(O.ramp_weights(P, delta, D)[mm] - direct) < 1e-9 * abs(direct) + 1e-3


# ---------------------------------------------------------------- CTF filter limits (Eq. 13-15)
def test_filter_at_zero_defocus_is_absorption_ct():
    """R = 0, eps = 0: H = -lambda/(4 pi sigma) for every q, i.e. mu = (4pi/lambda) sigma delta
    = -ln(I/I_in) slice by slice: Eq. 15."""
    lam, sigma = 3.9e-11, 0.3
    H = O.ctf_filter(32, 1e-6, lam, 0.0, sigma, 0.0)
    assert np.allclose(H, -lam / (4 * math.pi * sigma), rtol=1e-13, atol=0)


def test_filter_small_defocus_is_homogeneous_tie():
    """Small R: (4 pi/lambda) sigma H(q) -> -1/(1 - pi lambda R q^2 / sigma) (Eq. 14), with the
    error shrinking like R^2."""
    lam, sigma, delta, P = 3.9e-11, -0.001, 1e-4, 64
    m = O.signed_freq(P).astype(float)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    errs = []
    for R in (0.02, 0.01):
        H = O.ctf_filter(P, delta, lam, R, sigma, 0.0)
        tie = -1.0 / (1.0 - math.pi * lam * R * q2 / sigma)
        errs.append(np.max(np.abs((4 * math.pi / lam) * sigma * H - tie)))
    assert errs[0] < 0.05
    assert 3.0 < errs[0] / errs[1] < 5.0  # second order in R


def test_filter_recovers_a_thin_slab_projection():
    """A weak thin object at depth z0, imaged by the multislice simulator (Fresnel
    propagator of Eq. 3, no CTF formula), is recovered by the filter of the layer at
    defocus R - z0 with eps -> 0 (Eq. 7 for a single slab; the layer filter of Eq. 11)."""
    n, delta, lam, sigma = 64, 1e-9, 1e-10, 0.5
    R = 2e-7
    phan = ph.Phantom("blob", np.array([[3.0, -2.0, 0.0], [-8.0, 5.0, 0.0]]), np.array([2.0, 3.0]),
                      np.array([2e-6, 1e-6]))
    rot = np.eye(3)[None]
    img = ph.multislice_images(phan, rot, n, n, delta, lam, np.array([R]), sigma, n_slabs=1,
                               dtype=__import__("torch").float64).numpy()[0]
    P = O.padded_size(n)
    o = (P - n) // 2
    g = np.zeros((P, P))
    g[o:o + n, o:o + n] = np.log(img)
    # the multislice slab sits at the phantom's centre depth plane; the simulator's only
    # slab is centred at z = 0 here, so the effective defocus is R
    H = O.ctf_filter(P, delta, lam, R, sigma, 1e-14)
    p = np.fft.ifft2(np.fft.fft2(g) * H).real[o:o + n, o:o + n]
    # true projection of the two blobs, in metres
    uu = np.arange(n) - (n - 1) / 2
    truth = np.zeros((n, n))
    for c, s, a in zip(phan.centre, phan.size, phan.amp):
        r2 = (uu[None, :] - c[0]) ** 2 + (uu[:, None] - c[1]) ** 2
        truth += a * math.sqrt(2 * math.pi) * s * np.exp(-r2 / (2 * s * s)) * delta
    err = np.linalg.norm(p - truth) / np.linalg.norm(truth)
    assert err < 2e-2, err


def _thin_slab_case(z0_vox, cs, thickness=40.0):
    """Two weak blobs at depth z0 (voxel units), imaged through a two-slab multislice run
    whose downstream slab is centred at +thickness/4: returns (ln I, truth, z_slab)."""
    n, delta, lam, sigma = 64, 1e-9, 1e-10, 0.5
    R = 2e-7
    phan = ph.Phantom("blob", np.array([[3.0, -2.0, z0_vox], [-8.0, 5.0, z0_vox]]), np.array([2.0, 3.0]),
                      np.array([2e-6, 1e-6]))
    img = ph.multislice_images(phan, np.eye(3)[None], n, n, delta, lam, np.array([R]), sigma, n_slabs=2,
                               cs=cs, thickness=thickness, dtype=__import__("torch").float64).numpy()[0]
    uu = np.arange(n) - (n - 1) / 2
    truth = np.zeros((n, n))
    for c, s, a in zip(phan.centre, phan.size, phan.amp):
        truth += a * math.sqrt(2 * math.pi) * s * np.exp(-((uu[None, :] - c[0]) ** 2 + (uu[:, None] - c[1]) ** 2)
                                                         / (2 * s * s)) * delta
    return np.log(img), truth, (thickness / 4.0) * delta, dict(delta=delta, lam=lam, sigma=sigma, R=R)


def _apply_layer_filter(lnI, r_eff, p, cs):
    n = lnI.shape[0]
    P = O.padded_size(n)
    o = (P - n) // 2
    g = np.zeros((P, P))
    g[o:o + n, o:o + n] = lnI
    H = O.ctf_filter(P, p["delta"], p["lam"], r_eff, p["sigma"], 1e-14, cs)
    return np.fft.ifft2(np.fft.fft2(g) * H).real[o:o + n, o:o + n]


def test_filter_focuses_at_defocus_minus_depth():
    """A slab downstream of the rotation centre (z0 > 0) is in focus at R - z0 (Eq. 5:
    slice m sits at defocus R - z_m), not at R + z0."""
    lnI, truth, z0, p = _thin_slab_case(10.0, 0.0)
    good = _apply_layer_filter(lnI, p["R"] - z0, p, 0.0)
    bad = _apply_layer_filter(lnI, p["R"] + z0, p, 0.0)
    e_good = np.linalg.norm(good - truth) / np.linalg.norm(truth)
    e_bad = np.linalg.norm(bad - truth) / np.linalg.norm(truth)
    assert e_good < 2e-2 and e_bad > 0.3, (e_good, e_bad)


def test_filter_spherical_aberration_term():
    """A Cs phase (pi/2) Cs lambda^3 q^4 added to the propagation phase (the per-view
    aberration Sec. 2 allows in the CTF argument) is undone only when the filter
    carries the same term."""
    cs = 3e-4
    lnI, truth, z0, p = _thin_slab_case(10.0, cs)
    good = _apply_layer_filter(lnI, p["R"] - z0, p, cs)
    bad = _apply_layer_filter(lnI, p["R"] - z0, p, 0.0)
    e_good = np.linalg.norm(good - truth) / np.linalg.norm(truth)
    e_bad = np.linalg.norm(bad - truth) / np.linalg.norm(truth)
    assert e_good < 2e-2 and e_bad > 0.3, (e_good, e_bad)


# ---------------------------------------------------------------- layer depths (Eq. 5)
@pytest.mark.parametrize("layer", [0, 3])
def test_layer_centres_refocus_each_layer_end_to_end(layer):
    """Through the whole operator: two weak blobs at the centre depth of one layer of
    Nz = 4 over a 40-voxel-thick volume (slabs [-20,-10), ..., [10,20) voxels, centres
    -15, -5, 5, 15), imaged along z by the multislice simulator whose 4 slabs have
    those centres.  Every volume slice of that layer must equal the ramp-filtered true
    projection (the filter-off operator applied to the projection itself): the layer's
    filter sits at defocus R - z_k (Eq. 5) and inverts its own slab exactly with
    eps -> 0 (Eq. 7, Eq. 11).  A half-layer slip of z_k (5 voxels, one DOF) gives 20-27 %."""
    n, nzv, nzl = 64, 40, 4
    delta, lam, sigma, R = 1e-9, 1e-10, 0.5, 2e-7
    z0 = -15.0 + 10.0 * layer
    phan = ph.Phantom("blob", np.array([[3.0, -2.0, z0], [-8.0, 5.0, z0]]), np.array([2.0, 3.0]),
                      np.array([2e-6, 1e-6]))
    rot = np.eye(3)[None]
    img = ph.multislice_images(phan, rot, n, n, delta, lam, np.array([R]), sigma, n_slabs=4, thickness=40.0,
                               dtype=__import__("torch").float64).numpy()
    vol = O.recon(img, rot, lam=lam, delta=delta, defocus=[R], nz_layers=nzl, grid=(n, n, nzv), sigma=sigma,
                  eps=1e-14)
    uu = np.arange(n) - (n - 1) / 2
    truth = np.zeros((n, n))
    for c, s, a in zip(phan.centre, phan.size, phan.amp):
        truth += a * math.sqrt(2 * math.pi) * s * np.exp(-((uu[None, :] - c[0]) ** 2 + (uu[:, None] - c[1]) ** 2)
                                                         / (2 * s * s)) * delta
    ref = O.recon(truth[None], rot, lam=lam, delta=delta, defocus=[R], nz_layers=1, grid=(n, n, 1),
                  filt=O.FILTER_OFF, input_mode=O.INPUT_CONTRAST)[0]
    for sl in vol[10 * layer:10 * layer + 10]:  # voxel centres -19.5 .. -10.5 (+10 per layer)
        err = np.linalg.norm(sl - ref) / np.linalg.norm(ref)
        assert err < 2e-2, err


# ---------------------------------------------------------------- opposite-pair form (Eq. 10, 11)
def _pair_case(layer, filt, views):
    """Two weak blobs at the centre depth of layer `layer` of Nz = 4 over a 40-voxel-thick
    volume, imaged along the given single-axis angles by the 4-slab multislice simulator;
    returns the worst relative L2 error over that layer's volume slices against the same
    scan's filter-off reconstruction of the true projections."""
    n, nzv, nzl = 64, 40, 4
    delta, lam, sigma, R = 1e-9, 1e-10, 0.5, 2e-7
    z0 = -15.0 + 10.0 * layer
    phan = ph.Phantom("blob", np.array([[3.0, -2.0, z0], [-8.0, 5.0, z0]]), np.array([2.0, 3.0]),
                      np.array([2e-6, 1e-6]))
    rot = np.stack([ph.single_axis_rotations(1, start=a, span=0.0)[0] for a in views])
    Rs = np.full(len(views), R)
    img = ph.multislice_images(phan, rot, n, n, delta, lam, Rs, sigma, n_slabs=4, thickness=40.0,
                               dtype=__import__("torch").float64).numpy()
    truth = ph.layer_projections(phan, rot, n, n, (n, n, nzv), 1, delta)[:, 0]
    vol = O.recon(img, rot, lam=lam, delta=delta, defocus=Rs, nz_layers=nzl, grid=(n, n, nzv), sigma=sigma,
                  eps=1e-14, filt=filt)
    ref = O.recon(truth, rot, lam=lam, delta=delta, defocus=Rs, nz_layers=1, grid=(n, n, nzv), filt=O.FILTER_OFF,
                  input_mode=O.INPUT_CONTRAST)
    return max(np.linalg.norm(vol[q] - ref[q]) / np.linalg.norm(ref[q]) for q in range(10 * layer, 10 * layer + 10))


@pytest.mark.parametrize("layer", [0, 1, 3])
def test_pair_form_recovers_a_slab_from_a_view_and_its_opposite(layer):
    """Eq. 10: the images at opposite directions (0 and 180 degrees about y) together
    determine F3 delta on the Ewald paraboloid; with eps -> 0 the pair filter (the real part
    of each view's Eq. 11 term at the layer depth) returns the slab's true projection at
    its depth, for slabs upstream, near and downstream of the centre (0.25 % here).  One
    view alone is not enough: its imaginary part has no partner (error far above 100 %)."""
    assert _pair_case(layer, O.FILTER_PAIR, (0.0, math.pi)) < 1e-2
    assert _pair_case(layer, O.FILTER_PAIR, (0.0,)) > 1.0


def test_pair_filter_at_the_image_plane_is_the_real_bracket_inverse():
    """With eps -> 0 at depth 0 the pair filter reduces to Re{2 e^{-i chi} / sin 2 chi} =
    1 / sin chi, Eq. 13's inverse at the image-plane defocus (the identity linking Eq. 10
    and Eq. 11), away from the zeros of sin chi and cos chi."""
    P, delta, lam, sigma, R = 64, 1e-9, 1e-10, 0.3, 1.3e-7
    m = O.signed_freq(P).astype(float)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    chi = math.pi * lam * R * q2 - math.atan(sigma)
    a = O.ctf_pair_filter(P, delta, lam, R, 0.0, sigma, 1e-15)
    b = O.ctf_filter(P, delta, lam, R, sigma, 1e-15)
    good = (np.abs(np.sin(chi)) > 1e-3) & (np.abs(np.cos(chi)) > 1e-3)
    assert good.sum() > P * P // 2
    assert np.allclose(a[good], b[good], rtol=1e-6, atol=0)


# ---------------------------------------------------------------- linear blend between layers
def test_layer_blend_is_affine_in_the_exact_depth():
    """Layers that are affine in their index, Y_k = k U + V, blend to (t - 1/2) U + V with t
    the FP64 depth in layer units, (z' + T/2) / h from the rotation itself (z' = d_n . (r -
    centre), T the bounding-box extent along d_n, h = T / Nz): so the blend sits between
    the two layer centres around the depth, with the weight on the right one.  Checked
    away from the outer half-layers (where a single layer is taken)."""
    rng = np.random.default_rng(21)
    grid, nu, nv, nzl = (23, 17, 19), 40, 36, 6
    rot = ph.cone_rotations(4, 80.0, seed=5)
    A, B = O.pixel_coefficients(rot, grid, nu, nv)
    T = O.layer_constants(rot, grid, nzl)
    U, V = rng.standard_normal((nv, nu)), rng.standard_normal((nv, nu))
    stack = np.stack([k * U + V for k in range(nzl)])
    i, j, k = (rng.integers(0, g, 4000) for g in grid)
    cen = (np.array(grid) - 1) / 2.0
    for n in range(rot.shape[0]):
        got = O.backproject_direction(stack, A[n], B[n], T[n], i, j, k, O.LAYER_LINEAR)
        a = A[n, 0] * i + A[n, 1] * j + A[n, 2] * k + A[n, 3]
        b = B[n, 0] * i + B[n, 1] * j + B[n, 2] * k + B[n, 3]
        zp = rot[n, 2] @ (np.stack([i, j, k]) - cen[:, None])
        ext = np.abs(rot[n, 2]) @ np.array(grid, float)
        t = (zp + ext / 2) / (ext / nzl)
        inner = (t > 0.5 + 1e-5) & (t < nzl - 0.5 - 1e-5) & (a > 0) & (a < nu - 1) & (b > 0) & (b < nv - 1)
        want = (t - 0.5) * O.bilinear(U, a, b) + O.bilinear(V, a, b)
        assert inner.sum() > 1000
        assert np.max(np.abs(got[inner] - want[inner])) < 1e-5


def test_layer_blend_of_equal_layers_is_the_layer_itself():
    """Filter off, every layer is the same ramp-filtered image: the blend's weights sum to
    one, so it equals the nearest-layer volume (Eq. 15 is untouched)."""
    cfg_rot = ph.single_axis_rotations(12)
    rng = np.random.default_rng(4)
    img = (1 + 1e-2 * rng.standard_normal((12, 24, 24))).astype(np.float64)
    kw = dict(lam=1e-10, delta=1e-9, defocus=np.full(12, 1e-7), nz_layers=5, grid=(24, 24, 24), filt=O.FILTER_OFF)
    a = O.recon(img, cfg_rot, layer_interp=O.LAYER_NEAREST, **kw)
    b = O.recon(img, cfg_rot, layer_interp=O.LAYER_LINEAR, **kw)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.slow
def test_layer_blend_lowers_the_worst_slice_error_once_layers_are_thinner_than_the_dof():
    """Two smooth blobs (s = 5, 6 voxels) in a thin slab at each of ten depths of a
    40-voxel-thick volume, imaged along z by the multislice simulator; Nz = 8 layers, so the
    layer pitch equals the DOF Delta^2 / (2 lambda) of Sec. 1 (5 voxels).  The volume slice
    at the slab's depth is compared with the ramp-filtered true projection: blending the two
    bracketing layers keeps the worst case below that of the nearest layer (0.042 against
    0.056 here).  (With layers thicker than the DOF the blend is no better: the refocused
    image then depends on depth through the CTF's oscillation, not smoothly.)"""
    n, nzv, nzl = 64, 40, 8
    delta, lam, sigma, R = 1e-9, 1e-10, 0.5, 2e-7
    rot = np.eye(3)[None]
    uu = np.arange(n) - (n - 1) / 2
    worst = {O.LAYER_NEAREST: 0.0, O.LAYER_LINEAR: 0.0}
    for z0 in np.arange(-19.5, 20, 4.0):
        phan = ph.Phantom("blob", np.array([[3.0, -2.0, z0], [-8.0, 5.0, z0]]), np.array([5.0, 6.0]),
                          np.array([2e-6, 1e-6]))
        img = ph.multislice_images(phan, rot, n, n, delta, lam, np.array([R - z0 * delta]), sigma, n_slabs=1,
                                   thickness=1.0, dtype=__import__("torch").float64).numpy()
        truth = np.zeros((n, n))
        for c, s, a in zip(phan.centre, phan.size, phan.amp):
            truth += a * math.sqrt(2 * math.pi) * s * np.exp(
                -((uu[None, :] - c[0]) ** 2 + (uu[:, None] - c[1]) ** 2) / (2 * s * s)) * delta
        ref = O.recon(truth[None], rot, lam=lam, delta=delta, defocus=[R], nz_layers=1, grid=(n, n, 1),
                      filt=O.FILTER_OFF, input_mode=O.INPUT_CONTRAST)[0]
        kk = int(round(z0 + (nzv - 1) / 2))
        for mode in worst:
            vol = O.recon(img, rot, lam=lam, delta=delta, defocus=[R], nz_layers=nzl, grid=(n, n, nzv),
                          sigma=sigma, eps=1e-14, layer_interp=mode)
            worst[mode] = max(worst[mode], np.linalg.norm(vol[kk] - ref) / np.linalg.norm(ref))
    assert worst[O.LAYER_LINEAR] < 0.85 * worst[O.LAYER_NEAREST], worst


# ---------------------------------------------------------------- layer decision
def test_layer_index_matches_fp64_depth_away_from_boundaries():
    rng = np.random.default_rng(3)
    grid = (20, 13, 17)
    rot = ph.cone_rotations(16, 80.0, seed=5)
    T = O.layer_constants(rot, grid, 6)
    ext = O.depth_extent(rot, grid)
    kk, jj, ii = np.meshgrid(*(np.arange(g) for g in grid[::-1]), indexing="ij")
    i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
    c = np.array([(g - 1) / 2 for g in grid])
    checked = 0
    for n in range(rot.shape[0]):
        zp = rot[n, 2, 0] * (i - c[0]) + rot[n, 2, 1] * (j - c[1]) + rot[n, 2, 2] * (k - c[2])
        t = (zp + ext[n] / 2) / (ext[n] / 6)
        far = np.abs(t - np.round(t)) > 1e-5
        ref = np.clip(np.floor(t), 0, 5).astype(np.int64)
        got = O.layer_index(T[n], 6, i, j, k)
        assert np.array_equal(got[far], ref[far])
        assert got.min() >= 0 and got.max() <= 5
        checked += far.sum()
    assert checked > 0.99 * rot.shape[0] * i.size
    del rng


# ---------------------------------------------------------------- backprojection brute force
def test_backprojection_matches_pure_python_loops():
    """Vectorised per-direction backprojection against per-voxel loops that go through
    the rotation directly (no precomputed coefficients)."""
    rng = np.random.default_rng(11)
    grid, nu, nv, nzl = (5, 4, 6), 7, 5, 3
    rot = ph.cone_rotations(3, 90.0, seed=2)
    stack = rng.standard_normal((rot.shape[0], nzl, nv, nu))
    A, B = O.pixel_coefficients(rot, grid, nu, nv)
    T = O.layer_constants(rot, grid, nzl)
    ext = O.depth_extent(rot, grid)
    c = np.array([(g - 1) / 2 for g in grid])
    kk, jj, ii = np.meshgrid(*(np.arange(g) for g in grid[::-1]), indexing="ij")
    i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
    for n in range(rot.shape[0]):
        got = O.backproject_direction(stack[n], A[n], B[n], T[n], i, j, k)
        for idx in range(i.size):
            r = np.array([i[idx], j[idx], k[idx]]) - c
            x, y, z = rot[n] @ r
            a, b = x + (nu - 1) / 2, y + (nv - 1) / 2
            t = (z + ext[n] / 2) / (ext[n] / nzl)
            if abs(t - round(t)) < 1e-6:
                continue
            lay = min(max(int(math.floor(t)), 0), nzl - 1)
            a0, b0 = math.floor(a), math.floor(b)
            val = 0.0
            for db in (0, 1):
                for da in (0, 1):
                    w = (a - a0 if da else 1 - (a - a0)) * (b - b0 if db else 1 - (b - b0))
                    if 0 <= a0 + da < nu and 0 <= b0 + db < nv:
                        val += w * stack[n, lay, b0 + db, a0 + da]
            assert abs(got[idx] - val) < 1e-12


# ---------------------------------------------------------------- closed-form ball (FBP)
def test_fbp_of_closed_form_ball_radon_recovers_delta():
    """Projection input of a uniform ball, filter off (Eq. 15 / conventional CT): the
    reconstruction inside the ball equals its decrement."""
    n, D = 64, 180
    grid = (n, n, n)
    ball = ph.Phantom("ball", np.array([[4.0, -3.0, 5.0]]), np.array([14.0]), np.array([1.0]))
    rot = ph.single_axis_rotations(D)
    proj = ph.ball_projections(ball, rot, n, n)  # voxel-length units (delta = 1)
    # voxels of the central y-slab through the ball centre
    j0 = int(round(ball.centre[0, 1] + (n - 1) / 2))
    kk, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, k = ii.ravel(), kk.ravel()
    j = np.full_like(i, j0)
    vals = O.recon(proj, rot, lam=1.0, delta=1.0, defocus=np.zeros(D), nz_layers=1, grid=grid,
                   filt=O.FILTER_OFF, input_mode=O.INPUT_CONTRAST, voxels=(i, j, k))
    c = ball.centre[0] + (n - 1) / 2
    rr = np.sqrt((i - c[0]) ** 2 + (j - c[1]) ** 2 + (k - c[2]) ** 2)
    inner = rr < 0.8 * ball.size[0]
    outer = rr > 1.25 * ball.size[0]
    assert np.linalg.norm(vals[inner] - 1.0) / np.sqrt(inner.sum()) < 1e-2
    assert np.sqrt(np.mean(vals[outer & (np.hypot(i - 31.5, k - 31.5) < 28)] ** 2)) < 2e-2


def test_filter_off_single_layer_is_textbook_fbp_slice_by_slice():
    """Nz = 1, filter off, a single-axis scan about y: the operator is parallel-beam FBP of
    each detector row (Eq. 15), written here independently: the band-limited Ram-Lak kernel
    convolved in real space over every shift the row needs (no DFT), scaled by pi/D and the
    pitch, then linear interpolation along the detector u axis of each view, zero outside."""
    rng = np.random.default_rng(21)
    D, nu, nx, ny, nz, delta = 16, 24, 20, 5, 17, 0.5
    rot = ph.single_axis_rotations(D, start=0.2)
    proj = rng.standard_normal((D, ny, nu))  # projection input, nv = ny: row v is slice j
    vol = O.recon(proj, rot, lam=1.0, delta=delta, defocus=np.zeros(D), nz_layers=1, grid=(nx, ny, nz),
                  filt=O.FILTER_OFF, input_mode=O.INPUT_CONTRAST)
    shifts = np.arange(-(nu - 1), nu)
    h = np.where(shifts == 0, 1 / (4 * delta ** 2),
                 np.where(shifts % 2 != 0, -1 / (shifts.astype(float) ** 2 * np.pi ** 2 * delta ** 2), 0.0))
    ref = np.zeros((nz, ny, nx))
    for n in range(D):
        # q[v, u] = (pi / D) * delta * sum_u' p[v, u'] h[u - u']
        q = np.zeros((ny, nu))
        for u in range(nu):
            for up in range(nu):
                q[:, u] += proj[n, :, up] * h[u - up + nu - 1]
        q *= np.pi / D * delta
        ux = rot[n, 0]  # the view's detector u axis in the volume frame
        for k in range(nz):
            for i in range(nx):
                r = np.array([i - (nx - 1) / 2, 0.0, k - (nz - 1) / 2])
                u = ux[0] * r[0] + ux[2] * r[2] + (nu - 1) / 2  # ux[1] = 0 about y
                u0 = int(np.floor(u))
                f = u - u0
                left = q[:, u0] if 0 <= u0 < nu else 0.0
                right = q[:, u0 + 1] if 0 <= u0 + 1 < nu else 0.0
                ref[k, :, i] += (1 - f) * left + f * right
    assert np.max(np.abs(vol - ref)) <= 1e-10 * np.max(np.abs(ref))


# ---------------------------------------------------------------- invariants
def _small_case(seed=4, D=12, grid=(10, 9, 8), nu=12, nv=11):
    rng = np.random.default_rng(seed)
    rot = ph.cone_rotations(D, 70.0, seed=seed)
    img = 1.0 + 1e-3 * rng.standard_normal((D, nv, nu))
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 80e-9, D), nz_layers=3, grid=grid,
              sigma=0.05, eps=0.01)
    return rot, img, kw


def test_linearity_in_contrast():
    rot, img, kw = _small_case()
    g1 = np.log(img)
    g2 = np.random.default_rng(9).standard_normal(g1.shape) * 1e-3
    r1 = O.recon(g1, rot, input_mode=O.INPUT_CONTRAST, **kw)
    r2 = O.recon(g2, rot, input_mode=O.INPUT_CONTRAST, **kw)
    r12 = O.recon(2.5 * g1 - 0.75 * g2, rot, input_mode=O.INPUT_CONTRAST, **kw)
    assert np.max(np.abs(r12 - (2.5 * r1 - 0.75 * r2))) <= 1e-12 * np.max(np.abs(r12))


def test_intensity_input_is_log_of_contrast():
    rot, img, kw = _small_case()
    a = O.recon(img, rot, input_mode=O.INPUT_INTENSITY, **kw)
    b = O.recon(np.log(img), rot, input_mode=O.INPUT_CONTRAST, **kw)
    assert np.array_equal(a, b)


def test_filter_off_layers_are_all_equal_to_single_layer():
    """With the CTF filter off every layer is the same ramp-filtered image, so Nz layers
    give exactly the Nz = 1 result (the conventional-FBP special case)."""
    rot, img, kw = _small_case()
    kw4 = dict(kw, nz_layers=4)
    kw1 = dict(kw, nz_layers=1)
    a = O.recon(img, rot, filt=O.FILTER_OFF, **kw4)
    b = O.recon(img, rot, filt=O.FILTER_OFF, **kw1)
    assert np.array_equal(a, b)


def test_rotating_every_view_rotates_the_volume():
    """Composing every direction with a 90-degree turn Q about z gives vol'(r) = vol(Q r)."""
    grid = (9, 9, 7)
    rot, img, kw = _small_case(grid=grid)
    kw = dict(kw, grid=grid)
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    a = O.recon(img, rot, **kw)
    b = O.recon(img, rot @ Q, **kw)
    # b[k, j, i] = a at Q (i-c, j-c, k-c): x' = -(j - c), y' = (i - c)
    c = (grid[0] - 1) // 2
    kk, jj, ii = np.meshgrid(np.arange(grid[2]), np.arange(grid[1]), np.arange(grid[0]), indexing="ij")
    expect = a[kk, ii, 2 * c - jj]
    assert np.max(np.abs(b - expect)) <= 1e-9 * np.max(np.abs(a))


def test_projection_sums_equal_volume_integral():
    """Mean preservation, exact part: every view of a ball inside the field of view
    carries its whole volume integral (4/3) pi r^3 delta."""
    ball = ph.Phantom("ball", np.array([[2.0, 1.0, -3.0]]), np.array([9.0]), np.array([1.0]))
    rot = ph.cone_rotations(5, 90.0, seed=1)
    proj = ph.ball_projections(ball, rot, 48, 48)
    vol = 4 / 3 * math.pi * 9.0 ** 3
    assert np.allclose(proj.sum(axis=(1, 2)), vol, rtol=2e-3)


# ---------------------------------------------------------------- physics (Sec. 3, Ewald on/off)
@pytest.mark.slow
def test_layering_beats_single_layer_when_dof_is_shallow():
    """With DOF = delta^2/(2 lambda) much smaller than the object, the layered
    reconstruction (Nz = 8) is closer to the phantom than the Nz = 1 one (the Ewald-off
    variant of Sec. 3), measured on the band-limited phantom."""
    n, D = 32, 48
    grid = (n, n, n)
    delta, lam, sigma = 1e-9, 1e-9, 0.3  # DOF = 0.5 nm vs 32 nm
    phan = ph.blob_phantom(grid, 30, seed=8, s_vox=1.0, amp_unit=5e-6)
    rot = ph.single_axis_rotations(D)
    R = np.full(D, 30e-9)
    img = ph.multislice_images(phan, rot, n, n, delta, lam, R, sigma, n_slabs=32,
                               dtype=__import__("torch").float64).numpy()
    kw = dict(lam=lam, delta=delta, defocus=R, grid=grid, sigma=sigma, eps=1e-2)
    r8 = O.recon(img, rot, nz_layers=8, **kw)
    r1 = O.recon(img, rot, nz_layers=1, **kw)
    kk, jj, ii = np.meshgrid(*(np.arange(n) - (n - 1) / 2,) * 3, indexing="ij")
    truth = np.zeros(grid)
    for c, s, a in zip(phan.centre, phan.size, phan.amp):
        truth += a * np.exp(-((ii - c[0]) ** 2 + (jj - c[1]) ** 2 + (kk - c[2]) ** 2) / (2 * s * s))
    e8 = np.linalg.norm(r8 - truth) / np.linalg.norm(truth)
    e1 = np.linalg.norm(r1 - truth) / np.linalg.norm(truth)
    assert e8 < 0.75 * e1, (e8, e1)


# ---------------------------------------------------------------- first Born forward model (Eq. 3, Eq. 7)
def _lowpass(v, qc):
    """The 3D spectrum of ``v`` kept below ``qc`` cycles per voxel."""
    f = [np.fft.fftfreq(m) for m in v.shape]
    q = np.sqrt(f[0][:, None, None] ** 2 + f[1][None, :, None] ** 2 + f[2][None, None, :] ** 2)
    return np.fft.ifftn(np.fft.fftn(v) * (q < qc)).real


def _born_spheres():
    """Six small uniform spheres (radius 2.5-4 voxels) in a 32^3 grid under a 48-view
    single-axis scan, imaged by the first-Born model.  The image planes sit 24 nm upstream
    of the rotation centre (negative defocus), 8-40 nm from every object plane, so within
    |q| <= 1/(2 Delta) the CTF phase stays within (-pi, 0): sin chi has no zero there and the
    inverse with a vanishing eps is well posed.  DOF = 6.25 nm against 32 nm of object."""
    n, D = 32, 48
    grid = (n, n, n)
    case = dict(delta=1e-9, lam=8e-11, sigma=0.3, grid=grid)
    rot = ph.single_axis_rotations(D)
    R = np.full(D, -24e-9)
    phan = ph.ball_phantom(grid, 6, seed=3, r_range=(2.5, 4.0), delta_range=(1e-6, 2e-6))
    img = ph.born_images(phan, rot, n, n, case["delta"], case["lam"], R, case["sigma"])
    kk, jj, ii = np.meshgrid(*(np.arange(n) - (n - 1) / 2,) * 3, indexing="ij")
    truth = np.zeros(grid)
    for c, r, a in zip(phan.centre, phan.size, phan.amp):
        truth += a * (((ii - c[0]) ** 2 + (jj - c[1]) ** 2 + (kk - c[2]) ** 2) <= r * r)
    return phan, rot, R, img, truth, case


def test_first_born_and_multislice_images_agree_to_first_order():
    """The two forward models share only the Fresnel propagator: for weak spheres their
    log-intensities agree to 1 %; at 100 times the decrement they part by over 5 % (the multislice keeps
    multiple scattering and the whole exponential), so the agreement is first-order."""
    import torch
    n, rot = 32, ph.single_axis_rotations(8)
    R = np.full(8, -24e-9)
    cases = []
    for amp, lo, hi in ((2e-6, 0.0, 0.01), (2e-4, 0.05, np.inf)):  # spheres: 0.2 % and 12.7 % measured
        cases.append((ph.ball_phantom((n, n, n), 6, seed=3, r_range=(2.5, 4.0), delta_range=(amp / 2, amp)), lo, hi))
    for amp, lo, hi in ((2e-6, 0.0, 0.01), (2e-4, 0.05, np.inf)):  # Gaussian blobs: 0.5 % and 59 %
        cases.append((ph.blob_phantom((n, n, n), 10, seed=4, s_vox=1.5, amp_unit=amp), lo, hi))
    for phan, lo, hi in cases:
        amp = float(phan.amp.max())
        born = ph.born_images(phan, rot, n, n, 1e-9, 8e-11, R, 0.3)
        ms = ph.multislice_images(phan, rot, n, n, 1e-9, 8e-11, R, 0.3, n_slabs=64, dtype=torch.float64).numpy()
        d = np.linalg.norm(np.log(born) - np.log(ms)) / np.linalg.norm(np.log(ms))
        assert lo <= d < hi, (amp, d)


def test_layered_operator_recovers_small_spheres_from_first_born_images():
    """The whole operator (contrast, per-layer CTF inverse at R - z_k, ramp, layered
    backprojection) on first-Born images of small spheres: within 8 % (13 % up to 0.3
    cycles per voxel) of the spheres, both low-passed alike (6.2 % and 10.8 % measured).
    Reconstructing with the defocus of the wrong sign, none, or twice the true one at least
    doubles the error, so the defocus enters with its sign and scale; layers refocused at
    R + z_k instead of R - z_k give 9.9 % (checked by mutation)."""
    phan, rot, R, img, truth, case = _born_spheres()
    kw = dict(lam=case["lam"], delta=case["delta"], nz_layers=16, grid=case["grid"], sigma=case["sigma"], eps=1e-6)

    def err(defocus, qc):
        r = O.recon(img, rot, defocus=defocus, **kw)
        t = _lowpass(truth, qc)
        return np.linalg.norm(_lowpass(r, qc) - t) / np.linalg.norm(t)

    e2, e3 = err(R, 0.2), err(R, 0.3)
    assert e2 < 0.08 and e3 < 0.13, (e2, e3)
    for wrong in (-R, 0 * R, 2 * R):
        assert err(wrong, 0.2) > 2 * e2


# ---------------------------------------------------------------- sampling density (Sec. 2, S(q))
def test_density_weights_reduce_to_the_ramp_for_a_single_axis_scan():
    """Gridded sampling density of a 180-degree single-axis scan: W -> pi |q_u| / D (the
    ramp that Sec. 2 says the sampling coefficients approximate), away from DC."""
    P, D, delta = 128, 180, 1e-9
    rot = ph.single_axis_rotations(D)
    W = O.density_weights(rot, P, delta)[::45]
    m = O.signed_freq(P)
    ideal = math.pi / D * np.abs(m) / (P * delta)
    band = (np.abs(m) >= 4) & (np.abs(m) <= P // 4)
    rows = np.abs(m) <= P // 4
    for w in W:
        ratio = w[np.ix_(rows, band)] / ideal[band][None, :]
        assert 0.9 < ratio.min() and ratio.max() < 1.05
    # even in q (needed for a real inverse transform)
    assert np.allclose(W[1], W[1][(-m) % P][:, (-m) % P], rtol=1e-12)


def test_density_weighted_fbp_of_a_ball_from_random_directions():
    """Any plane-wave scan (Sec. 2): projections of a uniform ball from 200 Haar-random
    directions, weighted by the inverse sampling density, reconstruct its decrement."""
    n, D = 32, 200
    grid = (n, n, n)
    ball = ph.Phantom("ball", np.array([[2.0, -1.5, 3.0]]), np.array([8.0]), np.array([1.0]))
    rot = ph.cone_rotations(D, 90.0, seed=3)
    proj = ph.ball_projections(ball, rot, n, n)
    vol = O.recon(proj, rot, lam=1.0, delta=1.0, defocus=np.zeros(D), nz_layers=1, grid=grid, filt=O.FILTER_OFF,
                  input_mode=O.INPUT_CONTRAST, density=True)
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = ball.centre[0] + (n - 1) / 2
    rr = np.sqrt((ii - c[0]) ** 2 + (jj - c[1]) ** 2 + (kk - c[2]) ** 2)
    inner = rr < 0.8 * 8
    assert abs(vol[inner].mean() - 1.0) < 0.03
    assert np.sqrt(np.mean((vol[inner] - 1.0) ** 2)) < 0.04


def test_density_weighting_is_invariant_to_repeating_the_scan():
    """S counts every view's samples, so recording each view twice doubles S (and the band
    mean that sets eps_S) and halves every weight: the reconstruction is unchanged.  A
    weight that is not the inverse of the gridded density would change with the repeat."""
    n, D = 24, 10
    grid = (n, n, n)
    ball = ph.Phantom("ball", np.array([[1.0, -2.0, 2.5]]), np.array([6.0]), np.array([1.0]))
    rot = ph.cone_rotations(D, 70.0, seed=11)
    proj = ph.ball_projections(ball, rot, n, n)
    kw = dict(lam=1.0, delta=1.0, nz_layers=1, grid=grid, filt=O.FILTER_OFF, input_mode=O.INPUT_CONTRAST,
              density=True)
    once = O.recon(proj, rot, defocus=np.zeros(D), **kw)
    twice = O.recon(np.concatenate([proj, proj]), np.concatenate([rot, rot]), defocus=np.zeros(2 * D), **kw)
    assert np.linalg.norm(twice - once) <= 1e-10 * np.linalg.norm(once)


def test_process_pool_sums_the_same_terms():
    """The spawned pool (used for the full-size parity cases) splits the directions over
    workers: the same terms summed in another order."""
    rot, img, kw = _small_case(seed=9, D=10)
    i = np.arange(10) % kw["grid"][0]
    j = (np.arange(10) * 3) % kw["grid"][1]
    k = (np.arange(10) * 7) % kw["grid"][2]
    a = O.recon(img, rot, voxels=(i, j, k), density=True, **kw)
    b = O.recon(img, rot, voxels=(i, j, k), density=True, workers=3, **kw)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_batch_workloads_span_the_stated_ranges():
    cfgs = ph.batch_workloads()
    assert len(cfgs) == 48
    assert all(64 <= c["grid"][0] <= 256 and c["grid"][0] % 32 == 0 and c["nu"] == c["grid"][0] for c in cfgs)
    assert all(60 <= c["n_dir"] <= 360 and 4 <= c["nz_layers"] <= 32 for c in cfgs)
    assert {c["phantom"] for c in cfgs} == {"balls", "blobs"} and len({c["lam"] for c in cfgs}) == 2
    assert all(c["rot"].shape == (c["n_dir"], 3, 3) and len(c["defocus"]) == c["n_dir"] for c in cfgs)
