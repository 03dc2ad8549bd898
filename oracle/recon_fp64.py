"""FP64 CPU oracle of the layered unified tomographic reconstruction (UTR).

TEST INFRASTRUCTURE ONLY.  Plain, slow, written to be checked against the paper by
eye.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the reconstruction library
never does, and this module shares no code with it.

What it computes, in the paper's order and notation (Sec. 2):

1. Contrast g_n = ln(I_n / I_in) (Eq. 4's left side), or the image as given.
2. G_n = 2D DFT of g_n zero-padded to P x P (F2 with kernel exp(-i 2 pi r.q), Eq. 3).
3. For each depth layer k of direction n, the real part of Eq. 11's bracket at the
   layer's own defocus R_n - z_k (Eq. 5 and Eq. 7 place a slice at depth z at
   defocus R - z; Eq. 13 is the single-layer case):
       chi_k(q) = pi*lambda*(R_n - z_k)*q^2 + (pi/2)*Cs*lambda^3*q^4 - omega,
       omega = atan(sigma)                                         (Eq. 7)
       H_k(q)   = lambda / (4 pi sqrt(1+sigma^2)) * sin chi / (sin^2 chi + eps)
   The Cs term is the per-view aberration that Sec. 2 allows in the sine argument.
4. The sampling-density weight of a single-axis scan, the ramp |q_x| (Sec. 2),
   discretised as the band-limited Ram-Lak kernel and scaled by pi/D.
5. Y_{n,k} = crop( Re IDFT[ G_n * H_k * W ] ): the layer stack.
6. Backprojection: every voxel takes, from each direction, a bilinear sample of the
   layer that contains its depth, and sums over directions.  Optionally (``layer_interp
   = LAYER_LINEAR``) it takes the linear blend of the samples of the two layers whose
   centres bracket its depth, which keeps the layers' defocus error below half a layer
   once the layers are thinner than the DOF Delta^2 / (2 lambda) of Sec. 1.

Readings where the paper is silent (each is listed in the design notes):
* layers are Nz equal slabs over the volume's bounding-box extent along the beam,
  centred on the rotation centre; the layer index is decided in 2^-24 fixed point
  (``layer_constants``), so that every implementation takes the same decision;
* P = smallest power of two >= 2*max(nu, nv), zero padding;
* pixel and voxel centres at (index - (n-1)/2) * delta; bilinear, zero outside the
  detector; nearest (containing) layer, or the blend of the two whose centres bracket
  the depth (layer k centred at k + 1/2 in layer units; beyond the outer centres the
  outer layer alone);
* intensities are floored at 1e-6 before the logarithm.

Every function states the passage it follows.  Pins (tests marked ``not gpu``) tie
each step to closed forms, brute force and invariants; none re-types these
formulas.
"""
from __future__ import annotations

import math

import numpy as np

INTENSITY_FLOOR = 1e-6
LAYER_FRAC_BITS = 24

LAYER_NEAREST = 0  # a voxel takes the layer that contains its depth
LAYER_LINEAR = 1   # a voxel takes the linear blend of the two layers whose centres bracket it

FILTER_OFF = 0
FILTER_TIKHONOV = 1
FILTER_PAIR = 2  # the complex bracket of Eq. 11, exact for opposite-view pairs (Eq. 10)
FILTER_DEPTH_COS = 3  # per layer cos(pi lambda z_k q^2): the real part of the Ewald placement
FILTER_DEPTH_SIN = 4  # per layer sin(pi lambda z_k q^2): minus its imaginary part
INPUT_INTENSITY = 0
INPUT_CONTRAST = 1


def padded_size(n: int) -> int:
    """Smallest power of two >= 2n (zero padding so that the circular filters act as
    linear ones on the n-pixel field of view)."""
    p = 1
    while p < 2 * n:
        p *= 2
    return p


def signed_freq(P: int) -> np.ndarray:
    """DFT bin index -> signed integer frequency m in [-P/2, P/2)."""
    m = np.arange(P)
    return np.where(m < P // 2, m, m - P)


# ----------------------------------------------------------------------------- geometry
def pixel_coefficients(rot: np.ndarray, grid, nu: int, nv: int) -> tuple[np.ndarray, np.ndarray]:
    """Affine maps voxel index -> detector pixel coordinate, a = A . (i, j, k, 1) and
    b = B . (i, j, k, 1), from the beam-frame position Rot_n (r - centre) (the
    plane-wave projection geometry of Sec. 2, any orientation)."""
    nx, ny, nz = grid
    c = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    A = np.zeros((rot.shape[0], 4))
    B = np.zeros((rot.shape[0], 4))
    A[:, :3] = rot[:, 0, :]
    B[:, :3] = rot[:, 1, :]
    A[:, 3] = (nu - 1) / 2.0 - rot[:, 0, :] @ c
    B[:, 3] = (nv - 1) / 2.0 - rot[:, 1, :] @ c
    return A, B


def depth_extent(rot: np.ndarray, grid) -> np.ndarray:
    """Extent, in voxel lengths, of the volume's bounding box along each beam axis:
    sum_i |d_n . e_i| * N_i."""
    nx, ny, nz = grid
    r2 = rot[:, 2, :]
    return np.abs(r2[:, 0]) * nx + np.abs(r2[:, 1]) * ny + np.abs(r2[:, 2]) * nz


def layer_centres(rot: np.ndarray, grid, nz_layers: int, delta: float) -> np.ndarray:
    """Depth z_k of each layer centre (metres, beam frame, rotation centre at 0): the
    slabs of Eq. 5 placed as Nz equal slabs over the bounding-box extent."""
    ext = depth_extent(rot, grid) * delta
    k = np.arange(nz_layers)
    return -ext[:, None] / 2.0 + (k[None, :] + 0.5) * (ext[:, None] / nz_layers)


def layer_constants(rot: np.ndarray, grid, nz_layers: int) -> np.ndarray:
    """Fixed-point (2^-24 layer) coefficients (T0, Ti, Tj, Tk) per direction, int64.

    t = (z' + T/2) / h in layer units is affine in the voxel index; its FP64
    coefficients are rounded to the nearest multiple of 2^-24 (ties to even), and
    the layer is floor(t) of the exact integer sum.  Written so that the operations
    and their order are fixed: ext, scale, ti/tj/tk, t0 as below."""
    nx, ny, nz = grid
    r2 = rot[:, 2, :]
    ext = (np.abs(r2[:, 0]) * float(nx) + np.abs(r2[:, 1]) * float(ny)) + np.abs(r2[:, 2]) * float(nz)
    scale = float(nz_layers) / ext
    ti = r2[:, 0] * scale
    tj = r2[:, 1] * scale
    tk = r2[:, 2] * scale
    t0 = 0.5 * float(nz_layers) - ((ti * (0.5 * (nx - 1)) + tj * (0.5 * (ny - 1))) + tk * (0.5 * (nz - 1)))
    one = float(1 << LAYER_FRAC_BITS)
    return np.stack([np.rint(t0 * one), np.rint(ti * one), np.rint(tj * one), np.rint(tk * one)],
                    axis=1).astype(np.int64)


def layer_index(T: np.ndarray, nz_layers: int, i, j, k) -> np.ndarray:
    """Layer of voxel (i, j, k) for one direction's constants ``T`` (exact integers)."""
    t = T[0] + T[1] * np.asarray(i, np.int64) + T[2] * np.asarray(j, np.int64) + T[3] * np.asarray(k, np.int64)
    return np.clip(t >> LAYER_FRAC_BITS, 0, nz_layers - 1)


def layer_blend(T: np.ndarray, nz_layers: int, i, j, k) -> tuple[np.ndarray, np.ndarray]:
    """Linear blend between adjacent layers: the two layers whose centres bracket the
    voxel's depth, k0 and k0 + 1, with weight w on k0 + 1.  In layer units the depth is
    t (the exact 2^-24 fixed-point sum of ``layer_index``) and layer k is centred at
    k + 1/2, so t' = t - 1/2, k0 = floor(t'), w = t' - k0; above the first centre (t' < 0)
    and below the last (k0 >= Nz - 1) a voxel takes that layer alone (w = 0).  Returns
    (k0, w) with w exact (a 24-bit fraction)."""
    t = T[0] + T[1] * np.asarray(i, np.int64) + T[2] * np.asarray(j, np.int64) + T[3] * np.asarray(k, np.int64)
    tp = t - (1 << (LAYER_FRAC_BITS - 1))
    k0 = tp >> LAYER_FRAC_BITS
    w = (tp - (k0 << LAYER_FRAC_BITS)).astype(np.float64) / float(1 << LAYER_FRAC_BITS)
    below = k0 < 0
    above = k0 >= nz_layers - 1
    k0 = np.where(below, 0, np.where(above, nz_layers - 1, k0))
    w = np.where(below | above, 0.0, w)
    return k0, w


# ----------------------------------------------------------------------------- filters
def ramp_weights(P: int, delta: float, n_dir: int) -> np.ndarray:
    """W[m], m = DFT bin: (pi/D) * delta * DFT_P[h](m) with the band-limited Ram-Lak
    kernel h[0] = 1/(4 delta^2), h[odd n] = -1/(n^2 pi^2 delta^2), h[even n != 0] = 0,
    for n in [-P/2, P/2).  This discretises the ramp |q_x| that Sec. 2 identifies as
    the sampling-matrix inverse of a 180-degree single-axis scan; pi/D is the
    angular step of the backprojection sum."""
    n = signed_freq(P)
    h = np.zeros(P)
    h[n == 0] = 1.0 / (4.0 * delta * delta)
    odd = (n % 2) != 0
    h[odd] = -1.0 / (n[odd].astype(np.float64) ** 2 * math.pi ** 2 * delta * delta)
    return (math.pi / n_dir) * delta * np.fft.fft(h).real


def ctf_filter(P: int, delta: float, lam: float, r_eff: float, sigma: float, eps: float,
               cs: float = 0.0) -> np.ndarray:
    """H(q) on the P x P DFT grid for one layer at effective defocus ``r_eff``:
    lambda / (4 pi sqrt(1+sigma^2)) * sin(chi) / (sin(chi)^2 + eps), the real part of
    the bracket of Eq. 11 with chi = pi*lambda*r_eff*q^2 + (pi/2)*Cs*lambda^3*q^4 - omega
    (omega = atan sigma, Eq. 7).  With eps = 0 it is Eq. 13's inverse sine."""
    m = signed_freq(P).astype(np.float64)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    chi = math.pi * lam * r_eff * q2 + 0.5 * math.pi * cs * lam ** 3 * q2 * q2 - math.atan(sigma)
    s = np.sin(chi)
    return lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma)) * s / (s * s + eps)


def ctf_pair_filter(P: int, delta: float, lam: float, r_n: float, z_k: float, sigma: float, eps: float,
                    cs: float = 0.0) -> np.ndarray:
    """Per-layer filter of the opposite-pair form: the real part of one view's Eq. 11 term
    carried to depth z_k,
        lambda / (4 pi sqrt(1+sigma^2)) * Re{ [sin chi / (sin^2 chi + eps)
                                               - i cos chi / (cos^2 chi + eps)] * exp(-i pi lambda z_k q^2) },
    chi = pi lambda R_n q^2 + (pi/2) Cs lambda^3 q^4 - omega at the view's own image plane
    (Eq. 11).  The complex term sits on the Ewald paraboloid (q, -lambda q^2 / 2) (Eq. 8);
    its inverse 3D transform at depth z carries the factor exp(-i pi lambda z q^2) (z
    positive downstream, so that the defocus of depth z is R - z as in Eq. 5).  A single
    view's term is complex; summed with the opposite view's (Eq. 9: its depth -z, mirrored
    u) the imaginary parts cancel and Eq. 10 follows, so the real part of each term is the
    term's share of the real reconstruction."""
    m = signed_freq(P).astype(np.float64)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    chi = math.pi * lam * r_n * q2 + 0.5 * math.pi * cs * lam ** 3 * q2 * q2 - math.atan(sigma)
    s, c = np.sin(chi), np.cos(chi)
    bracket = s / (s * s + eps) - 1j * c / (c * c + eps)
    depth = np.exp(-1j * math.pi * lam * z_k * q2)
    return lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma)) * (bracket * depth).real


def depth_phase_filter(P: int, delta: float, lam: float, z_k: float, sine: bool) -> np.ndarray:
    """cos or sin of pi lambda z_k q^2 on the P x P DFT grid: the real part and minus the
    imaginary part of exp(-i pi lambda z_k q^2), which carries a sample of the Ewald
    paraboloid (q, -lambda q^2 / 2) to depth z_k (Eq. 8).  With these per-layer filters and
    no CTF bracket the layered reconstruction is the CT step of Eq. 12 (the Ewald-placed
    reconstruction of the contrasts, as two real volumes)."""
    m = signed_freq(P).astype(np.float64)
    q2 = (m[None, :] ** 2 + m[:, None] ** 2) / (P * delta) ** 2
    ph = math.pi * lam * z_k * q2
    return np.sin(ph) if sine else np.cos(ph)


# ----------------------------------------------------------------------------- density
DENSITY_EPS_REL = 1e-3


def density_geometry(P: int) -> tuple[int, int]:
    """Sampling step s (in DFT bins) and half-width Gh of the 3D density grid: the grid
    has (2 Gh + 1)^3 cells of s bins, covering every slice point of norm <= sqrt(2) P/2."""
    s = max(1, P // 128)
    Gh = int(math.ceil(math.sqrt(2.0) * (P / 2) / s)) + 2
    return s, Gh


def density_grid(rot: np.ndarray, P: int) -> np.ndarray:
    """S: the sampling matrix of Sec. 2.  Every image's 2D DFT samples (m_u, m_v), taken
    every s bins with weight s^2, sit at m_u u_n + m_v v_n in 3D frequency space (u_n, v_n:
    the detector axes, rows 0 and 1 of Rot_n) and are spread over the 8 surrounding cells
    of the grid with trilinear weights summing to one; each sample is entered at q and at
    -q with half weight, so that S (and the weight) are even in q."""
    s, Gh = density_geometry(P)
    G = 2 * Gh + 1
    S = np.zeros(G * G * G)
    m = np.arange(-P // 2, P // 2, s, dtype=np.float64)
    mu, mv = np.meshgrid(m, m, indexing="ij")
    mu, mv = mu.ravel(), mv.ravel()
    for n in range(rot.shape[0]):
        q0 = (mu[:, None] * rot[n, 0][None, :] + mv[:, None] * rot[n, 1][None, :]) / s  # grid units
        for q in (q0, -q0):  # the sample and its mirror, half weight each (S even in q)
            base = np.floor(q).astype(np.int64)
            f = q - base
            idx = base + Gh
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                             * (f[:, 2] if dz else 1 - f[:, 2]))
                        cell = ((idx[:, 2] + dz) * G + (idx[:, 1] + dy)) * G + (idx[:, 0] + dx)
                        np.add.at(S, cell, w * 0.5 * s * s)
    return S.reshape(G, G, G)  # [z][y][x]


def density_ball_count(Gh: int) -> tuple[np.ndarray, int]:
    """Cells within Gh - 2 of the grid centre (the band): mask and count."""
    G = 2 * Gh + 1
    c = np.arange(G) - Gh
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    mask = (xx * xx + yy * yy + zz * zz) <= (Gh - 2) ** 2
    return mask, int(mask.sum())


def density_weights(rot: np.ndarray, P: int, delta: float, dirs=None) -> np.ndarray:
    """W_n(q) = g / (S(m_u u_n + m_v v_n) + eps_S) on each direction's P x P DFT grid
    (for the directions ``dirs`` only when given, in that order; S is always the density of
    every direction of ``rot``)
    (Sec. 2: the regularised inverse S_eps^-1 of the sampling matrix replaces the 1/n_q of
    Eq. 11).  S is interpolated trilinearly; g = s^3 / (P delta) turns sample counts into
    the density of slices per unit frequency, so that a 180-degree single-axis scan gives
    pi |q_u| / D; eps_S = 1e-3 times the mean of S over the band.  On the Nyquist row and
    column (bin -P/2, which is also +P/2) the weight is the mean over both aliases, so
    that it is even on the DFT grid."""
    s, Gh = density_geometry(P)
    G = 2 * Gh + 1
    S = density_grid(rot, P)
    mask, count = density_ball_count(Gh)
    eps_s = DENSITY_EPS_REL * S[mask].sum() / count
    g = s ** 3 / (P * delta)
    m = signed_freq(P).astype(np.float64)
    mv, mu = np.meshgrid(m, m, indexing="ij")  # [v][u]
    dirs = list(range(rot.shape[0])) if dirs is None else list(dirs)
    out = np.empty((len(dirs), P, P))
    Sf = S.ravel()

    def weight(n, a, b):
        q = (a[..., None] * rot[n, 0] + b[..., None] * rot[n, 1]) / s
        base = np.floor(q).astype(np.int64)
        f = q - base
        idx = base + Gh
        val = np.zeros(a.shape)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[..., 0] if dx else 1 - f[..., 0]) * (f[..., 1] if dy else 1 - f[..., 1])
                         * (f[..., 2] if dz else 1 - f[..., 2]))
                    cell = ((idx[..., 2] + dz) * G + (idx[..., 1] + dy)) * G + (idx[..., 0] + dx)
                    val += w * Sf[cell]
        return g / (val + eps_s)

    # the Nyquist bin -P/2 is also +P/2: there the weight is the mean over both aliases,
    # which keeps it even on the DFT grid (a real inverse transform)
    nyq_u = mu == -(P // 2)
    nyq_v = (mv == -(P // 2)) & ~nyq_u
    for o, n in enumerate(dirs):
        w0 = weight(n, mu, mv)
        w1 = weight(n, np.where(nyq_u, -mu, mu), np.where(nyq_v, -mv, mv))
        out[o] = np.where(nyq_u | nyq_v, 0.5 * (w0 + w1), w0)
    return out


# ----------------------------------------------------------------------------- stage A
def contrast(image: np.ndarray, input_mode: int) -> np.ndarray:
    """g = ln(I/I_in) (left side of Eq. 4), intensities floored at 1e-6, or the image
    itself when it already is a contrast or a projection."""
    img = np.asarray(image, dtype=np.float64)
    if input_mode == INPUT_INTENSITY:
        return np.log(np.maximum(img, INTENSITY_FLOOR))
    return img


def layer_stack(image: np.ndarray, *, delta: float, lam: float, r_n: float, z_layers: np.ndarray,
                n_dir: int, sigma: float, eps: float, cs: float, filt: int, input_mode: int,
                weight: np.ndarray | None = None) -> np.ndarray:
    """Layer stack Y_k (k over ``z_layers``) of one image, float64 ``(Nz, nv, nu)``:
    crop(Re IDFT[G * H_k * W]) with G the DFT of the zero-padded contrast, image
    centred in the P x P frame; W is the single-axis ramp, or ``weight`` (P x P, the
    density weighting of an arbitrary scan); H_k the real-bracket layer filter
    (``FILTER_TIKHONOV``), the opposite-pair one (``FILTER_PAIR``) or 1 (``FILTER_OFF``)."""
    nv, nu = image.shape
    P = padded_size(max(nu, nv))
    ou, ov = (P - nu) // 2, (P - nv) // 2
    g = np.zeros((P, P))
    g[ov:ov + nv, ou:ou + nu] = contrast(image, input_mode)
    G = np.fft.fft2(g)
    W = ramp_weights(P, delta, n_dir)[None, :] if weight is None else weight
    out = np.empty((len(z_layers), nv, nu))
    for k, z in enumerate(z_layers):
        if filt == FILTER_TIKHONOV:
            F = W * ctf_filter(P, delta, lam, r_n - z, sigma, eps, cs)
        elif filt == FILTER_PAIR:
            F = W * ctf_pair_filter(P, delta, lam, r_n, z, sigma, eps, cs)
        elif filt in (FILTER_DEPTH_COS, FILTER_DEPTH_SIN):
            F = W * depth_phase_filter(P, delta, lam, z, filt == FILTER_DEPTH_SIN)
        else:
            F = W
        out[k] = np.fft.ifft2(G * F).real[ov:ov + nv, ou:ou + nu]
    return out


# ----------------------------------------------------------------------------- stage B
def bilinear(img: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Bilinear sample of img[v][u] at (u, v) = (a, b), zero outside the detector."""
    nv, nu = img.shape
    a0 = np.floor(a).astype(np.int64)
    b0 = np.floor(b).astype(np.int64)
    fa = a - a0
    fb = b - b0

    def tap(ii, jj):
        ok = (ii >= 0) & (ii < nu) & (jj >= 0) & (jj < nv)
        return np.where(ok, img[np.clip(jj, 0, nv - 1), np.clip(ii, 0, nu - 1)], 0.0)

    return ((1 - fb) * ((1 - fa) * tap(a0, b0) + fa * tap(a0 + 1, b0))
            + fb * ((1 - fa) * tap(a0, b0 + 1) + fa * tap(a0 + 1, b0 + 1)))


def backproject_direction(stack: np.ndarray, A: np.ndarray, B: np.ndarray, T: np.ndarray,
                          i, j, k, interp: int = LAYER_NEAREST) -> np.ndarray:
    """One direction's contribution to voxels (i, j, k): bilinear sample of the layer
    containing each voxel's depth (the real-space counterpart of gridding onto the
    direction's Ewald patch, Sec. 2), or with ``interp = LAYER_LINEAR`` the linear blend
    of the bilinear samples of the two layers whose centres bracket the depth
    (``layer_blend``)."""
    nz_layers = stack.shape[0]
    a = A[0] * i + A[1] * j + A[2] * k + A[3]
    b = B[0] * i + B[1] * j + B[2] * k + B[3]
    out = np.zeros(np.shape(a))
    if interp == LAYER_NEAREST:
        lay = layer_index(T, nz_layers, i, j, k)
        for L in np.unique(lay):
            sel = lay == L
            out[sel] = bilinear(stack[L], a[sel], b[sel])
        return out
    k0, w = layer_blend(T, nz_layers, i, j, k)
    for L in np.unique(k0):
        sel = k0 == L
        lo = bilinear(stack[L], a[sel], b[sel])
        hi = bilinear(stack[min(L + 1, nz_layers - 1)], a[sel], b[sel])
        out[sel] = (1.0 - w[sel]) * lo + w[sel] * hi
    return out


def _partial_recon(args):
    """Sum over directions ``dirs`` of their contributions to voxels (i, j, k)."""
    (images, rot, dirs, lam, delta, defocus, nz_layers, grid, sigma, eps, cs, filt, input_mode, i, j, k,
     n_dir, density, interp) = args
    nu, nv = images.shape[2], images.shape[1]
    dens = density_weights(rot, padded_size(max(nu, nv)), delta, dirs) if density else None
    A, B = pixel_coefficients(rot, grid, nu, nv)
    T = layer_constants(rot, grid, nz_layers)
    zc = layer_centres(rot, grid, nz_layers, delta)
    acc = np.zeros(i.shape)
    chunk = 1 << 21
    for o, n in enumerate(dirs):
        st = layer_stack(images[n], delta=delta, lam=lam, r_n=float(defocus[n]), z_layers=zc[n], n_dir=n_dir,
                         sigma=sigma, eps=eps, cs=cs, filt=filt, input_mode=input_mode,
                         weight=None if dens is None else dens[o])
        for s0 in range(0, i.size, chunk):
            sl = slice(s0, s0 + chunk)
            acc[sl] += backproject_direction(st, A[n], B[n], T[n], i[sl], j[sl], k[sl], interp)
    return acc


def recon(images, rot, *, lam: float, delta: float, defocus, nz_layers: int, grid, sigma: float = 0.0,
          eps: float = 0.1, cs: float = 0.0, filt: int = FILTER_TIKHONOV, input_mode: int = INPUT_INTENSITY,
          voxels=None, dirs=None, workers: int = 1, density: bool = False,
          layer_interp: int = LAYER_NEAREST) -> np.ndarray:
    """The whole operator, FP64.  ``images`` (D, nv, nu); ``rot`` (D, 3, 3);
    ``defocus`` (D,).  Returns vol[z][y][x] float64, or, when ``voxels = (i, j, k)``
    index arrays are given, the values at those voxels only.  ``dirs`` restricts the
    sum to a subset of the directions (the ramp keeps its pi/D for all D);
    ``workers`` > 1 splits the directions over a spawned process pool (the same
    arithmetic, summed in a different order).  ``density`` selects the sampling-density
    weighting of an arbitrary scan instead of the single-axis ramp; ``layer_interp`` picks
    the nearest layer or the linear blend of the two bracketing layers."""
    images = np.asarray(images)
    rot = np.asarray(rot, dtype=np.float64)
    D = images.shape[0]
    nx, ny, nz = grid
    if voxels is None:
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
    else:
        i, j, k = (np.asarray(x, np.int64) for x in voxels)
    dirs = list(range(D)) if dirs is None else list(dirs)
    common = (lam, delta, np.asarray(defocus, np.float64), nz_layers, tuple(grid), sigma, eps, cs, filt,
              input_mode, i, j, k, D, density, layer_interp)
    if workers <= 1 or len(dirs) < 2:
        acc = _partial_recon((images, rot, dirs) + common)
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        groups = [dirs[w::workers] for w in range(workers) if dirs[w::workers]]
        with ProcessPoolExecutor(max_workers=len(groups), mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_partial_recon, [(images, rot, g) + common for g in groups]))
        acc = np.sum(parts, axis=0)
    if voxels is None:
        return acc.reshape(nz, ny, nx)
    return acc
