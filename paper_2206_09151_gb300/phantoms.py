"""Seeded synthetic inputs: scan geometries, phantoms and simulated transmission images.

This module draws every random number the workloads use and turns phantoms into
images with a forward simulator. It holds none of the reconstruction's arithmetic
(no CTF inversion, no ramp, no layering, no backprojection); the reconstruction
library and the FP64 oracle both consume what it produces.

Conventions (shared by the C-ABI, the oracle and this module):

* Volume ``vol[z][y][x]``; voxel ``(i, j, k)`` has its centre at
  ``((i-(nx-1)/2)*delta, (j-(ny-1)/2)*delta, (k-(nz-1)/2)*delta)``.
* ``rot[n]`` is a 3x3 row-major rotation, volume frame -> beam frame: its rows are
  the detector ``u`` axis, the detector ``v`` axis and the beam direction, each
  written in volume coordinates.
* Image ``img[n][v][u]``; pixel ``(u, v)`` sits at beam-frame
  ``((u-(nu-1)/2)*delta, (v-(nv-1)/2)*delta)``.
* Defocus ``R_n`` is the distance from the plane through the rotation centre to
  the image plane, positive downstream (the reading of Sec. 3, where the image
  planes lie downstream of the object).

The simulator is a multislice model (Fig. 1(a)): the object is cut into thin slabs
normal to the beam, each slab multiplies the wave by its transmission function
exp(-a + i*phi) with phi = (2*pi/lambda) * int delta dz and a = sigma * phi (the
monomorphous object of Sec. 2), and free space between slabs and on to the image
plane is crossed with the Fresnel propagator of Eq. 3, exp(-i*pi*lambda*R*q^2),
optionally with a spherical-aberration phase (pi/2)*Cs*lambda^3*q^4 on the last
leg.  Intensities get Poisson shot noise at a stated dose.

A second, independent forward model (``born_images``) keeps single scattering only
(the first Born approximation): every thin plane of the object is lit by the unscattered
plane wave, its weak perturbation is carried to the image plane on its own, and the
perturbations add.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

__all__ = [
    "single_axis_rotations",
    "cone_rotations",
    "Phantom",
    "ball_phantom",
    "blob_phantom",
    "multislice_images",
    "born_images",
    "ball_projections",
    "config_workload",
    "mlp_init",
    "layer_projections",
]


# ----------------------------------------------------------------------------- geometry
def single_axis_rotations(n_dir: int, span: float = math.pi, start: float = 0.0, axis=None) -> np.ndarray:
    """Rotations for ``n_dir`` tilts about one fixed axis, evenly over ``[start, start+span)``.

    The axis is the volume y axis by default, else the unit vector along ``axis``; it
    stays the detector v axis for every view (row 1 of every rotation), which is the
    single-axis scan of Sec. 2 whose sampling density reduces to the ramp |q_x|.
    """
    th = start + span * np.arange(n_dir, dtype=np.float64) / max(n_dir, 1)
    c, s = np.cos(th), np.sin(th)
    rot = np.zeros((n_dir, 3, 3), dtype=np.float64)
    rot[:, 0, 0] = c
    rot[:, 0, 2] = s
    rot[:, 1, 1] = 1.0
    rot[:, 2, 0] = -s
    rot[:, 2, 2] = c
    if axis is not None:
        v = np.asarray(axis, np.float64) / np.linalg.norm(axis)
        # Q: a rotation taking e_y to v (Rodrigues about e_y x v); rot_n Q^T has row 1 = v
        ey = np.array([0.0, 1.0, 0.0])
        w = np.cross(ey, v)
        sn, cs = np.linalg.norm(w), float(ey @ v)
        K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]) / (sn if sn > 0 else 1.0)
        Q = np.eye(3) + sn * K + (1 - cs) * (K @ K)
        rot = rot @ Q.T
    return rot


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.empty((q.shape[0], 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def cone_rotations(n_dir: int, max_tilt_deg: float, seed: int) -> np.ndarray:
    """Haar-random rotations (uniform unit quaternions, Shoemake 1992) kept when the beam
    direction lies within ``max_tilt_deg`` of the volume z axis (a slab's normal)."""
    rng = np.random.default_rng(seed)
    out = []
    cos_max = math.cos(math.radians(max_tilt_deg))
    while sum(len(o) for o in out) < n_dir:
        u1, u2, u3 = rng.random((3, 4 * n_dir + 16))
        q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                      np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
        r = _quat_to_rot(q)
        out.append(r[np.abs(r[:, 2, 2]) >= cos_max])
    return np.concatenate(out)[:n_dir].copy()


# ----------------------------------------------------------------------------- phantoms
@dataclass
class Phantom:
    """Sum of primitives. ``kind`` is ``"ball"`` (uniform ball, delta inside radius) or
    ``"blob"`` (isotropic Gaussian, delta(r) = amp * exp(-|r-c|^2 / (2 s^2))).
    Centres and sizes are in voxel units relative to the volume centre."""
    kind: str
    centre: np.ndarray   # (K, 3) voxel units, relative to the volume centre
    size: np.ndarray     # (K,) radius (ball) or Gaussian s (blob), voxel units
    amp: np.ndarray      # (K,) delta inside the ball, or the blob's peak delta


def ball_phantom(grid, count: int, seed: int, r_range=(2.0, 8.0), delta_range=(1e-6, 1e-5)) -> Phantom:
    """``count`` uniform balls with radii U[r_range] voxels and decrement U[delta_range],
    centres inside the cylinder about y of radius n/2 - r (so every ball stays in the
    field of view of a single-axis scan); overlaps add."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_range[0], r_range[1], count)
    cen = np.zeros((count, 3))
    rad_xz = 0.5 * min(nx, nz) - r
    for n in range(count):
        while True:
            x, z = rng.uniform(-rad_xz[n], rad_xz[n], 2)
            if x * x + z * z <= rad_xz[n] ** 2:
                break
        y = rng.uniform(-(0.5 * ny - r[n]), 0.5 * ny - r[n])
        cen[n] = (x, y, z)
    d = rng.uniform(delta_range[0], delta_range[1], count)
    return Phantom("ball", cen, r, d)


def blob_phantom(grid, count: int, seed: int, s_vox: float, w_range=(1.0, 8.0), amp_unit=1.0,
                 margin: float = 3.0, region: str = "cylinder") -> Phantom:
    """``count`` Gaussian pseudo-atoms of width ``s_vox`` voxels, weights U[w_range] times
    ``amp_unit`` peak decrement, centres uniform inside the box shrunk by ``margin*s``
    and, for ``region = "cylinder"``, inside the y-axis cylinder (a single-axis scan's
    field of view); ``region = "box"`` fills the whole shrunk box (a slab)."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    m = margin * s_vox
    if region == "box":
        lo = -0.5 * np.array([nx, ny, nz], np.float64) + m
        cen = rng.uniform(lo, -lo, (count, 3))
    else:
        rc = 0.5 * min(nx, nz) - m
        cen = np.empty((0, 3))
        while cen.shape[0] < count:
            c = np.stack([rng.uniform(-rc, rc, 2 * count), rng.uniform(-(0.5 * ny - m), 0.5 * ny - m, 2 * count),
                          rng.uniform(-rc, rc, 2 * count)], axis=1)
            c = c[c[:, 0] ** 2 + c[:, 2] ** 2 <= rc * rc]
            cen = np.concatenate([cen, c])
    cen = cen[:count]
    w = rng.uniform(w_range[0], w_range[1], count) * amp_unit
    return Phantom("blob", cen, np.full(count, float(s_vox)), w)


# ----------------------------------------------------------------------------- images
def _pow2_at_least(x: int) -> int:
    p = 1
    while p < x:
        p *= 2
    return p


def born_images(ph: Phantom, rot: np.ndarray, nu: int, nv: int, delta: float, lam: float, defocus: np.ndarray,
                sigma: float, *, dz_vox: float = 0.25) -> np.ndarray:
    """Flat-fielded intensities ``(D, nv, nu)`` (float64) in the first Born approximation,
    by brute force over depth planes: for every primitive and every plane of thickness
    ``dz_vox`` voxels that it crosses (beam frame), the plane's share t(u, v) of the ray
    integral of delta (a ball's chord clipped to the plane, exactly; a blob's Gaussian depth
    profile integrated over the plane with erf) perturbs the incident wave by
    (i - sigma) (2 pi / lambda) t -- the first-order term of the transmission
    exp((i - sigma) phi) of a monomorphous object -- and that perturbation alone is carried
    to the image plane by the Fresnel propagator of Eq. 3 over R_n - z, z the plane's
    centre.  The perturbations of all planes add (no plane sees another's scattered wave);
    I = |1 + psi|^2.  Same geometry and units as ``multislice_images``."""
    D = rot.shape[0]
    P = _pow2_at_least(2 * max(nu, nv))
    ou, ov = (P - nu) // 2, (P - nv) // 2
    f = np.fft.fftfreq(P, d=delta)
    q2 = f[None, :] ** 2 + f[:, None] ** 2
    uu = np.arange(P) - ou - (nu - 1) / 2.0  # padded-grid pixel centres, voxel units
    vv = np.arange(P) - ov - (nv - 1) / 2.0
    k = 2.0 * math.pi / lam
    out = np.empty((D, nv, nu))
    for n in range(D):
        c = ph.centre @ rot[n].T
        Psi = np.zeros((P, P), dtype=np.complex128)
        for b in range(c.shape[0]):
            size, amp = float(ph.size[b]), float(ph.amp[b])
            rho2 = (uu[None, :] - c[b, 0]) ** 2 + (vv[:, None] - c[b, 1]) ** 2
            if ph.kind == "ball":
                half = np.sqrt(np.maximum(size * size - rho2, 0.0))  # half chord, voxel units
                reach = size
            else:
                lateral = np.exp(-rho2 / (2.0 * size * size))
                reach = 6.0 * size
            for z0 in np.arange(c[b, 2] - reach, c[b, 2] + reach, dz_vox):
                z1 = z0 + dz_vox
                if ph.kind == "ball":
                    t = np.clip(np.minimum(z1, c[b, 2] + half) - np.maximum(z0, c[b, 2] - half), 0.0, None)
                else:
                    w = math.sqrt(2.0) * size
                    t = lateral * (size * math.sqrt(math.pi / 2.0)
                                   * (math.erf((z1 - c[b, 2]) / w) - math.erf((z0 - c[b, 2]) / w)))
                if not t.any():
                    continue
                zm = 0.5 * (z0 + z1)
                Psi += np.fft.fft2(t * (amp * delta)) * np.exp(-1j * math.pi * lam * (float(defocus[n]) - zm * delta) * q2)
        psi = np.fft.ifft2(Psi * (k * (1j - sigma)))
        out[n] = (np.abs(1.0 + psi) ** 2)[ov:ov + nv, ou:ou + nu]
    return out


def ball_projections(ph: Phantom, rot: np.ndarray, nu: int, nv: int) -> np.ndarray:
    """Straight-ray line integrals of a ball phantom, in voxel-length units:
    p(u, v) = sum over balls of 2 * delta * sqrt(r^2 - rho^2) (the Radon transform of a
    uniform ball, sampled at pixel centres).  Returns float64 ``(D, nv, nu)``."""
    assert ph.kind == "ball"
    uu = np.arange(nu) - (nu - 1) / 2.0
    vv = np.arange(nv) - (nv - 1) / 2.0
    out = np.zeros((rot.shape[0], nv, nu))
    for n in range(rot.shape[0]):
        c = ph.centre @ rot[n].T  # beam-frame centres, voxel units
        for b in range(ph.centre.shape[0]):
            du = uu[None, :] - c[b, 0]
            dv = vv[:, None] - c[b, 1]
            rho2 = du * du + dv * dv
            out[n] += 2.0 * ph.amp[b] * np.sqrt(np.maximum(ph.size[b] ** 2 - rho2, 0.0))
    return out


def _slab_projection(ph: Phantom, c_beam: np.ndarray, sel: np.ndarray, P: int, off: int, nu: int, nv: int,
                     device) -> torch.Tensor:
    """Projected decrement (voxel-length units) of the primitives ``sel`` on a P x P grid
    whose pixel (off + u, off + v) is image pixel (u, v).  Evaluated with torch on
    ``device`` (float64), in chunks of primitives."""
    out = torch.zeros((P, P), dtype=torch.float64, device=device)
    if sel.size == 0:
        return out
    if ph.kind == "ball":
        rad = int(math.ceil(float(ph.size[sel].max()))) + 1
    else:
        rad = int(math.ceil(4.0 * float(ph.size[sel].max()))) + 1
    offs = torch.arange(-rad, rad + 1, device=device, dtype=torch.float64)
    chunk = max(1, (1 << 22) // (2 * rad + 1) ** 2)
    for a in range(0, sel.size, chunk):
        sl = sel[a:a + chunk]
        cu = torch.as_tensor(c_beam[sl, 0] + (nu - 1) / 2.0 + off, device=device)
        cv = torch.as_tensor(c_beam[sl, 1] + (nv - 1) / 2.0 + off, device=device)
        size = torch.as_tensor(ph.size[sl], device=device)[:, None, None]
        amp = torch.as_tensor(ph.amp[sl], device=device)[:, None, None]
        iu = torch.floor(cu)[:, None, None] + offs[None, None, :]
        iv = torch.floor(cv)[:, None, None] + offs[None, :, None]
        du = iu - cu[:, None, None]
        dv = iv - cv[:, None, None]
        rho2 = du * du + dv * dv
        if ph.kind == "ball":
            val = 2.0 * amp * torch.sqrt(torch.clamp(size * size - rho2, min=0.0))
        else:
            val = amp * math.sqrt(2.0 * math.pi) * size * torch.exp(-rho2 / (2.0 * size * size))
        iu_b = torch.remainder(iu.expand_as(val).to(torch.int64), P)
        iv_b = torch.remainder(iv.expand_as(val).to(torch.int64), P)
        out.view(-1).index_add_(0, (iv_b * P + iu_b).reshape(-1), val.reshape(-1))
    return out


def multislice_images(ph: Phantom, rot: np.ndarray, nu: int, nv: int, delta: float, lam: float,
                      defocus: np.ndarray, sigma: float, *, cs: float = 0.0, n_slabs: int = 16,
                      photons: float | None = None, seed: int = 0, device="cpu",
                      dtype=torch.float32, thickness: float | None = None) -> torch.Tensor:
    """Flat-fielded intensities I/I_in, shape ``(D, nv, nu)``, of ``ph`` under plane-wave
    illumination along each ``rot[n]`` beam axis, by the multislice model described in
    the module docstring.  The slabs tile ``[-thickness/2, thickness/2]`` (voxel units,
    beam frame; default: the phantom's enclosing sphere) and a primitive belongs to the
    slab holding its centre.  ``delta`` is the voxel and pixel pitch, ``lam`` the
    wavelength, ``defocus[n]`` the image-plane distance R_n, ``sigma`` = beta/delta.
    ``photons`` (per pixel) adds Poisson noise when given."""
    D = rot.shape[0]
    P = _pow2_at_least(2 * max(nu, nv))
    off_u = (P - nu) // 2
    off_v = (P - nv) // 2
    f = torch.fft.fftfreq(P, d=delta, device=device, dtype=torch.float64)
    q2 = f[None, :] ** 2 + f[:, None] ** 2
    reach = ph.size * (1.0 if ph.kind == "ball" else 4.0)
    thick = thickness if thickness is not None else \
        2.0 * float(np.max(np.linalg.norm(ph.centre, axis=1) + reach)) + 1.0  # voxel units
    dz = thick / n_slabs
    zc = -thick / 2.0 + (np.arange(n_slabs) + 0.5) * dz
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    step = torch.exp(-1j * math.pi * lam * (dz * delta) * q2)
    out = torch.empty((D, nv, nu), dtype=dtype, device=device)
    for n in range(D):
        c_beam = ph.centre @ rot[n].T
        slab = np.clip(np.floor((c_beam[:, 2] + thick / 2.0) / dz), 0, n_slabs - 1).astype(np.int64)
        U = torch.ones((P, P), dtype=torch.complex128, device=device)
        for m in range(n_slabs):
            sel = np.nonzero(slab == m)[0]
            if sel.size:
                proj = _slab_projection(ph, c_beam, sel, P, off_u, nu, nv, device) * delta  # length units
                phi = (2.0 * math.pi / lam) * proj
                U = U * torch.exp(torch.complex(-sigma * phi, phi))
            if m + 1 < n_slabs:
                U = torch.fft.ifft2(torch.fft.fft2(U) * step)
            else:
                chi = math.pi * lam * (float(defocus[n]) - zc[m] * delta) * q2
                if cs != 0.0:
                    chi = chi + 0.5 * math.pi * cs * lam ** 3 * q2 * q2
                U = torch.fft.ifft2(torch.fft.fft2(U) * torch.exp(-1j * chi))
        I = (U.real ** 2 + U.imag ** 2)[off_v:off_v + nv, off_u:off_u + nu]
        if photons is not None:
            I = torch.poisson(I * photons, generator=gen) / photons
        out[n] = I.to(dtype)
    return out


# ----------------------------------------------------------------------------- learned filter
def mlp_init(seed: int, eps0: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of the 3 -> 64 -> 64 -> 1 regulariser network (4481 floats,
    layout W1[64][3], b1, W2[64][64], b2, w3, b3): He-uniform weights, zero hidden biases,
    and an output bias at softplus^-1(eps0) so that the untrained network sits near the
    Tikhonov value eps0."""
    rng = np.random.default_rng(seed)
    h = 64
    W1 = rng.uniform(-1, 1, (h, 3)) * math.sqrt(6.0 / 3)
    W2 = rng.uniform(-1, 1, (h, h)) * math.sqrt(6.0 / h)
    w3 = rng.uniform(-1, 1, h) * math.sqrt(6.0 / h) * 0.01
    b3 = math.log(math.expm1(eps0))
    return np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), w3, [b3]]).astype(np.float64)


def layer_projections(ph: Phantom, rot: np.ndarray, nu: int, nv: int, grid, nz_layers: int,
                      delta: float) -> np.ndarray:
    """True projections (metres) of the parts of the phantom that fall in each depth layer
    (Nz equal slabs over the volume's bounding-box extent along the beam), float64
    (D, Nz, nv, nu): the targets of the learned regulariser.  A primitive is assigned to
    the layer holding its centre."""
    nx, ny, nz = grid
    out = np.zeros((rot.shape[0], nz_layers, nv, nu))
    uu = np.arange(nu) - (nu - 1) / 2.0
    vv = np.arange(nv) - (nv - 1) / 2.0
    for n in range(rot.shape[0]):
        d = rot[n, 2]
        ext = abs(d[0]) * nx + abs(d[1]) * ny + abs(d[2]) * nz
        c = ph.centre @ rot[n].T
        layer = np.clip(np.floor((c[:, 2] + ext / 2) / (ext / nz_layers)), 0, nz_layers - 1).astype(int)
        for b in range(c.shape[0]):
            r2 = (uu[None, :] - c[b, 0]) ** 2 + (vv[:, None] - c[b, 1]) ** 2
            s = ph.size[b]
            if ph.kind == "ball":
                p = 2.0 * ph.amp[b] * np.sqrt(np.maximum(s * s - r2, 0.0))
            else:
                p = ph.amp[b] * math.sqrt(2.0 * math.pi) * s * np.exp(-r2 / (2.0 * s * s))
            out[n, layer[b]] += p * delta
    return out


def layer_projections_device(ph: Phantom, rot: np.ndarray, nu: int, nv: int, grid, nz_layers: int,
                             delta: float, device="cuda") -> torch.Tensor:
    """:func:`layer_projections` evaluated with torch on ``device`` (all primitives of a
    direction splatted at once): float32 ``(D, Nz, nv, nu)`` true projections (metres) of
    the parts of the phantom in each depth layer, a primitive assigned to the layer
    holding its centre."""
    nx, ny, nz = grid
    D = rot.shape[0]
    out = torch.zeros((D, nz_layers, nv, nu), dtype=torch.float32, device=device)
    if ph.centre.shape[0] == 0:
        return out
    rad = int(math.ceil(float(ph.size.max()) * (1.0 if ph.kind == "ball" else 4.0))) + 1
    offs = torch.arange(-rad, rad + 1, device=device, dtype=torch.float64)
    size = torch.as_tensor(ph.size, device=device)[:, None, None]
    amp = torch.as_tensor(ph.amp, device=device)[:, None, None]
    for n in range(D):
        d = rot[n, 2]
        ext = abs(d[0]) * nx + abs(d[1]) * ny + abs(d[2]) * nz
        c = ph.centre @ rot[n].T
        layer = np.clip(np.floor((c[:, 2] + ext / 2) / (ext / nz_layers)), 0, nz_layers - 1).astype(np.int64)
        cu = torch.as_tensor(c[:, 0] + (nu - 1) / 2.0, device=device)
        cv = torch.as_tensor(c[:, 1] + (nv - 1) / 2.0, device=device)
        iu = torch.floor(cu)[:, None, None] + offs[None, None, :]
        iv = torch.floor(cv)[:, None, None] + offs[None, :, None]
        rho2 = (iu - cu[:, None, None]) ** 2 + (iv - cv[:, None, None]) ** 2
        if ph.kind == "ball":
            val = 2.0 * amp * torch.sqrt(torch.clamp(size * size - rho2, min=0.0))
        else:
            val = amp * math.sqrt(2.0 * math.pi) * size * torch.exp(-rho2 / (2.0 * size * size))
        iu_b, iv_b = iu.expand_as(val), iv.expand_as(val)
        ok = (iu_b >= 0) & (iu_b < nu) & (iv_b >= 0) & (iv_b < nv)
        lay = torch.as_tensor(layer, device=device)[:, None, None].expand_as(val)
        idx = (lay * nv + iv_b.to(torch.int64)) * nu + iu_b.to(torch.int64)
        acc = torch.zeros(nz_layers * nv * nu, dtype=torch.float64, device=device)
        acc.index_add_(0, idx[ok], val[ok])
        out[n] = (acc * delta).view(nz_layers, nv, nu).to(torch.float32)
    return out


def training_set(first: int, count: int, physics: str = "c3", n: int = 128, views: int = 4, nz_layers: int = 16,
                 device="cuda", photons: float | None = None) -> dict:
    """Seeded training data of the learned regulariser: ``count`` phantoms of n^3 voxels
    (seeds first .. first + count - 1), alternately Gaussian pseudo-atoms and uniform balls,
    each seen from ``views`` random directions, with their multislice images (Poisson
    noise) and the true projections of each of Nz depth layers.

    ``physics = "c3"``: 0.1 nm voxels, lambda 1.97 pm, R ~ U[0.5, 1.5] um, Cs 2.7 mm,
    sigma 0.07, 100 e/px, pseudo-atoms of s = 0.1 nm at the density of the 512^3 scan,
    random single-axis angles.  ``"c5"``: 0.05 nm voxels, R ~ U[0.75, 1.25] um, 50 e/px,
    pseudo-atoms of s = 0.1 nm at the density of the 1024 x 1024 x 256 slab filling the box,
    Haar-random directions within 60 deg of z.  Balls: 20 of radius U[2, 8] voxels with a
    decrement giving 0.02-0.1 rad of peak phase.  ``photons`` overrides the dose per pixel."""
    grid = (n, n, n)
    dose = photons
    if physics == "c3":
        delta, photons, s_vox, blobs, region = 1e-10, 100.0, 1.0, int(round(160000 / 64 * (n / 128) ** 3)), "cylinder"
        r_range = (0.5e-6, 1.5e-6)
    elif physics == "c5":
        delta, photons, s_vox, region = 5e-11, 50.0, 2.0, "box"
        blobs = int(round(200000 * n ** 3 / (1024 * 1024 * 256)))
        r_range = (0.75e-6, 1.25e-6)
    else:
        raise ValueError(physics)
    if dose is not None:
        photons = float(dose)
    lam, sigma, cs = 1.97e-12, 0.07, 2.7e-3
    amp = 0.01 * lam / (2 * math.pi * math.sqrt(2 * math.pi) * s_vox * delta)
    ball_delta = (0.02 * lam / (2 * math.pi * 2 * 5 * delta), 0.1 * lam / (2 * math.pi * 2 * 5 * delta))
    imgs, tgts, rots, Rs = [], [], [], []
    for p in range(first, first + count):
        rng = np.random.default_rng(50000 + p)
        if p % 2 == 0:
            phan = blob_phantom(grid, blobs, seed=60000 + p, s_vox=s_vox, amp_unit=amp, region=region)
        else:
            phan = ball_phantom(grid, 20, seed=60000 + p, delta_range=ball_delta)
        if physics == "c3":
            rot = np.stack([single_axis_rotations(1, start=float(a), span=0.0)[0]
                            for a in rng.uniform(0, math.pi, views)])
        else:
            rot = cone_rotations(views, 60.0, seed=70000 + p)
        R = rng.uniform(r_range[0], r_range[1], views)
        imgs.append(multislice_images(phan, rot, n, n, delta, lam, R, sigma, cs=cs, photons=photons,
                                      seed=80000 + p, device=device, dtype=torch.float32))
        tgts.append(layer_projections_device(phan, rot, n, n, grid, nz_layers, delta, device))
        rots.append(rot)
        Rs.append(R)
    return dict(images=torch.cat(imgs), targets=torch.cat(tgts), rot=np.concatenate(rots), defocus=np.concatenate(Rs),
                grid=grid, nz_layers=nz_layers, lam=lam, delta=delta, sigma=sigma, cs=cs, nsr=photons ** -0.5)


# ----------------------------------------------------------------------------- workloads
def config_workload(name: str, *, scale_dirs: int | None = None):
    """Parameters of the named synthetic workloads (all seeded).

    ``"small"``: 64^3 voxels of 1 nm, 90 single-axis directions over 180 deg, 64x64
    images, lambda = 0.1 nm, Nz = 8, 20 uniform balls (radii U[2,8] voxels, delta
    U[1e-6,1e-5], sigma = beta/delta = 0.01), R_n ~ U[100,120] nm, 1e4 photons/pixel.

    ``"mid"``: 256^3 voxels of 0.1 nm, 360 single-axis directions over 180 deg,
    256x256 images, lambda = 1.97 pm (300 keV electrons), Nz = 32, defocus 1 um,
    Cs = 2.7 mm, 2e4 Gaussian pseudo-atoms (s = 0.1 nm, weights U[1,8], peak phase
    0.01 rad per unit weight), sigma = 0.07, 100 electrons/pixel.

    ``"learned"``: 512^3, 720 single-axis directions, 512x512 images, Nz = 64, the
    physics of "mid" with R_n ~ U[0.5, 1.5] um, 1.6e5 pseudo-atoms (the density of "mid").

    ``"slab"``: a 1024 x 1024 x 256 slab of 0.05 nm voxels, 1500 Haar-random directions
    within 60 deg of its normal, 1024x1024 images, Nz = 64, lambda = 1.97 pm, R = 1 um,
    Cs = 2.7 mm, 2e5 pseudo-atoms of s = 0.1 nm filling the slab, 50 electrons/pixel,
    sampling-density weighting (``ramp = "density"``).

    ``scale_dirs`` keeps the first directions only (a scan of its own).
    """
    if name == "small":
        n, D = 64, 90
        cfg = dict(grid=(n, n, n), nu=n, nv=n, n_dir=D, delta=1e-9, lam=1e-10, nz_layers=8, sigma=0.01,
                   eps=1e-2, cs=0.0, photons=1e4, seed=1001, phantom="balls", count=20)
        rng = np.random.default_rng(cfg["seed"] + 7)
        cfg["defocus"] = rng.uniform(100e-9, 120e-9, D)
    elif name == "mid":
        n, D = 256, 360
        cfg = dict(grid=(n, n, n), nu=n, nv=n, n_dir=D, delta=1e-10, lam=1.97e-12, nz_layers=32, sigma=0.07,
                   eps=0.1, cs=2.7e-3, photons=100.0, seed=2001, phantom="blobs", count=20000)
        cfg["defocus"] = np.full(D, 1e-6)
    elif name == "learned":
        # 512^3 / 720 views / Nz = 64 in bfloat16, the physics of "mid" with R_n ~ U[0.5, 1.5] um
        n, D = 512, 720
        cfg = dict(grid=(n, n, n), nu=n, nv=n, n_dir=D, delta=1e-10, lam=1.97e-12, nz_layers=64, sigma=0.07,
                   eps=0.1, cs=2.7e-3, photons=100.0, seed=3001, phantom="blobs", count=160000)
        cfg["defocus"] = np.random.default_rng(cfg["seed"] + 7).uniform(0.5e-6, 1.5e-6, D)
    elif name == "slab":
        # 1024 x 1024 x 256 slab, 1500 Haar-random views within 60 deg of its normal, 1024^2
        # images, 0.05 nm voxels (DOF 0.63 nm against 12.8 nm of thickness), Nz = 64 in bfloat16,
        # sampling-density weighting, 2e5 pseudo-atoms of s = 0.1 nm in the whole box, 50 e/px
        D = 1500
        cfg = dict(grid=(1024, 1024, 256), nu=1024, nv=1024, n_dir=D, delta=5e-11, lam=1.97e-12, nz_layers=64,
                   sigma=0.07, eps=0.1, cs=2.7e-3, photons=50.0, seed=5001, phantom="blobs", count=200000,
                   region="box", ramp="density")
        cfg["defocus"] = np.full(D, 1e-6)
        cfg["rot"] = cone_rotations(D, 60.0, cfg["seed"] + 11)
    else:
        raise ValueError(name)
    cfg.setdefault("ramp", "single_axis")
    if "rot" not in cfg:
        cfg["rot"] = single_axis_rotations(cfg["n_dir"])
    if scale_dirs is not None:
        cfg["n_dir"] = scale_dirs
        cfg["defocus"] = cfg["defocus"][:scale_dirs]
        cfg["rot"] = cfg["rot"][:scale_dirs].copy()
    return cfg


def batch_workloads(count: int = 48, seed: int = 4001) -> list:
    """``count`` uneven tomograms for a batched run: grids n^3 with n ~ U{64, 96, ..., 256}
    (n x n images), D ~ U[60, 360] single-axis views, Nz ~ U[4, 32]; the phantom alternates
    between balls and Gaussian blobs and, independently, the physics between the "small"
    (soft X-ray, 1 nm voxels) and "mid" (300 keV electrons, 0.1 nm voxels, Cs) settings.
    Each entry has the keys of :func:`config_workload`; images take 4 multislice slabs."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(rng.choice(np.arange(64, 257, 32)))
        D = int(rng.integers(60, 361))
        nzl = int(rng.integers(4, 33))
        balls = q % 2 == 0
        electrons = (q // 2) % 2 == 1
        cfg = dict(grid=(n, n, n), nu=n, nv=n, n_dir=D, nz_layers=nzl, seed=seed + 10 * q, n_slabs=4,
                   ramp="single_axis", start=float(rng.uniform(0, math.pi)))
        if electrons:
            cfg.update(delta=1e-10, lam=1.97e-12, sigma=0.07, eps=0.1, cs=2.7e-3, photons=100.0,
                       defocus=np.full(D, 1e-6), delta_range=(2e-7, 2e-6))
        else:
            cfg.update(delta=1e-9, lam=1e-10, sigma=0.01, eps=1e-2, cs=0.0, photons=1e4,
                       defocus=rng.uniform(100e-9, 120e-9, D), delta_range=(1e-6, 1e-5))
        if balls:
            cfg.update(phantom="balls", count=20)
        else:
            cfg.update(phantom="blobs", count=max(200, int(20000 * (n / 256) ** 3)),
                       s_vox=max(1.0, 1e-10 / cfg["delta"]))
        cfg["rot"] = single_axis_rotations(D, start=cfg["start"])
        out.append(cfg)
    return out


def make_phantom(cfg) -> Phantom:
    """The phantom that ``cfg`` (from :func:`config_workload`) names."""
    if cfg["phantom"] == "balls":
        return ball_phantom(cfg["grid"], cfg["count"], cfg["seed"], delta_range=cfg.get("delta_range", (1e-6, 1e-5)))
    # peak phase per unit weight 0.01 rad: (2 pi / lam) * amp * sqrt(2 pi) * s * delta = 0.01
    s = cfg.get("s_vox", 1e-10 / cfg["delta"])
    amp = 0.01 * cfg["lam"] / (2 * math.pi * math.sqrt(2 * math.pi) * s * cfg["delta"])
    return blob_phantom(cfg["grid"], cfg["count"], cfg["seed"], s, amp_unit=amp,
                        region=cfg.get("region", "cylinder"))


def make_images(cfg, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """Multislice images of :func:`make_phantom` ``(cfg)`` for the scan ``cfg`` names."""
    phan = make_phantom(cfg)
    return multislice_images(phan, cfg["rot"], cfg["nu"], cfg["nv"], cfg["delta"], cfg["lam"], cfg["defocus"],
                             cfg["sigma"], cs=cfg["cs"], photons=cfg["photons"], seed=cfg["seed"], device=device,
                             dtype=dtype, n_slabs=cfg.get("n_slabs", 16))
