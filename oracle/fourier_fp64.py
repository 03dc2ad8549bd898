"""FP64 oracle of the paper's two 3D-Fourier-space forms (test infrastructure only; the
same rules as ``recon_fp64``: only tests, ``smoke()`` and ``bench.py``'s CPU legs use it,
and it shares no code with the CUDA library).

1. ``recon_swapped`` -- Eq. 12: with one defocus R for every view, the CT reconstruction
   comes first and the CTF inversion is one 3D filter after it.  The CT step is the layered
   reconstruction of the contrasts with the Ewald placement and no CTF bracket (per layer
   cos and sin of pi lambda z_k q^2: two real volumes V_c, V_s, the real part and minus
   the imaginary part of the complex Ewald-placed volume).  The 3D step multiplies the 3D
   DFT of the complex volume V_c - i V_s by the bracket of Eq. 11 at the 3D frequency
   and keeps the real part:
       F3 delta = lambda / (4 pi sqrt(1+sigma^2)) [s'(q) F3 V_c - c'(q) F3 V_s],
       s' = sin chi / (sin^2 chi + eps),  c' = cos chi / (cos^2 chi + eps),
   chi = pi lambda R q_perp^2 + (pi/2) Cs lambda^3 q_perp^4 - omega, with q_perp^2 the
   in-plane part of a point q of the Ewald paraboloid (|q|^2 = q_perp^2 + lambda^2
   q_perp^4 / 4).  Volumes are zero-padded, centred, to the next power of two >= 2 n per
   axis (the reading of the 2D padding).

2. ``recon_gridding`` -- the UTR of Sec. 2 after Eq. 11: every view's 2D DFT coefficient
   times the bracket of Eq. 11 (its own R_n) is spread with trilinear weights (summing to
   one) onto the 8 cells around its point Rot_n^T (q_u, q_v, -lambda q_perp^2 / 2) of a 3D
   grid of the padded volume's DFT bins; S(q) sums the weights, and the result is
   divided by S_eps = S + eps_S (eps_S = 1e-3 x the mean of S over the cells with S > 0,
   the regularised inverse of the sampling matrix).  Optional noise filter of Sec. 3:
   a coefficient is zeroed where the gridded contrast spectrum (the same splat without
   the bracket, divided by S_eps) has a magnitude below NSR M / sqrt(S) (M^2 pixels per
   image; Parseval).  delta = Re of the inverse 3D DFT, cropped."""
from __future__ import annotations

import math

import numpy as np

from . import recon_fp64 as R


def padded3(grid) -> tuple[int, int, int]:
    """Per axis the smallest power of two >= 2 n (nx, ny, nz order)."""
    return tuple(R.padded_size(int(n)) for n in grid)


def _freq3(P3, delta):
    """Signed 3D frequencies (cycles / m) of the P3 grid, arrays shaped [z][y][x]."""
    fx = R.signed_freq(P3[0]) / (P3[0] * delta)
    fy = R.signed_freq(P3[1]) / (P3[1] * delta)
    fz = R.signed_freq(P3[2]) / (P3[2] * delta)
    return fx[None, None, :], fy[None, :, None], fz[:, None, None]


def q_perp2(q2, lam):
    """In-plane squared frequency of the Ewald-paraboloid point of squared norm q2:
    the root of p + lambda^2 p^2 / 4 = q2."""
    return 2.0 * (np.sqrt(1.0 + lam * lam * q2) - 1.0) / (lam * lam)


def bracket_parts(qp2, lam, r, sigma, eps, cs):
    """s' = sin chi / (sin^2 chi + eps) and c' = cos chi / (cos^2 chi + eps) of Eq. 11."""
    chi = math.pi * lam * r * qp2 + 0.5 * math.pi * cs * lam ** 3 * qp2 * qp2 - math.atan(sigma)
    s, c = np.sin(chi), np.cos(chi)
    return s / (s * s + eps), c / (c * c + eps)


def _pad_centred(vol, P3):
    nz, ny, nx = vol.shape
    out = np.zeros((P3[2], P3[1], P3[0]), dtype=vol.dtype)
    oz, oy, ox = (P3[2] - nz) // 2, (P3[1] - ny) // 2, (P3[0] - nx) // 2
    out[oz:oz + nz, oy:oy + ny, ox:ox + nx] = vol
    return out, (oz, oy, ox)


def swap_ct(images, rot, *, lam, delta, defocus, nz_layers, grid, input_mode=R.INPUT_INTENSITY, density=False,
            workers=1):
    """CT step of Eq. 12: the two real volumes (V_c, V_s)."""
    kw = dict(lam=lam, delta=delta, defocus=defocus, nz_layers=nz_layers, grid=grid, input_mode=input_mode,
              density=density, workers=workers)
    vc = R.recon(images, rot, filt=R.FILTER_DEPTH_COS, **kw)
    vs = R.recon(images, rot, filt=R.FILTER_DEPTH_SIN, **kw)
    return vc, vs


def swap_phase(vc, vs, *, lam, delta, defocus, sigma, eps, cs=0.0):
    """3D step of Eq. 12 on the CT volumes: the CTF inversion at one R for every view."""
    nz, ny, nx = vc.shape
    P3 = padded3((nx, ny, nz))
    pc, (oz, oy, ox) = _pad_centred(np.asarray(vc, np.float64), P3)
    ps, _ = _pad_centred(np.asarray(vs, np.float64), P3)
    fx, fy, fz = _freq3(P3, delta)
    q2 = fx * fx + fy * fy + fz * fz
    sp, cp = bracket_parts(q_perp2(q2, lam), lam, float(defocus), sigma, eps, cs)
    pref = lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma))
    F = pref * (sp * np.fft.fftn(pc) - cp * np.fft.fftn(ps))
    return np.fft.ifftn(F).real[oz:oz + nz, oy:oy + ny, ox:ox + nx]


def recon_swapped(images, rot, *, lam, delta, defocus, nz_layers, grid, sigma, eps, cs=0.0,
                  input_mode=R.INPUT_INTENSITY, density=False, workers=1):
    """Eq. 12: ``swap_ct`` then ``swap_phase``; ``defocus`` is the one R of every view."""
    D = np.asarray(images).shape[0]
    vc, vs = swap_ct(images, rot, lam=lam, delta=delta, defocus=np.full(D, float(defocus)), nz_layers=nz_layers,
                     grid=grid, input_mode=input_mode, density=density, workers=workers)
    return swap_phase(vc, vs, lam=lam, delta=delta, defocus=defocus, sigma=sigma, eps=eps, cs=cs)


GRID_EPS_REL = 1e-3


def recon_gridding(images, rot, *, lam, delta, defocus, grid, sigma, eps, cs=0.0, nsr=None,
                   input_mode=R.INPUT_INTENSITY) -> np.ndarray:
    """The UTR of Sec. 2 (Eq. 11 by 3D Fourier gridding), with the NSR noise filter of
    Sec. 3 when ``nsr`` is given.  Returns vol[z][y][x]."""
    images = np.asarray(images)
    rot = np.asarray(rot, np.float64)
    D, nv, nu = images.shape
    nx, ny, nz = grid
    P = R.padded_size(max(nu, nv))
    P3 = padded3(grid)
    acc = np.zeros(P3[2] * P3[1] * P3[0], complex)
    raw = np.zeros_like(acc)
    S = np.zeros(P3[2] * P3[1] * P3[0])
    m = R.signed_freq(P).astype(np.float64)
    mv, mu = np.meshgrid(m, m, indexing="ij")  # [v][u]
    qu, qv = mu / (P * delta), mv / (P * delta)
    qp2 = qu * qu + qv * qv
    pref = lam / (4.0 * math.pi * math.sqrt(1.0 + sigma * sigma))
    ou, ov = (P - nu) // 2, (P - nv) // 2
    for n in range(D):
        g = np.zeros((P, P))
        g[ov:ov + nv, ou:ou + nu] = R.contrast(images[n], input_mode)
        # DFT about the detector centre (frame position ou + (nu-1)/2): the Fourier slice
        # relation holds between transforms taken about the rotation centre
        cu, cv = ou + (nu - 1) / 2.0, ov + (nv - 1) / 2.0
        G = np.fft.fft2(g) * np.exp(2j * math.pi * (mu * cu + mv * cv) / P)
        sp, cp = bracket_parts(qp2, lam, float(defocus[n]), sigma, eps, cs)
        Z = pref * G * (sp - 1j * cp)
        # the sample's point on the Ewald paraboloid, beam frame -> object frame (rows of
        # Rot_n are the detector u, v axes and the beam), in grid units of each axis
        qz = -0.5 * lam * qp2
        q = (qu[..., None] * rot[n, 0] + qv[..., None] * rot[n, 1] + qz[..., None] * rot[n, 2])
        gpos = [q[..., a] * (P3[a] * delta) for a in range(3)]
        base = [np.floor(x).astype(np.int64) for x in gpos]
        frac = [x - b for x, b in zip(gpos, base)]
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((frac[0] if dx else 1 - frac[0]) * (frac[1] if dy else 1 - frac[1])
                         * (frac[2] if dz else 1 - frac[2]))
                    ix = (base[0] + dx) % P3[0]
                    iy = (base[1] + dy) % P3[1]
                    iz = (base[2] + dz) % P3[2]
                    cell = ((iz * P3[1] + iy) * P3[0] + ix).ravel()
                    np.add.at(S, cell, w.ravel())
                    np.add.at(acc, cell, (w * Z).ravel())
                    if nsr is not None:
                        np.add.at(raw, cell, (w * G).ravel())
    eps_s = GRID_EPS_REL * S[S > 0].mean() if np.any(S > 0) else 1.0
    F = acc / (S + eps_s)
    if nsr is not None:
        M = math.sqrt(nu * nv)
        keep = np.abs(raw / (S + eps_s)) >= nsr * M / np.sqrt(np.maximum(S, 1e-300))
        F = np.where(keep & (S > 0), F, 0.0)
    # DFT bin -> volume scale: F3 delta / Delta^3 with F2 g ~ Delta^2 DFT2 (see the module notes)
    F = F.reshape(P3[2], P3[1], P3[0]) / delta
    # back from the volume centre (frame position o + (n-1)/2 per axis) to the frame origin
    oz, oy, ox = (P3[2] - nz) // 2, (P3[1] - ny) // 2, (P3[0] - nx) // 2
    mx = R.signed_freq(P3[0])[None, None, :]
    my = R.signed_freq(P3[1])[None, :, None]
    mz = R.signed_freq(P3[2])[:, None, None]
    F = F * np.exp(-2j * math.pi * (mx * (ox + (nx - 1) / 2.0) / P3[0] + my * (oy + (ny - 1) / 2.0) / P3[1]
                                    + mz * (oz + (nz - 1) / 2.0) / P3[2]))
    vol = np.fft.ifftn(F).real
    return vol[oz:oz + nz, oy:oy + ny, ox:ox + nx]
