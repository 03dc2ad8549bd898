"""Reconstruction error against the phantom as a function of the number of depth layers.

The depth of field Delta^2 / (2 lambda) of Sec. 1 sets how thin the layers must be: a
voxel filtered at the defocus of a layer centre up to h/2 away from its own depth is
blurred once h/2 approaches the DOF.  This study reconstructs one seeded workload at a
list of layer counts Nz, with the nearest layer and with the blend of the two layers whose
centres bracket each voxel, and reports for each the relative L2 error against the
phantom itself (Gaussian pseudo-atoms sampled at the voxel centres) inside the
single-axis field of view, and against the finest layering of the list.

    python -m paper_2206_09151_gb300.layer_study --workload mid --slabs 64

Every reconstruction runs through the library (``Reconstructor``); the images come from
the seeded multislice simulator of ``phantoms`` (``--slabs`` slabs through the object, so
that the simulated object itself is resolved in depth more finely than the layers)."""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import phantoms as ph
from .recon import Reconstructor


def phantom_volume(phan: ph.Phantom, grid, device) -> torch.Tensor:
    """delta(r) of a blob phantom at the voxel centres, vol[z][y][x] (each blob summed over
    the voxels within 4 s of its centre)."""
    nx, ny, nz = grid
    vol = torch.zeros(nz * ny * nx, dtype=torch.float64, device=device)
    cen = torch.as_tensor(phan.centre, dtype=torch.float64, device=device)
    size = torch.as_tensor(phan.size, dtype=torch.float64, device=device)
    amp = torch.as_tensor(phan.amp, dtype=torch.float64, device=device)
    rad = int(math.ceil(4.0 * float(phan.size.max())))
    offs = torch.arange(-rad, rad + 1, device=device, dtype=torch.float64)
    half = torch.tensor([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2], dtype=torch.float64, device=device)
    chunk = max(1, (1 << 22) // (2 * rad + 1) ** 3)
    for a in range(0, cen.shape[0], chunk):
        c = cen[a:a + chunk] + half  # voxel index of each centre
        base = torch.floor(c)
        ix = base[:, 0, None, None, None] + offs[None, None, None, :]
        iy = base[:, 1, None, None, None] + offs[None, None, :, None]
        iz = base[:, 2, None, None, None] + offs[None, :, None, None]
        r2 = (ix - c[:, 0, None, None, None]) ** 2 + (iy - c[:, 1, None, None, None]) ** 2 + \
            (iz - c[:, 2, None, None, None]) ** 2
        s = size[a:a + chunk, None, None, None]
        val = amp[a:a + chunk, None, None, None] * torch.exp(-r2 / (2 * s * s))
        ok = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny) & (iz >= 0) & (iz < nz)
        idx = (iz * ny + iy) * nx + ix
        vol.index_add_(0, idx[ok].to(torch.int64), val[ok])
    return vol.view(nz, ny, nx)


def run(workload: str = "mid", nz_list=(1, 2, 4, 8, 16, 32, 64, 96), slabs: int = 64, photons: float | None = None,
        stack: str = "f32", device: str = "cuda") -> list[dict]:
    cfg = ph.config_workload(workload)
    cfg["n_slabs"] = slabs
    if photons is not None:
        cfg["photons"] = photons if photons > 0 else None
    phan = ph.make_phantom(cfg)
    img = ph.make_images(cfg, device=device, dtype=torch.float32)
    nx, ny, nz = cfg["grid"]
    truth = phantom_volume(phan, cfg["grid"], device)
    xx = torch.arange(nx, device=device, dtype=torch.float64) - (nx - 1) / 2
    zz = torch.arange(nz, device=device, dtype=torch.float64) - (nz - 1) / 2
    fov = ((xx[None, :] ** 2 + zz[:, None] ** 2) <= (0.5 * min(nx, nz) - 2) ** 2)[:, None, :].expand(nz, ny, nx)
    dof = cfg["delta"] ** 2 / (2 * cfg["lam"])
    vols = {}
    rows = []
    for nzl in nz_list:
        for interp in ("nearest", "linear"):
            r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                              defocus=cfg["defocus"], nz_layers=nzl, sigma=cfg["sigma"], eps=cfg["eps"],
                              cs=cfg["cs"], stack_dtype=stack, ramp=cfg["ramp"], layer_interp=interp,
                              device=device)
            vol = r.run(img).double()
            torch.cuda.synchronize()
            h = float(np.max(np.abs(cfg["rot"][:, 2, :]) @ np.array(cfg["grid"], float))) * cfg["delta"] / nzl
            r.close()
            err = float(torch.linalg.norm((vol - truth)[fov]) / torch.linalg.norm(truth[fov]))
            vols[(nzl, interp)] = vol
            rows.append({"nz": nzl, "interp": interp, "layer_pitch_over_dof": h / dof, "rel_l2_vs_phantom": err})
    ref = vols[(nz_list[-1], "linear")]
    for row in rows:
        v = vols[(row["nz"], row["interp"])]
        row["rel_l2_vs_finest"] = float(torch.linalg.norm((v - ref)[fov]) / torch.linalg.norm(ref[fov]))
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="mid", choices=["small", "mid"])
    ap.add_argument("--nz", default="1,2,4,8,16,32,64,96")
    ap.add_argument("--slabs", type=int, default=64, help="multislice slabs through the object")
    ap.add_argument("--photons", type=float, default=None, help="electrons per pixel (0: noise-free)")
    ap.add_argument("--stack", default="f32", choices=["f32", "bf16"])
    args = ap.parse_args()
    rows = run(args.workload, tuple(int(x) for x in args.nz.split(",")), args.slabs, args.photons, args.stack)
    for row in rows:
        print(json.dumps(row))


if __name__ == "__main__":
    main()
