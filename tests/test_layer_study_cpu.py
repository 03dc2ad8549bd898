"""The layer-count study's phantom sampler (CPU): Gaussian pseudo-atoms sampled at the
voxel centres sums to its continuous integral amp (2 pi)^(3/2) s^3, and lands where its
centre is (the grid centre convention of the reconstruction, (n - 1)/2)."""
import math

import numpy as np
import torch

from paper_2206_09151_gb300 import phantoms as ph
from paper_2206_09151_gb300.layer_study import phantom_volume


def test_blob_sums_to_its_integral_and_sits_at_its_centre():
    grid = (40, 33, 36)
    phan = ph.Phantom("blob", np.array([[2.25, -3.5, 1.0], [-9.0, 6.0, -4.5]]), np.array([1.5, 2.0]),
                      np.array([1e-6, 3e-6]))
    vol = phantom_volume(phan, grid, "cpu").numpy()
    want = sum(a * (2 * math.pi) ** 1.5 * s ** 3 for a, s in zip(phan.amp, phan.size))
    assert abs(vol.sum() - want) < 2e-4 * want  # the stencil stops 4 s out
    one = ph.Phantom("blob", phan.centre[:1], phan.size[:1], phan.amp[:1])
    v1 = phantom_volume(one, grid, "cpu").numpy()
    kk, jj, ii = np.meshgrid(*(np.arange(g) for g in grid[::-1]), indexing="ij")
    w = v1 / v1.sum()
    cen = [(ii * w).sum() - (grid[0] - 1) / 2, (jj * w).sum() - (grid[1] - 1) / 2, (kk * w).sum() - (grid[2] - 1) / 2]
    assert np.allclose(cen, phan.centre[0], atol=1e-3)
    assert torch.is_tensor(phantom_volume(one, grid, "cpu"))
