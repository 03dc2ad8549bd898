"""recon_run_host: the images in host memory, each direction block uploaded on the plan's
copy stream while the previous block is reconstructed.  The volume must be the one
recon_run gives for the same images, bit for bit (to the learned filter's float-atomic
variation with that filter), over several blocks with a ragged last one, from pinned and
from pageable memory, and on two calls in a row (the slots and events are reused)."""
import numpy as np
import pytest
import torch

from paper_2206_09151_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_2206_09151_gb300.build import build
    build()


def _case(filt):
    from paper_2206_09151_gb300.recon import Reconstructor
    rng = np.random.default_rng(21)
    D, n = 23, 40
    rot = ph.single_axis_rotations(D, start=0.2)
    img = (1.0 + 1e-2 * rng.standard_normal((D, n, n))).astype(np.float32)
    kw = dict(lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 80e-9, D), nz_layers=5, sigma=0.05, eps=0.02,
              dir_block=6)  # blocks of 6, 6, 6 and 5 directions
    if filt == "mlp":
        kw.update(filter="mlp", mlp_weights=ph.mlp_init(3).astype(np.float32), nsr=1e-2)
    return Reconstructor(rot, n, n, (n, n + 3, 24), **kw), img


@pytest.mark.parametrize("filt", ["tikhonov", "mlp"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_input_run_equals_the_device_input_run(filt, pinned):
    r, img = _case(filt)
    assert r.n_blocks == 4
    ref = r.run(torch.from_numpy(img).cuda()).cpu()
    host = torch.from_numpy(img)
    if pinned:
        host = host.pin_memory()
    for _ in range(2):
        got = r.run_host(host)
        torch.cuda.synchronize()
        if filt == "mlp":  # the power spectrum sums with float atomics: last-bit run-to-run variation
            assert torch.allclose(got.cpu(), ref, rtol=1e-6, atol=1e-6 * float(ref.abs().max()))
        else:
            assert torch.equal(got.cpu(), ref)
    r.close()


def test_host_input_run_on_the_general_geometry():
    """Cone views with density weights and the TMA-staged backprojection: within the float
    atomics' run-to-run variation of the density weights."""
    from paper_2206_09151_gb300.recon import Reconstructor
    rng = np.random.default_rng(22)
    D, n = 17, 32
    rot = ph.cone_rotations(D, 60.0, seed=4)
    img = (1.0 + 1e-2 * rng.standard_normal((D, n, n))).astype(np.float32)
    r = Reconstructor(rot, n, n, (n, n, 16), lam=1e-10, delta=1e-9, defocus=rng.uniform(50e-9, 80e-9, D),
                      nz_layers=4, sigma=0.05, eps=0.02, ramp="density", dir_block=5)
    ref = r.run(torch.from_numpy(img).cuda()).cpu().numpy()
    got = r.run_host(torch.from_numpy(img).pin_memory()).cpu().numpy()
    r.close()
    rel = np.linalg.norm(got.astype(np.float64) - ref) / np.linalg.norm(ref)
    assert rel <= 1e-6, rel
