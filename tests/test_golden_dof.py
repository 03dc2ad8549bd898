"""The plan's depth-of-field report against the figures Sec. 3 prints for its two examples.

DOF = Delta^2 / (2 lambda) (Sec. 1).  ``tests/golden/dof_sec3_examples.txt`` holds, per
example, the wavelength, the resolution, the thickness the paper compares the DOF with and the
printed DOF; the plan is built on the host (no CUDA call) at a voxel pitch equal to that
resolution over a cube as thick as the object.
"""
import math
import os

import numpy as np
import pytest

from __graft_entry__ import build
from paper_2206_09151_gb300 import _abi
from paper_2206_09151_gb300 import phantoms as ph

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dof_sec3_examples.txt")


def _examples():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            name, lam, delta, thick, dof, tol = line
            rows[name] = dict(lam=float(lam), delta=float(delta), thickness=float(thick), dof_printed=float(dof),
                              rel_tol=None if tol == "-" else float(tol))
    return rows


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load_library()


def _plan(rot, n, lam, delta, defocus, nz):
    return _abi.recon_plan(rot, n, n, lam, delta, np.full(rot.shape[0], defocus), nz, (n, n, n))


def test_fixture_holds_both_examples():
    ex = _examples()
    assert set(ex) == {"electron_200kev", "xray_32kev"}
    # the electron example's resolution is the 40 mrad aperture's lambda / alpha
    e = ex["electron_200kev"]
    assert e["delta"] == pytest.approx(e["lam"] / 0.040, rel=1e-12)
    # the X-ray wavelength is hc / E at 32 keV (hc = 12.39842 keV Angstrom)
    assert ex["xray_32kev"]["lam"] == pytest.approx(12.39842 / 32.0 * 1e-10, rel=1e-4)


def test_electron_example_dof_is_about_8_angstrom_and_needs_layers(lib):
    """Sec. 3, first example: DOF about 8 Angstrom, much less than the 70 Angstrom particle, so
    the Ewald curvature matters and one layer is not enough."""
    e = _examples()["electron_200kev"]
    n = int(round(e["thickness"] / e["delta"]))  # 112 voxels of 0.625 Angstrom
    beam_z = np.eye(3)[None]
    # image planes 300-350 Angstrom from the cube's z = 0 face, i.e. 200-250 Angstrom downstream of
    # the rotation centre, from which R is measured here (the DOF does not depend on R)
    p = _plan(beam_z, n, e["lam"], e["delta"], 2.25e-8, 1)
    h, dof = _abi.recon_plan_dof(p)
    assert dof == pytest.approx(e["delta"] ** 2 / (2 * e["lam"]), rel=1e-12)
    assert abs(dof - e["dof_printed"]) <= e["rel_tol"] * e["dof_printed"]
    assert h == pytest.approx(e["thickness"], rel=1e-9) and h > 8 * dof
    assert _abi.recon_plan_warning(p) != ""
    _abi.recon_destroy(p)
    nz = _abi.recon_layers_for_dof(beam_z, (n, n, n), e["lam"], e["delta"])
    assert nz == math.ceil(e["thickness"] / dof) == 9
    p = _plan(beam_z, n, e["lam"], e["delta"], 2.25e-8, nz)
    assert _abi.recon_plan_warning(p) == ""
    _abi.recon_destroy(p)
    # the paper's scan: orientations uniform on the sphere; any view sees at least the cube's side
    rot = ph.cone_rotations(16, 90.0, seed=5)
    assert _abi.recon_layers_for_dof(rot, (n, n, n), e["lam"], e["delta"]) >= nz


def test_xray_example_dof_is_far_above_the_sample_one_layer_suffices(lib):
    """Sec. 3, second example: the DOF is metres against 0.11 m of sample, so the curvature is
    irrelevant and the layered method reduces to one layer (Eq. 13)."""
    x = _examples()["xray_32kev"]
    n = int(math.ceil(x["thickness"] / x["delta"]))  # 734 voxels of 150 um
    rot = ph.single_axis_rotations(8)  # the 180-degree single-axis scan
    assert _abi.recon_layers_for_dof(rot, (n, n, n), x["lam"], x["delta"]) == 1
    p = _plan(rot, n, x["lam"], x["delta"], 6.0, 1)  # R = 6 m
    h, dof = _abi.recon_plan_dof(p)
    assert dof == pytest.approx(x["delta"] ** 2 / (2 * x["lam"]), rel=1e-12)
    # under either figure (printed 29 m, computed 290 m) the DOF exceeds the sample 100-fold
    assert min(dof, x["dof_printed"]) > 100 * x["thickness"]
    assert h <= n * x["delta"] * math.sqrt(2) * (1 + 1e-12)
    assert _abi.recon_plan_warning(p) == ""
    _abi.recon_destroy(p)
