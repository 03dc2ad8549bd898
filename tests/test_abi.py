"""The C-ABI library loads and exports every entry point include/recon.h declares,
and its host-side plan validation works without a GPU (recon_plan makes no CUDA
call).  CPU only: no compute call here."""
import ctypes

import numpy as np
import pytest

from paper_2206_09151_gb300 import _abi, phantoms as ph
from paper_2206_09151_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load_library()


def test_every_declared_entry_point_is_exported(lib):
    names = _abi.header_entry_points()
    assert {"recon_plan", "recon_run", "recon_destroy", "recon_workspace_size", "recon_error_string"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def _plan(**kw):
    args = dict(rot=ph.single_axis_rotations(12), nu=40, nv=33, lam=1e-10, delta=1e-9,
                defocus=np.full(12, 1e-7), nz_layers=4, grid=(30, 20, 10))
    args.update(kw)
    opts = args.pop("opts", None)
    return _abi.recon_plan(args["rot"], args["nu"], args["nv"], args["lam"], args["delta"], args["defocus"],
                           args["nz_layers"], args["grid"], opts)


def test_plan_builds_on_the_host_and_reports_its_layout(lib):
    p = _plan()
    P, db, nb, sb = _abi.recon_plan_info(p)
    assert P == 128 and 1 <= db <= 12 and nb == -(-12 // db) and 1 <= sb <= db
    ws = _abi.recon_workspace_size(p)
    assert ws > 0 and ws % 256 == 0
    _abi.recon_destroy(p)
    assert lib.recon_destroy(None) == 0


def test_workspace_grows_with_the_direction_block(lib):
    o1 = _abi.recon_default_options()
    o1.dir_block = 1
    o4 = _abi.recon_default_options()
    o4.dir_block = 4
    p1, p4 = _plan(opts=o1), _plan(opts=o4)
    assert _abi.recon_plan_info(p1)[1:3] == (1, 12) and _abi.recon_plan_info(p4)[1:3] == (4, 3)
    assert _abi.recon_workspace_size(p4) > _abi.recon_workspace_size(p1)
    _abi.recon_destroy(p1)
    _abi.recon_destroy(p4)


def test_block_sizing_follows_the_per_direction_intermediates(lib):
    """Small images: stage A runs the whole direction block (as many directions as 4 GiB
    holds, balanced).  Large images (one direction's spectra and intermediates above 64 MiB):
    stage A runs in sub-blocks within 2 GiB, and the rest of a 16 GiB budget holds stacks."""
    o = _abi.recon_default_options()
    # 256^2 images, Nz = 32, float32 stacks: 120 directions per block, whole-block stage A
    p = _plan(rot=ph.single_axis_rotations(360), nu=256, nv=256, defocus=np.full(360, 1e-6), nz_layers=32,
              grid=(256, 256, 256), opts=o)
    assert _abi.recon_plan_info(p) == (512, 120, 3, 120)
    _abi.recon_destroy(p)
    # 1024^2 images, Nz = 64, bfloat16 stacks, density weights: 546 MB of intermediates per
    # direction, so sub-blocks of 3 (1.64 GB) and 56 directions per block (15.1 GB of stacks;
    # 57 fit, balanced over 27 blocks)
    o.stack_dtype = _abi.RECON_STACK_BF16
    o.ramp_mode = _abi.RECON_RAMP_DENSITY
    rot = ph.cone_rotations(1500, 60.0, seed=3)
    p = _plan(rot=rot, nu=1024, nv=1024, defocus=np.full(1500, 1e-6), nz_layers=64, grid=(1024, 1024, 256),
              delta=5e-11, lam=1.97e-12, opts=o)
    P, db, nb, sb = _abi.recon_plan_info(p)
    assert (P, sb) == (2048, 3) and db == 56 and nb == 27
    assert _abi.recon_workspace_size(p) < (16 << 30) + (256 << 20)
    _abi.recon_destroy(p)
    # an explicit stage_block still wins
    o.stage_block = 3
    p = _plan(rot=rot, nu=1024, nv=1024, defocus=np.full(1500, 1e-6), nz_layers=64, grid=(1024, 1024, 256),
              delta=5e-11, lam=1.97e-12, opts=o)
    assert _abi.recon_plan_info(p)[3] == 3
    _abi.recon_destroy(p)


def test_default_options(lib):
    o = _abi.recon_default_options()
    assert (o.sigma, o.eps, o.cs, o.filter, o.input_mode, o.stack_dtype, o.accumulate, o.dir_block,
            o.check_finite, o.layer_interp) == (0.0, 0.1, 0.0, 1, 0, 0, 0, 0, 0, 0)


@pytest.mark.parametrize("kw,code", [
    (dict(nu=0), _abi.RECON_E_INVALID_ARG),
    (dict(nu=1025), _abi.RECON_E_UNSUPPORTED_SIZE),
    (dict(nz_layers=-1), _abi.RECON_E_INVALID_ARG),
    (dict(nz_layers=97), _abi.RECON_E_UNSUPPORTED_SIZE),
    (dict(lam=0.0), _abi.RECON_E_INVALID_ARG),
    (dict(delta=-1.0), _abi.RECON_E_INVALID_ARG),
    (dict(grid=(5000, 2, 2)), _abi.RECON_E_UNSUPPORTED_SIZE),
    (dict(rot=ph.single_axis_rotations(12) * 1.01), _abi.RECON_E_INVALID_ARG),
    (dict(rot=ph.cone_rotations(12, 40.0, seed=1)), _abi.RECON_E_INVALID_ARG),
    (dict(defocus=np.full(12, np.nan)), _abi.RECON_E_INVALID_ARG),
])
def test_plan_rejects_bad_arguments(lib, kw, code):
    with pytest.raises(_abi.ReconError) as e:
        _plan(**kw)
    assert e.value.code == code
    assert _abi.recon_last_error() != ""


def test_density_weighting_accepts_any_geometry(lib):
    o = _abi.recon_default_options()
    o.ramp_mode = _abi.RECON_RAMP_DENSITY
    p = _plan(rot=ph.cone_rotations(12, 40.0, seed=1), opts=o)
    assert _abi.recon_workspace_size(p) > 0
    _abi.recon_destroy(p)


def test_plan_rejects_bad_options(lib):
    o = _abi.recon_default_options()
    o.eps = 0.0
    with pytest.raises(_abi.ReconError):
        _plan(opts=o)
    o = _abi.recon_default_options()
    o.filter = 7
    with pytest.raises(_abi.ReconError):
        _plan(opts=o)


def test_null_arguments_are_errors_not_crashes(lib):
    out = ctypes.c_void_p()
    assert lib.recon_plan(None, 1.0, 1.0, None, 1, None, None, ctypes.byref(out)) == _abi.RECON_E_INVALID_ARG
    assert lib.recon_workspace_size(None, None) == _abi.RECON_E_INVALID_ARG
    assert lib.recon_run(None, None, None, None, 0, None) == _abi.RECON_E_INVALID_ARG
    p = _plan()
    # a misaligned or short workspace is refused before any CUDA call
    assert lib.recon_run(p, 16, 16, 8, 1 << 40, None) == _abi.RECON_E_WORKSPACE
    assert lib.recon_run(p, 16, 16, 256, 1, None) == _abi.RECON_E_WORKSPACE
    _abi.recon_destroy(p)


def test_host_input_run_is_validated_before_any_cuda_call(lib):
    """recon_run_host: its workspace is recon_workspace_size plus two 256-aligned slots of a
    direction block's images; null host images, check_finite plans and short or misaligned
    workspaces are refused on the host."""
    o = _abi.recon_default_options()
    o.dir_block = 5
    p = _plan(opts=o)
    ws, wh = _abi.recon_workspace_size(p), _abi.recon_run_host_workspace_size(p)
    slot = -(-(4 * 5 * 33 * 40) // 256) * 256
    assert wh == ws + 2 * slot
    assert lib.recon_run_host(p, None, 16, 256, wh, None) == _abi.RECON_E_INVALID_ARG
    assert lib.recon_run_host(p, 16, 16, 256, wh - 256, None) == _abi.RECON_E_WORKSPACE
    assert lib.recon_run_host(p, 16, 16, 8, 1 << 40, None) == _abi.RECON_E_WORKSPACE
    _abi.recon_destroy(p)
    o.check_finite = 1
    p = _plan(opts=o)
    assert lib.recon_run_host(p, 16, 16, 256, 1 << 40, None) == _abi.RECON_E_INVALID_ARG
    _abi.recon_destroy(p)


def test_error_strings(lib):
    texts = {_abi.recon_error_string(c) for c in (0, -1, -2, -3, -4, -5, -6, -7, -8)}
    assert len(texts) == 9 and "unknown status" not in texts


def test_learned_filter_without_weights_is_its_own_error(lib):
    o = _abi.recon_default_options()
    o.filter = _abi.RECON_FILTER_MLP
    o.nsr = 0.1
    with pytest.raises(_abi.ReconError) as e:
        _plan(opts=o)
    assert e.value.code == _abi.RECON_E_NO_WEIGHTS
    w = (ctypes.c_float * _abi.RECON_MLP_PARAMS)()
    o.mlp_weights = ctypes.cast(w, ctypes.POINTER(ctypes.c_float))
    o.nsr = 0.0
    with pytest.raises(_abi.ReconError) as e:
        _plan(opts=o)
    assert e.value.code == _abi.RECON_E_INVALID_ARG


def test_check_finite_option_is_validated(lib):
    o = _abi.recon_default_options()
    o.check_finite = 2
    with pytest.raises(_abi.ReconError) as e:
        _plan(opts=o)
    assert e.value.code == _abi.RECON_E_INVALID_ARG
    o.check_finite = 1
    _abi.recon_destroy(_plan(opts=o))


def test_backprojection_kernel_choice_is_reported_and_validated(lib):
    """AUTO resolves to the single-axis direct kernel for a scan about y with the nearest
    layer, to the TMA-staged kernel for a tilted axis or the layer blend; the tile depth of
    the TMA kernel is 0, 8 or 16."""
    rot_y = ph.single_axis_rotations(12)
    rot_t = ph.single_axis_rotations(12, axis=(0.3, 1.0, 0.2))
    for rot, interp, want in ((rot_y, _abi.RECON_LAYER_NEAREST, _abi.RECON_BP_DIRECT),
                              (rot_t, _abi.RECON_LAYER_NEAREST, _abi.RECON_BP_TMA),
                              (rot_y, _abi.RECON_LAYER_LINEAR, _abi.RECON_BP_TMA)):
        o = _abi.recon_default_options()
        o.layer_interp = interp
        p = _plan(rot=rot, opts=o)
        assert _abi.recon_plan_bp_kernel(p) == want
        _abi.recon_destroy(p)
    for bad in (4, 12, -1, 32):
        o = _abi.recon_default_options()
        o.bp_tile_z = bad
        with pytest.raises(_abi.ReconError) as e:
            _plan(rot=rot_t, opts=o)
        assert e.value.code == _abi.RECON_E_INVALID_ARG
    for ok in (0, 8, 16):
        o = _abi.recon_default_options()
        o.bp_tile_z = ok
        o.bp_kernel = _abi.RECON_BP_TMA
        p = _plan(rot=rot_y, opts=o)
        assert _abi.recon_plan_bp_kernel(p) == _abi.RECON_BP_TMA
        _abi.recon_destroy(p)


def test_depth_of_field_report_and_layer_count(lib):
    """DOF = Delta^2 / (2 lambda) (Sec. 1).  A 64^3 single-axis scan with Delta = 1 nm,
    lambda = 0.1 nm: DOF = 5 nm; the bounding-box extent along a beam at angle t in the
    x-z plane is 64 (|cos t| + |sin t|) nm, largest (64 sqrt 2 = 90.5 nm) at 45 degrees."""
    rot = ph.single_axis_rotations(4)  # 0, 45, 90, 135 degrees
    grid, lam, delta = (64, 64, 64), 1e-10, 1e-9
    assert _abi.recon_layers_for_dof(rot, grid, lam, delta) == 19  # ceil(90.51 / 5)
    assert _abi.recon_layers_for_dof(rot[:1], grid, lam, delta) == 13  # ceil(64 / 5)
    assert _abi.recon_layers_for_dof(rot, grid, lam, 1e-8) == 2  # 905 nm thick, DOF 500 nm
    assert _abi.recon_layers_for_dof(rot, grid, lam, 2e-8) == 1  # 1810 nm thick, DOF 2000 nm
    assert _abi.recon_layers_for_dof(rot, (4096, 4096, 4096), 1e-10, 1e-9) == _abi.RECON_MAX_LAYERS
    for nz, warn in ((8, True), (19, False)):
        p = _plan(rot=rot, nu=64, nv=64, defocus=np.full(4, 1e-7), nz_layers=nz, grid=grid)
        h, dof = _abi.recon_plan_dof(p)
        assert dof == pytest.approx(5e-9, rel=1e-12)
        assert h == pytest.approx(64 * np.sqrt(2) * 1e-9 / nz, rel=1e-9)
        assert (_abi.recon_plan_warning(p) != "") == warn
        _abi.recon_destroy(p)


def test_training_config_is_validated_on_the_host(lib):
    rot = ph.single_axis_rotations(2)
    cfg, keep = _abi.make_train_cfg(rot, np.zeros(2), 16, 16, 2, (8, 8, 8), 1e-10, 1e-9, 0.1, 0.0, 0.0, 0, 16, 16,
                                    10, 1e-3)
    with pytest.raises(_abi.ReconError) as e:
        _abi.recon_mlp_train_workspace_size(cfg)  # nsr = 0
    assert e.value.code == _abi.RECON_E_INVALID_ARG
    cfg.nsr = 1e-2
    assert _abi.recon_mlp_train_workspace_size(cfg) > 0
    cfg.steps = -1
    with pytest.raises(_abi.ReconError):
        _abi.recon_mlp_train_workspace_size(cfg)
    del keep


def test_learned_filter_needs_weights_and_nsr(lib):
    o = _abi.recon_default_options()
    o.filter = _abi.RECON_FILTER_MLP
    with pytest.raises(_abi.ReconError):
        _plan(opts=o)


def test_layer_interp_is_validated_and_nz_zero_follows_the_depth_of_field(lib):
    o = _abi.recon_default_options()
    o.layer_interp = 2
    with pytest.raises(_abi.ReconError) as e:
        _plan(opts=o)
    assert e.value.code == _abi.RECON_E_INVALID_ARG
    o.layer_interp = _abi.RECON_LAYER_LINEAR
    _abi.recon_destroy(_plan(opts=o))
    # Nz = 0: the smallest layer count whose layers are no thicker than the DOF
    rot = ph.single_axis_rotations(4)
    p = _plan(rot=rot, nu=64, nv=64, defocus=np.full(4, 1e-7), nz_layers=0, grid=(64, 64, 64))
    assert _abi.recon_plan_layers(p) == _abi.recon_layers_for_dof(rot, (64, 64, 64), 1e-10, 1e-9) == 19
    assert _abi.recon_plan_warning(p) == ""
    _abi.recon_destroy(p)


def test_fourier_forms_validate_on_the_host(lib):
    """Eq. 12 needs the pair filter's depth tables and one defocus; both 3D-Fourier forms
    refuse grids whose padded side would exceed 2048; the workspace sizes are queries."""
    rot = ph.single_axis_rotations(12, span=2 * np.pi)
    o = _abi.recon_default_options()
    o.filter = _abi.RECON_FILTER_PAIR
    p = _plan(rot=rot, defocus=np.full(12, 1e-7), opts=o)
    P3 = (64, 64, 32)  # grid (30, 20, 10) padded to the next power of two >= 2 n
    ws = _abi.recon_swap_workspace_size(p)
    assert ws >= 2 * 8 * P3[0] * P3[1] * P3[2]
    assert _abi.recon_grid_workspace_size(p) >= 3 * 8 * P3[0] * P3[1] * P3[2]
    assert lib.recon_swap_ct(p, 16, None, 0, None) == _abi.RECON_E_WORKSPACE
    assert lib.recon_swap_phase(p, 0.1, 0.0, 16, 256, ws, None) == _abi.RECON_E_INVALID_ARG  # eps = 0
    assert lib.recon_grid_run(p, 16, 16, -1.0, 256, 1 << 40, None) == _abi.RECON_E_INVALID_ARG  # nsr < 0
    _abi.recon_destroy(p)
    p = _plan(rot=rot, defocus=np.linspace(1e-7, 2e-7, 12), opts=o)  # several defocus values
    assert lib.recon_swap_ct(p, 16, 256, 1 << 40, None) == _abi.RECON_E_INVALID_ARG
    _abi.recon_destroy(p)
    p = _plan(rot=rot, defocus=np.full(12, 1e-7))  # Tikhonov plan: no depth tables for Eq. 12
    assert lib.recon_swap_ct(p, 16, 256, 1 << 40, None) == _abi.RECON_E_INVALID_ARG
    _abi.recon_destroy(p)
    p = _plan(rot=rot, defocus=np.full(12, 1e-7), grid=(1100, 8, 8))
    with pytest.raises(_abi.ReconError) as e:
        _abi.recon_grid_workspace_size(p)
    assert e.value.code == _abi.RECON_E_UNSUPPORTED_SIZE
    _abi.recon_destroy(p)
