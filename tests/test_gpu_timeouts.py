"""Bounded waits of the tensor-core kernels, through the C ABI.

Every wait of the tcgen05 back-projection and of the tensor-core range
table is bounded by a clock budget. A test hook (pl_options
debug_unsatisfiable) makes one wait depend on a barrier that nothing
completes -- the back-projection's MMA warp (1), the range table's first
stage (2) or the MMA warp of the inverse z transform at off-grid heights (3)
-- with a short budget (wait_timeout_us). The kernel must then give
up, drain its own copies and products, release tensor memory and return: the
next pl_execute reports PL_ERR_TIMEOUT, no CUDA error is raised, and the same
device goes on to produce a correct image. Nothing here faults, traps or
hangs the GPU: the waits end by their budgets.
"""
import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PL_ERR_TIMEOUT = 8


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


def echo_of(w):
    clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
    return wl.add_noise(clean, w.snr_db, wl.rng_for(130, 0)).astype(np.complex64)


@pytest.mark.parametrize("hook,fine,dense", [(1, False, True), (1, False, False), (1, True, False),
                                              (2, False, False), (3, False, False)])
def test_unsatisfiable_wait_times_out_and_device_stays_usable(binding, hook, fine, dense):
    # hook 1 in the dense kernel (6.25 mm grid, dense products), the sparse
    # kernel with planar 32-row windows (6.25 mm) and with 16-row windows
    # (2 mm)
    w = wl.small_mono(seed=0)
    if hook == 3:
        # 24 voxel heights off the scan grid: the tensor-core inverse DFT
        w.grid = dict(w.grid, nz=24, z0=-0.071, dz=0.0061)
    if fine:
        # a 2 mm grid: 16-row windows, the back-projection's sparse products
        x0, dx = wl.centred_axis(0.128, 64)
        w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    echo = torch.from_numpy(echo_of(w)).cuda()
    plan = binding.Plan.from_workload(w, block_config=4, debug_unsatisfiable=hook,
                                      wait_timeout_us=2000, dense_products=dense)
    assert plan.info["block_config"] == 4 and plan.info["table_exact"] == 1
    if hook == 3:
        assert plan.info["z_transform_fft"] == 0
    assert plan.info["sparse_products"] == (0 if dense else 1)
    assert plan.info["slab_rows"] == (16 if fine else 32)
    plan.execute(echo)
    torch.cuda.synchronize()            # the kernels returned: no CUDA error
    with pytest.raises(binding.PolylineError) as ei:
        plan.execute(echo)              # reports the expired wait of the first call
    assert ei.value.status == PL_ERR_TIMEOUT
    plan.close()
    # the same context reconstructs correctly afterwards (a short budget alone
    # changes nothing)
    good = binding.Plan.from_workload(w, block_config=4, wait_timeout_us=2000)
    img = good.execute(echo).cpu().numpy().reshape(w.grid["nz"], -1)
    img2 = good.execute(echo).cpu().numpy().reshape(w.grid["nz"], -1)   # no timeout left over
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo.cpu().numpy(), w.z_scan, w.f_hz,
                              w.n_pad, w.pix_xy(), w.axis("z"))
    err = float(np.linalg.norm(img - ref) / np.linalg.norm(ref))
    print("hook %d: image after the timeout, rel L2 %.3e" % (hook, err))
    assert err < 1e-4 and np.array_equal(img, img2)


def test_debug_hook_is_validated(binding):
    w = wl.small_mono(seed=0)
    with pytest.raises(binding.PolylineError) as ei:
        binding.Plan.from_workload(w, block_config=4, debug_unsatisfiable=4)
    assert ei.value.status == 1
    with pytest.raises(binding.PolylineError) as ei:
        binding.Plan.from_workload(w, block_config=4, wait_timeout_us=-1)
    assert ei.value.status == 1
