"""Host-side failure modes of a plan, through the C ABI: NaN / Inf in the echo
data (pl_options check_nonfinite) and device allocation failure while a plan
is built (pl_options debug_fail_alloc, a test hook). Neither faults the GPU:
the echo scan sets a flag in mapped host memory, and the allocation failure is
reported by the host wrapper before cudaMalloc is called.
"""
import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PL_ERR_NONFINITE = 5
PL_ERR_OOM = 7


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


@pytest.fixture(scope="module")
def scene():
    w = wl.small_mono(seed=3)
    clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
    echo = wl.add_noise(clean, w.snr_db, wl.rng_for(140, 0)).astype(np.complex64)
    return w, echo


def poisoned(echo, flat_index, value, imag=False):
    e = echo.copy().reshape(-1)
    if imag:
        e[flat_index] = complex(e[flat_index].real, value)
    else:
        e[flat_index] = complex(value, e[flat_index].imag)
    return e.reshape(echo.shape)


def same(a, b):
    """Two reconstructions of the same echo by plans built alike."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b)) <= 1e-6 * float(np.linalg.norm(b))


def status_of(fn, binding):
    try:
        fn()
    except binding.PolylineError as e:
        return e.status
    return 0


@pytest.mark.parametrize("block_config", [0, 1])
def test_scan_is_transparent_on_finite_echo(binding, scene, block_config):
    w, echo = scene
    d = torch.from_numpy(echo).cuda()
    a = binding.Plan.from_workload(w, block_config=block_config)
    b = binding.Plan.from_workload(w, block_config=block_config, check_nonfinite=True)
    ia = a.execute(d).cpu().numpy()
    ib = b.execute(d).cpu().numpy()
    ib2 = b.execute(d).cpu().numpy()         # nothing reported by the clean first call
    torch.cuda.synchronize()
    assert same(ia, ib) and same(ib2, ib)
    a.close()
    b.close()


@pytest.mark.parametrize("where,value,imag", [("first", np.nan, False), ("last", np.inf, True),
                                              ("middle", -np.inf, False),
                                              ("middle", np.nan, True)])
@pytest.mark.parametrize("block_config", [0, 1])
def test_host_call_reports_nonfinite_echo_in_the_same_call(binding, scene, where, value, imag,
                                                           block_config):
    w, echo = scene
    n = echo.size
    idx = {"first": 0, "last": n - 1, "middle": n // 2 + 3}[where]
    bad = poisoned(echo, idx, value, imag)
    plan = binding.Plan.from_workload(w, block_config=block_config, check_nonfinite=True)
    assert status_of(lambda: plan.execute_host(bad), binding) == PL_ERR_NONFINITE
    # the flag was taken: a clean echo goes through and gives the usual image
    img = plan.execute_host(echo)
    ref = binding.Plan.from_workload(w, block_config=block_config).execute_host(echo)
    assert same(img, ref)
    plan.close()


@pytest.mark.parametrize("offset", [0, 1])
def test_device_call_reports_on_the_next_call(binding, scene, offset):
    # offset 1: the echo starts 8 bytes past a 16-byte boundary (the scan's
    # leading-element path); the poisoned value is the buffer's last
    w, echo = scene
    n = echo.size
    big = torch.zeros(n + offset, dtype=torch.complex64, device="cuda")
    view = big[offset:].view(echo.shape)
    assert view.data_ptr() % 16 == 8 * offset
    plan = binding.Plan.from_workload(w, check_nonfinite=True)
    for idx in (n - 1, 0):
        view.copy_(torch.from_numpy(poisoned(echo, idx, np.inf)))
        plan.execute(view)                   # asynchronous: no report yet
        torch.cuda.synchronize()
        view.copy_(torch.from_numpy(echo))
        assert status_of(lambda: plan.execute(view), binding) == PL_ERR_NONFINITE
        plan.execute(view)                   # the flag was cleared by the report
        torch.cuda.synchronize()
        assert status_of(lambda: plan.execute(view), binding) == 0
        torch.cuda.synchronize()
    plan.close()


def test_unchecked_plan_does_not_report(binding, scene):
    w, echo = scene
    plan = binding.Plan.from_workload(w)
    plan.execute_host(poisoned(echo, 5, np.nan))
    plan.execute_host(echo)                  # no scan, no report
    plan.close()


def test_host_stream_reports_a_poisoned_scan(binding, scene):
    w, echo = scene
    plan = binding.Plan.from_workload(w, check_nonfinite=True)
    scans = [echo, echo, poisoned(echo, 77, np.nan, imag=True), echo]
    assert status_of(lambda: plan.execute_host_stream(scans), binding) == PL_ERR_NONFINITE
    imgs = plan.execute_host_stream([echo, echo, echo])          # both plans' flags taken
    ref = plan.execute_host(echo)
    assert all(same(i, ref) for i in imgs)
    plan.close()


def test_batch_reports_a_poisoned_scene(binding):
    ws = [wl.small_mono(seed=s) for s in (4, 5)]
    echos = []
    for i, w in enumerate(ws):
        clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
        echos.append(wl.add_noise(clean, w.snr_db, wl.rng_for(141, i)).astype(np.complex64))
    b = binding.Batch(ws, check_nonfinite=True)
    good = [torch.from_numpy(e).cuda() for e in echos]
    first = [im.clone() for im in b.execute(good)]
    bad = [good[0], torch.from_numpy(poisoned(echos[1], 11, np.inf)).cuda()]
    assert status_of(lambda: b.execute(bad), binding) == PL_ERR_NONFINITE
    again = b.execute(good)
    assert all(same(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(first, again))
    b.close()


@pytest.mark.parametrize("block_config", [0, 1])
def test_every_plan_allocation_failure_is_reported_and_cleaned_up(binding, scene, block_config):
    w, echo = scene
    binding.Plan.from_workload(w, block_config=block_config).close()    # warm: modules loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for n in range(1, 200):
        st = status_of(lambda: binding.Plan.from_workload(w, block_config=block_config,
                                                          debug_fail_alloc=n).close(),
                       binding)
        if st == 0:
            break
        assert st == PL_ERR_OOM, (n, st)
        failures += 1
    else:
        raise AssertionError("the plan never completed")
    print("block_config %d: %d plan-time device allocations, each failure reported"
          % (block_config, failures))
    assert failures >= 10
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= 4 << 20          # nothing left allocated
    # the device and the library are fine afterwards
    plan = binding.Plan.from_workload(w, block_config=block_config)
    img = plan.execute_host(echo)
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo, w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    err = float(np.linalg.norm(img.reshape(ref.shape) - ref) / np.linalg.norm(ref))
    assert err < 2e-4
    plan.close()


def test_options_are_validated(binding, scene):
    w, _ = scene
    for kw in (dict(debug_fail_alloc=-1),):
        with pytest.raises(binding.PolylineError) as ei:
            binding.Plan.from_workload(w, **kw)
        assert ei.value.status == 1
