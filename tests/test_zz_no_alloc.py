"""pl_synth_echo_static: the entry point for callers that cannot allocate
device memory (it keeps its scratch in a static device array instead of
calling cudaMalloc). Its echo must match pl_synth_echo's on the same inputs,
call after call, since every call reuses the same scratch.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6   # both entry points run the same kernel on the same FP32 inputs


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


def _pair(binding, w, pts, amp):
    ref = binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, pts, amp)
    got = binding.synth_echo_static(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, pts, amp)
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.cpu().numpy()


def test_static_scratch_matches_allocating_entry_point_twice(binding):
    # first call: small monostatic scene; second call: a different,
    # multistatic geometry with more points (the scratch keeps the first
    # call's contents, which must not leak into the second result)
    w1 = wl.small_mono(seed=3)
    got, ref = _pair(binding, w1, w1.pts, w1.amp)
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)

    w2 = wl.small_mono(seed=4, n_pts=40)
    xy, sec, ptx, prx, _ = wl.multistatic_array(0.5, 4, 60.0, 2, 16)
    w2.mode, w2.elem_xy, w2.pair_tx, w2.pair_rx = 1, xy, ptx, prx
    w2.f_hz = w2.f_hz[:11]
    got, ref = _pair(binding, w2, w2.pts, w2.amp * (0.5 - 0.25j))
    assert got.shape == (w2.n_chan, w2.n_scan, 11)
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


def test_static_scratch_rejects_sizes_beyond_its_limit(binding):
    w = wl.small_mono(seed=0)
    too_many = np.zeros((16385, 3))
    with pytest.raises(binding.PolylineError) as ei:
        binding.synth_echo_static(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, too_many,
                                  np.ones(16385))
    assert ei.value.status == 1
    assert "static scratch" in str(ei.value)
