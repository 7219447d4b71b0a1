"""Sampling / resolution figures of Sec. II-C/D (pl_design, host code): the
angles come from the array the generator built, the monostatic limit is half
the multistatic one (two-way paths), limits shrink with the target size and
the scan aperture, and the paper's own Table I array meets its limits."""
import math

import pytest

from paper_2109_02842_gb300 import workloads as wl

C0 = 299792458.0


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    return b


def test_angles_and_band_follow_the_array(binding):
    w = wl.small_mono(seed=0)               # 4 chords over 60 degrees, 28-33 GHz
    d = binding.design(w)
    assert abs(d["theta_h_deg"] - 60.0) < 1e-9
    assert abs(d["bandwidth"] - 5e9) < 1.0
    assert abs(d["lambda_min"] - C0 / 33e9) < 1e-12
    span = (w.n_scan - 1) * w.dz
    assert abs(math.radians(d["theta_z_deg"]) - 2 * math.atan(span / 2 / w.radius)) < 1e-12
    # a beam narrower than the scan aperture limits theta_z
    assert binding.design(w, beamwidth_z_deg=5.0)["theta_z_deg"] == pytest.approx(5.0)


def test_monostatic_limit_is_half_and_shrinks_with_target(binding):
    w = wl.paper_table1(0)
    m = wl.paper_table1(1)
    dm, dx = binding.design(w, 0.2), binding.design(m, 0.2)
    assert dm["max_elem_spacing"] == pytest.approx(0.5 * dx["max_rx_spacing"])
    assert dx["max_elem_spacing"] == pytest.approx(dx["max_rx_spacing"])
    assert binding.design(w, 0.5)["max_rx_spacing"] < dm["max_rx_spacing"]
    # resolutions do not depend on the target size; finer with a wider band
    assert binding.design(w, 0.5)["res_x"] == dm["res_x"]
    w2 = wl.paper_table1(0)
    w2.f_hz = w2.f_hz * 1.0
    w2.f_hz[-1] = 40e9
    assert binding.design(w2)["res_y"] < dm["res_y"]


def test_paper_table1_arrays_meet_their_limits(binding):
    # Table I: 0.48 cm monostatic spacing, 20 receivers per 0.192 m section
    for mode in (0, 1):
        d = binding.design(wl.paper_table1(mode), target_dim=0.2)
        assert d["spacing_ok"] == 1 and d["scan_step_ok"] == 1, d
    assert binding.design(wl.paper_table1(0))["elem_spacing"] == pytest.approx(0.0048, rel=1e-6)


def test_bad_inputs_are_rejected(binding):
    w = wl.small_mono(seed=0)
    w.f_hz = w.f_hz * -1.0
    with pytest.raises(binding.PolylineError):
        binding.design(w)
