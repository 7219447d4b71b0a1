"""ctypes binding of libpolyline (include/polyline.h): argument marshalling only.

Every computation runs in the CUDA library. Device buffers are torch CUDA
tensors (complex64), streams are torch streams. If the library has not been
built, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpolyline.so")

PL_STAGE_ZFFT, PL_STAGE_RANGE_TABLE, PL_STAGE_BACKPROJECT, PL_STAGE_ZIFFT = range(4)
STAGE_NAMES = ("zfft", "range_table", "backproject", "zifft")

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


class PlGeometry(ctypes.Structure):
    _fields_ = [("mode", _I), ("radius", _D), ("n_sections", _I), ("chord_len", _D),
                ("n_elem", _I), ("elem_xy", _P), ("elem_section", _P), ("n_pairs", _I),
                ("pair_tx", _P), ("pair_rx", _P)]


class PlScan(ctypes.Structure):
    _fields_ = [("z0", _D), ("dz", _D), ("n", _I), ("n_pad", _I)]


class PlFreqs(ctypes.Structure):
    _fields_ = [("f_hz", _P), ("n", _I)]


class PlGrid(ctypes.Structure):
    _fields_ = [("x0", _D), ("dx", _D), ("y0", _D), ("dy", _D), ("z0", _D), ("dz", _D),
                ("nx", _I), ("ny", _I), ("nz", _I)]


class PlOptions(ctypes.Structure):
    _fields_ = [("precision", _I), ("nufft_sigma", _D), ("nufft_w", _I), ("tile_u", _I),
                ("block_config", _I), ("debug_unsatisfiable", _I), ("wait_timeout_us", _I),
                ("one_block_per_sm", _I), ("check_nonfinite", _I), ("debug_fail_alloc", _I),
                ("dense_products", _I), ("sparse_window_rows", _I), ("reserved", _I * 1)]


class PlInfo(ctypes.Structure):
    _fields_ = [("mode", _I), ("n_chan", _I), ("n_scan", _I), ("n_pad", _I), ("n_f", _I),
                ("nx", _I), ("ny", _I), ("nz", _I), ("table_len", _I), ("fine_len", _I),
                ("slab_rows", _I), ("nufft_w", _I), ("nufft_sigma", _D), ("table_h", _D),
                ("table_l0", _D), ("z_transform_fft", _I), ("launches_per_execute", _I),
                ("workspace_bytes", ctypes.c_size_t), ("updates_per_execute", _D),
                ("block_config", _I), ("tile_u", _I), ("bp_launches", _I),
                ("es_beta", _D), ("band_group", _I), ("table_layout", _I), ("table_cols", _I),
                ("table_exact", _I), ("precision", _I), ("sparse_products", _I)]


class PlBatchOptions(ctypes.Structure):
    _fields_ = [("tile_u", _I), ("block_config", _I), ("autotune", _I),
                ("wait_timeout_ms", _D), ("debug_unsatisfiable", _I), ("tc_launch", _I),
                ("reserved", _I * 6)]


class PlBatchInfo(ctypes.Structure):
    _fields_ = [("n_scenes", _I), ("tile_u", _I), ("block_config", _I), ("autotuned", _I),
                ("persistent", _I), ("persistent_blocks", _I), ("work_items", _I),
                ("launches_per_execute", _I), ("tune_best_ms", _D), ("tune_default_ms", _D),
                ("updates_per_execute", _D), ("workspace_bytes", ctypes.c_size_t)]


EXPORTED = ("pl_plan_create", "pl_execute", "pl_execute_host", "pl_execute_host_stream",
            "pl_execute_exact",
            "pl_execute_bp_direct", "pl_design", "pl_plan_destroy",
            "pl_plan_get_info", "pl_plan_workspace", "pl_plan_set_timing",
            "pl_plan_stage_times", "pl_synth_echo", "pl_synth_echo_static",
            "pl_batch_create", "pl_execute_batch", "pl_batch_get_info", "pl_batch_destroy",
            "pl_nn_padded_k", "pl_nn_conv3d", "pl_nn_wgrad_workspace", "pl_nn_conv3d_wgrad",
            "pl_nn_weight_flip", "pl_nn_elementwise", "pl_nn_resample", "pl_nn_features",
            "pl_nn_loss", "pl_nn_residual", "pl_nn_check", "pl_nn_to_complex", "pl_nn_adam",
            "pl_measure_peak", "pl_status_string", "pl_last_error", "pl_version")

_lib = None


class PlDesignInfo(ctypes.Structure):
    _fields_ = [("lambda_min", _D), ("lambda_c", _D), ("bandwidth", _D),
                ("theta_h_deg", _D), ("theta_z_deg", _D),
                ("max_rx_spacing", _D), ("max_elem_spacing", _D), ("max_scan_step", _D),
                ("res_x", _D), ("res_y", _D), ("res_z", _D),
                ("elem_spacing", _D), ("scan_step", _D),
                ("spacing_ok", _I), ("scan_step_ok", _I)]


class PolylineError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (status_string(status), status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load libpolyline.so; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpolyline.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    lib.pl_plan_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(PlGeometry),
                                   ctypes.POINTER(PlScan), ctypes.POINTER(PlFreqs),
                                   ctypes.POINTER(PlGrid), ctypes.POINTER(PlOptions)]
    lib.pl_execute.argtypes = [_P, _P, _P, _P]
    lib.pl_execute_host.argtypes = [_P, _P, _P, _P]
    lib.pl_execute_host_stream.argtypes = [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]
    lib.pl_execute_exact.argtypes = [_P, _P, _P, _P]
    lib.pl_execute_bp_direct.argtypes = [_P, _P, _P, _P]
    lib.pl_plan_destroy.argtypes = [_P]
    lib.pl_plan_get_info.argtypes = [_P, ctypes.POINTER(PlInfo)]
    lib.pl_plan_workspace.argtypes = [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]
    lib.pl_plan_set_timing.argtypes = [_P, _I]
    lib.pl_plan_stage_times.argtypes = [_P, ctypes.POINTER(_D), ctypes.POINTER(_I)]
    lib.pl_synth_echo.argtypes = [_I, _P, _P, _D, _D, _I, _P, _I, _I, _P, _P, _P, _P]
    lib.pl_synth_echo_static.argtypes = [_I, _P, _P, _D, _D, _I, _P, _I, _I, _P, _P, _P, _P]
    lib.pl_batch_create.argtypes = [ctypes.POINTER(_P), _I, ctypes.POINTER(PlGeometry),
                                    ctypes.POINTER(PlScan), ctypes.POINTER(PlFreqs),
                                    ctypes.POINTER(PlGrid), ctypes.POINTER(PlOptions),
                                    ctypes.POINTER(PlBatchOptions)]
    lib.pl_execute_batch.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]
    lib.pl_batch_get_info.argtypes = [_P, ctypes.POINTER(PlBatchInfo)]
    lib.pl_batch_destroy.argtypes = [_P]
    lib.pl_measure_peak.argtypes = [_I, _P, ctypes.POINTER(_D)]
    lib.pl_measure_peak.restype = _I
    lib.pl_status_string.restype = ctypes.c_char_p
    lib.pl_status_string.argtypes = [_I]
    lib.pl_last_error.restype = ctypes.c_char_p
    lib.pl_version.restype = _I
    for name in ("pl_plan_create", "pl_execute", "pl_execute_host", "pl_execute_host_stream",
                 "pl_plan_destroy",
                 "pl_plan_get_info", "pl_plan_workspace", "pl_plan_set_timing",
                 "pl_plan_stage_times", "pl_synth_echo", "pl_synth_echo_static",
                 "pl_batch_create", "pl_execute_batch", "pl_batch_get_info", "pl_batch_destroy"):
        getattr(lib, name).restype = _I
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().pl_status_string(s).decode()


def _check(status: int):
    if status != 0:
        raise PolylineError(status, load().pl_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream)


class _DevArray:
    """Exposes a raw device pointer to torch via __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _descriptors(keep, mode, elem_xy, scan_z0, scan_dz, n_scan, f_hz, grid, n_pad, pair_tx,
                 pair_rx, radius, n_sections, chord_len, elem_section, precision, nufft_sigma,
                 nufft_w, tile_u, block_config, debug_unsatisfiable=0, wait_timeout_us=0,
                 one_block_per_sm=0, check_nonfinite=0, debug_fail_alloc=0, dense_products=0,
                 sparse_window_rows=0):
    exy = _f64(elem_xy).reshape(-1, 2)
    sec = None if elem_section is None else _i32(elem_section)
    ptx = None if pair_tx is None else _i32(pair_tx)
    prx = None if pair_rx is None else _i32(pair_rx)
    f = _f64(f_hz).ravel()
    keep += [exy, sec, ptx, prx, f]
    geom = PlGeometry(int(mode), float(radius), int(n_sections), float(chord_len),
                      exy.shape[0], _ptr(exy), _ptr(sec),
                      0 if ptx is None else ptx.size, _ptr(ptx), _ptr(prx))
    scan = PlScan(float(scan_z0), float(scan_dz), int(n_scan), int(n_pad))
    freqs = PlFreqs(_ptr(f), f.size)
    g = PlGrid(float(grid["x0"]), float(grid["dx"]), float(grid["y0"]), float(grid["dy"]),
               float(grid["z0"]), float(grid["dz"]), int(grid["nx"]), int(grid["ny"]),
               int(grid["nz"]))
    opt = PlOptions(int(precision), float(nufft_sigma), int(nufft_w), int(tile_u),
                    int(block_config), int(debug_unsatisfiable), int(wait_timeout_us),
                    int(one_block_per_sm), 1 if check_nonfinite else 0, int(debug_fail_alloc),
                    1 if dense_products else 0, int(sparse_window_rows))
    return geom, scan, freqs, g, opt


def _workload_args(w):
    return (w.mode, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.grid, w.n_pad,
            w.pair_tx if w.mode == 1 else None, w.pair_rx if w.mode == 1 else None, w.radius,
            w.n_sections, w.chord_len, w.elem_section)


class Plan:
    """A reconstruction plan (pl_plan_create / pl_execute / pl_plan_destroy)."""

    def __init__(self, mode, elem_xy, scan_z0, scan_dz, n_scan, f_hz, grid, n_pad=0,
                 pair_tx=None, pair_rx=None, radius=0.0, n_sections=0, chord_len=0.0,
                 elem_section=None, precision=0, nufft_sigma=0.0, nufft_w=0, tile_u=0,
                 block_config=0, debug_unsatisfiable=0, wait_timeout_us=0, one_block_per_sm=0,
                 check_nonfinite=False, debug_fail_alloc=0, dense_products=False,
                 sparse_window_rows=0):
        lib = load()
        self._keep = []
        geom, scan, freqs, g, opt = _descriptors(
            self._keep, mode, elem_xy, scan_z0, scan_dz, n_scan, f_hz, grid, n_pad, pair_tx,
            pair_rx, radius, n_sections, chord_len, elem_section, precision, nufft_sigma,
            nufft_w, tile_u, block_config, debug_unsatisfiable, wait_timeout_us,
            one_block_per_sm, check_nonfinite, debug_fail_alloc, dense_products,
            sparse_window_rows)
        h = _P()
        _check(lib.pl_plan_create(ctypes.byref(h), geom, scan, freqs, g, opt))
        self._h = h
        self.info = self.get_info()

    @classmethod
    def from_workload(cls, w, **opts):
        return cls(w.mode, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.grid, n_pad=w.n_pad,
                   pair_tx=w.pair_tx if w.mode == 1 else None,
                   pair_rx=w.pair_rx if w.mode == 1 else None, radius=w.radius,
                   n_sections=w.n_sections, chord_len=w.chord_len, elem_section=w.elem_section,
                   **opts)

    def get_info(self) -> dict:
        i = PlInfo()
        _check(load().pl_plan_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in PlInfo._fields_}

    @property
    def echo_shape(self):
        return (self.info["n_chan"], self.info["n_scan"], self.info["n_f"])

    @property
    def image_shape(self):
        return (self.info["nz"], self.info["ny"], self.info["nx"])

    def execute(self, echo, image=None, stream=None):
        """echo: CUDA complex64 [n_chan][n_scan][n_f]; returns image [nz][ny][nx]."""
        import torch
        assert echo.is_cuda and echo.dtype == torch.complex64 and echo.is_contiguous()
        assert tuple(echo.shape) == self.echo_shape
        if image is None:
            image = torch.empty(self.image_shape, dtype=torch.complex64, device=echo.device)
        assert image.is_cuda and image.dtype == torch.complex64 and image.is_contiguous()
        assert tuple(image.shape) == self.image_shape
        _check(load().pl_execute(self._h, _P(echo.data_ptr()), _P(image.data_ptr()),
                                 _stream_handle(stream)))
        return image

    def execute_host(self, echo, image=None, stream=None):
        """Host buffers in and out (copies inside the call); returns a NumPy image."""
        if image is None:
            image = np.empty(self.image_shape, dtype=np.complex64)
        import torch
        if isinstance(echo, torch.Tensor):
            assert not echo.is_cuda and echo.dtype == torch.complex64 and echo.is_contiguous()
            eptr = echo.data_ptr()
        else:
            assert echo.dtype == np.complex64 and echo.flags.c_contiguous
            eptr = echo.ctypes.data
        if isinstance(image, torch.Tensor):
            iptr = image.data_ptr()
        else:
            iptr = image.ctypes.data
        _check(load().pl_execute_host(self._h, _P(eptr), _P(iptr), _stream_handle(stream)))
        return image

    def execute_host_stream(self, echoes, images=None, stream=None):
        """A sequence of scans from host buffers with the copies overlapped
        with the reconstruction; returns the list of host images."""
        import torch
        n = len(echoes)
        if images is None:
            images = [np.empty(self.image_shape, dtype=np.complex64) for _ in range(n)]
        assert len(images) == n

        def ptr(a, shape):
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.dtype == torch.complex64 and a.is_contiguous()
                assert tuple(a.shape) == shape
                return a.data_ptr()
            assert a.dtype == np.complex64 and a.flags.c_contiguous and a.shape == shape
            return a.ctypes.data

        ep = (_P * max(n, 1))(*[ptr(e, self.echo_shape) for e in echoes])
        ip = (_P * max(n, 1))(*[ptr(i, self.image_shape) for i in images])
        _check(load().pl_execute_host_stream(self._h, n, ep, ip, _stream_handle(stream)))
        return images

    def execute_exact(self, echo, image=None, stream=None):
        """The exact-sum hybrid ("omega-K-BP", Sec. III): same buffers as execute."""
        return self._execute_with(load().pl_execute_exact, echo, image, stream)

    def execute_bp_direct(self, echo, image=None, stream=None):
        """Direct back-projection (the "BP" of Sec. III): same buffers as execute."""
        return self._execute_with(load().pl_execute_bp_direct, echo, image, stream)

    def _execute_with(self, fn, echo, image, stream):
        import torch
        assert echo.is_cuda and echo.dtype == torch.complex64 and echo.is_contiguous()
        assert tuple(echo.shape) == self.echo_shape
        if image is None:
            image = torch.empty(self.image_shape, dtype=torch.complex64, device=echo.device)
        _check(fn(self._h, _P(echo.data_ptr()), _P(image.data_ptr()), _stream_handle(stream)))
        return image

    def workspace(self, stage):
        """Torch view (complex64) of an intermediate buffer."""
        import torch
        ptr = _P()
        nbytes = ctypes.c_size_t()
        _check(load().pl_plan_workspace(self._h, int(stage), ctypes.byref(ptr),
                                        ctypes.byref(nbytes)))
        i = self.info
        if stage == PL_STAGE_ZFFT:
            shape = (i["n_chan"], i["n_pad"], i["n_f"])
            if nbytes.value == np.prod(shape) * 4:        # BF16 spectrum (precision 2)
                raw = torch.as_tensor(_DevArray(ptr.value, shape + (2,), "<i2"), device="cuda")
                return raw.view(torch.bfloat16)
        elif stage == PL_STAGE_RANGE_TABLE:
            lay = i["table_layout"]
            if lay in (2, 3):
                # tensor-core layout [c][hi/lo][row][column] (BF16; columns
                # 2u + (re, im), or planar: Re of the bins, then Im)
                shape = (i["n_chan"], 2, i["table_len"], i["table_cols"])
            else:
                # rows of planar bin pairs {re_u, re_u+1, im_u, im_u+1}
                shape = (i["n_chan"], i["table_len"], (i["n_pad"] + 1) // 2, 4)
            esize = 4 if lay == 0 else 2
            assert nbytes.value == np.prod(shape) * esize, (nbytes.value, shape, lay)
            if esize == 2:
                raw = torch.as_tensor(_DevArray(ptr.value, shape, "<i2"), device="cuda")
                return raw.view(torch.bfloat16)
            return torch.as_tensor(_DevArray(ptr.value, shape, "<f4"), device="cuda")
        else:
            # [parts][n_pad][ny][nx]; the spectrum is the sum over parts
            plane = i["n_pad"] * i["ny"] * i["nx"] * 8
            shape = (nbytes.value // plane, i["n_pad"], i["ny"], i["nx"])
        return torch.as_tensor(_DevArray(ptr.value, shape, "<c8"), device="cuda")

    def set_timing(self, enable: bool = True):
        _check(load().pl_plan_set_timing(self._h, 1 if enable else 0))

    def stage_times(self):
        """{stage: (total_ms, launches)} since the last call / set_timing."""
        ms = (_D * 4)()
        n = (_I * 4)()
        _check(load().pl_plan_stage_times(self._h, ms, n))
        return {STAGE_NAMES[s]: (ms[s], n[s]) for s in range(4)}

    def close(self):
        if getattr(self, "_h", None):
            load().pl_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def design(w, target_dim=0.0, beamwidth_z_deg=0.0) -> dict:
    """Sampling and resolution figures of Sec. II-C/D (pl_design) for a
    workload's array, scan and band (host computation)."""
    lib = load()
    keep = []
    geom, scan, freqs, _, _ = _descriptors(keep, *_workload_args(w), 0, 0.0, 0, 0, 0)
    d = PlDesignInfo()
    lib.pl_design.argtypes = [ctypes.POINTER(PlGeometry), ctypes.POINTER(PlScan),
                              ctypes.POINTER(PlFreqs), _D, _D, ctypes.POINTER(PlDesignInfo)]
    _check(lib.pl_design(ctypes.byref(geom), ctypes.byref(scan), ctypes.byref(freqs),
                         float(target_dim), float(beamwidth_z_deg), ctypes.byref(d)))
    return {k: getattr(d, k) for k, _ in PlDesignInfo._fields_}


def synth_echo(tx_xy, rx_xy, z0, dz, n_scan, f_hz, pts, amp, out=None, stream=None):
    """Point-scatterer echo on the GPU (Eq. 1 / Eq. 10); returns CUDA complex64."""
    import torch
    tx = _f64(tx_xy).reshape(-1, 2)
    rx = _f64(rx_xy).reshape(-1, 2)
    f = _f64(f_hz).ravel()
    p = _f64(pts).reshape(-1, 3)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(amp, np.complex128), (p.shape[0],)))
    a = _f64(np.stack([a.real, a.imag], 1))
    if out is None:
        out = torch.empty((tx.shape[0], n_scan, f.size), dtype=torch.complex64, device="cuda")
    _check(load().pl_synth_echo(tx.shape[0], _ptr(tx), _ptr(rx), float(z0), float(dz),
                                int(n_scan), _ptr(f), f.size, p.shape[0], _ptr(p), _ptr(a),
                                _P(out.data_ptr()), _stream_handle(stream)))
    return out


def synth_echo_static(tx_xy, rx_xy, z0, dz, n_scan, f_hz, pts, amp, out=None, stream=None):
    """Same as synth_echo through pl_synth_echo_static, which allocates no
    device memory (for callers that cannot allocate; see include/polyline.h).
    Asynchronous on `stream`."""
    import torch
    tx = _f64(tx_xy).reshape(-1, 2)
    rx = _f64(rx_xy).reshape(-1, 2)
    f = _f64(f_hz).ravel()
    p = _f64(pts).reshape(-1, 3)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(amp, np.complex128), (p.shape[0],)))
    a = _f64(np.stack([a.real, a.imag], 1))
    if out is None:
        out = torch.empty((tx.shape[0], n_scan, f.size), dtype=torch.complex64, device="cuda")
    _check(load().pl_synth_echo_static(tx.shape[0], _ptr(tx), _ptr(rx), float(z0), float(dz),
                                       int(n_scan), _ptr(f), f.size, p.shape[0], _ptr(p),
                                       _ptr(a), _P(out.data_ptr()), _stream_handle(stream)))
    return out


PEAK_UNITS = ("TFLOP/s", "Gsin/s", "GB/s")


def measure_peak(which: int, stream=None) -> float:
    """pl_measure_peak: 0 FP32 FMA (TFLOP/s), 1 MUFU sine (G/s), 2 shared-memory
    load bandwidth (GB/s), measured on the current device."""
    v = _D()
    _check(load().pl_measure_peak(int(which), _stream_handle(stream), ctypes.byref(v)))
    return v.value


class Batch:
    """Uneven scans reconstructed together (pl_batch_create / pl_execute_batch):
    per-scene z transforms around one persistent range-table + back-projection
    launch, replayed as a CUDA graph."""

    def __init__(self, workloads, precision=0, nufft_sigma=0.0, nufft_w=0, tile_u=0,
                 block_config=0, autotune=False, wait_timeout_ms=0.0, debug_unsatisfiable=0,
                 tc_launch=0, tc_debug_unsatisfiable=0, tc_wait_timeout_us=0,
                 check_nonfinite=False):
        lib = load()
        self._keep = []
        n = len(workloads)
        G, S, F, R, O = ((PlGeometry * n)(), (PlScan * n)(), (PlFreqs * n)(), (PlGrid * n)(),
                         (PlOptions * n)())
        for i, w in enumerate(workloads):
            G[i], S[i], F[i], R[i], O[i] = _descriptors(
                self._keep, *_workload_args(w), precision, nufft_sigma, nufft_w, 0, 0,
                tc_debug_unsatisfiable, tc_wait_timeout_us, 0, check_nonfinite)
        bo = PlBatchOptions(int(tile_u), int(block_config), 1 if autotune else 0,
                            float(wait_timeout_ms), int(debug_unsatisfiable), int(tc_launch))
        h = _P()
        _check(lib.pl_batch_create(ctypes.byref(h), n, G, S, F, R, O, ctypes.byref(bo)))
        self._h = h
        self.n = n
        self.echo_shapes = [(w.n_chan, w.n_scan, w.n_f) for w in workloads]
        self.image_shapes = [(w.grid["nz"], w.grid["ny"], w.grid["nx"]) for w in workloads]
        self.info = self.get_info()

    def get_info(self) -> dict:
        i = PlBatchInfo()
        _check(load().pl_batch_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in PlBatchInfo._fields_}

    def execute(self, echos, images=None, stream=None):
        import torch
        if images is None:
            images = [torch.empty(s, dtype=torch.complex64, device=e.device)
                      for s, e in zip(self.image_shapes, echos)]
        for e, s in zip(echos, self.echo_shapes):
            assert e.is_cuda and e.dtype == torch.complex64 and tuple(e.shape) == s
        ep = (_P * self.n)(*[e.data_ptr() for e in echos])
        ip = (_P * self.n)(*[im.data_ptr() for im in images])
        _check(load().pl_execute_batch(self._h, ep, ip, _stream_handle(stream)))
        return images

    def close(self):
        if getattr(self, "_h", None):
            load().pl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
