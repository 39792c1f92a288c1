"""Python binding of the SRP C ABI (``include/srp.h``).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libsrp.so``.  The functions keep the C names; tensors are torch
CUDA tensors passed by ``data_ptr()``; streams default to torch's current
stream.  There is no CPU fallback: loading fails loudly if the library has
not been built (``python -m paper_2012_09499_gb300.build_lib``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsrp.so")

SRP_OK, SRP_ERR_INVALID_ARG, SRP_ERR_OOM, SRP_ERR_CUDA, SRP_ERR_UNSUPPORTED, SRP_ERR_TIMEOUT = range(6)
MODES = {"conventional": 1, "nyquist": 2}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2}
INPUTS = {"stft": 0, "cross": 1}
ENGINES = {"auto": 0, "cuda_cores": 1}
WEIGHTINGS = {"phat": 0, "none": 1}
STAGES = ("cross_spectra", "gcc_samples", "map", "argmax")


class SrpError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class srp_plan_desc(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32), ("mic_xyz", ctypes.POINTER(ctypes.c_double)),
        ("grid_kind", ctypes.c_int), ("J", ctypes.c_int64),
        ("grid_xyz", ctypes.POINTER(ctypes.c_double)),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("K", ctypes.c_int32),
        ("mode", ctypes.c_int), ("n_aux", ctypes.c_int32), ("precision", ctypes.c_int),
        ("input_kind", ctypes.c_int), ("max_frames", ctypes.c_int32),
        ("host_io", ctypes.c_int32), ("engine", ctypes.c_int), ("weighting", ctypes.c_int),
        ("resident_fraction", ctypes.c_float), ("argmax", ctypes.c_int),
    ]


class srp_plan_info(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32), ("Q", ctypes.c_int32), ("K", ctypes.c_int32),
        ("Kb", ctypes.c_int32), ("J", ctypes.c_int64), ("n_aux", ctypes.c_int32),
        ("S", ctypes.c_int32), ("max_nq", ctypes.c_int32), ("x_frac_bits", ctypes.c_int32),
        ("max_frames", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
        ("device_bytes", ctypes.c_size_t), ("weight_bytes", ctypes.c_size_t),
        ("argmax_rescored", ctypes.c_int32), ("accum_promotion", ctypes.c_int32),
        ("gcc_tensor_cores", ctypes.c_int32),
    ]


class srp_complexity(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_double), ("P", ctypes.c_int32), ("K_b", ctypes.c_int32),
        ("J", ctypes.c_int64), ("C_samp", ctypes.c_double), ("C_int", ctypes.c_double),
        ("C_conv", ctypes.c_double), ("R_samp", ctypes.c_double), ("R_int", ctypes.c_double),
        ("R", ctypes.c_double),
    ]


class srp_refine_desc(ctypes.Structure):
    _fields_ = [
        ("n_offsets", ctypes.c_int32), ("offsets", ctypes.POINTER(ctypes.c_double)),
        ("levels", ctypes.c_int32), ("shrink", ctypes.c_double), ("keep_grid", ctypes.c_int32),
    ]


class srp_batch_tiles(ctypes.Structure):
    _fields_ = [("frames_per_tile", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("operand_a", ctypes.c_int32),
                ("accumulators", ctypes.c_int32)]


class srp_batch_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("items", ctypes.c_int32), ("ctas", ctypes.c_int32),
        ("tiles", srp_batch_tiles), ("launches", ctypes.c_int32), ("tuned", ctypes.c_int32),
        ("tuned_ms", ctypes.c_float), ("device_bytes", ctypes.c_size_t),
    ]


class srp_server_desc(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_size_t), ("host_budget_bytes", ctypes.c_size_t),
                ("max_inflight", ctypes.c_int32), ("no_batching", ctypes.c_int32)]


class srp_completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("tag", ctypes.c_uint64),
                ("stream", ctypes.c_int32), ("L", ctypes.c_int32), ("status", ctypes.c_int32),
                ("iteration_streams", ctypes.c_int32), ("iteration_frames", ctypes.c_int32),
                ("iteration", ctypes.c_int64),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("t_gpu_start_ms", ctypes.c_double),
                ("t_gpu_end_ms", ctypes.c_double)]


class srp_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "completed", "frames_completed", "rejected", "timed_out", "failed",
        "iterations", "kernel_launches", "admission_waits", "queued")] + [
        ("device_budget_bytes", ctypes.c_size_t), ("device_bytes_in_use", ctypes.c_size_t),
        ("device_bytes_peak", ctypes.c_size_t), ("batched_streams", ctypes.c_int32),
        ("max_iteration_streams", ctypes.c_int32), ("overlapped_iterations", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libsrp.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2012_09499_gb300.build_lib`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
        dp = ctypes.POINTER(srp_plan_desc)
        sigs = {
            "srp_plan_describe": [dp, ctypes.POINTER(srp_plan_info), vp],
            "srp_plan_footprint": [dp, ctypes.POINTER(ctypes.c_size_t)],
            "srp_plan_complexity": [dp, ctypes.POINTER(srp_complexity)],
            "srp_plan": [dp, ctypes.POINTER(vp)],
            "srp_plan_get_info": [vp, ctypes.POINTER(srp_plan_info)],
            "srp_plan_tdoa": [vp, vp],
            "srp_map": [vp, vp, i32, vp, vp, vp, vp],
            "srp_map_host": [vp, vp, i32, vp, vp, vp, vp],
            "srp_map_host_async": [vp, vp, i32, vp, vp, vp, vp],
            "srp_map_host_wait": [vp],
            "srp_cross_spectra": [vp, vp, i32, vp, vp],
            "srp_gcc_samples": [vp, vp, i32, vp, vp],
            "srp_set_timing": [vp, i32],
            "srp_stage_times": [vp, vp, i32],
            "srp_last_launch_count": [vp, ctypes.POINTER(i32)],
            "srp_destroy": [vp],
            "srp_poll_device_status": [vp, vp],
            "srp_refiner_create": [vp, dp, ctypes.POINTER(srp_refine_desc), ctypes.POINTER(vp)],
            "srp_refine": [vp, i32, vp, vp, vp, vp, vp, vp],
            "srp_refiner_destroy": [vp],
            "srp_batch_create": [vp, i32, vp, ctypes.POINTER(vp)],
            "srp_map_batch": [vp, vp, vp, vp, vp, vp, vp],
            "srp_batch_tune": [vp, vp, vp, vp, vp, vp, vp],
            "srp_batch_get_info": [vp, ctypes.POINTER(srp_batch_info)],
            "srp_batch_stage_times": [vp, vp, i32],
            "srp_batch_set_timing": [vp, i32],
            "srp_batch_poll_device_status": [vp, vp],
            "srp_batch_destroy": [vp],
            "srp_server_create": [vp, i32, ctypes.POINTER(srp_server_desc), ctypes.POINTER(vp)],
            "srp_server_submit": [vp, i32, vp, i32, vp, vp, vp, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_uint64)],
            "srp_server_poll": [vp, vp, i32, ctypes.POINTER(i32), i32],
            "srp_server_get_stats": [vp, ctypes.POINTER(srp_server_stats)],
            "srp_server_hold": [vp, i32],
            "srp_server_destroy": [vp],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = st
        L.srp_status_string.argtypes = [st]
        L.srp_status_string.restype = ctypes.c_char_p
        L.srp_last_error_message.argtypes = []
        L.srp_last_error_message.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != SRP_OK:
        L = lib()
        detail = (L.srp_status_string(status) or b"").decode()
        msg = (L.srp_last_error_message() or b"").decode()
        raise SrpError(status, where, f"{detail}: {msg}" if msg else detail)


def _ptr(t):
    """Device address of a tensor (or None for NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _host_ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_desc(mic_xyz, grid_xyz, fs, c, K, mode="nyquist", n_aux=2, precision="fp32",
              input_kind="stft", max_frames=64, far_field=False, host_io=False, engine="auto",
              weighting="phat", resident_weights=False, resident_fraction=None,
              argmax="rescore"):
    """Fill an srp_plan_desc; returns (desc, keep-alive arrays).  argmax:
    "rescore" (reduced-precision plans choose the maximiser in FP32) or
    "map" (the reduced-precision map's own first maximiser)."""
    mic = np.ascontiguousarray(mic_xyz, np.float64)
    grid = np.ascontiguousarray(grid_xyz, np.float64)
    d = srp_plan_desc()
    d.M = mic.shape[0]
    d.mic_xyz = mic.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.grid_kind = 1 if far_field else 0
    d.J = grid.shape[0]
    d.grid_xyz = grid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.fs, d.c, d.K = float(fs), float(c), int(K)
    d.mode = MODES[mode]
    d.n_aux = int(n_aux)
    d.precision = PRECISIONS[precision]
    d.input_kind = INPUTS[input_kind]
    d.max_frames = int(max_frames)
    d.host_io = int(host_io)  # 0, 1 (srp_map_host) or 2 (also srp_map_host_async)
    d.engine = ENGINES[engine]
    d.weighting = WEIGHTINGS[weighting]
    # resident_weights=True streams the whole matrix; resident_fraction a part of it
    d.resident_fraction = float(resident_fraction if resident_fraction is not None
                                else (1.0 if resident_weights else 0.0))
    d.argmax = {"rescore": 0, "map": 1}[argmax]
    return d, (mic, grid)


def srp_plan_describe(desc):
    info = srp_plan_info()
    nq = np.zeros(max(desc.M * (desc.M - 1) // 2, 1), np.int32)
    _check(lib().srp_plan_describe(ctypes.byref(desc), ctypes.byref(info), nq.ctypes.data),
           "srp_plan_describe")
    return info, nq[: info.Q]


def srp_plan_complexity(desc) -> dict:
    """Operation counts and reduction factors of Sec. 3.3 for a descriptor."""
    c = srp_complexity()
    _check(lib().srp_plan_complexity(ctypes.byref(desc), ctypes.byref(c)), "srp_plan_complexity")
    return {k: getattr(c, k) for k, _ in srp_complexity._fields_}


def srp_plan_footprint(desc) -> int:
    b = ctypes.c_size_t()
    _check(lib().srp_plan_footprint(ctypes.byref(desc), ctypes.byref(b)), "srp_plan_footprint")
    return int(b.value)


def srp_plan(desc):
    h = ctypes.c_void_p()
    _check(lib().srp_plan(ctypes.byref(desc), ctypes.byref(h)), "srp_plan")
    return h


def srp_plan_get_info(h):
    info = srp_plan_info()
    _check(lib().srp_plan_get_info(h, ctypes.byref(info)), "srp_plan_get_info")
    return info


def srp_plan_tdoa(h):
    info = srp_plan_get_info(h)
    x = np.zeros((info.J, info.Q), np.float64)
    _check(lib().srp_plan_tdoa(h, x.ctypes.data), "srp_plan_tdoa")
    return x


def srp_map(h, d_in, L, d_maps, d_argmax, d_peak=None, stream=None):
    _check(lib().srp_map(h, _ptr(d_in), int(L), _ptr(d_maps), _ptr(d_argmax), _ptr(d_peak),
                         _stream(stream)), "srp_map")


def srp_map_host(h, h_in, L, h_maps, h_argmax, h_peak=None, stream=None):
    _check(lib().srp_map_host(h, _host_ptr(h_in), int(L), _host_ptr(h_maps),
                              _host_ptr(h_argmax), _host_ptr(h_peak), _stream(stream)),
           "srp_map_host")


def srp_map_host_async(h, h_in, L, h_maps, h_argmax, h_peak=None, stream=None):
    _check(lib().srp_map_host_async(h, _host_ptr(h_in), int(L), _host_ptr(h_maps),
                                    _host_ptr(h_argmax), _host_ptr(h_peak), _stream(stream)),
           "srp_map_host_async")


def srp_map_host_wait(h):
    _check(lib().srp_map_host_wait(h), "srp_map_host_wait")


def srp_cross_spectra(h, d_y, L, d_psi, stream=None):
    _check(lib().srp_cross_spectra(h, _ptr(d_y), int(L), _ptr(d_psi), _stream(stream)),
           "srp_cross_spectra")


def srp_gcc_samples(h, d_in, L, d_xi, stream=None):
    _check(lib().srp_gcc_samples(h, _ptr(d_in), int(L), _ptr(d_xi), _stream(stream)),
           "srp_gcc_samples")


def srp_set_timing(h, enable=True):
    _check(lib().srp_set_timing(h, 1 if enable else 0), "srp_set_timing")


def srp_stage_times(h):
    ms = (ctypes.c_float * len(STAGES))()
    _check(lib().srp_stage_times(h, ctypes.addressof(ms), len(STAGES)), "srp_stage_times")
    return dict(zip(STAGES, list(ms)))


def srp_last_launch_count(h) -> int:
    n = ctypes.c_int32()
    _check(lib().srp_last_launch_count(h, ctypes.byref(n)), "srp_last_launch_count")
    return int(n.value)


def srp_poll_device_status(h, stream=None):
    _check(lib().srp_poll_device_status(h, _stream(stream)), "srp_poll_device_status")


def srp_destroy(h):
    _check(lib().srp_destroy(h), "srp_destroy")


class Plan:
    """Owns one plan handle; allocates outputs with torch for convenience."""

    def __init__(self, mic_xyz, grid_xyz, fs, c, K, **kw):
        self.desc, self._keep = make_desc(mic_xyz, grid_xyz, fs, c, K, **kw)
        self.handle = srp_plan(self.desc)
        self.info = srp_plan_get_info(self.handle)

    def map(self, d_in, L=None, maps=True, stream=None):
        """Run the hot path on a complex64 CUDA tensor ([L][M][Kb] STFT or
        [L][Q][Kb] cross spectra); returns (maps[L][J] or None, argmax[L], peak[L])."""
        import torch
        L = d_in.shape[0] if L is None else L
        dev = d_in.device
        out_maps = torch.empty((L, self.info.J), dtype=torch.float32, device=dev) if maps else None
        am = torch.empty(L, dtype=torch.int32, device=dev)
        pk = torch.empty(L, dtype=torch.float32, device=dev)
        srp_map(self.handle, d_in, L, out_maps, am, pk, stream)
        return out_maps, am, pk

    def close(self):
        if self.handle is not None:
            srp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Refiner:
    """Coarse-to-fine search around per-frame centres on a Nyquist Plan (see
    srp_refine): offsets [F][3], levels, shrink per level; keep_grid lets
    refine() take the plan's argmax as centres."""

    def __init__(self, plan, offsets, levels=1, shrink=0.5, keep_grid=True):
        self.plan = plan
        self.offsets = np.ascontiguousarray(offsets, np.float64).reshape(-1, 3)
        d = srp_refine_desc(self.offsets.shape[0],
                            self.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            int(levels), float(shrink), 1 if keep_grid else 0)
        h = ctypes.c_void_p()
        _check(lib().srp_refiner_create(plan.handle, ctypes.byref(plan.desc), ctypes.byref(d),
                                        ctypes.byref(h)), "srp_refiner_create")
        self.handle = h

    def refine(self, L, argmax=None, centres=None, values=False, stream=None):
        """Returns (best_xyz [L][3] float64, best_val [L], values [L][F] or
        None) as CUDA tensors; argmax: int32 [L] or centres: float64 [L][3]."""
        import torch
        dev = (argmax if argmax is not None else centres).device
        xyz = torch.empty((L, 3), dtype=torch.float64, device=dev)
        val = torch.empty(L, dtype=torch.float32, device=dev)
        vals = (torch.empty((L, self.offsets.shape[0]), dtype=torch.float32, device=dev)
                if values else None)
        _check(lib().srp_refine(self.handle, int(L), _ptr(argmax), _ptr(centres), _ptr(xyz),
                                _ptr(val), _ptr(vals), _stream(stream)), "srp_refine")
        return xyz, val, vals

    def close(self):
        if self.handle is not None:
            lib().srp_refiner_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srp_gcc_samples_static(M, K, n_aux, Nq, d_y, L, d_xi, stream=None):
    """srp_gcc_samples without a plan or any device allocation (scratch in a
    fixed 8 MiB device array inside the library); Nq is a host int32 [Q]."""
    fn = lib().srp_gcc_samples_static
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    nq = np.ascontiguousarray(Nq, np.int32).reshape(-1)
    if nq.size != int(M) * (int(M) - 1) // 2:
        raise ValueError(f"Nq must hold M(M-1)/2 = {int(M) * (int(M) - 1) // 2} lag counts, "
                         f"got {nq.size}")
    _check(fn(int(M), int(K), int(n_aux), nq.ctypes.data, _ptr(d_y), int(L), _ptr(d_xi),
              _stream(stream)), "srp_gcc_samples_static")


# --------------------------------------------------------------------------
# batched uneven instances
# --------------------------------------------------------------------------
BATCH_STAGES = ("operands", "map", "argmax")


def _ptr_array(items):
    """ctypes array of device addresses (NULL for None)."""
    arr = (ctypes.c_void_p * len(items))()
    for k, t in enumerate(items):
        arr[k] = _ptr(t)
    return arr


def srp_batch_create(handles, tiles=None):
    """Batch over plan handles; tiles = (frames_per_tile, stages, ctas_per_sm
    [, operand_a: 1 TMEM, 2 shared memory [, accumulators: 1 or 2]]), zeros for
    defaults, or None."""
    hs = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                            for h in handles])
    t = None
    if tiles is not None:
        t = srp_batch_tiles(*[int(v) for v in tiles] + [0] * (5 - len(tiles)))
    b = ctypes.c_void_p()
    _check(lib().srp_batch_create(hs, len(handles), ctypes.byref(t) if t is not None else None,
                                  ctypes.byref(b)), "srp_batch_create")
    return b


def _batch_args(d_in, L, d_maps, d_argmax, d_peak):
    n = len(L)
    Ls = (ctypes.c_int32 * n)(*[int(v) for v in L])
    return (_ptr_array(d_in), Ls, None if d_maps is None else _ptr_array(d_maps),
            _ptr_array(d_argmax), None if d_peak is None else _ptr_array(d_peak))


def srp_map_batch(b, d_in, L, d_maps, d_argmax, d_peak=None, stream=None):
    a = _batch_args(d_in, L, d_maps, d_argmax, d_peak)
    _check(lib().srp_map_batch(b, *a, _stream(stream)), "srp_map_batch")


def srp_batch_tune(b, d_in, L, d_maps, d_argmax, d_peak=None, stream=None):
    a = _batch_args(d_in, L, d_maps, d_argmax, d_peak)
    _check(lib().srp_batch_tune(b, *a, _stream(stream)), "srp_batch_tune")


def srp_batch_get_info(b):
    info = srp_batch_info()
    _check(lib().srp_batch_get_info(b, ctypes.byref(info)), "srp_batch_get_info")
    return info


def srp_batch_set_timing(b, enable=True):
    _check(lib().srp_batch_set_timing(b, 1 if enable else 0), "srp_batch_set_timing")


def srp_batch_stage_times(b):
    ms = (ctypes.c_float * len(BATCH_STAGES))()
    _check(lib().srp_batch_stage_times(b, ctypes.addressof(ms), len(BATCH_STAGES)),
           "srp_batch_stage_times")
    return dict(zip(BATCH_STAGES, list(ms)))


def srp_batch_poll_device_status(b, stream=None):
    _check(lib().srp_batch_poll_device_status(b, _stream(stream)), "srp_batch_poll_device_status")


def srp_batch_destroy(b):
    _check(lib().srp_batch_destroy(b), "srp_batch_destroy")


class Batch:
    """Owns one batch over Plan objects (kept alive with it); allocates
    outputs with torch for convenience."""

    def __init__(self, plans, tiles=None):
        self.plans = list(plans)
        self.handle = srp_batch_create([p.handle for p in self.plans], tiles)

    @property
    def info(self):
        return srp_batch_get_info(self.handle)

    def outputs(self, L, device, maps=True):
        """Fresh per-plan (maps, argmax, peak) tensors for frame counts L."""
        import torch
        outs = []
        for p, l in zip(self.plans, L):
            outs.append((torch.empty((l, p.info.J), dtype=torch.float32, device=device)
                         if maps else None,
                         torch.empty(max(l, 1), dtype=torch.int32, device=device),
                         torch.empty(max(l, 1), dtype=torch.float32, device=device)))
        return outs

    def map(self, d_in, L=None, outs=None, maps=True, stream=None, tune=False):
        """Map every plan: d_in list of complex64 CUDA tensors (None where
        L[i] = 0); returns the list of (maps or None, argmax, peak)."""
        L = [x.shape[0] if x is not None else 0 for x in d_in] if L is None else list(L)
        dev = next(x.device for x in d_in if x is not None)
        outs = self.outputs(L, dev, maps) if outs is None else outs
        fn = srp_batch_tune if tune else srp_map_batch
        fn(self.handle, d_in, L, [o[0] for o in outs] if maps else None,
           [o[1] for o in outs], [o[2] for o in outs], stream)
        return outs

    def close(self):
        if self.handle is not None:
            srp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

class Server:
    """Continuous-batching server over Plan objects (stream i maps with
    plans[i]).  submit() copies the input frames at once; results land in
    numpy arrays owned by this object and are returned by poll()."""

    def __init__(self, plans, device_budget_bytes, host_budget_bytes=256 << 20, max_inflight=2,
                 batching=True):
        self.plans = list(plans)
        d = srp_server_desc(int(device_budget_bytes), int(host_budget_bytes), int(max_inflight),
                            0 if batching else 1)
        hs = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().srp_server_create(hs, len(self.plans), ctypes.byref(d), ctypes.byref(h)),
               "srp_server_create")
        self.handle = h
        self._pending = {}  # request id -> (argmax, peak, maps) buffers
        self._buf = (srp_completion * 256)()

    def submit(self, stream, frames, tag=0, want_maps=False, deadline_ms=0.0):
        """Queue frames (complex64 [L][M][Kb] numpy array); returns the request id."""
        x = np.ascontiguousarray(frames, np.complex64)
        L = x.shape[0]
        am = np.empty(L, np.int32)
        pk = np.empty(L, np.float32)
        mp = np.empty((L, self.plans[stream].info.J), np.float32) if want_maps else None
        rid = ctypes.c_uint64()
        _check(lib().srp_server_submit(self.handle, int(stream), x.ctypes.data, L, am.ctypes.data,
                                       pk.ctypes.data, None if mp is None else mp.ctypes.data,
                                       int(tag), float(deadline_ms), ctypes.byref(rid)),
               "srp_server_submit")
        self._pending[rid.value] = (am, pk, mp)
        return rid.value

    def poll(self, wait_ms=0):
        """Finished requests as dicts (id, tag, stream, L, status, times and
        the result arrays)."""
        n = ctypes.c_int32()
        _check(lib().srp_server_poll(self.handle, self._buf, len(self._buf), ctypes.byref(n),
                                     int(wait_ms)), "srp_server_poll")
        out = []
        for c in self._buf[: n.value]:
            am, pk, mp = self._pending.pop(c.request_id)
            out.append(dict(id=c.request_id, tag=c.tag, stream=c.stream, L=c.L, status=c.status,
                            t_submit=c.t_submit_ms, t_start=c.t_start_ms, t_done=c.t_done_ms,
                            iteration=c.iteration, iteration_streams=c.iteration_streams,
                            iteration_frames=c.iteration_frames,
                            t_gpu_start=c.t_gpu_start_ms, t_gpu_end=c.t_gpu_end_ms,
                            argmax=am, peak=pk, maps=mp))
        return out

    def hold(self, on=True):
        """Queue submissions without starting iterations (on) or resume (off)."""
        _check(lib().srp_server_hold(self.handle, 1 if on else 0), "srp_server_hold")

    def drain(self, timeout_s=60.0):
        """Poll until every submitted request has finished."""
        import time
        out = []
        t_end = time.monotonic() + timeout_s
        while self._pending and time.monotonic() < t_end:
            out += self.poll(wait_ms=50)
        if self._pending:
            raise TimeoutError(f"{len(self._pending)} requests still pending")
        return out

    @property
    def stats(self):
        st = srp_server_stats()
        _check(lib().srp_server_get_stats(self.handle, ctypes.byref(st)), "srp_server_get_stats")
        return st

    def close(self):
        if self.handle is not None:
            srp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srp_server_destroy(h):
    _check(lib().srp_server_destroy(h), "srp_server_destroy")
