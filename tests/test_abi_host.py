"""The C ABI without a GPU: the library loads, exports every declared entry
point, and its host-only planner (validation, pair table, lag counts, sizes)
agrees with the oracle and the paper's worked example."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle import oracle
from paper_2012_09499_gb300 import build_lib, srp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib.build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^SRP_API\s+[\w\s\*]+?\b(srp_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(srp.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    L = srp.lib()
    assert L.srp_status_string(0) == b"ok"
    assert L.srp_status_string(5) == b"timeout"
    assert L.srp_destroy(None) == 0


def _desc(**kw):
    rng = np.random.default_rng(kw.pop("seed", 0))
    mic = kw.pop("mic", rng.uniform(-0.25, 0.25, (kw.pop("M", 6), 3)))
    grid = kw.pop("grid", rng.uniform(-2, 2, (kw.pop("J", 100), 3)))
    base = dict(fs=16000.0, c=343.0, K=512)
    base.update({k: kw.pop(k) for k in list(kw) if k in base})
    return srp.make_desc(mic, grid, base["fs"], base["c"], base["K"], **kw)


@pytest.mark.parametrize("seed", range(5))
def test_describe_matches_oracle_lag_counts(seed):
    rng = np.random.default_rng(100 + seed)
    M = int(rng.integers(2, 17))
    mic = rng.uniform(-0.5, 0.5, (M, 3))
    n_aux = int(rng.integers(0, 4))
    d, keep = srp.make_desc(mic, np.zeros((3, 3)), 16000.0, 343.0, 1024, n_aux=n_aux)
    info, nq = srp.srp_plan_describe(d)
    ref, _ = oracle.lag_counts(mic, 16000.0, 343.0)
    assert nq.tolist() == ref.tolist()
    assert info.Q == M * (M - 1) // 2
    assert info.S == int(np.sum(2 * ref + 2 * n_aux + 1))
    assert info.max_nq == int(ref.max())


def test_describe_paper_example():
    """Sec. 4 array: N_q in {4 (x6), 8 (x6), 9 (x3)}, so S = 2*99 + 15(2 N_aux + 1)."""
    mic = synth.circular_array(6, 0.1)
    dirs = synth.half_sphere_directions(2.0)
    for n_aux in range(4):
        d, keep = srp.make_desc(mic, dirs, 16000.0, 340.0, 2048, n_aux=n_aux, far_field=True)
        info, nq = srp.srp_plan_describe(d)
        assert sorted(nq.tolist()) == [4] * 6 + [8] * 6 + [9] * 3
        assert info.S == 198 + 15 * (2 * n_aux + 1)
        assert info.J == 8101


@pytest.mark.parametrize("seed", range(4))
def test_complexity_matches_oracle(seed):
    """srp_plan_complexity (host only) gives the oracle's Sec. 3.3 counts, in
    both modes, for random arrays and for the paper's circle."""
    rng = np.random.default_rng(300 + seed)
    M = int(rng.integers(2, 17))
    cases = [(rng.uniform(-0.4, 0.4, (M, 3)), int(rng.integers(1, 5000)), 2 * int(rng.integers(8, 2049)),
              int(rng.integers(0, 5)), mode) for mode in ("nyquist", "conventional")]
    cases.append((synth.circular_array(6, 0.05 * (seed + 1)), 8101, 2048, seed % 3, "nyquist"))
    for mic, J, K, naux, mode in cases:
        grid = rng.uniform(-2, 2, (J, 3))
        d, keep = srp.make_desc(mic, grid, 16000.0, 343.0, K, mode=mode, n_aux=naux)
        got = srp.srp_plan_complexity(d)
        ref = oracle.complexity(mic, 16000.0, 343.0, K // 2, J, naux)
        assert (got["P"], got["K_b"], got["J"]) == (ref["P"], ref["K_b"], ref["J"])
        for k in ("N", "C_samp", "C_int", "C_conv", "R_samp", "R_int", "R"):
            assert got[k] == pytest.approx(ref[k], rel=1e-14, abs=0), k
    with pytest.raises(srp.SrpError):
        d, keep = _desc(K=7)
        srp.srp_plan_complexity(d)


def test_exact_integer_lag_bound():
    mic = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    d, keep = srp.make_desc(mic, np.zeros((1, 3)), 8192.0, 256.0, 64)
    _, nq = srp.srp_plan_describe(d)
    assert nq.tolist() == [16]


def test_footprint_counts_every_buffer():
    d, keep = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2)
    info, nq = srp.srp_plan_describe(d)
    fp = srp.srp_plan_footprint(d)
    assert fp == info.device_bytes
    Q, Jp, Lp = 28, 1024, 64
    Sc = int(np.sum(-(-(2 * nq + 5) // 64) * 64))  # each pair padded to 64-lag chunks
    # status, pairs, N_q, pair offsets, cross spectra, argmax partials
    common = 4 + 8 * Q + 4 * Q + 4 * Q + 8 * 64 * Q * 513 + 8 * Lp * (Jp // 128)
    x_tab = 4 * Q * Jp  # int32 TDOA table of the CUDA-core kernels
    # tensor-core engine: twiddles, 8-aligned pair offsets, split 16-bit GCC samples
    tc_tables = 4 * Q + 8 * Q * Jp + 16 * (Sc // 64)  # pair offsets, (TDOA, sp), chunk table
    # the tensor-core IDFT's twiddle operand: (hi, lo) x N lag columns x K slots,
    # N = 2 (max N_q + N_aux) + 1 rounded up to 32
    Ng = -(-(2 * (int(nq.max()) + 2) + 1) // 32) * 32
    tc_tables += 2 * 2 * Ng * 1024
    assert fp == common + 8 * 1024 + tc_tables + 2 * 2 * Lp * Sc
    d3, keep3 = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2, engine="cuda_cores")
    Sp = -(-info.S // 64) * 64
    assert srp.srp_plan_footprint(d3) == common + x_tab + 8 * 1024 + 4 * Sp * Lp
    d4, keep4 = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2, precision="bf16",
                      argmax="map")
    assert srp.srp_plan_footprint(d4) == common + 8 * 1024 + tc_tables + 2 * Lp * Sc
    # re-scoring the maximiser in FP32 keeps the FP32 GCC samples too
    d6, keep6 = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2, precision="bf16")
    assert srp.srp_plan_describe(d6)[0].argmax_rescored == 1
    rescore = 4 * Lp * Sp + (17 * 8 + 4) * Lp  # FP32 samples, frame keys, slots, counters
    assert srp.srp_plan_footprint(d6) == common + 8 * 1024 + tc_tables + 2 * Lp * Sc + rescore
    d2, keep2 = _desc(M=8, J=1000, K=1024, max_frames=64, mode="conventional",
                      engine="cuda_cores")
    assert srp.srp_plan_footprint(d2) == common + x_tab
    # conventional on the tensor cores: 2 Kb = 1026 slots per pair, padded to 1088
    Scc = Q * 1088
    d5, keep5 = _desc(M=8, J=1000, K=1024, max_frames=64, mode="conventional")
    assert srp.srp_plan_footprint(d5) == (common + 4 * Q + 8 * Q * Jp + 16 * (Scc // 64)
                                          + 2 * 2 * Lp * Scc)


@pytest.mark.parametrize("field,value", [
    ("M", 1), ("M", 65), ("K", 7), ("K", 2), ("K", 16384), ("J", 0), ("fs", 0.0),
    ("c", -1.0), ("n_aux", -1), ("max_frames", 0), ("mode", 3), ("precision", 7),
    ("input_kind", 5), ("grid_kind", 4), ("engine", 2), ("host_io", 3), ("host_io", -1),
    ("weighting", 2), ("argmax", 2), ("argmax", -1),
])
def test_invalid_descriptors_rejected(field, value):
    d, keep = _desc()
    setattr(d, field, value)
    with pytest.raises(srp.SrpError) as e:
        srp.srp_plan_describe(d)
    assert e.value.status == srp.SRP_ERR_INVALID_ARG


@pytest.mark.parametrize("kw", [dict(mode="conventional", precision="bf16", engine="cuda_cores"),
                                dict(engine="cuda_cores", precision="fp16"),
                                dict(precision="fp16", weighting="none")])
def test_half_precision_needs_tensor_cores(kw):
    d, keep = _desc(**kw)
    with pytest.raises(srp.SrpError) as e:
        srp.srp_plan_describe(d)
    assert e.value.status == srp.SRP_ERR_UNSUPPORTED


def test_nonfinite_geometry_rejected():
    mic = np.zeros((3, 3))
    mic[1, 0] = np.nan
    d, keep = srp.make_desc(mic, np.zeros((4, 3)), 16000.0, 343.0, 64)
    with pytest.raises(srp.SrpError) as e:
        srp.srp_plan_describe(d)
    assert e.value.status == srp.SRP_ERR_INVALID_ARG


def test_null_handle_rejected():
    with pytest.raises(srp.SrpError) as e:
        srp.srp_map(None, 1, 1, None, 1, stream=0)
    assert e.value.status == srp.SRP_ERR_INVALID_ARG


def test_engine_choice_by_accumulation_bias():
    """FP32 conventional plans with a long reduction stay on the tensor cores
    and promote their accumulators every 128 chunks (with up to 64 frames per
    call; more frames take the CUDA cores); the benchmark's 3D workload and
    every Nyquist plan use the tensor cores without promotion."""
    rng = np.random.default_rng(5)
    mic8 = rng.uniform(-0.25, 0.25, (8, 3))
    mic16 = rng.uniform(-0.5, 0.5, (16, 3))
    grid = rng.uniform(0, 5, (100, 3))
    cases = [(mic8, 1024, "conventional", "fp32", 1, 0), (mic16, 2048, "conventional", "fp32", 1, 128),
             (mic16, 2048, "conventional", "bf16", 1, 0), (mic16, 2048, "nyquist", "fp32", 1, 0),
             (mic8, 1024, "nyquist", "fp32", 1, 0)]
    for mic, K, mode, prec, tc, promo in cases:
        d, keep = srp.make_desc(mic, grid, 16000.0, 343.0, K, mode=mode, precision=prec)
        info, _ = srp.srp_plan_describe(d)
        assert info.tensor_cores == tc, (mic.shape[0], K, mode, prec)
        assert info.accum_promotion == promo, (mic.shape[0], K, mode, prec)
    d, keep = srp.make_desc(mic16, grid, 16000.0, 343.0, 2048, mode="conventional",
                            max_frames=65)
    info, _ = srp.srp_plan_describe(d)
    assert info.tensor_cores == 0 and info.accum_promotion == 0
    d, keep = srp.make_desc(mic8, grid, 16000.0, 343.0, 1024, engine="cuda_cores")
    assert srp.srp_plan_describe(d)[0].tensor_cores == 0


def test_batch_entry_points_reject_bad_arguments():
    """Argument checks of the batch entry points run before any CUDA call."""
    L = srp.lib()
    out = ctypes.c_void_p()
    assert L.srp_batch_create(None, 0, None, ctypes.byref(out)) == srp.SRP_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.srp_batch_create(arr, 2, None, ctypes.byref(out)) == srp.SRP_ERR_INVALID_ARG
    assert L.srp_batch_create(arr, 1, None, None) == srp.SRP_ERR_INVALID_ARG
    assert L.srp_map_batch(None, None, None, None, None, None, None) == srp.SRP_ERR_INVALID_ARG
    info = srp.srp_batch_info()
    assert L.srp_batch_get_info(None, ctypes.byref(info)) == srp.SRP_ERR_INVALID_ARG
    assert L.srp_batch_destroy(None) == srp.SRP_OK


def test_server_entry_points_reject_bad_arguments():
    """Argument checks of the serving entry points run before any CUDA call."""
    L = srp.lib()
    out = ctypes.c_void_p()
    d = srp.srp_server_desc(1 << 20, 1 << 20, 2, 0)
    assert L.srp_server_create(None, 0, ctypes.byref(d), ctypes.byref(out)) == \
        srp.SRP_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert L.srp_server_create(arr, 1, ctypes.byref(d), ctypes.byref(out)) == \
        srp.SRP_ERR_INVALID_ARG
    bad = srp.srp_server_desc(0, 1 << 20, 2, 0)
    assert L.srp_server_create(arr, 1, ctypes.byref(bad), ctypes.byref(out)) == \
        srp.SRP_ERR_INVALID_ARG
    bad = srp.srp_server_desc(1 << 20, 1 << 20, 9, 0)
    assert L.srp_server_create(arr, 1, ctypes.byref(bad), ctypes.byref(out)) == \
        srp.SRP_ERR_INVALID_ARG
    n = ctypes.c_int32()
    assert L.srp_server_poll(None, None, 0, ctypes.byref(n), 0) == srp.SRP_ERR_INVALID_ARG
    assert L.srp_server_submit(None, 0, None, 1, None, None, None, 0, 0.0, None) == \
        srp.SRP_ERR_INVALID_ARG
    assert L.srp_server_destroy(None) == srp.SRP_OK


def test_footprint_counts_host_staging_slots():
    """host_io slots of staging: input, maps, argmax and peak per slot, each
    rounded up to 256 bytes."""
    up = lambda v: -(-v // 256) * 256
    d0, k0 = _desc(M=6, J=1000, K=512, max_frames=20)
    base = srp.srp_plan_footprint(d0)
    for slots in (1, 2):
        d, k = _desc(M=6, J=1000, K=512, max_frames=20, host_io=slots)
        stage = up(8 * 20 * 6 * 257) + up(4 * 20 * 1000) + 2 * up(4 * 32)
        assert srp.srp_plan_footprint(d) == base + slots * stage


def test_resident_weights_footprint_and_limits():
    """A resident interpolation matrix adds J_pad x (16-slot steps holding
    lags) x 2 bytes (twice for FP32) and a chunk-offset table; it exists for
    Nyquist tensor-core plans only."""
    for prec, hs in (("fp32", 2), ("bf16", 1)):
        d0, k0 = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2, precision=prec)
        info, nq = srp.srp_plan_describe(d0)
        d1, k1 = _desc(M=8, J=1000, K=1024, max_frames=64, n_aux=2, precision=prec,
                       resident_weights=True)
        info1, _ = srp.srp_plan_describe(d1)
        spans = 2 * nq + 5
        steps = int(np.sum(-(-spans // 16)))
        chunks = int(np.sum(-(-spans // 64)))
        w = (1024 // 128) * steps * hs * 4096
        assert info1.weight_bytes == w and info.weight_bytes == 0
        assert srp.srp_plan_footprint(d1) == srp.srp_plan_footprint(d0) + w + 4 * chunks
    for kw in (dict(mode="conventional"), dict(engine="cuda_cores")):
        d, k = _desc(resident_weights=True, **kw)
        with pytest.raises(srp.SrpError) as e:
            srp.srp_plan_describe(d)
        assert e.value.status == srp.SRP_ERR_UNSUPPORTED


def test_partial_resident_fraction():
    """A resident fraction keeps whole pairs' weights, about that fraction of
    the 16-slot steps; out-of-range fractions are refused."""
    d1, k1 = _desc(M=8, J=1000, K=1024, n_aux=2, precision="bf16", resident_fraction=1.0)
    dh, kh = _desc(M=8, J=1000, K=1024, n_aux=2, precision="bf16", resident_fraction=0.5)
    full = srp.srp_plan_describe(d1)[0].weight_bytes
    half = srp.srp_plan_describe(dh)[0].weight_bytes
    assert 0.3 * full < half < 0.7 * full
    for bad in (-0.1, 1.5, float("nan")):
        d, k = _desc(resident_fraction=bad)
        with pytest.raises(srp.SrpError) as e:
            srp.srp_plan_describe(d)
        assert e.value.status == srp.SRP_ERR_INVALID_ARG


def test_static_gcc_samples_checks_before_any_cuda_call():
    """srp_gcc_samples_static validates its arguments on the host: a lag
    table of the wrong length is refused by the binding, and sizes beyond its
    limits by the library, before anything touches a device."""
    with pytest.raises(ValueError):
        srp.srp_gcc_samples_static(4, 64, 0, np.zeros(5, np.int32), None, 1, None)
    L = srp.lib()
    nq = np.zeros(6, np.int32)
    for M, K, n_aux, frames in [(17, 64, 0, 1), (4, 63, 0, 1), (4, 64, -1, 1), (4, 64, 0, -1),
                                (4, 64, 0, 65536), (4, 8192, 0, 200)]:
        args = (M, K, n_aux, nq.ctypes.data if M == 4 else np.zeros(136, np.int32).ctypes.data,
                None, frames, None, None)
        assert L.srp_gcc_samples_static(*args) == srp.SRP_ERR_INVALID_ARG, (M, K, frames)


def test_gcc_engine_choice():
    """The critical GCC samples run as the tensor cores' partial inverse DFT
    for Nyquist tensor-core plans with PHAT-weighted STFT input, K a multiple
    of 64 and at most 128 lag columns (2 (max N_q + N_aux) + 1); every other
    plan forms them on the CUDA cores."""
    rng = np.random.default_rng(7)
    mic = rng.uniform(-0.25, 0.25, (8, 3))
    grid = rng.uniform(0, 5, (100, 3))

    def engine(mic_=mic, K=1024, **kw):
        d, keep = srp.make_desc(mic_, grid, 16000.0, 343.0, K, **kw)
        return srp.srp_plan_describe(d)[0].gcc_tensor_cores

    assert engine() == 1
    assert engine(precision="bf16") == 1 and engine(precision="fp16") == 1
    assert engine(K=2048) == 1 and engine(K=64 * 15) == 1
    assert engine(weighting="none") == 0
    assert engine(input_kind="cross") == 0
    assert engine(mode="conventional") == 0
    assert engine(engine="cuda_cores") == 0
    assert engine(K=1000) == 0  # not a multiple of 64
    # lag columns 2 (max N_q + N_aux) + 1 against the limit of 128: apertures
    # of 0.9 m (87 columns), 1.5 m (143) and 5 m at 16 kHz
    for width, tc in ((0.9, 1), (1.5, 0), (5.0, 0)):
        wide = np.array([[0.0, 0.0, 0.0], [width, 0.0, 0.0], [0.0, 0.3, 0.0]])
        info, nq = srp.srp_plan_describe(srp.make_desc(wide, grid, 16000.0, 343.0, 1024)[0])
        assert (2 * (int(nq.max()) + 2) + 1 <= 128) == bool(tc)
        assert info.gcc_tensor_cores == tc, width
