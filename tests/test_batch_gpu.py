"""Batched uneven instances through the C ABI: srp_map_batch over plans with
different M, J, K and grids must give, for every plan, the map srp_map
defines, within the same tolerances against the FP64 oracle (FP32 path:
1e-4 x peak, argmax exact except documented ties; BF16/FP16: 1e-2 x peak).
Frame counts vary per plan and per call, including plans skipped (L = 0)."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2012_09499_gb300 import build_lib, srp, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "bf16": 1e-2, "fp16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_mix(seed, n, J_range, L, **fix):
    return [synth.uneven_instance(seed * 1000 + i, J_range, L, **fix) for i in range(n)]


def make_plans(cfgs, mode, precision, max_frames):
    return [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], mode=mode, n_aux=2,
                     precision=precision, max_frames=max_frames) for c in cfgs]


def oracle_maps(cfg, mode, L, sub=None):
    grid = cfg["grid"] if sub is None else cfg["grid"][sub]
    maps, _, _ = oracle.srp_map(cfg["Y"][:L], cfg["mic"], grid, cfg["fs"], cfg["c"], cfg["K"],
                                mode=mode, n_aux=2)
    return maps


def check(maps, idx, peak, ref, tol, exact_argmax=True, rescored=False):
    pk = np.abs(ref).max(axis=1)
    err = np.abs(maps.astype(np.float64) - ref).max(axis=1)
    assert np.all(err <= tol * pk), (err / pk).max()
    if rescored:
        # BF16 / FP16 Nyquist plans choose the maximiser in FP32: the oracle's
        # first maximiser except on FP32 ties, the peak its FP32 value
        rows = np.arange(ref.shape[0])
        assert np.all(np.abs(peak.astype(np.float64) - ref[rows, idx]) <= TOL["fp32"] * pk)
        ridx = np.argmax(ref, axis=1)
        for l in np.nonzero(idx != ridx)[0]:
            assert ref[l, ridx[l]] - ref[l, idx[l]] < TOL["fp32"] * pk[l]
        return (err / pk).max()
    assert np.array_equal(idx, np.argmax(maps, axis=1))  # first maximiser of its own map
    assert np.array_equal(peak, maps[np.arange(maps.shape[0]), idx])
    if exact_argmax:
        ridx = np.argmax(ref, axis=1)
        for l in np.nonzero(idx != ridx)[0]:  # documented ties only
            assert ref[l, ridx[l]] - ref[l, idx[l]] < tol * pk[l]
    return (err / pk).max()


def run_batch(batch, cfgs, L, tune=False):
    d_in = [dev(c["Y"][:l]) if l > 0 else None for c, l in zip(cfgs, L)]
    outs = batch.map(d_in, L=L, tune=tune)
    torch.cuda.synchronize()
    srp.srp_batch_poll_device_status(batch.handle)
    return [(m.cpu().numpy(), a.cpu().numpy()[:l], p.cpu().numpy()[:l])
            for (m, a, p), l in zip(outs, L)]


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_nyquist_batch_matches_oracle(precision):
    cfgs = small_mix(1, 5, (800, 4000), 32)
    plans = make_plans(cfgs, "nyquist", precision, 32)
    batch = srp.Batch(plans)
    L = [32, 17, 0, 5, 32]
    res = run_batch(batch, cfgs, L)
    for c, (m, a, p), l in zip(cfgs, res, L):
        if l == 0:
            continue
        check(m, a, p, oracle_maps(c, "nyquist", l), TOL[precision],
              exact_argmax=precision == "fp32", rescored=precision != "fp32")
    batch.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_rescored_batch_argmax_equals_per_plan_map(precision):
    """A batch of BF16 / FP16 Nyquist plans re-scores each frame's maximiser
    in FP32 as srp_map does for those plans: every plan's argmax equals its
    own srp_map call's (or both are FP32 near-ties) and the peaks agree to
    1e-6 (the batch's operand kernel forms the same FP32 samples, up to
    rounding), on a full and on a partial call."""
    cfgs = small_mix(9, 4, (2000, 9000), 16)
    plans = make_plans(cfgs, "nyquist", precision, 16)
    assert all(p.info.argmax_rescored == 1 for p in plans)
    batch = srp.Batch(plans)
    for L in ([16, 16, 16, 16], [16, 0, 9, 3]):
        res = run_batch(batch, cfgs, L)
        for c, pl, (m, a, p), l in zip(cfgs, plans, res, L):
            if l == 0:
                continue
            m1, a1, p1 = pl.map(dev(c["Y"][:l]), L=l)
            torch.cuda.synchronize()
            a1, p1 = a1.cpu().numpy()[:l], p1.cpu().numpy()[:l]
            assert np.all(np.abs(p - p1) <= 1e-6 * np.abs(p1))
            assert np.mean(a == a1) >= 0.9  # any other frame is an FP32 near-tie (peaks above)
    # without maps the whole selected tiles are scored: the same maximisers
    L = [16, 16, 16, 16]
    full = run_batch(batch, cfgs, L)
    d_in = [dev(c["Y"][:l]) for c, l in zip(cfgs, L)]
    bare = batch.map(d_in, L=L, maps=False)
    torch.cuda.synchronize()
    for (m, a, p), (m2, a2, p2) in zip(full, bare):
        assert m2 is None
        assert np.array_equal(a, a2.cpu().numpy()) and np.array_equal(p, p2.cpu().numpy())
    batch.close()
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_conventional_batch_matches_oracle(precision):
    # few pairs and bins, so that the FP32 plans run on the tensor cores
    cfgs = [synth.uneven_instance(50 + i, (600, 1500), 6, M=M, K=K)
            for i, (M, K) in enumerate([(4, 512), (6, 1024), (5, 2048), (4, 1024)])]
    plans = make_plans(cfgs, "conventional", precision, 8)
    assert all(p.info.tensor_cores == 1 for p in plans)
    batch = srp.Batch(plans)
    L = [6, 3, 6, 1]
    res = run_batch(batch, cfgs, L)
    for c, (m, a, p), l in zip(cfgs, res, L):
        check(m, a, p, oracle_maps(c, "conventional", l), TOL[precision],
              exact_argmax=precision == "fp32")
    batch.close()


def test_batch_equals_per_plan_map():
    cfgs = small_mix(2, 4, (2000, 9000), 16)
    plans = make_plans(cfgs, "nyquist", "fp32", 16)
    batch = srp.Batch(plans)
    L = [16, 9, 16, 3]
    res = run_batch(batch, cfgs, L)
    for c, pl, (m, a, p), l in zip(cfgs, plans, res, L):
        m1, a1, p1 = pl.map(dev(c["Y"][:l]), L=l)
        torch.cuda.synchronize()
        m1 = m1.cpu().numpy()
        pk = np.abs(m1).max(axis=1)
        assert np.all(np.abs(m - m1).max(axis=1) <= 1e-6 * pk)
    batch.close()


def test_batch_repeated_calls_and_varying_frames():
    cfgs = small_mix(3, 3, (1000, 3000), 24)
    plans = make_plans(cfgs, "nyquist", "bf16", 24)
    batch = srp.Batch(plans)
    first = run_batch(batch, cfgs, [24, 24, 24])
    again = run_batch(batch, cfgs, [24, 24, 24])
    for (m0, a0, p0), (m1, a1, p1) in zip(first, again):
        assert np.array_equal(m0, m1) and np.array_equal(a0, a1)
    # fewer frames, one plan skipped: the leading frames are unchanged
    part = run_batch(batch, cfgs, [7, 0, 13])
    for (m0, a0, _), (m1, a1, _), l in zip(first, part, [7, 0, 13]):
        assert np.array_equal(m0[:l], m1) and np.array_equal(a0[:l], a1)
    batch.close()


def test_batch_tuner_and_explicit_tiles():
    cfgs = small_mix(4, 4, (3000, 12000), 32)
    plans = make_plans(cfgs, "nyquist", "fp32", 32)
    batch = srp.Batch(plans)
    L = [32, 32, 20, 32]
    res = run_batch(batch, cfgs, L, tune=True)
    info = batch.info
    assert info.tuned == 1 and info.tuned_ms > 0.0 and info.launches == 3
    assert info.tiles.frames_per_tile in (16, 32)
    refs = [oracle_maps(c, "nyquist", l) for c, l in zip(cfgs, L)]
    for (m, a, p), ref in zip(res, refs):
        check(m, a, p, ref, TOL["fp32"])
    # the chosen tiles keep serving ordinary calls
    for (m, a, p), ref in zip(run_batch(batch, cfgs, L), refs):
        check(m, a, p, ref, TOL["fp32"])
    batch.close()
    # a fixed tile shape: 16 frames per item, two stages, one CTA per SM, with
    # operand A in tensor memory (1) and in shared memory (2): same results
    outs = {}
    for where in (1, 2):
        b2 = srp.Batch(plans, tiles=(16, 2, 1, where))
        assert (b2.info.tiles.frames_per_tile, b2.info.tiles.stages,
                b2.info.tiles.ctas_per_sm, b2.info.tiles.operand_a) == (16, 2, 1, where)
        outs[where] = run_batch(b2, cfgs, L)
        for (m, a, p), ref in zip(outs[where], refs):
            check(m, a, p, ref, TOL["fp32"])
        b2.close()
    for (m1, a1, _), (m2, a2, _) in zip(outs[1], outs[2]):
        assert np.array_equal(m1, m2) and np.array_equal(a1, a2)


def test_one_and_two_accumulators_agree():
    """The 16-slot steps summed by one MMA warp into one accumulator, or by two
    warps into two that the epilogue adds, give the same maps up to the order
    of the FP32 sums; with 64 frames per item and A in tensor memory only the
    single accumulator lets two CTAs share an SM, and the default picks it."""
    cfgs = small_mix(6, 3, (3000, 9000), 64)
    L = [64, 40, 64]
    for precision in ("fp32", "bf16"):
        plans = make_plans(cfgs, "nyquist", precision, 64)
        refs = [oracle_maps(c, "nyquist", l) for c, l in zip(cfgs, L)]
        outs = {}
        for mw in (1, 2):
            b = srp.Batch(plans, tiles=(32, 2, 2, 1, mw))
            assert (b.info.tiles.operand_a, b.info.tiles.accumulators) == (1, mw)
            outs[mw] = run_batch(b, cfgs, L)
            for (m, a, p), ref in zip(outs[mw], refs):
                check(m, a, p, ref, TOL[precision], exact_argmax=precision == "fp32",
                      rescored=precision != "fp32")
            b.close()
        # the FP32 accumulation bias of tcgen05 (about 1.5e-8 relative per MMA
        # into one accumulator) grows with the steps one accumulator sums
        steps = max(p.info.S // 16 + p.info.Q for p in plans)  # 16-lag steps, padded per pair
        bound = 4 * 3 * steps * 1.5e-8 if precision == "fp32" else 1e-2
        for (m1, _, _), (m2, _, _) in zip(outs[1], outs[2]):
            pk = np.abs(m2).max(axis=1, keepdims=True)
            assert np.all(np.abs(m1 - m2) <= bound * pk), (np.abs(m1 - m2) / pk).max()
        b = srp.Batch(plans, tiles=(64, 0, 2, 1))
        t = b.info.tiles
        assert (t.ctas_per_sm, t.accumulators) == (2, 1)
        for (m, a, p), ref in zip(run_batch(b, cfgs, L), refs):
            check(m, a, p, ref, TOL[precision], exact_argmax=precision == "fp32",
                  rescored=precision != "fp32")
        b.close()
        for pl in plans:
            pl.close()


def test_batch_full_scale_sampled():
    """Arrays of the uneven mix at full size (J up to 500k, K up to 2048,
    M up to 16): sampled candidates and frames against the oracle."""
    cfgs = synth.uneven_mix(7, 6, L=32)
    plans = make_plans(cfgs, "nyquist", "fp32", 32)
    batch = srp.Batch(plans)
    L = [32] * len(cfgs)
    d_in = [dev(c["Y"]) for c in cfgs]
    outs = batch.map(d_in, L=L)
    torch.cuda.synchronize()
    srp.srp_batch_poll_device_status(batch.handle)
    for c, (m, a, p) in zip(cfgs, outs):
        J = c["grid"].shape[0]
        sub = np.arange(0, J, max(1, J // 1500))
        frames = [0, 31]
        ref = np.stack([oracle_maps({**c, "Y": c["Y"][[f]]}, "nyquist", 1, sub)[0]
                        for f in frames])
        got = m[frames][:, sub].cpu().numpy().astype(np.float64)
        full = m[frames].cpu().numpy()
        pk = np.abs(full).max(axis=1)
        assert np.all(np.abs(got - ref).max(axis=1) <= TOL["fp32"] * pk)
        assert np.array_equal(a[frames].cpu().numpy(), np.argmax(full, axis=1))
    batch.close()


def test_batch_rejects_mixed_modes_and_cuda_core_plans():
    cfgs = small_mix(5, 2, (500, 800), 4)
    a = make_plans(cfgs[:1], "nyquist", "fp32", 4)[0]
    b = make_plans(cfgs[1:], "conventional", "fp32", 4)[0]
    with pytest.raises(srp.SrpError) as e:
        srp.Batch([a, b])
    assert e.value.status == srp.SRP_ERR_UNSUPPORTED
    c = srp.Plan(cfgs[0]["mic"], cfgs[0]["grid"], 16000.0, 343.0, cfgs[0]["K"],
                 engine="cuda_cores", max_frames=4)
    with pytest.raises(srp.SrpError) as e:
        srp.Batch([a, c])
    assert e.value.status == srp.SRP_ERR_UNSUPPORTED
    batch = srp.Batch([a])
    with pytest.raises(srp.SrpError) as e:  # more frames than the plan takes
        srp.srp_map_batch(batch.handle, [None], [5], None, [None])
    assert e.value.status == srp.SRP_ERR_INVALID_ARG
    batch.close()


def test_batch_promoted_conventional_fp32():
    """FP32 conventional plans with long reductions (M = 16: 120 pairs, K =
    2048) promote their accumulators every 128 chunks inside the persistent
    kernel too: a batch of such plans with ordinary ones meets 1e-4 x peak
    against the oracle, equals each plan's own srp_map to 1e-6 x peak, and
    keeps doing so when a call skips the promoted plan or maps fewer frames."""
    long_cfgs = [synth.uneven_instance(77 + i, (500, 900), 4, M=16, K=2048) for i in range(2)]
    short_cfgs = [synth.uneven_instance(90 + i, (600, 1500), 4, M=M, K=K)
                  for i, (M, K) in enumerate([(4, 512), (6, 1024)])]
    cfgs = [long_cfgs[0], short_cfgs[0], long_cfgs[1], short_cfgs[1]]
    plans = make_plans(cfgs, "conventional", "fp32", 4)
    assert [p.info.accum_promotion > 0 for p in plans] == [True, False, True, False]
    assert all(p.info.tensor_cores == 1 for p in plans)
    batch = srp.Batch(plans)
    assert batch.info.tiles.operand_a == 1  # the promoting kernel keeps A in TMEM
    refs = [oracle_maps(c, "conventional", 4) for c in cfgs]
    for L in ([4, 4, 4, 4], [3, 4, 0, 2]):
        res = run_batch(batch, cfgs, L)
        for c, pl, (m, a, p), ref, l in zip(cfgs, plans, res, refs, L):
            if l == 0:
                continue
            check(m, a, p, ref[:l], TOL["fp32"])
            m1, a1, p1 = pl.map(dev(c["Y"][:l]), L=l)
            torch.cuda.synchronize()
            m1 = m1.cpu().numpy()
            pk = np.abs(m1).max(axis=1)
            assert np.all(np.abs(m - m1).max(axis=1) <= 1e-6 * pk)
    batch.close()
    for pl in plans:
        pl.close()


def test_batch_timing_mode_same_outputs():
    cfgs = small_mix(6, 3, (1000, 3000), 16)
    plans = make_plans(cfgs, "nyquist", "fp32", 16)
    batch = srp.Batch(plans)
    L = [16, 8, 16]
    graph = run_batch(batch, cfgs, L)
    with pytest.raises(srp.SrpError):
        srp.srp_batch_stage_times(batch.handle)  # timing is off
    srp.srp_batch_set_timing(batch.handle, True)
    timed = run_batch(batch, cfgs, L)
    st = srp.srp_batch_stage_times(batch.handle)
    assert all(v > 0.0 for v in st.values()), st
    for (m0, a0, _), (m1, a1, _) in zip(graph, timed):
        assert np.array_equal(m0, m1) and np.array_equal(a0, a1)
    batch.close()


def test_batch_mixes_weightings():
    """A batch may hold PHAT and unweighted plans (the weighting is per plan)."""
    cfgs = small_mix(8, 3, (800, 2000), 8)
    plans = [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], n_aux=2, max_frames=8,
                      weighting=w) for c, w in zip(cfgs, ["phat", "none", "none"])]
    batch = srp.Batch(plans)
    res = run_batch(batch, cfgs, [8, 8, 5])
    for c, w, (m, a, p), l in zip(cfgs, ["phat", "none", "none"], res, [8, 8, 5]):
        ref, _, _ = oracle.srp_map(c["Y"][:l], c["mic"], c["grid"], c["fs"], c["c"], c["K"],
                                   mode="nyquist", n_aux=2, weighting=w)
        check(m, a, p, ref, TOL["fp32"])
    batch.close()


def test_batch_far_field_and_cross_spectrum_input():
    """Far-field direction grids and plans fed with ready cross spectra in one
    batch, against the oracle."""
    far = synth.paper_circle_setup(7, L=6, step_deg=6.0)
    near = synth.uneven_instance(900, (900, 1500), 6, M=5, K=512)
    psi = oracle.phat(near["Y"]).astype(np.complex64)
    plans = [srp.Plan(far["mic"], far["grid"], far["fs"], far["c"], far["K"], n_aux=2,
                      far_field=True, max_frames=6),
             srp.Plan(near["mic"], near["grid"], near["fs"], near["c"], near["K"], n_aux=2,
                      input_kind="cross", max_frames=6)]
    batch = srp.Batch(plans)
    d_in = [dev(far["Y"]), dev(psi)]
    outs = batch.map(d_in, L=[6, 4])
    torch.cuda.synchronize()
    srp.srp_batch_poll_device_status(batch.handle)
    ref_far, _, _ = oracle.srp_map(far["Y"], far["mic"], far["grid"], far["fs"], far["c"],
                                   far["K"], mode="nyquist", n_aux=2, far_field=True)
    ref_near, _, _ = oracle.srp_map(None, near["mic"], near["grid"], near["fs"], near["c"],
                                    near["K"], mode="nyquist", n_aux=2, psi=psi[:4])
    for (m, a, p), ref, l in zip(outs, [ref_far, ref_near], [6, 4]):
        check(m.cpu().numpy(), a.cpu().numpy()[:l], p.cpu().numpy()[:l], ref, TOL["fp32"])
    batch.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_with_resident_weights(precision):
    """Plans that stream their precomputed interpolation matrix, batched with
    plans that generate it: the same maps as an all-generating batch."""
    cfgs = small_mix(9, 4, (1500, 5000), 16)
    gen = make_plans(cfgs, "nyquist", precision, 16)
    mixed = [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], n_aux=2,
                      precision=precision, max_frames=16, resident_fraction=[1.0, 0.0, 0.5, 0.3][k])
             for k, c in enumerate(cfgs)]
    L = [16, 11, 16, 3]
    b0, b1 = srp.Batch(gen), srp.Batch(mixed)
    assert b1.info.tiles.operand_a == 2  # streamed A blocks live in shared memory
    r0, r1 = run_batch(b0, cfgs, L), run_batch(b1, cfgs, L)
    for (m0, a0, _), (m1, a1, _) in zip(r0, r1):
        assert np.array_equal(m0, m1) and np.array_equal(a0, a1)
    b0.close()
    b1.close()
