"""The serving engine through the C ABI: frame blocks from many arrays,
mapped by continuous batching with admission by device memory.  Each
request's result must be the same when it runs alone and when it runs in a
mix of other requests, and within tolerance of the FP64 oracle."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2012_09499_gb300 import build_lib, srp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def mix(seed, n, J_range, L, **fix):
    return [synth.uneven_instance(seed * 1000 + i, J_range, L, **fix) for i in range(n)]


def check_fp32_maximiser(idx, peak, ref):
    """BF16 / FP16 plans choose the maximiser in FP32: the oracle's first
    maximiser except on FP32 ties (gap below 1e-4 x peak), the peak its FP32
    value within 1e-4 x peak."""
    pk = np.abs(ref).max(axis=1)
    rows = np.arange(ref.shape[0])
    assert np.all(np.abs(peak.astype(np.float64) - ref[rows, idx]) <= 1e-4 * pk)
    ridx = np.argmax(ref, axis=1)
    for l in np.nonzero(idx != ridx)[0]:
        assert ref[l, ridx[l]] - ref[l, idx[l]] < 1e-4 * pk[l]


def plans_for(cfgs, mode="nyquist", precision="bf16", max_frames=32):
    return [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], mode=mode, n_aux=2,
                     precision=precision, max_frames=max_frames) for c in cfgs]


def oracle_maps(cfg, frames, mode="nyquist"):
    maps, _, _ = oracle.srp_map(frames, cfg["mic"], cfg["grid"], cfg["fs"], cfg["c"], cfg["K"],
                                mode=mode, n_aux=2)
    return maps


def test_result_alone_equals_result_in_the_mix():
    cfgs = mix(11, 6, (1500, 6000), 40)
    plans = plans_for(cfgs, max_frames=32)
    srv = srp.Server(plans, device_budget_bytes=256 << 20, max_inflight=2)
    probe = cfgs[2]["Y"][8:16]
    srv.submit(2, probe, tag=1, want_maps=True)
    alone = srv.drain()
    assert len(alone) == 1 and alone[0]["status"] == srp.SRP_OK
    # the same block again, amid bursts from every stream
    rng = np.random.default_rng(0)
    tags = {}
    for burst in range(6):
        for k in range(10):
            s = int(rng.integers(0, len(cfgs)))
            f0 = int(rng.integers(0, 32)) & ~7
            tags[srv.submit(s, cfgs[s]["Y"][f0:f0 + 8], tag=100 + burst * 10 + k,
                            want_maps=(k % 3 == 0))] = (s, f0)
        if burst == 3:
            srv.submit(2, probe, tag=2, want_maps=True)
        time.sleep(0.002)
    done = srv.drain()
    st = srv.stats
    srv.close()
    assert all(d["status"] == srp.SRP_OK for d in done)
    assert st.completed == 62 and st.iterations >= 2 and st.batched_streams == 6
    again = [d for d in done if d["tag"] == 2][0]
    a0 = alone[0]
    assert np.array_equal(again["maps"], a0["maps"])
    assert np.array_equal(again["argmax"], a0["argmax"])
    assert np.array_equal(again["peak"], a0["peak"])
    # every map that came back is within the BF16 tolerance of the oracle, and
    # the maximiser, chosen in FP32, is the oracle's (up to FP32 ties)
    ref = oracle_maps(cfgs[2], probe)
    pk = np.abs(ref).max(axis=1)
    assert np.all(np.abs(a0["maps"] - ref).max(axis=1) <= 1e-2 * pk)
    check_fp32_maximiser(a0["argmax"], a0["peak"], ref)
    for d in done:
        if d["maps"] is None or d["tag"] < 100:
            continue
        s, f0 = tags[d["id"]]
        ref = oracle_maps(cfgs[s], cfgs[s]["Y"][f0:f0 + 8])
        pk = np.abs(ref).max(axis=1)
        assert np.all(np.abs(d["maps"] - ref).max(axis=1) <= 1e-2 * pk)
        check_fp32_maximiser(d["argmax"], d["peak"], ref)
    # latencies are ordered and positive
    for d in done:
        assert d["t_submit"] <= d["t_start"] <= d["t_done"]


def test_iterations_carry_many_streams_and_overlap_on_the_gpu():
    """Continuous batching on the device: requests from 8 streams queued
    together (a hold, then a release) are mapped as iterations that each
    carry every stream's group, the probe's iteration carries the other
    streams' groups too, and the next iteration is on the GPU while the
    previous one still is (their GPU intervals intersect).  The probe's
    result equals the one it gets alone."""
    cfgs = mix(15, 8, (20000, 40000), 32)
    plans = plans_for(cfgs, max_frames=32)
    srv = srp.Server(plans, device_budget_bytes=2 << 30, host_budget_bytes=512 << 20,
                     max_inflight=2)
    probe = cfgs[5]["Y"][16:24]
    srv.submit(5, probe, tag=1)
    alone = srv.drain()
    assert len(alone) == 1 and alone[0]["status"] == srp.SRP_OK
    for s_ in range(len(cfgs)):  # first launches of every plan before the measured part
        srv.submit(s_, cfgs[s_]["Y"][:8], tag=3)
    srv.drain()
    srv.hold(True)
    for rnd in range(3):  # 3 x 32 frames per stream: three iterations of 8 groups each
        for s_ in range(len(cfgs)):
            for b in range(4):
                if rnd == 0 and s_ == 5 and b == 2:
                    srv.submit(5, probe, tag=2)
                else:
                    srv.submit(s_, cfgs[s_]["Y"][8 * b:8 * b + 8], tag=10)
    srv.hold(False)
    done = srv.drain()
    st = srv.stats
    srv.close()
    assert all(d["status"] == srp.SRP_OK for d in done) and len(done) == 96
    again = [d for d in done if d["tag"] == 2][0]
    assert np.array_equal(again["argmax"], alone[0]["argmax"])
    assert np.array_equal(again["peak"], alone[0]["peak"])
    # the probe's iteration mapped the other streams' frames in the same launch
    mates = {d["stream"] for d in done if d["iteration"] == again["iteration"]}
    assert again["iteration_streams"] == 8 and mates == set(range(8))
    assert st.max_iteration_streams == 8
    # two iterations were on the GPU at the same time
    iv = {}
    for d in done:
        iv[d["iteration"]] = (d["t_gpu_start"], d["t_gpu_end"])
    assert len(iv) >= 3
    its = sorted(iv)
    pairs = [(a, b) for a in its for b in its if a < b and
             iv[a][0] < iv[b][1] and iv[b][0] < iv[a][1]]
    assert pairs, iv
    assert st.overlapped_iterations >= 2
    for a, b in iv.values():
        assert 0.0 < a < b


def group_bytes(cfg, L):
    """Device working set of one group of L frames: input, maps, argmax, peak,
    each rounded up to 256 bytes."""
    up = lambda v: -(-v // 256) * 256
    M, Kb, J = cfg["mic"].shape[0], cfg["K"] // 2 + 1, cfg["grid"].shape[0]
    return up(8 * M * Kb * L) + up(4 * L * J) + 2 * up(4 * L)


def test_admission_by_device_budget():
    base = synth.uneven_instance(12, (5000, 5001), 16, M=8, K=1024, dims=3)
    cfgs = [dict(base, Y=synth.uneven_instance(120 + i, (5000, 5001), 16, M=8, K=1024,
                                               dims=3)["Y"]) for i in range(3)]
    plans = plans_for([base] * 3, max_frames=16)
    g8 = group_bytes(base, 8)
    budget = g8 + g8 // 2  # one 8-frame group at a time; 16 frames never fit
    assert group_bytes(base, 16) > budget
    srv = srp.Server(plans, device_budget_bytes=budget, max_inflight=2)
    with pytest.raises(srp.SrpError) as e:  # 16 frames can never fit
        srv.submit(0, cfgs[0]["Y"][:16])
    assert e.value.status == srp.SRP_ERR_OOM
    for k in range(12):
        srv.submit(k % 3, cfgs[k % 3]["Y"][:8], tag=k)
    done = srv.drain()
    st = srv.stats
    srv.close()
    assert len(done) == 12 and all(d["status"] == srp.SRP_OK for d in done)
    assert st.rejected == 1
    assert st.device_bytes_peak <= st.device_budget_bytes
    assert st.admission_waits > 0
    # same input, same plan: same answer whenever it ran
    by_stream = {}
    for d in done:
        by_stream.setdefault(d["stream"], []).append(d["argmax"])
    for v in by_stream.values():
        assert all(np.array_equal(v[0], x) for x in v)


def test_deadline_expires_while_queued():
    big = synth.uneven_instance(13, (400_000, 450_000), 32, M=12, K=2048)
    small = synth.uneven_instance(14, (1000, 2000), 8)
    plans = plans_for([big, small], precision="fp32", max_frames=32)
    srv = srp.Server(plans, device_budget_bytes=1 << 30, max_inflight=1)
    srv.submit(0, big["Y"], tag=0)                           # keeps the only slot busy
    srv.submit(1, small["Y"][:4], tag=1, deadline_ms=1e-6)   # cannot start within 1 ns
    srv.submit(1, small["Y"][:4], tag=2)
    done = {d["tag"]: d for d in srv.drain()}
    st = srv.stats
    srv.close()
    assert done[0]["status"] == srp.SRP_OK and done[2]["status"] == srp.SRP_OK
    assert done[1]["status"] == srp.SRP_ERR_TIMEOUT and st.timed_out == 1


def test_unbatched_and_cuda_core_streams():
    """CUDA-core plans, and every plan when batching is off, map with their
    own srp_map calls (results equal srp_map); tensor-core plans, those whose
    FP32 accumulators are promoted included, go through the batched kernels
    (results within 1e-6 x peak of srp_map)."""
    cfgs = [synth.uneven_instance(20 + i, (800, 1500), 8, M=M, K=K)
            for i, (M, K) in enumerate([(12, 2048), (4, 512), (9, 1024)])]
    plans = plans_for(cfgs, mode="conventional", precision="fp32", max_frames=8)
    assert [p.info.tensor_cores for p in plans] == [1, 1, 1]
    assert [p.info.accum_promotion > 0 for p in plans] == [True, False, True]
    plans[2].close()  # the third stream on the CUDA cores instead
    plans[2] = srp.Plan(cfgs[2]["mic"], cfgs[2]["grid"], cfgs[2]["fs"], cfgs[2]["c"],
                        cfgs[2]["K"], mode="conventional", n_aux=2, precision="fp32",
                        max_frames=8, engine="cuda_cores")
    for batching in (True, False):
        srv = srp.Server(plans, device_budget_bytes=64 << 20, max_inflight=2,
                         batching=batching)
        for k in range(9):
            srv.submit(k % 3, cfgs[k % 3]["Y"][:8], tag=k, want_maps=True)
        done = srv.drain()
        srv.close()
        assert all(d["status"] == srp.SRP_OK for d in done)
        for d in done:
            s = d["stream"]
            m, a, p = plans[s].map(torch.from_numpy(cfgs[s]["Y"][:8]).cuda())
            torch.cuda.synchronize()
            m = m.cpu().numpy()
            if batching and plans[s].info.tensor_cores:
                # the batched kernels
                pk = np.abs(m).max(axis=1)
                assert np.all(np.abs(d["maps"] - m).max(axis=1) <= 1e-6 * pk)
            else:  # the plan's own srp_map call
                assert np.array_equal(d["maps"], m)
                assert np.array_equal(d["argmax"], a.cpu().numpy())
