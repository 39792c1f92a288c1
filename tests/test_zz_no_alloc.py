"""srp_gcc_samples_static: the allocation-free variant of srp_gcc_samples,
for callers that may not call cudaMalloc (an allocator owned by a host
application, a real-time audio thread).  Its scratch is a fixed 8 MiB device
array inside the library.  Checked against the plan-based entry on two calls
in a row, and for its size limit.  Kept in a file collected last."""
import numpy as np
import pytest
import torch

from paper_2012_09499_gb300 import build_lib, srp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _reference(cfg, n_aux, L):
    plan = srp.Plan(cfg["mic"], cfg["grid"], cfg["fs"], cfg["c"], cfg["K"], n_aux=n_aux,
                    max_frames=L)
    y = torch.from_numpy(cfg["Y"][:L]).cuda()
    xi = torch.empty((L, plan.info.S), dtype=torch.float32, device="cuda")
    srp.srp_gcc_samples(plan.handle, y, L, xi)
    torch.cuda.synchronize()
    _, nq = srp.srp_plan_describe(plan.desc)
    plan.close()
    return y, xi, nq


def test_static_scratch_matches_plan_entry_twice():
    cases = [(synth.room_3d(seed=11, L=5, shape=(3, 3, 3), spacing=1.0), 2, 5),
             (synth.tiny_2d(seed=12, L=16, K=1024), 1, 16)]
    outs = []
    for cfg, n_aux, L in cases:  # two calls in a row, different shapes
        y, ref, nq = _reference(cfg, n_aux, L)
        out = torch.full_like(ref, float("nan"))
        srp.srp_gcc_samples_static(cfg["mic"].shape[0], cfg["K"], n_aux, nq, y, L, out)
        outs.append((out, ref))
    torch.cuda.synchronize()
    for out, ref in outs:
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=3e-6)


def test_static_scratch_rejects_oversize():
    M, K = 16, 2048  # 120 pairs x 1025 bins x 8 B = 984000 B per frame
    nq = np.zeros(120, np.int32)
    y = torch.zeros((9, M, K // 2 + 1), dtype=torch.complex64, device="cuda")
    xi = torch.zeros((9, 120), dtype=torch.float32, device="cuda")
    with pytest.raises(srp.SrpError) as e:
        srp.srp_gcc_samples_static(M, K, 0, nq, y, 9, xi)
    assert e.value.status == srp.SRP_ERR_INVALID_ARG
    srp.srp_gcc_samples_static(M, K, 0, nq, y, 8, xi)  # 8 frames fit
    torch.cuda.synchronize()
    assert torch.all(xi[:8] == 0)


def test_static_scratch_rejects_frame_count_beyond_grid_limit():
    # M = 2, K = 4: 24 bytes of scratch per frame, so 65536 frames would fit
    # the array, but the frame index is a grid dimension (at most 65535)
    y = torch.zeros((1, 2, 3), dtype=torch.complex64, device="cuda")
    xi = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(srp.SrpError) as e:
        srp.srp_gcc_samples_static(2, 4, 0, np.zeros(1, np.int32), y, 65536, xi)
    assert e.value.status == srp.SRP_ERR_INVALID_ARG
