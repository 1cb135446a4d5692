"""The allocation-free SNSD entry point (for callers that cannot allocate
device memory: a host framework holding the device pool, a real-time loop, a
plugin limited to start-up allocation) gives the same results as the regular
entry point, through the C ABI, on two calls in a row that reuse its fixed
scratch; and it rejects a body count above its scratch limit.  Collected last
(file name) so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest
import torch

from paper_2506_14097_gb300 import scenes

pytestmark = pytest.mark.gpu


def _case(seed, n, side):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * side
    q = scenes.random_quaternions(rng, n)
    axes = rng.uniform(0.4, 1.0, (n, 3))
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, min(n, i + 12))], dtype=np.int32)
    box = np.array([side] * 3)
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    return dev(pairs, torch.int32), dev(x), dev(q), dev(axes), box


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-12)])
def test_noalloc_matches_regular_entry_point_twice(relcp_gpu, precision, tol):
    R = relcp_gpu
    for call, (seed, n, side) in enumerate(((31, 600, 9.0), (32, 900, 11.0))):
        pairs, x, q, axes, box = _case(seed, n, side)
        ref, ref_it = R.relcp_snsd_eval(pairs, x, q, axes, box, precision)
        out = torch.full((pairs.shape[0], 10), float("nan"), dtype=torch.float64, device="cuda")
        it = torch.full((pairs.shape[0],), -999, dtype=torch.int32, device="cuda")
        R.relcp_snsd_eval_noalloc(pairs, x, q, axes, box, out, it, precision)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all(), call
        err = float((out - ref).abs().max())
        assert err <= tol * (1.0 + float(ref.abs().max())), (call, err)
        assert torch.equal(it, ref_it), call


def test_noalloc_rejects_too_many_bodies(relcp_gpu):
    R = relcp_gpu
    n = R.NOALLOC_MAX_BODIES + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    q[:, 0] = 1.0
    axes = torch.ones((n, 3), dtype=torch.float64, device="cuda")
    pairs = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda")
    out = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(R.RelcpError) as e:
        R.relcp_snsd_eval_noalloc(pairs, x, q, axes, np.zeros(3), out)
    assert e.value.status == R.RELCP_ERR_CAPACITY
