"""The allocation-free reduction entry point, qtm_ensemble_reduce_static.

Some callers cannot let a library allocate device memory -- a host framework
whose memory planner owns every buffer, or a service with a device footprint
fixed at start-up.  For them the library offers one entry point that reduces
per-trajectory values the caller already holds, keeping its scratch in a fixed
array inside the library.  This test calls it through the C ABI twice in a row
(different ensemble sizes, so stale scratch from the first call would show in
the second) and checks each result against what the context-based entry points
(qtm_expect, qtm_sums) return for the same trajectories.  It runs on its own and
after the rest of the suite alike: it builds all of its own data.
"""

import numpy as np
import pytest

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

pytestmark = pytest.mark.gpu

TOL = 1e-8  # the ensemble tolerance of the GPU parity tests


def _context_results(prob, ntraj, seed):
    ctx = Q.qtm_create(prob)
    Q.qtm_run(ctx, ntraj, seed)
    mean, se = Q.qtm_expect(ctx)
    s1, s2, n = Q.qtm_sums(ctx)
    values = Q.qtm_traj_expect(ctx)
    Q.qtm_destroy(ctx)
    assert n == ntraj
    return values, mean, se, s1, s2


def test_static_scratch_reduction_matches_context_path():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    prob = S.jaynes_cummings_driven()
    stream = torch.cuda.current_stream()
    for ntraj, seed in ((3000, 1), (777, 5)):
        values, mean, se, s1, s2 = _context_results(prob, ntraj, seed)
        P = values.shape[1] * values.shape[2]
        dev_values = torch.from_numpy(values.reshape(ntraj, P)).to("cuda")
        out = torch.full((4, P), float("nan"), dtype=torch.float64, device="cuda")
        Q.qtm_ensemble_reduce_static(dev_values.data_ptr(), ntraj, P, out[0].data_ptr(), out[1].data_ptr(),
                                     out[2].data_ptr(), out[3].data_ptr(), int(stream.cuda_stream))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got[2] - mean.ravel()).max() <= TOL
        assert np.abs(got[3] - se.ravel()).max() <= TOL
        assert np.abs(got[0] - s1.ravel()).max() <= TOL * max(1.0, np.abs(s1).max())
        assert np.abs(got[1] - s2.ravel()).max() <= TOL * max(1.0, np.abs(s2).max())


def test_static_scratch_rejects_oversized_problems():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_ensemble_reduce_static(p, 1, (1 << 18) + 1, p, p, p, p, 0)
    assert ei.value.status == Q.QTM_ERR_ARG
    assert "n_values" in str(ei.value)
