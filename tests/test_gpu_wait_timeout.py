"""A bounded device wait that runs out.  The cooperative FP64 Jacobi SVD
(more than 128 columns) meets at a grid barrier after every round of column
pairs; with the context's wait limit set to 0 every block but the last to
arrive gives up at once: the kernel records SEEMPS_ERR_TIMEOUT in the status
word and returns without trapping or hanging.  The host reads status 5; with
the default limit restored the same context computes the split correctly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_reports_status_and_context_stays_usable():
    import torch
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    ctx = pkg.Context(0, chi_max=256, d=2, D_max=1, krylov_dim=2)
    rng = np.random.default_rng(5)
    M = torch.from_numpy(rng.standard_normal((300, 256))).cuda()
    assert ctx.device_status() == 0
    ctx.set_wait_limit(0)
    ctx.svd_truncate(M, 256, 1e-14, precision=pkg.FP64)  # returns; its results are invalid
    torch.cuda.synchronize()
    assert ctx.device_status() == 5  # SEEMPS_ERR_TIMEOUT (reading it also clears it)
    ctx.set_wait_limit(-1)
    res = ctx.svd_truncate(M, 256, 1e-14, precision=pkg.FP64)
    s_ref = np.linalg.svd(M.cpu().numpy(), compute_uv=False)
    assert np.abs(res.S.cpu().numpy() - s_ref).max() <= 1e-13 * s_ref[0]
    assert ctx.device_status() == 0
    ctx.close()
