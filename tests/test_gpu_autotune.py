"""The tile autotuner: both tile kernels of the bf16x3 GEMM form every output
from the same products in the same order, so switching a shape to the timed
winner changes no result bit; the table is filled by seemps_autotune and
read only by contexts that turned autotuning on."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.mark.parametrize("chi", [200, 384, 700])
def test_autotuned_heff_is_bit_identical(pkg, chi):
    import torch
    ctx = pkg.Context(0, chi_max=chi, d=2, D_max=5, krylov_dim=4)
    rng = np.random.default_rng(chi)
    W = wl.mpo.xxz(4, 1.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    L, R = t(rng.standard_normal((chi, 5, chi))), t(rng.standard_normal((chi, 5, chi)))
    th = t(rng.standard_normal((chi, 2, 2, chi)))
    A = t(rng.standard_normal((chi, 2, chi)))
    W1, W2 = t(W[1]), t(W[2])
    y0 = ctx.heff_apply(L, W1, W2, R, th, precision=pkg.BF16X3)
    E0 = ctx.env_update(pkg.LEFT, L, A, W1, precision=pkg.BF16X3)
    n = ctx.autotune(chi, chi, 2, 5, 5, 5)
    st0 = ctx.autotune_stats()
    assert st0["table_size"] >= 1 and st0["shapes_timed"] == n
    ctx.set_autotune(True)
    y1 = ctx.heff_apply(L, W1, W2, R, th, precision=pkg.BF16X3)
    E1 = ctx.env_update(pkg.LEFT, L, A, W1, precision=pkg.BF16X3)
    st1 = ctx.autotune_stats()
    print(f"chi={chi}: {n} shapes timed, table {st1['table_size']}, lookups hit {st1['hits']}")
    assert st1["hits"] >= 2  # both GEMMs of H_n (the environment update's six-product GEMM has one tile)
    assert torch.equal(y0, y1)
    assert torch.equal(E0, E1)
    # a second tuning call finds every shape recorded
    assert ctx.autotune(chi, chi, 2, 5, 5, 5) == 0
    assert ctx.device_status() == 0
    ctx.close()
