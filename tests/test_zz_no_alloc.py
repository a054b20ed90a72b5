"""tp_energy_static: the energy entry point that allocates nothing.

It is meant for callers that cannot call cudaMalloc (code running where device allocation is
forbidden, or after all free memory went to the caller's own pool); its scratch is a fixed-size
__device__ array inside the library.  Checked through the C ABI against the context-based
tp_energy, on two calls in a row (the scratch keeps the previous call's contents, so the second call
shows that nothing stale leaks into the result).  This file is collected last."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["trefoil256", "knot3000", "scene2"])
def test_static_energy_matches_context_energy_twice(name):
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    c = {"trefoil256": S.trefoil_256(),
         "knot3000": S.single(S.fourier_knot(3000, 6, 8)),
         "scene2": S.scene([S.fourier_knot(700, 4, 1), S.fourier_knot(1300, 5, 2)])}[name]
    g = dev(c.gamma)
    edges = torch.as_tensor(c.edges).cuda()
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=tpe.TP_PRECOND_JACOBI)
    ref = host(tpe.tp_energy(ctx, g))[0]
    for call in range(2):
        E = host(tpe.tp_energy_static(g, edges))[0]
        # same arithmetic, different chunking of the sums: relative 1e-9
        assert abs(E - ref) <= 1e-9 * abs(ref), (call, E, ref)


def test_static_energy_rejects_oversize_graph():
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    n = 65537
    g = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    edges = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(tpe.TpError) as ei:
        tpe.tp_energy_static(g, edges)
    assert ei.value.status == tpe.TP_ERR_INVALID_ARG
