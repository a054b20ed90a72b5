"""tp_energy_static: the energy entry point that allocates nothing.

It is meant for callers that cannot call cudaMalloc (code running where device allocation is
forbidden, or after all free memory went to the caller's own pool); its scratch is a fixed-size
__device__ array inside the library.  Checked through the C ABI against the FP64 oracle and against
the context-based tp_energy, on two calls in a row (the scratch keeps the previous call's contents,
so the second call shows that nothing stale leaks into the result), on an empty graph and on a graph
at the scratch's size limit.  This file is collected last."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


@pytest.mark.parametrize("name", ["trefoil256", "knot3000", "scene2"])
def test_static_energy_matches_oracle_and_context_energy_twice(orc, name):
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    c = {"trefoil256": S.trefoil_256(),
         "knot3000": S.single(S.fourier_knot(3000, 6, 8)),
         "scene2": S.scene([S.fourier_knot(700, 4, 1), S.fourier_knot(1300, 5, 2)])}[name]
    g = dev(c.gamma)
    edges = torch.as_tensor(c.edges).cuda()
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=tpe.TP_PRECOND_JACOBI)
    ref = host(tpe.tp_energy(ctx, g))[0]
    Eo = orc.energy(c.gamma, c.edges)
    for call in range(2):
        E = host(tpe.tp_energy_static(g, edges))[0]
        # the FP64 oracle: mixed precision keeps the energy to ~1e-7 relative
        assert abs(E - Eo) <= 1e-6 * abs(Eo), (call, E, Eo)
        # same arithmetic as the context's pass, different chunking of the sums: relative 1e-9
        assert abs(E - ref) <= 1e-9 * abs(ref), (call, E, ref)


def test_static_energy_of_empty_graph_is_zero():
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    g = dev(S.unit_square())
    edges = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    E = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        assert host(tpe.tp_energy_static(g, edges, E=E))[0] == 0.0


def test_static_energy_at_the_size_limit():
    """65,536 edges (the largest graph the fixed scratch holds), two calls, against the context's pass;
    rows of the oracle on a sample pin the scale of the result."""
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(65536, 8, 31))
    g = dev(c.gamma)
    edges = torch.as_tensor(c.edges).cuda()
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=tpe.TP_PRECOND_JACOBI)
    rows = torch.empty(c.n_edges, dtype=torch.float64, device="cuda")
    ref = host(tpe.tp_energy(ctx, g, rows=rows))[0]
    for call in range(2):
        E = host(tpe.tp_energy_static(g, edges))[0]
        assert abs(E - ref) <= 1e-9 * abs(ref), (call, E, ref)
    from oracle import oracle as O
    O.build_library()
    idx = np.arange(0, c.n_edges, 4099, dtype=np.int32)
    ro = O.energy_rows(c.gamma, c.edges, idx)
    assert np.abs(host(rows)[idx] - ro).max() <= 1e-6 * np.abs(ro).max()


def test_static_energy_rejects_oversize_graph():
    torch = need_gpu()
    from paper_2006_07859_gb300 import tpe
    n = 65537
    g = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    edges = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(tpe.TpError) as ei:
        tpe.tp_energy_static(g, edges)
    assert ei.value.status == tpe.TP_ERR_INVALID_ARG
