"""Batching machinery (row A10): CG blocks replayed as captured CUDA graphs, and the autotuner of the
pair passes' targets per thread, each checked against the direct path and the FP64 oracle."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import cosine, dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def _batch():
    sizes = S.batch_sizes(24, 64, 700, 77)
    return S.batch_of_knots(sizes, 8, 77)


@pytest.mark.parametrize("precond", [1, 4])
@pytest.mark.parametrize("profile", [False, True])
def test_graph_replay_is_bitwise_identical(torch, precond, profile):
    """The same gradient solve with CG blocks as captured graphs and as direct launches: the same
    kernels in the same order with deterministic reductions give bitwise equal results, and the
    launch count and (when profiling) the number of timed apply launches agree."""
    from paper_2006_07859_gb300 import tpe
    b = _batch()
    out = {}
    for graphs in (0, 1):
        ctx = tpe.Context.from_curves(b, precision=tpe.TP_MIXED, precond=precond, independent=1, cg_rtol=1e-6,
                                      cg_maxit=3000, cg_check_every=8, use_graphs=graphs, warm_start=0)
        g = dev(b.gamma)
        dE = tpe.tp_differential(ctx, g)
        ctx.profile(profile)
        l0 = ctx.launch_count()
        gg, info = tpe.sobolev_gradient(ctx, g, dE)
        # a second solve reuses the cached graphs
        gg2, info2 = tpe.sobolev_gradient(ctx, g, dE)
        torch.cuda.synchronize()
        out[graphs] = (host(gg), host(gg2), info["iters"], ctx.launch_count() - l0,
                       ctx.profile_read(4)[1] if profile else 0)
        ctx.close()
    a, g1 = out[0], out[1]
    assert a[2] == g1[2]
    assert np.array_equal(a[0], g1[0]) and np.array_equal(a[1], g1[1])
    assert np.array_equal(g1[0], g1[1])
    assert a[3] == g1[3]
    if profile:
        assert a[4] == g1[4] > 0


def test_warm_start_repeats_a_solve_in_fewer_iterations(torch):
    """With warm starts (the default) a second gradient solve on the same input starts from the first
    one's solution: it stops after fewer iterations at the same tolerance and lands within that
    tolerance of the first solution.  With warm_start = 0 the two solves are bitwise identical."""
    from paper_2006_07859_gb300 import tpe
    b = _batch()
    res = {}
    for warm in (0, 1):
        ctx = tpe.Context.from_curves(b, precision=tpe.TP_MIXED, precond=4, independent=1, cg_rtol=1e-6,
                                      cg_maxit=3000, warm_start=warm)
        g = dev(b.gamma)
        dE = tpe.tp_differential(ctx, g)
        g1, i1 = tpe.sobolev_gradient(ctx, g, dE)
        g2, i2 = tpe.sobolev_gradient(ctx, g, dE)
        res[warm] = (host(g1), host(g2), i1, i2)
        ctx.close()
    c1, c2, ci1, ci2 = res[0]
    assert np.array_equal(c1, c2) and ci1["iters"] == ci2["iters"]
    w1, w2, wi1, wi2 = res[1]
    assert np.array_equal(w1, c1)                        # nothing to start from on the first call
    assert wi2["converged"] and wi2["iters"] < wi1["iters"]
    assert wi2["rel_res"] <= 1e-4
    assert rel(w2, w1) <= 1e-4


def test_autotune_keeps_parity(torch, orc):
    """After the autotuner picks targets per thread, the passes still match the FP64 oracle."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(3000, 8, 5))
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=1)
    g = dev(c.gamma)
    res = tpe.tp_autotune(ctx, g)
    # gather passes: targets per thread; symmetric passes: 0 (off) or the variant the timing picked
    valid = {"energy": {1, 2, 4}, "diff": {1, 2, 4}, "apply": {1, 2, 4}, "apply_symmetric": {0, 1, 2},
             "energy_symmetric": {0, 1, 2}, "diff_symmetric": {0, 1, 2, 3, 4}}
    assert all(res["tpt"][k] in v for k, v in valid.items()), res["tpt"]
    assert all(len(v) >= 2 for v in res["ms"].values())
    rows = torch.empty(c.n_edges, dtype=torch.float64, device="cuda")
    tpe.tp_energy(ctx, g, rows=rows)
    dE = host(tpe.tp_differential(ctx, g))
    u = np.random.default_rng(3).normal(size=(c.n_vertices, 3))
    Au = host(tpe.sobolev_apply(ctx, g, dev(u)))
    idx = np.sort(np.random.default_rng(4).choice(c.n_edges, 48, replace=False)).astype(np.int32)
    assert rel(host(rows)[idx], orc.energy_rows(c.gamma, c.edges, idx)) <= 1e-6
    ref = orc.differential_at(c.gamma, c.edges, idx)
    assert cosine(dE[idx], ref) >= 0.9999 and rel(dE[idx], ref) <= 1e-5
    assert rel(Au[idx], orc.gram_apply_at(c.gamma, c.edges, 0.75, u, idx)) <= 1e-6


@pytest.mark.parametrize("tpt", [1, 2])
@pytest.mark.parametrize("case", ["single_ragged", "batch"])
def test_symmetric_apply_matches_gather_and_oracle(torch, orc, tpt, case):
    """The symmetric apply (each unordered pair once, both rows fed) against the gather apply and the
    oracle: single curve with a ragged last block and a batch of independent curves of mixed sizes."""
    from paper_2006_07859_gb300 import tpe
    if case == "single_ragged":
        c = S.single(S.fourier_knot(1000, 8, 9))
        indep = 0
    else:
        c = _batch()
        indep = 1
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=1, independent=indep)
    g = dev(c.gamma)
    u = np.random.default_rng(11).normal(size=(c.n_vertices, 3))
    Au_gather = host(tpe.sobolev_apply(ctx, g, dev(u)))
    tpe.tp_set_apply_variant(ctx, tpt)
    Au_sym = host(tpe.sobolev_apply(ctx, g, dev(u)))
    Au_sym2 = host(tpe.sobolev_apply(ctx, g, dev(u)))
    assert np.array_equal(Au_sym, Au_sym2)          # deterministic
    assert rel(Au_sym, Au_gather) <= 1e-6
    if case == "single_ragged":
        idx = np.sort(np.random.default_rng(12).choice(c.n_vertices, 40, replace=False)).astype(np.int32)
        assert rel(Au_sym[idx], orc.gram_apply_at(c.gamma, c.edges, 0.75, u, idx)) <= 1e-6
    else:
        for k in range(4):
            gk, ek = c.curve(k)
            v0, v1 = c.vertex_offsets[k], c.vertex_offsets[k + 1]
            ref = orc.gram_apply(gk, ek, 0.75, u[v0:v1])
            assert rel(Au_sym[v0:v1], ref) <= 1e-6


@pytest.mark.parametrize("tpt", [1, 2])
@pytest.mark.parametrize("case", ["single_ragged", "batch", "near"])
def test_symmetric_energy_matches_gather_and_oracle(torch, orc, tpt, case):
    """Energy rows of the symmetric pass (each unordered pair once, both rows fed; FP64 cross
    products for near pairs) against the gather pass and the oracle."""
    from paper_2006_07859_gb300 import tpe
    if case == "single_ragged":
        c = S.single(S.fourier_knot(1000, 8, 9))
    elif case == "near":
        c = S.single(S.fourier_knot(3000, 16, 4))   # fine sampling: many pairs inside the near cutoff
    else:
        c = _batch()
    indep = 1 if case == "batch" else 0
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=1, independent=indep)
    g = dev(c.gamma)
    rows_g = torch.empty(c.n_edges, dtype=torch.float64, device="cuda")
    rows_s = torch.empty_like(rows_g)
    E_g = host(tpe.tp_energy(ctx, g, rows=rows_g))
    tpe.tp_set_energy_variant(ctx, tpt)
    E_s = host(tpe.tp_energy(ctx, g, rows=rows_s))
    E_s2 = host(tpe.tp_energy(ctx, g))
    assert np.array_equal(E_s, E_s2)
    # Both passes add a tile's pair terms in plain FP32 (128 sources here, up to 512 in the gather)
    # before folding into FP64, so they differ by the rounding of those partial sums: a few 1e-6 of
    # the largest row at n = 1000.  The oracle decides.
    assert rel(host(rows_s), host(rows_g)) <= 2e-5
    assert rel(E_s, E_g) <= 1e-6
    idx = np.sort(np.random.default_rng(13).choice(c.n_edges, 48, replace=False)).astype(np.int32)
    if case != "batch":
        assert rel(host(rows_s)[idx], orc.energy_rows(c.gamma, c.edges, idx)) <= 1e-6
    else:
        for k in range(3):
            gk, ek = c.curve(k)
            assert abs(E_s[k] - orc.energy(gk, ek)) <= 1e-6 * abs(E_s[k])


@pytest.mark.parametrize("tpt", [1, 2, 3, 4])
@pytest.mark.parametrize("case", ["single_ragged", "batch", "near"])
def test_symmetric_differential_matches_gather_and_oracle(torch, orc, tpt, case):
    """The symmetric differential (row J's terms of a pair mirrored from row I's; near pairs FP64 on both
    sides) against the gather pass and the oracle; translation invariance sum_v dE_v = 0 per curve."""
    from paper_2006_07859_gb300 import tpe
    if case == "single_ragged":
        c = S.single(S.fourier_knot(1000, 8, 9))
    elif case == "near":
        c = S.single(S.fourier_knot(3000, 16, 4))
    else:
        c = _batch()
    indep = 1 if case == "batch" else 0
    ctx = make_ctx(c, precision=tpe.TP_MIXED, precond=1, independent=indep)
    g = dev(c.gamma)
    dE_g = host(tpe.tp_differential(ctx, g))
    tpe.tp_set_diff_variant(ctx, tpt)
    dE_s = host(tpe.tp_differential(ctx, g))
    dE_s2 = host(tpe.tp_differential(ctx, g))
    assert np.array_equal(dE_s, dE_s2)
    assert rel(dE_s, dE_g) <= 1e-5
    assert cosine(dE_s, dE_g) >= 1 - 1e-10
    for k in range(min(4, len(c.vertex_offsets) - 1)):
        v0, v1 = c.vertex_offsets[k], c.vertex_offsets[k + 1]
        assert np.abs(dE_s[v0:v1].sum(0)).max() <= 1e-4 * np.abs(dE_s[v0:v1]).max()
    if case != "batch":
        idx = np.sort(np.random.default_rng(14).choice(c.n_vertices, 32, replace=False)).astype(np.int32)
        ref = orc.differential_at(c.gamma, c.edges, idx)
        assert cosine(dE_s[idx], ref) >= 0.9999
        assert rel(dE_s[idx], ref) <= 1e-5
