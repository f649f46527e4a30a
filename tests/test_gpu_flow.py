"""The dataflow epoch (GMF_FLAG_PERSIST for blocks of more than 16 tiles): one
cooperative launch per sweep range in which tile and update items, taken in
ticket order, wait only for the updates of the strips they read. Every result
equals the per-sweep tile and update launches bit for bit (same functions,
same sums in the same order), for every item order (lag), with rows or
columns moving, with 16- and 32-bit counts, ragged blocks, a per-sweep NB
shape estimate (whose update is taken by the CTA that finishes a sweep's last
tile) and sweep ranges shorter than an epoch. The bounded waits end the launch
with GMF_ERR_TIMEOUT when a dependency count can never be met."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


def _pair(gmf, prob, d, nbr, nbc, seed, **settings):
    n, m = prob.Y.shape
    rp, cp = synth.partitions(n, m, seed)
    start = synth.crude_start(prob, d, seed=seed)
    Y = torch.from_numpy(prob.Y.view(np.int16) if prob.Y.dtype == np.uint16 else prob.Y).cuda()
    kw = dict(family=prob.family, nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp,
              settings=synth.fit_settings(**settings), precision="mixed")
    flow = gmf.Model(Y, prob.X, prob.Z, prob.offset, start, flags=gmf.GMF_FLAG_PERSIST, **kw)
    ref = gmf.Model(Y, prob.X, prob.Z, prob.offset, start, **kw)
    if flow.epoch_mode != "persistent":
        pytest.skip("the dataflow epoch cannot keep every CTA resident on this device")
    assert ref.epoch_mode == "separate"
    return flow, ref


def _same(a, b):
    pa, pb = a.get_params(), b.get_params()
    for k in ("U", "V", "B", "Gamma"):
        np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)
    assert pa["alpha"] == pb["alpha"]
    ea, eb = a.get_ema(), b.get_ema()
    for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col", "cnt_row", "cnt_col", "t"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    assert a.deviance() == b.deviance()


# (n, m, y dtype, blocks): rows moving (r > s) with ragged row and column tails; columns moving (r < s);
# 32-bit counts (one CTA per SM, no Ddot over the counts)
SHAPES = [(6000, 2000, "uint16", 1024, 512), (2048, 6000, "uint16", 512, 1024), (5000, 1600, "int32", 1024, 512)]


@pytest.mark.parametrize("shape", SHAPES, ids=["rows-move", "columns-move", "int32"])
@pytest.mark.parametrize("alpha_mode", [0, 1])
def test_flow_epoch_equals_per_sweep_launches(gmf, shape, alpha_mode):
    n, m, ydt, nbr, nbc = shape
    prob = synth.make_problem(n, m, 3, 1, 12, "negbin", seed=3, zero_frac=0.85, offset=True, y_dtype=ydt)
    flow, ref = _pair(gmf, prob, 12, nbr, nbc, 3, alpha_mode=alpha_mode)
    assert flow.launches_per_sweep == 0
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 3)
    for e in range(3):
        flow.epoch(sig[e])
        ref.epoch(sig[e])
    _same(flow, ref)


def test_flow_item_order_and_sweep_ranges(gmf):
    """Lags 0, 1, 5 and 64 give the same bits; sweep ranges [0, 2), [2, 3),
    [3, S) of an epoch equal the whole epoch; Poisson."""
    n, m, nbr, nbc = 4500, 2048, 768, 512
    prob = synth.make_problem(n, m, 2, 2, 6, "poisson", seed=8, offset=True, y_dtype="uint16")
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 8)
    ref = None
    for lag in (0, 1, 5, 64):
        flow, ref0 = _pair(gmf, prob, 6, nbr, nbc, 8)
        flow.set_flow_lag(lag)
        S = len(sig[0])
        flow.epoch(sig[0])
        flow.sweeps(sig[1], 0, 2)
        flow.sweeps(sig[1], 2, 3)
        flow.sweeps(sig[1], 3, S)
        flow.epoch(sig[2])
        if ref is None:
            for e in range(3):
                ref0.epoch(sig[e])
            ref = ref0
        _same(flow, ref)
    with pytest.raises(gmf.GmfError):
        flow.set_flow_lag(65)


def test_flow_waits_time_out_and_the_context_survives(gmf):
    n, m, nbr, nbc = 4000, 1536, 1024, 512
    prob = synth.make_problem(n, m, 2, 1, 8, "negbin", seed=5, zero_frac=0.6, offset=True, y_dtype="uint16")
    sig = synth.sweep_orders(n, m, nbr, nbc, 2, 5)
    flow, ref = _pair(gmf, prob, 8, nbr, nbc, 5)
    flow.set_wait_limit(2_000_000, 1)       # 2 ms per wait; every moving-strip count one visit short
    torch.cuda.synchronize()
    flow.epoch(sig[0])
    torch.cuda.synchronize()                 # the launch ends by itself
    with pytest.raises(gmf.GmfError) as e:
        flow.deviance()
    assert e.value.code == gmf.GMF_ERR_TIMEOUT
    del flow
    fresh, _ = _pair(gmf, prob, 8, nbr, nbc, 5)
    for s in sig:
        fresh.epoch(s)
        ref.epoch(s)
    _same(fresh, ref)
