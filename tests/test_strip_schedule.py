"""Host-side checks of the persistent epoch's dependency counts
(gmf_strip_schedule) and of the waiting protocol built on them, without a GPU.

Algorithm 1 visits, in sweep w, the blocks (I_{(sigma[w]+k) mod r}, J_k),
k < per = min(r, s) (roles swapped when r < s). Block k always keeps the fixed
strip k; its moving strip m(w, k) = (sigma[w] + k) mod max(r, s) passes between
blocks. In the persistent launch block k of sweep w waits until the moving
strip has been written back by every earlier visit of the launch's range."""
import itertools
import random

import numpy as np
import pytest


@pytest.fixture(scope="module")
def gmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


def moving(r, s, sig_w, k):
    return (sig_w + k) % max(r, s)


def need_brute(r, s, sigma, w0, w1):
    """Count, for every (w, k), the sweeps w' in [w0, w) with some block on m(w, k)."""
    per = min(r, s)
    out = np.zeros((w1 - w0, per), dtype=np.int32)
    for w in range(w0, w1):
        for k in range(per):
            mw = moving(r, s, sigma[w], k)
            out[w - w0, k] = sum(any(moving(r, s, sigma[v], kk) == mw for kk in range(per)) for v in range(w0, w))
    return out


CASES = [(40, 4), (4, 40), (3, 2), (2, 3), (5, 5), (1, 1), (7, 1), (1, 6), (12, 2), (9, 4)]


@pytest.mark.parametrize("r,s", CASES)
def test_need_counts_equal_brute_force(gmf, r, s):
    S = max(r, s)
    rng = np.random.default_rng(r * 100 + s)
    for _ in range(3):
        sigma = rng.permutation(S).astype(np.int32)
        for w0, w1 in [(0, S), (0, 0), (S // 2, S), (min(1, S), max(min(1, S), S - 1))]:
            got = gmf.strip_schedule(r, s, sigma, w0, w1)
            np.testing.assert_array_equal(got, need_brute(r, s, sigma, w0, w1), err_msg=f"{r}x{s} [{w0},{w1})")


@pytest.mark.parametrize("r,s", CASES)
def test_need_counts_special_cases(gmf, r, s):
    """Closed forms: the first sweep of a range waits for nothing; the blocks of
    one sweep move along distinct strips; over a whole epoch each of the S strips
    is visited per times, so the counts of a strip are 0, 1, ..., per-1 in sweep
    order and sum to S * per * (per - 1) / 2."""
    S, per = max(r, s), min(r, s)
    sigma = np.random.default_rng(7).permutation(S).astype(np.int32)
    need = gmf.strip_schedule(r, s, sigma, 0, S)
    assert (need[0] == 0).all()
    for w in range(S):
        assert len({moving(r, s, sigma[w], k) for k in range(per)}) == per
    assert int(need.sum()) == S * per * (per - 1) // 2
    seen = {}
    for w in range(S):
        for k in range(per):
            mw = moving(r, s, sigma[w], k)
            assert need[w, k] == seen.get(mw, 0)
            seen[mw] = seen.get(mw, 0) + 1
    assert all(v == per for v in seen.values())


def test_strip_schedule_rejects_bad_arguments(gmf):
    sigma = np.arange(4, dtype=np.int32)
    for args in [(0, 4, sigma, 0, 4), (4, 0, sigma, 0, 4), (4, 2, sigma, 0, 5), (4, 2, sigma, 3, 2),
                 (4, 2, sigma, -1, 2)]:
        with pytest.raises(gmf.GmfError) as e:
            gmf.strip_schedule(*args)
        assert e.value.code == gmf.GMF_ERR_ARG
    with pytest.raises(gmf.GmfError):
        gmf.strip_schedule(4, 2, np.array([0, 1, 2, 4], dtype=np.int32), 0, 4)


def simulate(r, s, sigma, w0, w1, seed, need_fn=need_brute):
    """The waiting protocol of the persistent launch with its clusters as
    independent workers in a random interleaving: cluster k runs block k of its
    next sweep once the moving strip's count reaches need, and the strip's
    count grows by one once the cluster has written the block back: published
    at the top of its next block, before that block's own wait, or never after
    its last block. Returns the order in which each strip's visits completed,
    or None if the workers stall."""
    per = min(r, s)
    need = need_fn(r, s, sigma, w0, w1)
    count = {}
    nxt = [w0] * per                    # next sweep of each cluster
    order = {}
    rnd = random.Random(seed)
    while any(w < w1 for w in nxt):
        ready = [k for k in range(per) if nxt[k] < w1
                 and count.get(moving(r, s, sigma[nxt[k]], k), 0) >= need[nxt[k] - w0, k]]
        if not ready:
            return None
        k = rnd.choice(ready)
        w = nxt[k]
        mw = moving(r, s, sigma[w], k)
        order.setdefault(mw, []).append(w)
        nxt[k] += 1
        if nxt[k] < w1:                       # the top of the next block publishes, then waits
            count[mw] = count.get(mw, 0) + 1
    return order


@pytest.mark.parametrize("r,s", CASES)
def test_protocol_never_stalls_and_keeps_sweep_order(r, s):
    """Every interleaving the counts allow completes, and each strip sees its
    visits in sweep order -- the order of the per-sweep launches, which is why
    the persistent launch reproduces their results bit for bit."""
    S = max(r, s)
    for seed, (w0, w1) in itertools.product(range(5), [(0, S), (S // 3, S)]):
        sigma = np.random.default_rng(seed).permutation(S)
        order = simulate(r, s, sigma, w0, w1, seed=seed)
        assert order is not None
        for visits in order.values():
            assert visits == sorted(visits)


def test_protocol_stalls_without_the_counts():
    """A plant in the protocol, not in the library: with every count raised by
    one visit the first sweep already waits for a strip nobody writes, and the
    simulation reports the stall (so the test above can fail)."""
    sigma = np.random.default_rng(0).permutation(6)
    assert simulate(6, 2, sigma, 0, 6, seed=0, need_fn=lambda *a: need_brute(*a) + 1) is None
