"""Host-side check, without a GPU, of the buffer and mbarrier protocol of the
tensor-core deviance (gmf_deviance_tc.cu). The CTA loop is restated as a
sequence of events per CTA (TMA issues into count buffers, eta MMA issues
into TMEM accumulators, operand builds, waits, epilogues, CTA barriers) for
both variants: ST = 1 (one count buffer, one accumulator, a serial tile loop)
and ST = 2 (two of each, the next tile's counts and MMAs in flight during the
current epilogue). The checks: every tile of the CTA (c, c + G, ...) is
reduced once, in order; every wait uses the parity of the phase it waits
for and no barrier ever has two phases outstanding (an mbarrier tracks one);
an epilogue reads a buffer and an accumulator only after waiting for the
copy and the MMA that filled them with its own tile; nothing writes a buffer,
an accumulator or the operands while an earlier tile still needs them; and
the clean-up finds nothing in flight."""
import pytest


def events(st, first, G, ntiles):
    """The kernel's event sequence for one CTA (variant st, first tile, grid G)."""
    ev = []
    t = first
    if st == 1:
        while t < ntiles:
            ev += [("tma", 0, t), ("build", t), ("sync",), ("mma", 0, t), ("wait", "mma"), ("wait", 0),
                   ("epi", 0, 0, t), ("sync",)]
            t += G
        return ev
    if t < ntiles:
        ev += [("tma", 0, t), ("build", t), ("sync",), ("mma", 0, t)]
    it = 0
    while t < ntiles:
        b = it & 1
        tn = t + G
        if tn < ntiles:
            ev.append(("tma", b ^ 1, tn))
        ev.append(("wait", "mma"))
        if tn < ntiles:
            ev += [("build", tn), ("sync",), ("mma", b ^ 1, tn)]
        ev += [("wait", b), ("epi", b, b, t), ("sync",)]
        it += 1
        t += G
    return ev


def check(st, first, G, ntiles, ev=None):
    issued = {0: [], 1: [], "mma": []}      # per barrier: tiles of the phases issued, in order
    waited = {0: 0, 1: 0, "mma": 0}
    ybuf = {0: None, 1: None}               # tile whose counts the buffer holds (or is receiving)
    acc = {0: None, 1: None}                # tile whose eta the accumulator holds (or is receiving)
    ops = None                               # tile whose operands are in shared memory
    ready_y, ready_acc = set(), set()        # (buffer, tile) pairs whose copy / MMA was waited for
    busy_y, busy_acc = {}, {}                # buffer -> tile still to be read by an epilogue
    mma_pending_ops = None
    done = []
    for e in (events(st, first, G, ntiles) if ev is None else ev):
        kind = e[0]
        if kind == "tma":
            _, b, t = e
            assert b not in busy_y, f"count buffer {b} overwritten while tile {busy_y.get(b)} needs it"
            assert len(issued[b]) == waited[b], "two phases outstanding on a count barrier"
            issued[b].append(t)
            ybuf[b] = t
            busy_y[b] = t
        elif kind == "build":
            assert mma_pending_ops is None, "operands rebuilt while an MMA may still read them"
            ops = e[1]
        elif kind == "mma":
            _, b, t = e
            assert ops == t, "MMA issued on another tile's operands"
            assert b not in busy_acc, f"accumulator {b} overwritten while tile {busy_acc.get(b)} needs it"
            assert len(issued["mma"]) == waited["mma"], "two phases outstanding on the MMA barrier"
            issued["mma"].append((b, t))
            acc[b] = t
            busy_acc[b] = t
            mma_pending_ops = t
        elif kind == "wait":
            bar = e[1]
            # the kernel waits with parity (phases waited so far) mod 2: that is the parity of the phase in
            # flight exactly when each phase is waited for once, in order, and never two are outstanding
            assert waited[bar] < len(issued[bar]), "wait on a barrier with nothing in flight"
            if bar == "mma":
                b, t = issued["mma"][waited[bar]]
                ready_acc.add((b, t))
                mma_pending_ops = None
            else:
                ready_y.add((bar, issued[bar][waited[bar]]))
            waited[bar] += 1
        elif kind == "epi":
            _, b, a, t = e
            assert ybuf[b] == t and (b, t) in ready_y, "epilogue before its counts arrived"
            assert acc[a] == t and (a, t) in ready_acc, "epilogue before its eta MMA completed"
            done.append(t)
            del busy_y[b]
            del busy_acc[a]
        elif kind == "sync":
            pass
    assert done == list(range(first, ntiles, G))
    for bar in issued:
        assert waited[bar] == len(issued[bar]), "a copy or an MMA still in flight at the end"


@pytest.mark.parametrize("st", [1, 2])
@pytest.mark.parametrize("ntiles,G", [(1, 1), (5, 304), (304, 304), (305, 304), (1000, 304), (61035, 456),
                                      (61035, 304), (7, 3), (8, 3)])
def test_every_cta_follows_the_protocol(st, ntiles, G):
    firsts = range(min(G, ntiles)) if ntiles < 4000 else range(0, min(G, ntiles), max(1, G // 17))
    for first in firsts:
        check(st, first, G, ntiles)


def test_a_broken_order_is_caught():
    """The check can fail: issuing the next tile's counts into the buffer the
    current epilogue still reads, or skipping the wait for an MMA, is reported."""
    ev = events(2, 0, 1, 3)
    bad = [("tma", 0, 1) if e == ("tma", 1, 1) else e for e in ev]
    with pytest.raises(AssertionError):
        check(2, 0, 1, 3, bad)
    no_wait = list(ev)
    no_wait.remove(("wait", "mma"))
    with pytest.raises(AssertionError):
        check(2, 0, 1, 3, no_wait)
