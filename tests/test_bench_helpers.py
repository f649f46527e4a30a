"""Host-side pieces of bench.py that the reported numbers depend on (no GPU):
the entries of a sweep, the algorithmic work and bytes of a sweep launch, the
host description, and the clock sampler's behaviour without a GPU driver."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


@pytest.mark.parametrize("n,m,nbr,nbc", [(20000, 2000, 500, 500), (200000, 5000, 2048, 1024), (1100, 704, 500, 384),
                                         (600, 2048, 300, 512), (5, 4, 2, 3), (1000, 500, 100, 100)])
def test_an_epoch_of_sweeps_covers_every_entry_once(n, m, nbr, nbc):
    r, s = -(-n // nbr), -(-m // nbc)
    sigma = np.random.default_rng(n + m).permutation(max(r, s))
    assert sum(bench.sweep_entries(n, m, nbr, nbc, int(sg)) for sg in sigma) == n * m


def test_sweep_algorithmic_matches_the_stated_nb_medium_figures():
    """One launch (sweep) of nb_medium: 4 blocks of 500 x 500 = 1.0e6 entries,
    126 flops per entry at d = 10 (K = 15), 5.392 MB of algorithmic bytes (4 B
    per count + factor, EMA and parameter traffic)."""
    w = synth.WORKLOADS["nb_medium"]
    K, fr, fc = 1 + w.p + w.q + w.d, w.q + w.d, w.p + w.d
    ent, flops, byts = bench.sweep_algorithmic(w, K, fr, fc)
    assert ent == 1_000_000
    assert flops == ent * (2 * K + 4 * fr + 4 * fc) == 126_000_000
    assert byts == 5_392_000


def test_host_cpu_names_the_host():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_clock_sampler_without_a_driver_reports_none():
    """No NVML library and no nvidia-smi on a CPU machine: the sampler still starts,
    stops and reports that nothing was sampled (the bench's clocks field)."""
    if os.path.exists("/usr/bin/nvidia-smi") or os.path.exists("/dev/nvidia0"):
        pytest.skip("a GPU driver is present")
    c = bench.ClockSampler(0)
    c.start()
    c.mark(True)
    c.mark(False)
    out = c.stop()
    assert out["sm_mhz"] is None and out["sm_max_mhz"] is None


def test_epoch_algorithmic_matches_the_stated_atlas_figures():
    """One epoch of nb_atlas (200000 x 5000 uint16, d = 20, p = 3, q = 1, 2048 x
    1024 blocks: r = 98, s = 5): 1e9 entries, 226 flops per entry, 2 B per count
    plus 5 visits of every row (4K + 24 fr bytes) and 98 of every column (4K +
    24 fc bytes) = 2.923 GB."""
    w = synth.WORKLOADS["nb_atlas"]
    K, fr, fc = 1 + w.p + w.q + w.d, w.q + w.d, w.p + w.d
    ent, flops, byts = bench.epoch_algorithmic(w.n, w.m, w.nb_row, w.nb_col, K, fr, fc, 2)
    assert ent == 10 ** 9 and flops == 226 * 10 ** 9
    assert byts == 2 * 10 ** 9 + 5 * 200000 * (4 * 25 + 24 * 21) + 98 * 5000 * (4 * 25 + 24 * 23) == 2_923_480_000


def test_epoch_algorithmic_equals_the_sum_of_its_sweeps():
    """The per-epoch bytes equal the sum over an epoch's blocks of the per-block
    traffic (ragged chunks included), so bytes per sweep = bytes per epoch / sweeps."""
    n, m, nbr, nbc, K, fr, fc = 4300, 2100, 2048, 1024, 25, 21, 23
    r, s = -(-n // nbr), -(-m // nbc)
    tot = 0
    for a in range(r):
        for b in range(s):
            nI, mJ = min(nbr, n - a * nbr), min(nbc, m - b * nbc)
            tot += nI * mJ * 2 + nI * (4 * K + 24 * fr) + mJ * (4 * K + 24 * fc)
    assert bench.epoch_algorithmic(n, m, nbr, nbc, K, fr, fc, 2)[2] == tot
