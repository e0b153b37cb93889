"""Pins of the oracle's four-phonon sampling estimate (no GPU).

The paper names combining the GPU with sampling estimation as future work (Results section)
without stating the scheme; the reading here: each partner pair (λ, q', q'') enters the sums with
probability f, decided by SplitMix64's output function on a counter, and the sums are scaled by
2^64 / threshold.  The pins: the hash against the published SplitMix64 outputs, the sampled
process list against a pair-by-pair filter of the full list, the inclusion rate, and the
estimate's mean over seeds against the exact rates (unbiasedness) within its standard error."""
import math

import numpy as np
import pytest

import oracle
from synth import morse_system

M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def _mix_py(z):
    """SplitMix64's output function, written from its published definition (independent of C)."""
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & M64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & M64
    return z ^ (z >> 31)


def test_hash_matches_published_splitmix64_outputs():
    # the generator's first three outputs from state 0 (state advances by the golden gamma)
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for k, v in enumerate(published, start=1):
        assert oracle.splitmix64_mix(k * GOLDEN_GAMMA & M64) == v
        assert _mix_py(k * GOLDEN_GAMMA & M64) == v


@pytest.fixture(scope="module")
def prob():
    return oracle.Problem(*morse_system(seed=0), (3, 3, 3))


def _sampled(seed, thr, m0, q1, q2, nq):
    key = (m0 * nq + q1) * nq + q2
    return _mix_py((seed + (key + 1) * GOLDEN_GAMMA) & M64) < thr


@pytest.mark.parametrize("ch", [2, 3, 4])
def test_sampled_list_is_the_full_list_filtered_by_pair(prob, ch):
    f, seed = 0.3, 12345
    ps = prob.with_sampling(f, seed)
    _, thr = oracle.sample_threshold(f)
    nq, nb = prob.nq, prob.nb
    n_full = n_keep = 0
    for m0 in sorted(set(range(3, nq * nb, 7)) | {9, 21, 27, 81}):   # -- lives on the optical j = 3
        full = prob.processes(ch, m0)
        keep = [w for w in full.tolist()
                if _sampled(seed, thr, m0, oracle.decode4(w, nb, nq)[0], oracle.decode4(w, nb, nq)[2], nq)]
        got = ps.processes(ch, m0)
        assert got.tolist() == keep
        n_full += len(full)
        n_keep += len(keep)
    assert 0 < n_keep < n_full


def test_f_one_takes_every_pair(prob):
    g0, wp0, c0 = prob.rates([7, 40, 101], channel_mask=0b11100)
    g1, wp1, c1 = prob.with_sampling(1.0, 99).rates([7, 40, 101], channel_mask=0b11100)
    assert np.array_equal(c0, c1) and np.array_equal(g0, g1) and np.array_equal(wp0, wp1)


def test_inclusion_rate(prob):
    f, seed = 0.25, 7
    _, thr = oracle.sample_threshold(f)
    nq = prob.nq
    n = sum(_sampled(seed, thr, m0, q1, q2, nq) for m0 in range(6, 30) for q1 in range(nq) for q2 in range(nq))
    total = 24 * nq * nq
    assert abs(n - f * total) <= 5 * math.sqrt(total * f * (1 - f))


def test_estimate_is_unbiased(prob):
    """Mean of the sampled +- rate over 120 seeds against the exact rate, within 4.5 standard
    errors of the mean (the spread measured from the same samples)."""
    modes = [40, 101]
    exact = prob.rates(modes, channel_mask=0b01000)[0][3]
    ests = np.array([prob.with_sampling(0.5, s).rates(modes, channel_mask=0b01000)[0][3] for s in range(120)])
    mean, sem = ests.mean(axis=0), ests.std(axis=0, ddof=1) / math.sqrt(len(ests))
    assert np.all(sem > 0)
    assert np.all(np.abs(mean - exact) <= 4.5 * sem), (mean, exact, sem)
    # and a plausible spread: far below the value itself at f = 0.5 on this mesh
    assert np.all(ests.std(axis=0) < exact)
