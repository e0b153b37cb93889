"""Host logic of the autotuner (no GPU): a cached choice is looked up by the context's shape and
applied without timing anything; other shapes miss the cache."""
import json

from paper_2510_00518_gb300.batch import _key, autotune


class _FakeEngine:
    nq = 64

    def __init__(self, n_atoms=4, N=64, precision=1):
        self._info = {"n_atoms": n_atoms, "N": N, "precision": precision}
        self.block_threads = None

    def info(self):
        return dict(self._info)

    def set_block_threads(self, n):
        self.block_threads = n

    def rates(self, *a, **k):                    # must not be reached on a cache hit
        raise AssertionError("timed a cached shape")


def test_cached_choice_is_applied_without_timing(tmp_path):
    e = _FakeEngine()
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({_key(e, 4): 96}))
    assert autotune(e, 300.0, 0.1, 31, [1, 2, 3, 4], cache=str(cache)) == 96
    assert e.block_threads == 96
    assert _key(e, 4) == "na4_N64_p1_nq4"
    assert _key(_FakeEngine(n_atoms=6), 4) != _key(e, 4)
    assert _key(e, 5) != _key(e, 4)
