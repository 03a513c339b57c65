"""Host-side checks of the Gram tile-order autotuner: bucketing, the library's tuning table
(first match wins, default 8), and tune() choosing the fastest candidate with a fake timer and
reusing its JSON cache. No GPU is touched."""
import json
import os

import pytest


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2510_08430_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2510_08430_gb300 import build
        build.build()
    yield _lib.load()
    _lib.load().nqs_set_gram_tuning(0, None, None, None)


def test_bucket_rounds_up_to_powers_of_two():
    from paper_2510_08430_gb300.tune import bucket
    assert bucket(6464, 16384) == (8192, 16384)
    assert bucket(4096, 4097) == (4096, 8192)
    assert bucket(1, 1) == (1, 1)


def test_table_first_match_and_default():
    from paper_2510_08430_gb300 import tune
    tune.install({})
    assert tune.group_edge(6464, 16384) == 8
    tune.install({(8192, 16384): 12, (1024, 1 << 20): 2, (1 << 20, 1 << 20): 4})
    assert tune.group_edge(6464, 16384) == 12      # inside the first bucket
    assert tune.group_edge(900, 300000) == 2       # only the small-block bucket matches first
    assert tune.group_edge(20000, 16384) == 4      # larger blocks
    assert tune.group_edge(1 << 21, 1) == 8        # no match: default
    tune.install({})


def test_rejects_bad_entries(lib):
    import ctypes as C
    nb = (C.c_int64 * 1)(100)
    ns = (C.c_int64 * 1)(100)
    g = (C.c_int32 * 1)(0)
    assert lib.nqs_set_gram_tuning(1, nb, ns, g) == -1
    assert lib.nqs_set_gram_tuning(-1, nb, ns, g) == -1


def test_tune_picks_fastest_and_caches(tmp_path):
    from paper_2510_08430_gb300 import tune
    calls = []

    def factory(blocks, n_s, precision):
        def f(G):
            calls.append((tuple(blocks), n_s, G))
            return {1: 5.0, 2: 4.0, 4: 3.0, 8: 2.5, 12: 2.6, 16: 3.5}[G]
        return f

    cache = str(tmp_path / "tune.json")
    shapes = [([6464, 4160, 65], 16384)]
    res = tune.tune(shapes, cache_path=cache, timer_factory=factory, gpu="fake-gpu")
    assert res[(8192, 16384)]["group"] == 8
    assert tune.group_edge(6464, 16384) == 8
    assert len(calls) == len(tune.CANDIDATES)
    data = json.load(open(cache))
    assert data["fake-gpu"]["8192x16384"]["group"] == 8
    # a second call reuses the cache: no timing
    tune.tune(shapes, cache_path=cache, timer_factory=factory, gpu="fake-gpu")
    assert len(calls) == len(tune.CANDIDATES)
    assert tune.load(cache, gpu="fake-gpu") == 1
    tune.install({})
