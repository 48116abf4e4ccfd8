"""Host logic of the tuner (coordinate search over N_lim and the direct/FFT thresholds), no GPU."""
from paper_1302_6945_gb300 import tikh


def test_coordinate_search_finds_the_separable_minimum():
    # a separable cost with its minimum inside the search space; no GPU involved
    want = {"n_lim": 24, "prod_direct_max": 72, "eval_direct_max": 40}
    calls = []

    def cost(o):
        calls.append(o)
        return sum(abs((o[k] or 1000) - want[k]) for k in want)

    best, seen = tikh.coordinate_search(cost, {"n_lim": 32, "prod_direct_max": 0, "eval_direct_max": 0})
    assert best == want
    assert len(seen) == len(calls) <= 1 + sum(len(v) for v in tikh.TUNE_SPACE.values())


def test_coordinate_search_keeps_the_start_when_nothing_is_faster():
    start = {"n_lim": 32, "prod_direct_max": 0, "eval_direct_max": 0}
    best, _ = tikh.coordinate_search(lambda o: 0.0 if o == start else 1.0, start)
    assert best == start


def test_coordinate_search_tunes_the_fft_radix_and_tile():
    want = {"n_lim": 32, "prod_direct_max": 0, "eval_direct_max": 0, "fft_radix": 4, "fft_tile": 1024}

    def cost(o):
        return sum(abs((o.get(k) or 0) - want[k]) for k in want)

    best, _ = tikh.coordinate_search(cost, {"n_lim": 32, "prod_direct_max": 0, "eval_direct_max": 0, "fft_radix": 0,
                                            "fft_tile": 0})
    assert best["fft_radix"] == 4 and best["fft_tile"] == 1024
