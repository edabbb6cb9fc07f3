"""Host logic of the autotuner: candidate plans respect the budget, the
fastest candidate wins, and choices round-trip through the JSON cache.
Timing is injected, so nothing runs on a GPU."""
import pytest

from paper_1911_05328_gb300 import autotune, mmsr
from paper_1911_05328_gb300 import build as mmsr_build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mmsr_build.build()


def test_split_candidates_fit_budget_and_are_distinct():
    n = 4096
    budget = 8 * n * n * 4
    cands = autotune.split_candidates(mmsr.MM_SR_MIN_PLUS_I32, n, n, n, budget)
    ss = [s for s, _ in cands]
    assert ss[0] == 1 and 9 in ss and len(set(ss)) == len(ss)
    for s, b in cands:
        assert b <= budget
        assert mmsr.mm_plan_query(mmsr.MM_SR_MIN_PLUS_I32, -1, n, n, n, b).split_k == s


def test_strassen_candidates_respect_shape_and_budget():
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    big = 1 << 40
    assert [L for L, _ in autotune.strassen_candidates(sr, 1024, 1024, 1024, big)] == [0, 1, 2, 3, 4]
    assert [L for L, _ in autotune.strassen_candidates(sr, 96, 96, 96, big)] == [0, 1, 2, 3, 4][:6]  # 96 = 3*32
    assert [L for L, _ in autotune.strassen_candidates(sr, 100, 100, 100, big)] == [0, 1, 2]
    w1 = mmsr.mm_plan_query(sr, 1, 1024, 1024, 1024, 0).workspace_min
    assert [L for L, _ in autotune.strassen_candidates(sr, 1024, 1024, 1024, int(w1))] == [0, 1]


def test_fastest_split_is_chosen_and_cached(tmp_path, monkeypatch):
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 2048
    sr = mmsr.MM_SR_MIN_PLUS_I32
    budget = 4 * n * n * 4
    calls = []

    def fake_timer(fn):
        # pretend s = 3 is fastest: read the budget the tuner is about to pass
        calls.append(1)
        s = fake_timer.order.pop(0)
        return {1: 5.0, 2: 4.0, 3: 3.0, 4: 3.5, 5: 3.8}[s]

    fake_timer.order = [s for s, _ in autotune.split_candidates(sr, n, n, n, budget)]
    best = autotune.tune_semiring(sr, n, n, n, 0, 0, 0, 0, budget, timer=fake_timer)
    assert best["split_k"] == 3 and len(calls) == 5
    # second call hits the cache: no timing
    again = autotune.tune_semiring(sr, n, n, n, 0, 0, 0, 0, budget, timer=None)
    assert again == best
    assert autotune.load_cache()[autotune.key("semiring", sr, n, n, n, budget)]["split_k"] == 3


def test_strassen_depth_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    times = iter([10.0, 8.0, 8.5, 12.0, 20.0])
    best = autotune.tune_strassen(sr, 4096, 4096, 4096, 0, 0, 0, 0, 1 << 40, timer=lambda fn: next(times))
    assert best["levels"] == 1


def test_key_buckets():
    k1 = autotune.key("semiring", 3, 1000, 1000, 1000, 12345)
    k2 = autotune.key("semiring", 3, 1024, 1024, 1024, 16384)
    assert k1 == k2
    assert autotune.key("semiring", 3, 1025, 1024, 1024, 16384) != k2


def test_star_candidates_trade_classic_levels_for_workspace():
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    n = 4096
    big = 1 << 40
    # unlimited budget: pure Strassen at every depth
    assert [(c, L) for c, L, _ in autotune.star_candidates(sr, n, n, n, big)] == [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4)]
    # a budget that holds one level of Strassen only at a quarter of the size
    w = int(mmsr.mm_star_strassen_query(1, 1, sr, n, n, n).workspace_min)
    assert w < int(mmsr.mm_plan_query(sr, 1, n, n, n).workspace_min)
    cands = autotune.star_candidates(sr, n, n, n, w)
    assert all(wc <= w for _, _, wc in cands)
    assert [(c, L) for c, L, _ in cands][0] == (1, 1)
    assert all(c >= 1 for c, L, _ in cands if L >= 1)
    # the classic FP32 product keeps two split copies of A and B (bf16 hi/lo,
    # 8 (m + n) k bytes), more than this budget: the mixed plan is the only
    # plan of depth <= 1 that fits.
    assert int(mmsr.mm_plan_query(sr, -1, n, n, n).workspace_min) > w
    assert (0, 0) not in [(c, L) for c, L, _ in cands]


def test_star_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    n = 4096
    w = int(mmsr.mm_star_strassen_query(1, 2, sr, n, n, n).workspace_min)
    cands = autotune.star_candidates(sr, n, n, n, w)
    times = iter([10.0 - i for i in range(len(cands))])
    best = autotune.tune_star_strassen(sr, n, n, n, 0, 0, 0, 0, w, timer=lambda fn: next(times))
    assert (best["classic"], best["levels"], best["workspace"]) == cands[-1]
