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


def test_batched_split_tuning(tmp_path, monkeypatch):
    """Coordinate descent over k buckets: the fastest hint per bucket wins,
    short-k and (min,+) problems keep the library's rule, candidates that need
    more workspace than given are skipped, and the choice is cached."""
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    F32, MP = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_MIN_PLUS_I32
    FAKE = 1 << 20
    probs = [(F32, 256, 256, 16384, FAKE, FAKE, FAKE), (F32, 128, 128, 3000, FAKE, FAKE, FAKE),
             (F32, 64, 64, 100, FAKE, FAKE, FAKE), (MP, 64, 64, 5000, FAKE, FAKE, FAKE)]
    assert [b for b, _ in autotune.batch_buckets(probs)] == [16384, 4096]
    budget = mmsr.mm_batched_query(autotune.apply_splits(probs, [8, 16, 0, 0]))
    seen = []
    # pretend the 16384 bucket likes 8 slices and the 4096 bucket 2
    cost = {16384: {0: 9.0, 1: 12.0, 2: 8.0, 4: 7.0, 8: 5.0, 16: 6.0}, 4096: {0: 3.0, 1: 2.5, 2: 1.0, 4: 2.0,
                                                                            8: 2.2, 16: 2.4}}

    def fake_timer(fn):
        sp = fake_timer.current
        seen.append(tuple(sp))
        return cost[16384][sp[0]] + cost[4096][sp[1]]

    real_run = mmsr.mm_batched

    def spy(table, *a, **k):
        fake_timer.current = [t[7] for t in table]
        return 0

    monkeypatch.setattr(mmsr, "mm_batched", spy)

    def timer(fn):
        fn()
        return fake_timer(fn)

    rec = autotune.tune_batched(probs, FAKE, budget, timer=timer)
    assert rec["buckets"] == {"16384": 8, "4096": 2}
    assert rec["splits"] == [8, 2, 0, 0]
    assert all(t[2] == 0 and t[3] == 0 for t in seen)  # untuned problems keep the rule
    # a smaller workspace rules out the widest candidates
    small = mmsr.mm_batched_query(autotune.apply_splits(probs, [4, 16, 0, 0])) - 1
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune2.json"))
    seen.clear()
    rec2 = autotune.tune_batched(probs, FAKE, small, timer=timer)
    assert seen and all(mmsr.mm_batched_query(autotune.apply_splits(probs, t)) <= small for t in seen)
    assert mmsr.mm_batched_query(autotune.apply_splits(probs, rec2["splits"])) <= small
    # cached: no timing on the second call
    seen.clear()
    assert autotune.tune_batched(probs, FAKE, small, timer=timer) == rec2 and not seen
    monkeypatch.setattr(mmsr, "mm_batched", real_run)


def test_batched_strassen_level_tuning(tmp_path, monkeypatch):
    """After the k-slices, the tuner tries one Strassen-Winograd level for the
    large FP32 problems (every dimension >= 1024 and even) and keeps it only if
    the batch gets faster."""
    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    F32 = mmsr.MM_SR_PLUS_TIMES_F32
    FAKE = 1 << 20
    probs = [(F32, 2048, 2048, 2048, FAKE, FAKE, FAKE), (F32, 1024, 1025, 2048, FAKE, FAKE, FAKE),
             (F32, 512, 512, 512, FAKE, FAKE, FAKE)]
    assert autotune.strassen_candidates_in_batch(probs) == [0]
    budget = mmsr.mm_batched_query(autotune.apply_splits(probs, [16, 16, 0], [1, 0, 0]))
    real_run = mmsr.mm_batched
    for faster in (True, False):
        seen = []

        def spy(table, *a, **k):
            seen.append([t[8] for t in table])
            return 0

        monkeypatch.setattr(mmsr, "mm_batched", spy)

        def timer(fn):
            fn()
            lv = seen[-1]
            return 1.0 if (lv[0] == 1) == faster else 2.0

        rec = autotune.tune_batched(probs, FAKE, budget, timer=timer, cache={}, persist=False)
        assert rec["levels"] == ([1, 0, 0] if faster else [0, 0, 0])
        assert any(lv == [1, 0, 0] for lv in seen)
    monkeypatch.setattr(mmsr, "mm_batched", real_run)
