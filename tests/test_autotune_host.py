"""Host logic of the autotuner's table (no GPU): which shapes apply() installs."""
import json

from paper_2211_12265_gb300 import autotune, dil


class FakeCtx:
    handle = 1234

    def __init__(self):
        self.calls = []

    def set_tuning(self, op, warps_per_cta, warps_per_task, level):
        self.calls.append((op, warps_per_cta, warps_per_task, level))


def _table(with_mixed=True):
    t = {"plain": {"2": {"sign": {"warps_per_cta": 2, "warps_per_task": 1},
                         "verify": {"warps_per_cta": 4, "warps_per_task": 1}},
                   "5": {"keygen": {"warps_per_cta": 8, "warps_per_task": 2}}},
         "persistent": {"2": {"warps_per_cta": 8, "warps_per_task": 1, "ctas_per_sm": 0, "chunk": 1,
                              "speculation": 8},
                        "5": {"warps_per_cta": 8, "warps_per_task": 2, "ctas_per_sm": 0, "chunk": 1,
                              "speculation": 4}}}
    if with_mixed:
        t["persistent"]["mixed"] = {"warps_per_cta": 4, "warps_per_task": 1, "ctas_per_sm": 0, "chunk": 2,
                                    "speculation": 4}
    return t


def _apply(monkeypatch, table, **kw):
    got = []
    monkeypatch.setattr(dil, "dil_set_persistent_tuning", lambda h, *shape: got.append((h, shape)))
    ctx = FakeCtx()
    autotune.apply(ctx, table, **kw)
    return ctx.calls, got


def test_plain_shapes_installed_per_level(monkeypatch):
    calls, _ = _apply(monkeypatch, _table())
    assert sorted(calls) == sorted([(1, 2, 1, 2), (2, 4, 1, 2), (0, 8, 2, 5)])


def test_persistent_choice(monkeypatch):
    _, got = _apply(monkeypatch, _table(), persistent_level=2)
    assert got == [(1234, (8, 1, 0, 1, 8))]
    _, got = _apply(monkeypatch, _table())                    # default: the mixed-launch shape
    assert got == [(1234, (4, 1, 0, 2, 4))]
    _, got = _apply(monkeypatch, _table(), persistent_level="mixed")
    assert got == [(1234, (4, 1, 0, 2, 4))]
    _, got = _apply(monkeypatch, _table(with_mixed=False))    # fallback: the slowest level
    assert got == [(1234, (8, 2, 0, 1, 4))]
    _, got = _apply(monkeypatch, _table(with_mixed=False), persistent_level=3)   # untuned level
    assert got == [(1234, (8, 2, 0, 1, 4))]


def test_committed_table_is_complete():
    t = autotune.load()
    assert t is not None
    for level in ("2", "3", "5"):
        assert set(t["plain"][level]) == {"keygen", "sign", "verify"}
        for v in t["plain"][level].values():
            assert v["warps_per_cta"] % v["warps_per_task"] == 0 and v["warps_per_task"] in (1, 2, 4)
        p = t["persistent"][level]
        assert p["warps_per_cta"] % p["warps_per_task"] == 0 and p["chunk"] >= 1
    json.dumps(t)
