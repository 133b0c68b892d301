"""Control flow of the autotuner (no GPU): the fastest candidate within the
margin wins, the fallback number format is tuned only when no candidate of the
requested one qualifies, and a request nothing reaches raises.  The solver and
its timing are replaced by a fake that reports a chosen time and error per
candidate."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_07021_gb300 import sfmm, tune


class FakeRef:
    def __init__(self, **kw):
        pass

    def deflection(self, src, q, tgt):
        n = tgt.shape[0]
        return torch.ones(n, dtype=torch.float64), torch.ones((n, 2), dtype=torch.float64)

    def close(self):
        pass


def run(monkeypatch, results, precision, stated, fallback=None):
    """results: {(precision, p): (ms, error)} for the candidates tried."""
    calls = []
    monkeypatch.setattr(sfmm, "Plan", FakeRef)

    def fake_tune(src, q, tgt, prec, st, cands, idx, r_psi, r_alpha, repeats, safety, q_f32, table):
        best = None
        for c in cands:
            kw = tune.plan_kwargs(c)
            ms, err = results[(prec, kw["p"])]
            calls.append((prec, kw["p"]))
            row = dict(kw, precision=prec, ms=ms, error=err, ok=err <= safety * st)
            table.append(row)
            if row["ok"] and (best is None or ms < best["ms"]):
                best = row
        return best

    monkeypatch.setattr(tune, "_tune", fake_tune)
    x = torch.zeros((50, 3), dtype=torch.float64)
    cands = {sfmm.SFMM_MIXED: [dict(p=16, leaf_size=64), dict(p=20, leaf_size=64, c_s=1.3)],
             sfmm.SFMM_MIXED_DF: [dict(p=28, leaf_size=64, c_t=0.45)]}
    out = tune.autotune(x, torch.ones(50), x, precision, stated, candidates=cands[precision], sample=10,
                        fallback=fallback, fallback_candidates=cands.get(fallback))
    return out, calls


def test_fastest_within_margin_wins_and_no_fallback_is_run(monkeypatch):
    res = {(sfmm.SFMM_MIXED, 16): (3.0, 4e-7), (sfmm.SFMM_MIXED, 20): (2.5, 4.5e-7),
           (sfmm.SFMM_MIXED_DF, 28): (10.0, 1e-12)}
    out, calls = run(monkeypatch, res, sfmm.SFMM_MIXED, 1e-6, fallback=sfmm.SFMM_MIXED_DF)
    assert out["precision"] == sfmm.SFMM_MIXED and out["best"]["p"] == 20 and out["best"]["c_s"] == 1.3
    assert calls == [(sfmm.SFMM_MIXED, 16), (sfmm.SFMM_MIXED, 20)]


def test_fallback_is_tuned_when_nothing_qualifies(monkeypatch):
    res = {(sfmm.SFMM_MIXED, 16): (3.0, 6e-7), (sfmm.SFMM_MIXED, 20): (2.5, 7e-7),
           (sfmm.SFMM_MIXED_DF, 28): (10.0, 1e-12)}
    out, calls = run(monkeypatch, res, sfmm.SFMM_MIXED, 1e-6, fallback=sfmm.SFMM_MIXED_DF)
    assert out["precision"] == sfmm.SFMM_MIXED_DF and out["best"]["p"] == 28
    assert [r["precision"] for r in out["table"]] == [sfmm.SFMM_MIXED] * 2 + [sfmm.SFMM_MIXED_DF]
    assert np.isclose(out["error"], 1e-12)


def test_nothing_reaches_the_target(monkeypatch):
    res = {(sfmm.SFMM_MIXED, 16): (3.0, 6e-7), (sfmm.SFMM_MIXED, 20): (2.5, 7e-7)}
    with pytest.raises(RuntimeError):
        run(monkeypatch, res, sfmm.SFMM_MIXED, 1e-6)


def test_candidates_take_the_plan_defaults():
    """A candidate that leaves out c_s or c_t runs (and is reported) with the
    defaults of Plan itself, and its own settings win over them."""
    import inspect
    sig = inspect.signature(sfmm.Plan.__init__).parameters
    kw = tune.plan_kwargs(dict(p=20, leaf_size=64))
    assert kw == dict(p=20, leaf_size=64, c_s=sig["c_s"].default, c_t=sig["c_t"].default)
    kw = tune.plan_kwargs(dict(p=16, leaf_size=32, c_s=1.3))
    assert kw["c_s"] == 1.3 and kw["c_t"] == sig["c_t"].default


def test_default_candidate_lists_are_valid():
    """Every default candidate names a known number format's settings within the library's ranges."""
    for prec, cands in tune.DEFAULT_CANDIDATES.items():
        assert prec in (sfmm.SFMM_FP64, sfmm.SFMM_MIXED, sfmm.SFMM_MIXED_DF, sfmm.SFMM_FP32)
        assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)
        for c in cands:
            kw = tune.plan_kwargs(c)
            assert 1 <= kw["p"] <= 32 and kw["leaf_size"] >= 1 and kw["c_s"] > 1 and 0 < kw["c_t"] < 1
