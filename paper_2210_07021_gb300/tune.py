"""Measured choice of the solver settings (leaf size m, MAC constants c_s and
c_t, order p) for a number format and a stated error.

Every candidate is timed on the caller's data (CUDA events, after a warm-up
solve) and its psi and alpha are compared, on a sample of targets, with an FP64
reference solve run with a tighter MAC (c_t = 0.35, p = 32: errors near 1e-13
on clustered skies).  The fastest candidate whose norm-wise relative error is
at most `safety` times the stated error wins.  When none does and a fallback
number format is given (e.g. the all-FP32 path, whose error has a floor near
eps_f32 Q / |alpha| on targets in smooth or empty sky, falling back to the
1e-6 path), the fallback's candidates are tuned the same way.  The result is a
dict of Plan keyword arguments, the chosen number format and the measured table.
"""
import inspect

import numpy as np

from . import sfmm


def _grid(ps, ms, css, cts):
    return [dict(p=p, leaf_size=m, c_s=cs, c_t=ct) for p in ps for m in ms for cs in css for ct in cts]


DEFAULT_CANDIDATES = {
    # the benchmark sky's best settings first, then their neighbours in p, c_s and leaf size
    sfmm.SFMM_MIXED: _grid((20,), (96,), (1.5, 1.3), (0.5,)) + _grid((20,), (64, 80, 128), (1.5,), (0.5,))
                     + _grid((16, 24), (96,), (1.5, 2.0), (0.5,)),
    sfmm.SFMM_FP32: _grid((20,), (64, 48, 80), (1.3,), (0.5,)) + _grid((16,), (32, 64, 96), (2.0,), (0.5,)),
    sfmm.SFMM_MIXED_DF: _grid((28,), (64,), (1.6, 1.7), (0.45,)) + _grid((30, 32), (64, 96), (1.5, 1.6), (0.45,))
                        + _grid((24, 26), (64,), (2.0,), (0.45,)),
    # FP64: the near field (set by c_s and m) dominates, so c_s is varied with p and c_t
    sfmm.SFMM_FP64: _grid((24, 28, 32), (32, 64), (1.3, 1.5, 2.0), (0.45,)) + _grid((28, 32), (32, 64), (2.0,), (0.5,)),
}


_PLAN_PARAMS = inspect.signature(sfmm.Plan.__init__).parameters


def plan_defaults():
    """The MAC constants a Plan uses when a candidate does not set them (read
    from Plan's own signature, so the tuner reports the settings actually run)."""
    return {"c_s": _PLAN_PARAMS["c_s"].default, "c_t": _PLAN_PARAMS["c_t"].default}


def plan_kwargs(candidate):
    """A candidate's full Plan keyword arguments: its own, then the Plan defaults."""
    kw = dict(plan_defaults())
    kw.update(candidate)
    return kw


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def autotune(src, q, tgt, precision, stated, candidates=None, sample=2000, repeats=2, safety=0.5, q_f32=False,
             seed=0, fallback=None, fallback_candidates=None):
    """src, q, tgt: device tensors.  Returns dict(best=Plan kwargs, precision=the number format
    chosen, ms, error, table=[...]); `fallback` (a precision) is tuned when no candidate of
    `precision` reaches `safety` x `stated`."""
    import torch
    M = tgt.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(M, size=min(sample, M), replace=False))
    idx_t = torch.as_tensor(idx, device=tgt.device)
    ref_plan = sfmm.Plan(p=32, leaf_size=32, c_t=0.35, precision=sfmm.SFMM_FP64, q_f32=q_f32)
    r_psi, r_alpha = ref_plan.deflection(src, q, tgt.index_select(0, idx_t).contiguous())
    r_psi, r_alpha = r_psi.cpu().numpy(), r_alpha.cpu().numpy()
    ref_plan.close()
    table = []
    best = None
    runs = [(precision, candidates or DEFAULT_CANDIDATES[precision])]
    if fallback is not None:
        runs.append((fallback, fallback_candidates or DEFAULT_CANDIDATES[fallback]))
    for prec, cands in runs:
        if best is not None:
            break
        best = _tune(src, q, tgt, prec, stated, cands, idx, r_psi, r_alpha, repeats, safety, q_f32, table)
    if best is None:
        raise RuntimeError(f"no candidate reached {safety} x {stated:g}: {table}")
    return dict(best={k: best[k] for k in ("p", "leaf_size", "c_t", "c_s")}, precision=best["precision"],
                ms=best["ms"], error=best["error"], table=table)


def _tune(src, q, tgt, precision, stated, cands, idx, r_psi, r_alpha, repeats, safety, q_f32, table):
    import torch
    best = None
    for c in cands:
        kw = plan_kwargs(c)
        plan = sfmm.Plan(precision=precision, q_f32=q_f32, **kw)
        psi, alpha = plan.deflection(src, q, tgt)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(repeats):
            psi, alpha = plan.deflection(src, q, tgt, psi=psi, alpha=alpha)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / repeats
        err = max(_rel(psi.cpu().numpy()[idx], r_psi), _rel(alpha.cpu().numpy()[idx], r_alpha))
        plan.close()
        row = dict(kw, precision=precision, ms=ms, error=err, ok=err <= safety * stated)
        table.append(row)
        if row["ok"] and (best is None or ms < best["ms"]):
            best = row
    return best
