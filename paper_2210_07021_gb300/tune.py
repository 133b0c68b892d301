"""Measured choice of the solver settings (leaf size m, MAC constants c_s and
c_t, order p) for a number format and a stated error.

Every candidate is timed on the caller's data (CUDA events, after a warm-up
solve) and its psi and alpha are compared, on a sample of targets, with an FP64
reference solve run with a tighter MAC (c_t = 0.35, p = 32: errors near 1e-13
on clustered skies).  The fastest candidate whose norm-wise relative error is
at most `safety` times the stated error wins.  When none does and a fallback
number format is given (the FP32 path cannot reach 1e-6 where the deflection
is small next to eps_f32 times the far mass, e.g. targets in empty sky), the
fallback's candidates are tuned the same way.  The result is a dict of Plan
keyword arguments, the chosen number format and the measured table.
"""
import numpy as np

from . import sfmm

DEFAULT_CANDIDATES = {
    # the benchmark sky's best settings and their neighbours, then smaller leaves and the
    # default MAC (on skies whose error is set by the FP32 far field, e.g. 6e-7 at every
    # setting above, the smaller leaves can land below the tuning margin)
    sfmm.SFMM_MIXED: [dict(p=p, leaf_size=m, c_s=cs, c_t=0.5)
                      for p, m, cs in ((20, 64, 1.3), (20, 48, 1.3), (20, 80, 1.3), (20, 64, 1.5), (24, 64, 1.3),
                                       (20, 32, 1.3), (16, 32, 2.0), (16, 48, 2.0), (16, 64, 2.0), (16, 96, 2.0))]
                     + [dict(p=14, leaf_size=64, c_s=2.0, c_t=0.45)],
    sfmm.SFMM_MIXED_DF: [dict(p=p, leaf_size=m, c_t=ct) for p, ct in ((24, 0.4), (26, 0.45), (28, 0.5))
                         for m in (48, 64, 96)],
    sfmm.SFMM_FP64: [dict(p=p, leaf_size=m, c_t=ct) for p, ct in ((28, 0.45), (32, 0.5)) for m in (16, 32, 64)],
}


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
        kw = dict(c)
        kw.setdefault("c_s", 2.0)                 # the library's default MAC constants
        kw.setdefault("c_t", 0.5)
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
