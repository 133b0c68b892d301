"""Measured choice of the solver settings (leaf size m, MAC constant c_t,
order p) for a number format and a stated error.

Every candidate is timed on the caller's data (CUDA events, after a warm-up
solve) and its psi and alpha are compared, on a sample of targets, with an FP64
reference solve run with a tighter MAC (c_t = 0.35, p = 32: errors near 1e-13
on clustered skies).  The fastest candidate whose norm-wise relative error is
at most `safety` times the stated error wins.  The result is a dict of Plan
keyword arguments plus the measured table.
"""
import numpy as np

from . import sfmm

DEFAULT_CANDIDATES = {
    sfmm.SFMM_MIXED: [dict(p=16, leaf_size=m, c_t=0.5) for m in (32, 48, 64, 96)] + [dict(p=14, leaf_size=64, c_t=0.45)],
    sfmm.SFMM_MIXED_DF: [dict(p=p, leaf_size=m, c_t=ct) for p, ct in ((24, 0.4), (26, 0.45), (28, 0.5))
                         for m in (48, 64, 96)],
    sfmm.SFMM_FP64: [dict(p=p, leaf_size=m, c_t=ct) for p, ct in ((28, 0.45), (32, 0.5)) for m in (16, 32, 64)],
}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def autotune(src, q, tgt, precision, stated, candidates=None, sample=2000, repeats=2, safety=0.5, q_f32=False,
             seed=0):
    """src, q, tgt: device tensors.  Returns dict(best=Plan kwargs, table=[...])."""
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
    for c in (candidates or DEFAULT_CANDIDATES[precision]):
        kw = dict(c)
        kw.setdefault("c_s", 2.0)
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
        row = dict(kw, ms=ms, error=err, ok=err <= safety * stated)
        table.append(row)
        if row["ok"] and (best is None or ms < best["ms"]):
            best = row
    if best is None:
        raise RuntimeError(f"no candidate reached {safety} x {stated:g}: {table}")
    return dict(best={k: best[k] for k in ("p", "leaf_size", "c_t", "c_s")}, ms=best["ms"], error=best["error"],
                table=table)
