"""Launch autotuner for the fused stage kernel.

Times a few steps per candidate launch form on the live handle (CUDA events
inside the library bracket the stage kernels) and keeps the fastest:
  persistent     0: one CTA per work item; 1: SMs x CTAs-per-SM CTAs loop
                 over the work items
  blocks_per_cta blocks per work item (consecutive blocks in leaf order, which
                 is a space-filling order, so neighbours' halos hit in L2)
  ctas_per_sm    persistent CTAs per SM (0 = the occupancy limit)
  staging        mixed form only: how the stage kernel stages each block's
                 padded stencil in shared memory -- 1 = the same-level face
                 slabs by tensor copies (TMA), 0 = gathered by the threads
                 (the block's own cells come by a tensor copy either way)
The state advances while tuning; callers tune during warm-up.
"""
from . import bats as B

DEFAULT_CANDIDATES = [
    (0, 1, 0),
    (0, 2, 0),
    (0, 4, 0),
    (0, 8, 0),
    (0, 16, 0),
    (1, 1, 0),
    (1, 2, 0),
    (1, 4, 0),
    (1, 8, 0),
    (1, 1, 1),
]
STAGING_LAYOUTS = (1, 0)


def _stagings(solver):
    if getattr(solver, "precision", None) == B.BATS_MIXED and hasattr(solver, "set_staging"):
        return STAGING_LAYOUTS
    return (None,)


def autotune(solver, cfl, steps=2, candidates=None, use_graph=1, stagings=None):
    """Returns ((persistent, blocks_per_cta, ctas_per_sm, staging), table) and
    leaves the solver configured with the best candidate (graph replay on when
    use_graph).  staging is None for handles without the knob (FP64 form)."""
    table = []
    for st in (stagings if stagings is not None else _stagings(solver)):
        if st is not None:
            solver.set_staging(st)
        for cand in candidates or DEFAULT_CANDIDATES:
            solver.set_launch(cand[0], cand[1], cand[2], 0)  # eager launches: per-stage events
            solver.step(1, cfl)
            solver.step(steps, cfl)
            ms = solver.timings()[B.BATS_PHASE_STAGE] / steps
            table.append((tuple(cand) + (st,), ms))
    best = min(table, key=lambda r: r[1])[0]
    if best[3] is not None:
        solver.set_staging(best[3])
    solver.set_launch(best[0], best[1], best[2], use_graph)
    return best, table
