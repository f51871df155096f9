"""Small, self-contained cases of the library's kernels for profiling
(e.g. under Nsight Compute): one assembly, one mortar or one transmission solve
on synthetic icosphere grids.

    python -m paper_2206_00708_gb300.profile_case assemble --level 4 --k 10
    python -m paper_2206_00708_gb300.profile_case solve --level 4 --k 10
    python -m paper_2206_00708_gb300.profile_case solve --level 5 --level-int 4 --mixed
    python -m paper_2206_00708_gb300.profile_case solve --level 4 --mixed --rhs 64
    python -m paper_2206_00708_gb300.profile_case mortar --level 4
    python -m paper_2206_00708_gb300.profile_case solve --level 4 --mixed --formulation 5
    python -m paper_2206_00708_gb300.profile_case screen --screen 60 --k 20 --mixed
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["assemble", "solve", "mortar", "screen"])
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--level-int", type=int, default=None, help="interior grid level (default: --level)")
    ap.add_argument("--k", type=float, default=10.0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--mixed", action="store_true", help="BEM_PREC_MIXED instead of FP64")
    ap.add_argument("--rhs", type=int, default=1, help="plane waves in the solve (batched)")
    ap.add_argument("--formulation", type=int, default=0, help="bem_solve_opts.formulation (BEM_FORM_*)")
    ap.add_argument("--screen", type=int, default=60, help="screen case: cells per side of the fine grid")
    a = ap.parse_args(argv)
    import bem_inputs as bi
    import paper_2206_00708_gb300 as bem

    ctx = bem.bem_context_create(0)
    li = a.level if a.level_int is None else a.level_int
    ve, te, vi, ti = bi.transmission_pair(a.level, li, seed=2)
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    for _ in range(a.repeat):
        if a.case == "assemble":
            m = bem.bem_assemble(ctx, bem.BEM_OP_V, a.k, ge,
                                 precision=bem.BEM_PREC_MIXED if a.mixed else bem.BEM_PREC_FP64)
            bem.bem_context_synchronize(ctx)
            bem.bem_matrix_destroy(m)
        elif a.case == "mortar":
            s = bem.bem_projection(ctx, gi, ge)
            bem.bem_sparse_destroy(s)
        elif a.case == "screen":
            vs, ts = bi.screen_grid(a.screen, a.screen, jitter=0.2, seed=71)
            vc, tc = bi.screen_grid(max(2, a.screen // 3), max(2, a.screen // 3), jitter=0.2, seed=72)
            gs, gc = bem.bem_grid_create(ctx, vs, ts), bem.bem_grid_create(ctx, vc, tc)
            _, rep = bem.bem_solve_screen(ctx, gs, a.k, np.array([[1.0, 0.0, 0.0]]), coarse=gc,
                                          precond=bem.BEM_SCREEN_OO, opts={"precision": 1 if a.mixed else 0})
            bem.bem_grid_destroy(gs)
            bem.bem_grid_destroy(gc)
            print("iterations", rep["iterations"])
        else:
            dirs = np.array([[0.0, 0.0, 1.0]]) if a.rhs == 1 else bi.plane_wave_directions(a.rhs, seed=40)
            out, rep = bem.bem_solve_transmission(ctx, ge, gi, 1.5 * a.k, a.k, 2.0, dirs,
                                                  opts={"precision": 1 if a.mixed else 0,
                                                        "formulation": a.formulation})
            print("iterations", rep["iterations"])
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    bem.bem_context_destroy(ctx)
    print("ok")


if __name__ == "__main__":
    main()
