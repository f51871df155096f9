/* Minimal C use of the library: a transmission solve on an octahedron (the same grid
 * inside and out), one plane wave, both precisions; prints the iteration counts and the
 * first exterior trace value.  Build (after the library is built in-tree):
 *
 *   gcc -std=c11 -O2 solve_octahedron.c -I../../include -L.. -lbem -Wl,-rpath,'$ORIGIN/..' -o solve_octahedron
 *
 * Runs on a GPU with the library's requirements (sm_103a). */
#include <stdio.h>
#include <stdlib.h>

#include "bem.h"

static int check(bem_status s, const char* what) {
    if (s != BEM_OK && s != BEM_E_NOT_CONVERGED) {
        fprintf(stderr, "%s failed (%d): %s\n", what, (int)s, bem_last_error());
        return 1;
    }
    return 0;
}

int main(void) {
    /* octahedron, triangles counter-clockwise seen from outside */
    const double xyz[6 * 3] = {1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1};
    const int32_t tri[8 * 3] = {0, 2, 4, 2, 1, 4, 1, 3, 4, 3, 0, 4, 2, 0, 5, 1, 2, 5, 3, 1, 5, 0, 3, 5};
    bem_context* ctx = NULL;
    bem_grid *ext = NULL, *intr = NULL;
    if (check(bem_context_create(0, NULL, &ctx), "bem_context_create")) return 1;
    if (check(bem_grid_create(ctx, xyz, 6, tri, 8, 0, &ext), "bem_grid_create") ||
        check(bem_grid_create(ctx, xyz, 6, tri, 8, 0, &intr), "bem_grid_create"))
        return 1;
    const double dir[3] = {0.0, 0.0, 1.0};
    bem_incident inc = {1, dir, NULL};
    bem_c128 v_ext[6], w_ext[6], v_int[6], w_int[6];
    const bem_c128 k_ext = {1.0, 0.0}, k_int = {2.0, 0.0};
    for (int precision = BEM_PREC_FP64; precision <= BEM_PREC_MIXED; ++precision) {
        bem_solve_opts opts;
        bem_solve_opts_default(&opts);
        opts.precision = precision;
        bem_solve_report rep;
        if (check(bem_solve_transmission(ctx, ext, intr, k_int, k_ext, 1.0, &inc, &opts, v_ext, w_ext, v_int, w_int,
                                         0, &rep),
                  "bem_solve_transmission"))
            return 1;
        printf("precision %d: %d iterations, residual %.2e, v_ext[0] = %.6f%+.6fi\n", precision, rep.iterations,
               rep.residual, v_ext[0].re, v_ext[0].im);
    }
    bem_grid_destroy(ext);
    bem_grid_destroy(intr);
    bem_context_destroy(ctx);
    return 0;
}
