/* A plain C99 client of the library's C ABI: it includes only include/rf.h
 * and calls, without a GPU, the entry points that need none -- defaults,
 * argument checks, the device query and the ensemble tuner's host model.
 * Prints "OK" and returns 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "rf.h"

static int failures = 0;

static void check(int ok, const char *what)
{
    if (!ok) {
        printf("FAIL: %s (%s)\n", what, rf_last_error());
        failures++;
    }
}

int main(int argc, char **argv)
{
    int expect_no_device = argc > 1 && strcmp(argv[1], "--no-device") == 0;

    rf_solver_params p;
    rf_default_params(&p);
    check(p.tol_picard == 1e-6 && p.tol_cg == 1e-10 && p.n_max == 8 && p.precond == RF_PRECOND_JACOBI &&
              p.precision == RF_PREC_FP64 && p.picard_form == RF_PICARD_CHORD,
          "documented defaults");

    rf_mesh_desc mesh = {4, 3, 5, 1.0, 1.0, 0.5, 0.0, NULL};
    rf_ctx *ctx = (rf_ctx *)&mesh;             /* any non-NULL value: must come back NULL */
    rf_solver_params bad = p;
    bad.f_shrink = 1.0;
    check(rf_mesh_create(&mesh, &bad, NULL, NULL, &ctx) == RF_ERR_ARG && ctx == NULL, "f_shrink = 1 refused");
    bad = p;
    bad.precond = RF_PRECOND_MG;               /* multigrid serves the FP32 inner solve only */
    check(rf_mesh_create(&mesh, &bad, NULL, NULL, &ctx) == RF_ERR_ARG, "multigrid with FP64 refused");
    rf_mesh_desc empty = {0, 3, 5, 1.0, 1.0, 0.5, 0.0, NULL};
    check(rf_mesh_create(&empty, &p, NULL, NULL, &ctx) == RF_ERR_ARG, "empty mesh refused");
    if (expect_no_device) {
        check(rf_mesh_create(&mesh, &p, NULL, NULL, &ctx) == RF_ERR_NO_DEVICE && ctx == NULL,
              "no device, no CPU fallback");
    }

    /* the tuner's model: times 3, 3, 2, 2, 2 heaviest first on two units -> 7 */
    const double wide[5] = {3.0, 3.0, 2.0, 2.0, 2.0};
    const int order[5] = {0, 1, 2, 3, 4};
    double makespan = 0.0;
    check(rf_ens_model_makespan(wide, NULL, order, 5, 5, 2, 1, &makespan) == RF_OK && makespan == 7.0,
          "list-scheduling makespan");
    check(rf_ens_model_makespan(wide, NULL, order, 5, 5, 0, 1, &makespan) == RF_ERR_ARG, "zero units refused");

    if (failures) return 1;
    printf("OK\n");
    return 0;
}
