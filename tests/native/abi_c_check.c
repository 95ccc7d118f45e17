/* The C ABI used from plain C (no C++, no Python, no torch): the header
 * compiles as C, the library links, and the entry points that need no GPU
 * behave as include/qbvm.h states -- version, status strings, descriptors
 * rejected on the host before any device work, NULL arguments refused. */
#include <stdio.h>
#include <string.h>

#include "qbvm.h"

static int failures = 0;

static void expect(int cond, const char* what) {
    if (!cond) {
        printf("FAIL: %s\n", what);
        ++failures;
    }
}

static qbvm_desc good_desc(void) {
    qbvm_desc d;
    memset(&d, 0, sizeof d);
    d.dim = 2;
    d.m[0] = 16;
    d.m[1] = 16;
    d.m[2] = 1;
    d.L = 1.0;
    d.T = 0.1;
    d.nt = 16;
    d.form = QBVM_FORM_PQ;
    d.alpha = 1e-3;
    d.precision = QBVM_FP64;
    d.rhs_kind = QBVM_RHS_DELTA;
    d.order = QBVM_ORDER_AUTO;
    return d;
}

int main(void) {
    qbvm_plan_t* plan = NULL;
    qbvm_desc d;
    double x = 0.0;

    expect(qbvm_version() >= 100, "version");
    expect(strcmp(qbvm_strerror(QBVM_OK), "success") == 0, "strerror(OK)");
    expect(strlen(qbvm_strerror(QBVM_ERR_UNSUPPORTED)) > 0, "strerror(UNSUPPORTED)");

    /* invalid descriptors: BAD_ARG, nothing allocated */
    d = good_desc();
    d.dim = 4;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_BAD_ARG && plan == NULL, "dim 4");
    d = good_desc();
    d.nt = 1;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_BAD_ARG, "nt 1");
    d = good_desc();
    d.alpha = 0.0;
    d.delta = 0.0;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_BAD_ARG, "no alpha and no delta");
    d = good_desc();
    d.form = 7;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_BAD_ARG, "form");
    /* sizes the kernels do not implement: UNSUPPORTED */
    d = good_desc();
    d.nt = 2048;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_UNSUPPORTED, "nt 2048");
    d = good_desc();
    d.m[0] = 2049;
    expect(qbvm_plan(&d, &plan) == QBVM_ERR_UNSUPPORTED, "m 2049 in 2D");
    /* NULL arguments */
    expect(qbvm_plan(NULL, &plan) == QBVM_ERR_BAD_ARG, "plan(NULL)");
    expect(qbvm_solve(NULL, &x, &x, 0, NULL) == QBVM_ERR_BAD_ARG, "solve(NULL)");
    expect(qbvm_residual(NULL, &x, &x, &x, NULL) == QBVM_ERR_BAD_ARG, "residual(NULL)");
    expect(qbvm_destroy(NULL) == QBVM_OK, "destroy(NULL) is accepted");
    expect(qbvm_batch_destroy(NULL) == QBVM_OK, "batch_destroy(NULL) is accepted");
    expect(qbvm_sweep_destroy(NULL) == QBVM_OK, "sweep_destroy(NULL) is accepted");
    expect(qbvm_solve_batched(NULL, &x, &x, 0, NULL) == QBVM_ERR_BAD_ARG, "solve_batched(NULL)");
    d = good_desc();
    expect(qbvm_batch_plan(&d, 0, NULL, NULL) == QBVM_ERR_BAD_ARG, "batch_plan(count 0)");
    expect(qbvm_sweep_plan(NULL, NULL) == QBVM_ERR_BAD_ARG, "sweep_plan(NULL)");

    printf("abi c check: %d failures\n", failures);
    return failures ? 1 : 0;
}
