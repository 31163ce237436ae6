/*
 * A plain C client of liblbm_pf: nothing but include/lbm_pf.h between it and
 * the library.
 *
 *   c_client host
 *       Calls that need no GPU.  Every one must return its documented status
 *       (bad parameters and sizes, NULL handles, workspace sizing); exit 0 when
 *       they all do, 1 otherwise.
 *   c_client run STORAGE IN OUT
 *       IN holds nx, ny (int32) and phi0 (nx*ny doubles, x fastest).  Runs the
 *       static-drop parameters (density ratio 1000, sigma = 0.01, W = 4,
 *       tau = 0.8) from phi0 at rest for 50 steps with storage STORAGE, then
 *       writes phi, rho, ux, uy, p (nx*ny doubles each) and the four lbm_diag
 *       results to OUT.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_pf.h"

static lbm_params drop_params(int storage) {
    lbm_params p;
    memset(&p, 0, sizeof p);
    p.rho_l = 1.0;
    p.rho_g = 1e-3;
    p.nu_l = p.nu_g = 0.1; /* (tau - 1/2) / 3 with tau = 0.8 */
    p.visc_mode = LBM_VISC_LINEAR_NU;
    p.sigma = 0.01;
    p.W = 4.0;
    p.tau_h = 0.8;
    p.bc_y = LBM_BC_PERIODIC;
    p.normal_scheme = LBM_NORMAL_CENTRAL;
    p.storage = storage;
    p.kernel = LBM_KERNEL_AUTO;
    return p;
}

static int failures = 0;

static void expect(const char* what, int got, int want) {
    if (got != want) {
        fprintf(stderr, "%s: got %d, want %d\n", what, got, want);
        ++failures;
    }
}

static int host_checks(void) {
    lbm_params p = drop_params(LBM_STORE_FP32);
    lbm_handle* h = (lbm_handle*)&p; /* must be overwritten with NULL on failure */
    lbm_params bad = p;
    size_t bytes = 0;
    bad.rho_g = 0.0;
    expect("create with rho_g = 0", lbm_create(16, 16, &bad, &h), LBM_ERR_INVALID);
    expect("handle left NULL", h == NULL, 1);
    bad = p;
    bad.tau_h = 0.5;
    expect("create with tau_h = 1/2", lbm_create(16, 16, &bad, &h), LBM_ERR_INVALID);
    expect("create with nx = 0", lbm_create(0, 16, &p, &h), LBM_ERR_INVALID);
    expect("create past the size limit", lbm_create(16384, 6554, &p, &h), LBM_ERR_INVALID);
    expect("create with NULL params", lbm_create(16, 16, NULL, &h), LBM_ERR_INVALID);
    expect("workspace sizing", lbm_workspace_bytes(64, 64, &p, &bytes), LBM_OK);
    expect("workspace holds the FP32 state", bytes >= (size_t)64 * 64 * 152, 1);
    p.storage = LBM_STORE_FP16_SHIFTED;
    {
        size_t b16 = 0;
        expect("workspace sizing, 16-bit", lbm_workspace_bytes(64, 64, &p, &b16), LBM_OK);
        expect("16-bit workspace is smaller", b16 < bytes, 1);
    }
    expect("step on NULL", lbm_step(NULL, 1), LBM_ERR_INVALID);
    expect("init on NULL", lbm_init(NULL, NULL, NULL, NULL, NULL), LBM_ERR_INVALID);
    expect("fields on NULL", lbm_get_fields(NULL, NULL, NULL, NULL, NULL, NULL), LBM_ERR_INVALID);
    expect("state bytes of NULL", (int)lbm_state_bytes(NULL), 0);
    expect("last error of NULL is a string", lbm_last_error(NULL) != NULL, 1);
    lbm_destroy(NULL);
    return failures ? 1 : 0;
}

static int run(int storage, const char* in, const char* out) {
    FILE* f = fopen(in, "rb");
    int dims[2];
    if (!f || fread(dims, sizeof(int), 2, f) != 2) {
        fprintf(stderr, "cannot read %s\n", in);
        return 1;
    }
    const size_t N = (size_t)dims[0] * dims[1];
    double* buf = (double*)malloc(6 * N * sizeof(double));
    if (!buf || fread(buf, sizeof(double), N, f) != N) {
        fprintf(stderr, "short input %s\n", in);
        return 1;
    }
    fclose(f);
    lbm_params p = drop_params(storage);
    lbm_handle* h = NULL;
    double d[4];
    lbm_status rc = lbm_create(dims[0], dims[1], &p, &h);
    if (rc == LBM_OK) rc = lbm_init(h, buf, NULL, NULL, NULL);
    if (rc == LBM_OK) rc = lbm_step(h, 50);
    if (rc == LBM_OK)
        rc = lbm_get_fields(h, buf + N, buf + 2 * N, buf + 3 * N, buf + 4 * N, buf + 5 * N);
    if (rc == LBM_OK) rc = lbm_diag(h, &d[0], &d[1], &d[2], &d[3]);
    if (rc != LBM_OK) {
        fprintf(stderr, "status %d: %s\n", (int)rc, h ? lbm_last_error(h) : "lbm_create failed");
        lbm_destroy(h);
        return 1;
    }
    lbm_destroy(h);
    f = fopen(out, "wb");
    if (!f || fwrite(buf + N, sizeof(double), 5 * N, f) != 5 * N || fwrite(d, sizeof(double), 4, f) != 4) {
        fprintf(stderr, "cannot write %s\n", out);
        return 1;
    }
    fclose(f);
    free(buf);
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 2 && !strcmp(argv[1], "host")) return host_checks();
    if (argc == 5 && !strcmp(argv[1], "run")) return run(atoi(argv[2]), argv[3], argv[4]);
    fprintf(stderr, "usage: %s host | run STORAGE IN OUT\n", argv[0]);
    return 2;
}
