/*
 * A plain C consumer of the solver library (include/lskum.h): reads a cloud
 * from raw binary files, solves 20 pseudo-time iterations at M 0.63, alpha
 * 2 deg, and prints the residue, Cl, Cd and the first state entries. Used by
 * the tests to exercise the ABI without Python.
 *
 *   solve_from_files DIR      (DIR/n.bin int64, xy.bin, normals.bin (n x 2
 *                              double), flags.bin (n int8), off.bin (n + 1
 *                              int32), idx.bin (int32))
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lskum.h"

static void* read_all(const char* dir, const char* name, size_t* bytes) {
    char path[4096];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE* f = fopen(path, "rb");
    if (!f) return NULL;
    fseek(f, 0, SEEK_END);
    long len = ftell(f);
    fseek(f, 0, SEEK_SET);
    void* buf = malloc(len > 0 ? (size_t)len : 1);
    if (buf && len > 0 && fread(buf, 1, (size_t)len, f) != (size_t)len) {
        free(buf);
        buf = NULL;
    }
    fclose(f);
    if (bytes) *bytes = (size_t)len;
    return buf;
}

int main(int argc, char** argv) {
    if (argc != 2) {
        fprintf(stderr, "usage: %s DIR\n", argv[0]);
        return 2;
    }
    size_t b = 0;
    int64_t* np = (int64_t*)read_all(argv[1], "n.bin", &b);
    double* xy = (double*)read_all(argv[1], "xy.bin", NULL);
    double* nrm = (double*)read_all(argv[1], "normals.bin", NULL);
    int8_t* flags = (int8_t*)read_all(argv[1], "flags.bin", NULL);
    int32_t* off = (int32_t*)read_all(argv[1], "off.bin", NULL);
    int32_t* idx = (int32_t*)read_all(argv[1], "idx.bin", NULL);
    if (!np || b != sizeof(int64_t) || !xy || !nrm || !flags || !off || !idx) {
        fprintf(stderr, "cannot read the cloud files\n");
        return 2;
    }
    const int64_t n = *np;
    lskum_options o;
    lskum_default_options(&o);
    lskum_ctx* ctx = NULL;
    int rc = lskum_create(n, xy, nrm, flags, off, idx, &o, &ctx);
    if (rc != LSKUM_OK) {
        printf("create %d %s\n", rc, lskum_last_error());
        return 3;
    }
    double res = 0.0, cl = 0.0, cd = 0.0;
    double* prim = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    if (!prim) return 2;
    if ((rc = lskum_set_freestream(ctx, 0.63, 2.0)) != LSKUM_OK ||
        (rc = lskum_step(ctx, 20)) != LSKUM_OK ||
        (rc = lskum_residual_norm(ctx, &res)) != LSKUM_OK ||
        (rc = lskum_forces(ctx, &cl, &cd)) != LSKUM_OK ||
        (rc = lskum_get_state(ctx, prim)) != LSKUM_OK) {
        printf("solve %d %s\n", rc, lskum_last_error());
        lskum_destroy(ctx);
        return 4;
    }
    printf("ok %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", res, cl, cd, prim[0], prim[1], prim[2],
           prim[3]);
    lskum_destroy(ctx);
    free(prim);
    free(np);
    free(xy);
    free(nrm);
    free(flags);
    free(off);
    free(idx);
    return 0;
}
