/* A plain C (C11) consumer of include/ifgf.h: builds a Fejer-weighted sphere point
 * set, sizes its plan with ifgf_plan_dry_run (host only, no GPU) and prints the
 * plan statistics as one line; then checks two error paths.  Compiled and run by
 * tests/test_c_consumer.py against the in-tree libifgf.so. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "ifgf.h"

int main(int argc, char **argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 24; /* points per cube-face side */
    const double k = argc > 2 ? atof(argv[2]) : 6.283185307179586;
    const int64_t N = 6LL * n * n;
    double *x = malloc(sizeof(double) * 3 * N), *nu = malloc(sizeof(double) * 3 * N), *w = malloc(sizeof(double) * N);
    int64_t i = 0;
    const double pi = 3.14159265358979323846;
    for (int f = 0; f < 6; f++)
        for (int a = 0; a < n; a++)
            for (int b = 0; b < n; b++, i++) {
                /* equiangular face point (tan(pi u / 4), tan(pi v / 4), +-1), projected on the unit sphere */
                const double u = -1.0 + (2.0 * a + 1.0) / n, v = -1.0 + (2.0 * b + 1.0) / n;
                const double X = tan(pi * u / 4.0), Y = tan(pi * v / 4.0), s = (f % 2) ? -1.0 : 1.0;
                double p[3];
                const int ax = f / 2;
                p[ax] = s;
                p[(ax + 1) % 3] = X;
                p[(ax + 2) % 3] = s * Y;
                const double r = sqrt(1.0 + X * X + Y * Y);
                for (int c = 0; c < 3; c++) x[3 * i + c] = nu[3 * i + c] = p[c] / r;
                /* area element of the projection times the midpoint weight (2/n)^2 */
                w[i] = (pi / 4.0) * (pi / 4.0) * (1.0 + X * X) * (1.0 + Y * Y) / (r * r * r) * (4.0 / ((double)n * n));
            }
    ifgf_params prm;
    ifgf_params_default(&prm, k);
    ifgf_info info;
    ifgf_status st = ifgf_plan_dry_run(x, nu, w, N, &prm, &info);
    if (st != IFGF_OK) {
        printf("error %d %s\n", (int)st, ifgf_last_error());
        return 1;
    }
    long long nrc = 0;
    for (int d = 0; d <= info.D; d++) nrc += info.nrc[d];
    printf("N=%lld D=%d nrc=%lld leaf_evals=%lld near_pairs=%lld orders=%s\n", (long long)info.N, info.D, nrc,
           (long long)info.leaf_evals, (long long)info.near_pairs, ifgf_supported_orders());
    /* error paths: no points; a non-unit normal */
    st = ifgf_plan_dry_run(x, nu, w, 0, &prm, &info);
    printf("N=0 -> %d (%s)\n", (int)st, ifgf_last_error());
    nu[0] *= 2.0;
    st = ifgf_plan_dry_run(x, nu, w, N, &prm, &info);
    printf("bad normal -> %d (%s)\n", (int)st, ifgf_last_error());
    free(x);
    free(nu);
    free(w);
    return 0;
}
