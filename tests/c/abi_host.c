/* Host-only use of the C ABI from C99 (no device call): plan creation and
 * validation, grids, exact phase constants, sharding, status strings.
 * Prints "ok" and returns 0 on success. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "lct.h"

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            return 1;                                                 \
        }                                                             \
    } while (0)

int main(void) {
    const double pi = 3.14159265358979323846;
    lct_plan p = NULL;
    /* a rotation: a = d = cos t, b = -c = sin t */
    const double t = 0.7;
    CHECK(lct_plan_create(&p, 256, cos(t), sin(t), -sin(t), cos(t), LCT_C128) == LCT_OK);
    double y[512], rho[256], x[256];
    CHECK(lct_output_grid(p, 0, y, rho) == LCT_OK);
    CHECK(lct_input_grid(256, x) == LCT_OK);
    for (int j = 0; j < 256; ++j) {
        /* y_j = 4 b x_j / pi, real, rho = 0 for real parameters */
        CHECK(fabs(y[2 * j] - 4.0 * sin(t) * x[j] / pi) <= 1e-12 * (1.0 + fabs(y[2 * j])));
        CHECK(y[2 * j + 1] == 0.0 && rho[j] == 0.0);
    }
    uint64_t turns[5];
    CHECK(lct_plan_phase_turns(p, 0, turns) == LCT_OK);
    CHECK(lct_plan_destroy(p) == LCT_OK);

    /* validation errors are status codes */
    CHECK(lct_plan_create(&p, 9000, 1.0, 2.0, 0.5, 2.0, LCT_C64) == LCT_ERR_N);   /* not a power of two, above 8192 */
    CHECK(lct_plan_create(&p, 64, 1.0, 2.0, 0.6, 2.0, LCT_C64) == LCT_ERR_NOT_SYMPLECTIC);
    CHECK(strcmp(lct_status_string(LCT_OK), "ok") == 0);

    /* sharding: every signal owned once, loads add up */
    const int64_t N[5] = {4096, 64, 65536, 1024, 16};
    int32_t owner[5];
    double load[2];
    CHECK(lct_partition(5, N, NULL, 2, owner, load) == LCT_OK);
    double total = 0.0, expect = 0.0;
    for (int s = 0; s < 5; ++s) {
        CHECK(owner[s] == 0 || owner[s] == 1);
        expect += (double)N[s] * log2((double)N[s]);
    }
    total = load[0] + load[1];
    CHECK(fabs(total - expect) <= 1e-9 * expect);
    printf("ok\n");
    return 0;
}
