/* The C ABI from plain C (no Python, no torch): host-only entry points of
 * libkl called through include/kl.h.  Prints one line per check and returns
 * non-zero on the first failure. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "kl.h"

#define CHECK(cond, what)                                                    \
    do {                                                                     \
        if (!(cond)) {                                                       \
            printf("FAIL %s: %s\n", what, kl_last_error());                  \
            return 1;                                                        \
        }                                                                    \
        printf("ok %s\n", what);                                             \
    } while (0)

int main(int argc, char **argv)
{
    const char *dir = argc > 1 ? argv[1] : ".";
    char buf[4096], path[1024];
    CHECK(strstr(kl_version(), "sm_103a") != NULL, "version");

    int64_t sj, sk, origin, extent;
    CHECK(kl_layout(256, 256, 256, 3, KL_F32, &sj, &sk, &origin, &extent) == KL_OK &&
              sj % 32 == 0 && origin % 32 == 0 && extent == sk * 262,
          "layout");

    kl_op op = {5, 1, KL_F32, 0, 0};
    CHECK(kl_config_normalize(&op, "default", buf, sizeof buf) == KL_OK &&
              strncmp(buf, "direct:bx=256,", 14) == 0,
          "config_normalize");
    CHECK(kl_config_normalize(&op, "direct:bx=512", buf, sizeof buf) == KL_ERR_INVALID_ARG,
          "config_reject");
    int64_t n = 0;
    CHECK(kl_space_size(&op, 0, &n) == KL_OK && n > 7000000, "space_size");

    snprintf(path, sizeof path, "%s/c.wisdom", dir);
    remove(path);
    CHECK(kl_wisdom_append(path, "GPU C", 10, 3, 1, 64, 64, 64, "direct:bx=64", 1.0, "") == KL_OK,
          "wisdom_append");
    int32_t rule = 0;
    CHECK(kl_wisdom_select(path, "GPU C", 10, 3, 1, 70, 64, 64, buf, sizeof buf, &rule) == KL_OK &&
              rule == 2 && strcmp(buf, "direct:bx=64") == 0,
          "wisdom_select");

    double X[3] = {0.0, 0.5, 1.0}, y[3] = {1.0, 0.0, 1.0}, q[1] = {0.5}, m, v, ls;
    CHECK(kl_bo_posterior(3, 1, X, y, 1, q, 0.3, 1e-10, &m, &v, &ls) == KL_OK &&
              fabs(m) < 1e-6 && v < 1e-8,
          "bo_posterior");
    double C[2] = {0.25, 0.75}, ei[2];
    int32_t choice = -1;
    CHECK(kl_bo_suggest(3, 1, X, y, 0, NULL, 2, C, 0.0, 0.0, 0.0, &choice, ei) == KL_OK &&
              choice >= 0 && choice < 2,
          "bo_suggest");

    int64_t pts[4] = {7, 5, 4, 2};
    int32_t own[4], cnt = 0;
    int64_t load = 0;
    CHECK(kl_batch_shard(4, pts, 2, 0, own, &cnt, &load) == KL_OK && cnt == 2 && load == 9 &&
              own[0] == 0 && own[1] == 3,
          "batch_shard");

    kl_def *d = NULL;
    CHECK(kl_def_create(&d, "twice", "extern \"C\" __global__ void k(float *x) {}", "k") == KL_OK,
          "def_create");
    int64_t vals[3] = {64, 128, 256};
    const char *block[3] = {"B", NULL, NULL}, *grid[3] = {"div_ceil(problem_x, B)", NULL, NULL};
    CHECK(kl_def_param(d, "B", 3, vals, 128) == KL_OK && kl_def_restrict(d, "B >= 128") == KL_OK &&
              kl_def_geometry(d, block, grid, "B * 4") == KL_OK,
          "def_build");
    int64_t raw = 0, valid = 0, prob[3] = {1000, 1, 1}, geo[7];
    CHECK(kl_def_space_size(d, &raw, &valid) == KL_OK && raw == 3 && valid == 2, "def_space");
    CHECK(kl_def_launch_geometry(d, "B=256", prob, geo) == KL_OK && geo[0] == 256 && geo[3] == 4 &&
              geo[6] == 1024,
          "def_geometry");
    CHECK(kl_def_normalize(d, "B=64", buf, sizeof buf) == KL_ERR_INVALID_ARG, "def_restriction");
    kl_def_destroy(d);
    printf("all ok\n");
    return 0;
}
