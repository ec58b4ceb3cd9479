/*
 * A plain C client of the library (no Python, no PyTorch): one neo-Hookean cube environment,
 * two recorded control steps from host buffers, the state read back, and the reverse pass of
 * a loss sum(x_final) back to the initial positions.  Prints "x_sum xb0_sum" on success.
 * Built and run by tests/test_c_abi.py, which compares the numbers with the Python binding.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mpm.h"

#define N 512

static int check(mpm_status s, mpm_ctx* ctx, const char* what)
{
    if (s != MPM_OK) {
        fprintf(stderr, "%s failed: status %d: %s\n", what, (int)s, ctx ? mpm_last_error(ctx) : "");
        return 1;
    }
    return 0;
}

int main(void)
{
    mpm_env_spec spec;
    memset(&spec, 0, sizeof spec);
    spec.n_particles = N;
    spec.grid_res = 32;
    spec.substeps = 5;
    spec.bound = 3;
    spec.material = MPM_MAT_NEOHOOKEAN;
    spec.collider = MPM_COLL_NONE;
    spec.reward = MPM_REWARD_NONE;
    spec.n_sub = N;
    spec.dt = 1e-4f;
    spec.gravity[2] = -9.8f;
    spec.E = 1e4f;
    spec.nu = 0.3f;
    spec.rho = 1e3f;
    spec.p_vol = 0.008f / N;
    spec.alpha = 666.0f;

    mpm_options opt;
    memset(&opt, 0, sizeof opt);
    opt.max_steps = 2;
    opt.use_graphs = 1;

    static float x[N * 3], v[N * 3], C[N * 9], F[N * 9], xf[N * 3], xb[N * 3], xb0[N * 3];
    for (int p = 0; p < N; p++) {
        int i = p % 8, j = (p / 8) % 8, k = p / 64;
        x[3 * p] = 0.4f + 0.025f * (i + 0.5f);
        x[3 * p + 1] = 0.4f + 0.025f * (j + 0.5f);
        x[3 * p + 2] = 0.4f + 0.025f * (k + 0.5f);
        v[3 * p] = 0.1f;
        v[3 * p + 1] = 0.0f;
        v[3 * p + 2] = -0.05f;
        for (int q = 0; q < 9; q++) {
            C[9 * p + q] = 0.0f;
            F[9 * p + q] = (q % 4 == 0) ? 1.0f : 0.0f;
        }
        xb[3 * p] = xb[3 * p + 1] = xb[3 * p + 2] = 1.0f;
    }

    mpm_ctx* ctx = NULL;
    if (check(mpm_create(&spec, 1, &opt, &ctx), ctx, "mpm_create")) return 1;
    int bad = check(mpm_set_state(ctx, x, v, C, F, NULL, NULL, NULL), ctx, "mpm_set_state");
    for (int t = 0; t < 2 && !bad; t++) bad = check(mpm_step(ctx, NULL, NULL, MPM_STEP_RECORD, NULL), ctx, "mpm_step");
    if (!bad) bad = check(mpm_get_state(ctx, xf, NULL, NULL, NULL, NULL, NULL), ctx, "mpm_get_state");
    if (!bad)
        bad = check(mpm_backward(ctx, xb, NULL, NULL, NULL, NULL, NULL, xb0, NULL, NULL, NULL, NULL, NULL), ctx,
                    "mpm_backward");
    if (!bad) {
        int32_t flags = 0;
        bad = check(mpm_check_status(ctx, &flags), ctx, "mpm_check_status");
    }
    if (!bad) {
        double sx = 0.0, sb = 0.0;
        for (int q = 0; q < N * 3; q++) {
            sx += xf[q];
            sb += xb0[q];
        }
        printf("%.9e %.9e\n", sx, sb);
    }
    mpm_destroy(ctx);
    return bad;
}
