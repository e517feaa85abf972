/*
 * A plain C99 client of the C ABI (include/stp.h): a 2-DoF point robot in the
 * unit square among two moving discs, planned with the interval-root planner
 * (FP32), then one edge validated on its own. Without a usable CUDA device the
 * library must refuse (STP_ERR_CUDA: there is no CPU fallback) and the client
 * reports that and exits 0; any other failure exits 1.
 */
#include <stdio.h>

#include "stp.h"

int main(void) {
    const double q_lo[2] = {0.0, 0.0}, q_hi[2] = {1.0, 1.0};
    const double spheres[5] = {0.0, 0.0, 0.0, 0.0, 0.02}; /* frame 0, centre 0, radius 0.02 */
    stp_robot robot = {2, 0, NULL, q_lo, q_hi, 1, spheres, 0.5};
    const double radius[2] = {0.05, 0.05};
    /* [obstacle][waypoint][t, x, y, z] */
    const double way[2][2][4] = {{{0.0, 0.3, 0.7, 0.0}, {20.0, 0.7, 0.3, 0.0}},
                                 {{0.0, 0.6, 0.2, 0.0}, {20.0, 0.4, 0.8, 0.0}}};
    stp_obstacles obstacles = {2, 2, radius, &way[0][0][0]};
    const double q_start[2] = {0.05, 0.05}, q_goal[2] = {0.95, 0.95};
    stp_params prm = {0};
    prm.variant = 0;
    prm.n_roots = 4;
    prm.ext_per_iter = 64;
    prm.max_iters = 400;
    prm.eta = 0.1;
    prm.edge_res = 0.01;
    prm.env_dt = 0.02;
    prm.p_new = 0.05;
    prm.p_guided = 0.95;
    prm.t_max = 20.0;
    prm.seed = 1;
    prm.precision = 0;

    stp_problem *p = NULL;
    stp_status s = stp_create_problem(&robot, &obstacles, q_start, q_goal, &prm, &p);
    printf("create: %s\n", stp_status_string(s));
    if (s == STP_ERR_CUDA) {
        printf("no usable CUDA device: %s\n", stp_last_error(NULL));
        return p == NULL ? 0 : 1;
    }
    if (s != STP_OK) return 1;

    double U = 0.0, C = 0.0, path[4096 * 3];
    int n = 0;
    stp_stats st;
    s = stp_plan(p, &U, &C, &n, path, 4096, &st);
    printf("plan: %s U=%.4f C=%.4f states=%d iterations=%d edges=%lld\n", stp_status_string(s), U, C, n,
           st.iterations, st.edges_validated + st.bridges_validated);
    int ok = (s == STP_OK || s == STP_NO_SOLUTION);

    /* One edge on its own: from the start, 0.1 along x over 1 s. */
    const float qa[2] = {0.05f, 0.05f}, qb[2] = {0.15f, 0.05f}, ta[1] = {0.0f}, tb[1] = {1.0f};
    unsigned char verdict = 2;
    int checks = 0;
    s = stp_check_edges(p, 1, qa, ta, qb, tb, 0, &verdict, NULL, &checks);
    printf("edge: %s free=%d checks=%d\n", stp_status_string(s), (int)verdict, checks);
    ok = ok && s == STP_OK && verdict == 1 && checks >= 50 && checks <= 51;  /* max(0.1, 0.5 * 1) / 0.01 */

    stp_free(p);
    stp_release_cached();
    return ok ? 0 : 1;
}
