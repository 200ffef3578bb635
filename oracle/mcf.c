/* Exact optimal transport value by successive shortest paths (min-cost flow).
 *
 * Test infrastructure only: part of the CPU oracle, never linked into the
 * product library.
 *
 * Solves the transportation problem eq. (1) of arXiv 2408.00598 (the full OT
 * problem, M sources and M sinks, cost c_{ij;kl} of eq. (2)):
 *     min sum_{s,t} C[s][t] F[s][t]  s.t.  sum_t F[s][t] = a[s],
 *                                          sum_s F[s][t] = b[t],  F >= 0.
 * Method: successive shortest augmenting paths with node potentials (the
 * textbook primal-dual min-cost-flow scheme).  Every iteration runs a dense
 * O(V^2) Dijkstra on the residual graph from all sources that still have
 * supply to the nearest sink that still has demand, using reduced costs
 * C[s][t] + p[s] - p[t] >= 0, then pushes the bottleneck amount along the path.
 * Forward arcs s->t are uncapacitated; the backward arc t->s carries F[s][t].
 *
 * Amounts are doubles; remaining supplies/demands below `eps` count as zero.
 * Returns 0 on success, -1 on bad input, -2 if the iteration cap was hit.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

int ot_mcf_solve(int ns, int nt, const double* C, const double* a, const double* b,
                 double eps, double* flow_out, double* value_out, int* iters_out)
{
    if (ns <= 0 || nt <= 0 || !C || !a || !b || !value_out) return -1;
    const int V = ns + nt;
    double* F = (double*)calloc((size_t)ns * nt, sizeof(double));
    double* sup = (double*)malloc(sizeof(double) * ns);
    double* dem = (double*)malloc(sizeof(double) * nt);
    double* pot = (double*)calloc(V, sizeof(double));
    double* dist = (double*)malloc(sizeof(double) * V);
    int* prev = (int*)malloc(sizeof(int) * V);
    char* done = (char*)malloc(V);
    if (!F || !sup || !dem || !pot || !dist || !prev || !done) return -1;
    for (int s = 0; s < ns; ++s) { if (a[s] < 0) return -1; sup[s] = a[s]; }
    for (int t = 0; t < nt; ++t) { if (b[t] < 0) return -1; dem[t] = b[t]; }

    const int max_iters = 200 * V + 1000;
    int it = 0, status = 0;
    for (;;) {
        int any = 0;
        for (int s = 0; s < ns; ++s) if (sup[s] > eps) { any = 1; break; }
        if (!any) break;
        if (++it > max_iters) { status = -2; break; }

        /* Dijkstra over nodes 0..ns-1 (sources) and ns..ns+nt-1 (sinks). */
        for (int v = 0; v < V; ++v) { dist[v] = INFINITY; prev[v] = -1; done[v] = 0; }
        for (int s = 0; s < ns; ++s) if (sup[s] > eps) dist[s] = 0.0;
        int target = -1;
        for (;;) {
            int u = -1;
            double best = INFINITY;
            for (int v = 0; v < V; ++v)
                if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
            if (u < 0) break;
            done[u] = 1;
            if (u >= ns && dem[u - ns] > eps) { target = u; break; }
            if (u < ns) {                       /* forward arcs s -> t */
                const int s = u;
                for (int t = 0; t < nt; ++t) {
                    const int v = ns + t;
                    if (done[v]) continue;
                    double rc = C[(size_t)s * nt + t] + pot[s] - pot[v];
                    if (rc < 0) rc = 0;          /* round-off guard */
                    if (dist[u] + rc < dist[v]) { dist[v] = dist[u] + rc; prev[v] = u; }
                }
            } else {                            /* backward arcs t -> s with F > 0 */
                const int t = u - ns;
                for (int s = 0; s < ns; ++s) {
                    if (done[s] || F[(size_t)s * nt + t] <= 0.0) continue;
                    double rc = -C[(size_t)s * nt + t] + pot[u] - pot[s];
                    if (rc < 0) rc = 0;
                    if (dist[u] + rc < dist[s]) { dist[s] = dist[u] + rc; prev[s] = u; }
                }
            }
        }
        if (target < 0) { status = -2; break; }  /* infeasible (unequal masses) */
        const double dt = dist[target];
        for (int v = 0; v < V; ++v) pot[v] += (dist[v] < dt ? dist[v] : dt);

        /* Bottleneck along the path target <- ... <- source. */
        double push = dem[target - ns];
        int v = target;
        while (prev[v] >= 0) {
            const int u = prev[v];
            if (u >= ns) {                      /* backward arc sink u -> source v */
                const double f = F[(size_t)v * nt + (u - ns)];
                if (f < push) push = f;
            }
            v = u;
        }
        if (sup[v] < push) push = sup[v];
        /* Apply. */
        v = target;
        while (prev[v] >= 0) {
            const int u = prev[v];
            if (u < ns) F[(size_t)u * nt + (v - ns)] += push;      /* forward */
            else        F[(size_t)v * nt + (u - ns)] -= push;      /* backward */
            v = u;
        }
        sup[v] -= push;
        dem[target - ns] -= push;
    }

    double val = 0.0;
    for (size_t q = 0; q < (size_t)ns * nt; ++q) val += C[q] * F[q];
    *value_out = val;
    if (flow_out) memcpy(flow_out, F, sizeof(double) * (size_t)ns * nt);
    if (iters_out) *iters_out = it;
    free(F); free(sup); free(dem); free(pot); free(dist); free(prev); free(done);
    return status;
}
