/*
 * oracle.c -- plain, slow FP64 CPU reference for the PageRank of
 * "Two Parallel PageRank Algorithms via Improving Forward Push" (IFP1 / IFP2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Notation follows the paper: graph G(V,E), out-lists D(v), in-lists S(v),
 * deg(v) = |D(v)| (the ORIGINAL out-degree), dangling indicator d
 * (deg(v) = 0), personalization p, damping c, transition matrix P
 * (p_ij = a_ij / deg(v_j), column j zero when v_j is dangling),
 * P' = P + p d^T (Sec. 2.1).
 *
 * Functions:
 *   orc_power           Power iteration on the Google matrix P'' (Eq. 1).
 *   orc_dense_solve     Gaussian elimination on (I - cP') pi = (1-c) p (Eq. 2).
 *   orc_eq2_residual    || (I - cP') pi - (1-c) p ||_1 for any pi (Eq. 2).
 *   orc_ifp_sequential  Alg. 2 (IFP1) / Alg. 3 (IFP2) with one thread.
 *   orc_ifp_rounds      IFP1 / IFP2 in synchronous snapshot rounds with a
 *                       (1-c) reserve: the round semantics the GPU library
 *                       implements (reading of Sec. 3.3.1's "iteration").
 *   orc_ifp2_levels     IFP2 in level-ordered rounds: the in-round
 *                       propagation of Sec. 3.2's asynchronous scans, with
 *                       levels scanned in a fixed order.
 *   orc_ifp_async       IFP1 / IFP2 rounds in which each vertex of the
 *                       round's frontier pushes all the residual it holds
 *                       when its turn comes (Sec. 3.2's threads), the
 *                       frontier taken in id order: one schedule of the
 *                       GPU's asynchronous rounds.
 *   orc_ifp_scan        IFP1 / IFP2 as full scans in id order with a (1-c)
 *                       reserve: every non-dangling vertex, at its turn,
 *                       pushes all it holds if that is above xi_act
 *                       (Alg. 2/3 with K = 1): one schedule of the GPU's
 *                       asynchronous pull rounds.
 *
 * Arrays: out_off[n+1] (int64), out_dst[m] (int32), vertex ids 0..n-1.
 * Every loop is the textbook one; nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_IFP1 1
#define ORC_IFP2 2

static int64_t outdeg(const int64_t *out_off, int32_t v) { return out_off[v + 1] - out_off[v]; }

/*
 * Power method on P'' = cP' + (1-c) p e^T (Eq. 1): pi_{k+1} = P'' pi_k,
 * written without forming P'':
 *   pi_{k+1} = c P pi_k + c (d^T pi_k) p + (1-c) (e^T pi_k) p.
 * Starts from pi_0 = p and stops when ||pi_{k+1} - pi_k||_1 <= tol or after
 * max_iter steps (Sec. 4 takes the 210th iterate as the truth).
 * Returns 0 on convergence, 1 otherwise.
 */
int orc_power(int32_t n, const int64_t *out_off, const int32_t *out_dst, double c,
              const double *p, double tol, int32_t max_iter, double *pi, int32_t *iters,
              double *delta_out) {
    double *next = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) pi[i] = p[i];
    int32_t k = 0;
    double delta = INFINITY;
    int status = 1;
    while (k < max_iter) {
        double dangling_mass = 0.0, total_mass = 0.0;
        for (int32_t j = 0; j < n; j++) next[j] = 0.0;
        for (int32_t i = 0; i < n; i++) {
            total_mass += pi[i];
            int64_t deg = outdeg(out_off, i);
            if (deg == 0) {
                dangling_mass += pi[i];
                continue;
            }
            for (int64_t e = out_off[i]; e < out_off[i + 1]; e++)
                next[out_dst[e]] += c * pi[i] / (double)deg;
        }
        double gamma = c * dangling_mass + (1.0 - c) * total_mass;
        delta = 0.0;
        for (int32_t j = 0; j < n; j++) {
            next[j] += gamma * p[j];
            delta += fabs(next[j] - pi[j]);
            pi[j] = next[j];
        }
        k++;
        if (delta <= tol) { status = 0; break; }
    }
    free(next);
    if (iters) *iters = k;
    if (delta_out) *delta_out = delta;
    return status;
}

/*
 * Dense solve of Eq. 2, (I - cP') pi = (1-c) p, with P' = P + p d^T built
 * entry by entry; Gaussian elimination with partial pivoting.  O(n^3): for
 * n up to a few hundred.  Returns 0, or 1 if a pivot vanished.
 */
int orc_dense_solve(int32_t n, const int64_t *out_off, const int32_t *out_dst, double c,
                    const double *p, double *pi) {
    size_t N = (size_t)n;
    double *M = (double *)calloc(N * N, sizeof(double)); /* row-major, M[row*N + col] */
    double *b = (double *)malloc(sizeof(double) * (N ? N : 1));
    for (size_t i = 0; i < N; i++) M[i * N + i] = 1.0;
    for (int32_t j = 0; j < n; j++) { /* column j of cP' */
        int64_t deg = outdeg(out_off, j);
        if (deg == 0) {
            for (int32_t i = 0; i < n; i++) M[(size_t)i * N + (size_t)j] -= c * p[i];
        } else {
            for (int64_t e = out_off[j]; e < out_off[j + 1]; e++)
                M[(size_t)out_dst[e] * N + (size_t)j] -= c / (double)deg;
        }
    }
    for (size_t i = 0; i < N; i++) b[i] = (1.0 - c) * p[i];
    int status = 0;
    for (size_t k = 0; k < N; k++) {
        size_t piv = k;
        for (size_t i = k + 1; i < N; i++)
            if (fabs(M[i * N + k]) > fabs(M[piv * N + k])) piv = i;
        if (M[piv * N + k] == 0.0) { status = 1; break; }
        if (piv != k) {
            for (size_t j = 0; j < N; j++) {
                double t = M[k * N + j]; M[k * N + j] = M[piv * N + j]; M[piv * N + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (size_t i = k + 1; i < N; i++) {
            double f = M[i * N + k] / M[k * N + k];
            if (f == 0.0) continue;
            for (size_t j = k; j < N; j++) M[i * N + j] -= f * M[k * N + j];
            b[i] -= f * b[k];
        }
    }
    if (status == 0) {
        for (size_t kk = N; kk-- > 0;) {
            double s = b[kk];
            for (size_t j = kk + 1; j < N; j++) s -= M[kk * N + j] * pi[j];
            pi[kk] = s / M[kk * N + kk];
        }
    }
    free(M);
    free(b);
    return status;
}

/*
 * || (I - cP') pi - (1-c) p ||_1 for a given pi (Eq. 2), by its definition:
 * y = pi - c P pi - c (d^T pi) p, residual = sum_j |y_j - (1-c) p_j|.
 * Since ||(I - cP')^{-1}||_1 <= 1/(1-c) (P' is column-stochastic), the L1
 * distance of pi from the exact PageRank is at most residual / (1-c).
 */
double orc_eq2_residual(int32_t n, const int64_t *out_off, const int32_t *out_dst, double c,
                        const double *p, const double *pi) {
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double dangling_mass = 0.0;
    for (int32_t j = 0; j < n; j++) y[j] = pi[j];
    for (int32_t i = 0; i < n; i++) {
        int64_t deg = outdeg(out_off, i);
        if (deg == 0) { dangling_mass += pi[i]; continue; }
        for (int64_t e = out_off[i]; e < out_off[i + 1]; e++)
            y[out_dst[e]] -= c * pi[i] / (double)deg;
    }
    double res = 0.0;
    for (int32_t j = 0; j < n; j++) res += fabs(y[j] - c * dangling_mass * p[j] - (1.0 - c) * p[j]);
    free(y);
    return res;
}

/* in-lists S(v) from the out-lists, for IFP2 phase 2 */
static void build_in_lists(int32_t n, const int64_t *out_off, const int32_t *out_dst,
                           int64_t **in_off_out, int32_t **in_src_out) {
    int64_t m = out_off[n];
    int64_t *in_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *in_src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; e++) in_off[out_dst[e] + 1]++;
    for (int32_t v = 0; v < n; v++) in_off[v + 1] += in_off[v];
    for (int32_t u = 0; u < n; u++)
        for (int64_t e = out_off[u]; e < out_off[u + 1]; e++) {
            int32_t v = out_dst[e];
            in_src[in_off[v] + fill[v]++] = u;
        }
    free(fill);
    *in_off_out = in_off;
    *in_src_out = in_src;
}

/* R = sum of |r_i| over the non-dangling vertices: the quantity whose bound
 * ends the rounds of Sec. 3.1 (dangling residuals are settled at the end). */
static double nd_residual(int32_t n, const int64_t *out_off, const double *r) {
    double R = 0.0;
    for (int32_t i = 0; i < n; i++)
        if (outdeg(out_off, i) > 0) R += fabs(r[i]);
    return R;
}

/*
 * The end of IFP1 / IFP2 rounds from reserves x and residuals r.  IFP2
 * (Alg. 3) first runs phase 2 once: a dangling d, which never pushed, gets
 * r_d = p_d + sum over in-neighbours u of c * x_u / ((1-c) deg(u)).  Then
 * z_i = x_i + (1-c) r_i for IFP1 (Alg. 2: pibar + h, scaled by 1-c); for
 * IFP2 z_i = x_i on non-dangling vertices and (1-c) r_d on dangling ones.
 * pi = z / sum z.
 */
static void ifp_finalise(int algo, int32_t n, const int64_t *out_off, const int32_t *out_dst, double c,
                         const double *p, const double *x, double *r, double *pi) {
    double total = 0.0;
    if (algo == ORC_IFP2) {
        int64_t *in_off;
        int32_t *in_src;
        build_in_lists(n, out_off, out_dst, &in_off, &in_src);
        for (int32_t d = 0; d < n; d++) {
            if (outdeg(out_off, d) != 0) continue;
            double s = p[d];
            for (int64_t e = in_off[d]; e < in_off[d + 1]; e++) {
                int32_t u = in_src[e];
                s += c * x[u] / ((1.0 - c) * (double)outdeg(out_off, u));
            }
            r[d] = s;
        }
        free(in_off);
        free(in_src);
        for (int32_t i = 0; i < n; i++)
            pi[i] = outdeg(out_off, i) > 0 ? x[i] : (1.0 - c) * r[i];
    } else {
        for (int32_t i = 0; i < n; i++) pi[i] = x[i] + (1.0 - c) * r[i];
    }
    for (int32_t i = 0; i < n; i++) total += pi[i];
    for (int32_t i = 0; i < n; i++) pi[i] /= total;
}

/*
 * Alg. 2 (IFP1) and Alg. 3 (IFP2) with K = 1: one Calculation thread scans
 * the vertices in id order, again and again; a vertex v_i with h_i > xi
 * reserves 100% of h_i and pushes c*h_i/deg(v_i) to each v_j in D(v_i).  The
 * Management test ("some non-dangling vertex holds h_i > xi") is taken after
 * each full scan.  Only non-dangling vertices are processed.
 *
 * IFP2 (Alg. 3): edges into dangling vertices are invalid during phase 1, so
 * dangling vertices keep their initial h; phase 2 then sets, once, for each
 * dangling v_d: pibar_d = h_d + sum_{u in S(v_d)} c*pibar_u/deg(u), h_d = 0.
 * deg(u) stays the original out-degree.
 *
 * Result: IFP1 pi_i = (pibar_i + h_i) / sum (pibar + h); IFP2 pi_i = pibar_i /
 * sum pibar.  h0 is the initial h (Alg. 2/3 use h_i = 1; Alg. 1 uses p).
 *
 * Reading: the pushed amount is taken from h_i before h_i is cleared, so a
 * self-loop keeps the share pushed to itself (the paper's graphs have none).
 * Returns 0, or 1 if max_scans ran out first.
 */
int orc_ifp_sequential(int algo, int32_t n, const int64_t *out_off, const int32_t *out_dst,
                       double c, double xi, const double *h0, int32_t max_scans, double *pi,
                       int32_t *scans_out, int64_t *pushes_out, int64_t *edges_out) {
    double *pibar = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *h = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) h[i] = h0[i];
    int32_t scans = 0;
    int64_t pushes = 0, edges = 0;
    int status = 1;
    for (;;) {
        int any = 0; /* Management: some non-dangling vertex with h_i > xi */
        for (int32_t i = 0; i < n; i++)
            if (outdeg(out_off, i) > 0 && h[i] > xi) { any = 1; break; }
        if (!any) { status = 0; break; }
        if (scans >= max_scans) break;
        for (int32_t i = 0; i < n; i++) { /* Calculation(1) */
            int64_t deg = outdeg(out_off, i);
            if (deg == 0 || !(h[i] > xi)) continue;
            double v = h[i];
            h[i] = 0.0;
            pibar[i] += v;
            pushes++;
            for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) {
                int32_t j = out_dst[e];
                if (algo == ORC_IFP2 && outdeg(out_off, j) == 0) continue; /* invalid edge */
                h[j] += c * v / (double)deg;
                edges++;
            }
        }
        scans++;
    }
    double total = 0.0;
    if (algo == ORC_IFP2) {
        int64_t *in_off;
        int32_t *in_src;
        build_in_lists(n, out_off, out_dst, &in_off, &in_src);
        for (int32_t d = 0; d < n; d++) { /* phase 2, once */
            if (outdeg(out_off, d) != 0) continue;
            pibar[d] = h[d];
            for (int64_t e = in_off[d]; e < in_off[d + 1]; e++) {
                int32_t u = in_src[e];
                pibar[d] += c * pibar[u] / (double)outdeg(out_off, u);
                edges++;
            }
            h[d] = 0.0;
        }
        free(in_off);
        free(in_src);
        for (int32_t i = 0; i < n; i++) total += pibar[i];
        for (int32_t i = 0; i < n; i++) pi[i] = pibar[i] / total;
    } else {
        for (int32_t i = 0; i < n; i++) total += pibar[i] + h[i];
        for (int32_t i = 0; i < n; i++) pi[i] = (pibar[i] + h[i]) / total;
    }
    free(pibar);
    free(h);
    if (scans_out) *scans_out = scans;
    if (pushes_out) *pushes_out = pushes;
    if (edges_out) *edges_out = edges;
    return status;
}

/*
 * IFP1 / IFP2 with the asynchronous pushes of Sec. 3.2, in one schedule.  A
 * round starts like a synchronous one: R = sum of |r| over non-dangling
 * vertices, the stop and cap tests, and the frontier F = {non-dangling i :
 * |r_i| > xi_act}.  Then the vertices of F are taken in increasing id, and
 * each pushes the residual it holds at that moment (its value at the round's
 * start plus what earlier vertices of this round pushed to it): (1-c) of it
 * to its reserve, c/deg of it to every out-neighbour (IFP2: non-dangling
 * ones only).  The rounds end in ifp_finalise.  Returns 0 when R <= eps, 1
 * at the round cap, 2 when F is empty while R > eps.
 */
int orc_ifp_async(int algo, int32_t n, const int64_t *out_off, const int32_t *out_dst, double c,
                  double eps, double xi_act, const double *p, int32_t max_rounds, double *x, double *r,
                  double *pi, int32_t *rounds_out, double *trace_R, int64_t *trace_F) {
    size_t N = (size_t)(n > 0 ? n : 1);
    unsigned char *in_f = (unsigned char *)calloc(N, 1);
    for (int32_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = p[i]; }
    int32_t t = 0;
    int status = 1;
    for (;;) {
        double R = nd_residual(n, out_off, r);
        if (trace_R) trace_R[t] = R;
        if (R <= eps) { status = 0; break; }
        if (t >= max_rounds) { status = 1; break; }
        int64_t nF = 0;
        for (int32_t i = 0; i < n; i++) {
            in_f[i] = outdeg(out_off, i) > 0 && fabs(r[i]) > xi_act;
            if (in_f[i]) nF++;
        }
        if (nF == 0) { status = 2; break; }
        for (int32_t i = 0; i < n; i++) {
            if (!in_f[i]) continue;
            double v = r[i]; /* everything i holds now */
            r[i] -= v;       /* i hands all of it on: r_i becomes 0 */
            x[i] += (1.0 - c) * v;
            int64_t deg = outdeg(out_off, i);
            for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) {
                int32_t j = out_dst[e];
                if (algo == ORC_IFP2 && outdeg(out_off, j) == 0) continue; /* dangling target */
                r[j] += c * v / (double)deg;
            }
        }
        if (trace_F) trace_F[t] = nF;
        t++;
    }
    if (rounds_out) *rounds_out = t;
    ifp_finalise(algo, n, out_off, out_dst, c, p, x, r, pi);
    free(in_f);
    return status;
}

/*
 * IFP2 with level-ordered rounds: the asynchronous propagation of Sec. 3.2
 * (a vertex pushes, within the same scan, mass it received earlier in that
 * scan), made deterministic by scanning blocks of vertices ("levels") in a
 * fixed order.  level[i] in [0, L] for every non-dangling i; dangling
 * vertices are not scanned in phase 1 (IFP2).
 *
 * Rounds 0 and 1 are the synchronous rounds of orc_ifp_rounds.  A push made
 * in any round is delivered to its target the first time the target is
 * scanned after the push.  From round 2 on, a round scans levels 0, 1, ..., L
 * in order; every vertex j of the level being scanned
 *   receives its undelivered pushes;
 *   if |r_j| > xi_act: v = r_j, x_j += (1-c) v, r_j = 0, and c v / deg(j) is
 *   pushed to each non-dangling out-neighbour (F += 1, E += 1 per edge).
 * A push to a vertex of a higher level arrives in the same round; one to a
 * vertex of the same or a lower level arrives in the next round.
 *
 * Decisions: R_0, R_1 are the synchronous residuals at the start of rounds 0
 * and 1.  For a round t >= 2, R_t is the residual after the round: sum over
 * non-dangling |r| plus the pushed mass not yet delivered.  Stop when
 * R_t <= eps (after round t >= 2 the round's pushes stand: rounds = t + 1);
 * status 1 when max_rounds rounds ran, 2 when F_t was empty while R_t > eps.
 * On return, r holds the delivered residual and r_pending (if not NULL) the
 * undelivered pushes per target, so r + r_pending is the state's residual
 * (the identity (I - cP~)(x/(1-c)) = p - (r + r_pending) holds).  Phase 2 and
 * the finalisation are those of orc_ifp_rounds (IFP2).
 * Traces (length >= max_rounds + 2): R_t, F_t, E_t as above.
 */
int orc_ifp2_levels(int32_t n, const int64_t *out_off, const int32_t *out_dst, double c, double eps,
                    double xi_act, const double *p, const int32_t *level, int32_t L, int32_t max_rounds,
                    double *x, double *r, double *r_pending, double *pi, int32_t *rounds_out, double *trace_R,
                    int64_t *trace_F, int64_t *trace_E) {
    size_t N = (size_t)(n > 0 ? n : 1);
    double *pend = (double *)calloc(N, sizeof(double)); /* undelivered pushes per target */
    double *v = (double *)calloc(N, sizeof(double));
    unsigned char *active = (unsigned char *)calloc(N, 1);
    for (int32_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = p[i]; }
    int32_t t = 0, rounds = 0;
    int status = 1;
    for (;;) {
        if (t < 2) { /* synchronous round: deliver, measure, snapshot, push into pend */
            for (int32_t i = 0; i < n; i++) { r[i] += pend[i]; pend[i] = 0.0; }
            double R = 0.0;
            for (int32_t i = 0; i < n; i++)
                if (outdeg(out_off, i) != 0) R += fabs(r[i]);
            if (trace_R) trace_R[t] = R;
            if (R <= eps) { status = 0; rounds = t; break; }
            if (t >= max_rounds) { status = 1; rounds = t; break; }
            int64_t nF = 0, nE = 0;
            for (int32_t i = 0; i < n; i++) {
                active[i] = outdeg(out_off, i) > 0 && fabs(r[i]) > xi_act;
                if (!active[i]) continue;
                v[i] = r[i];
                x[i] += (1.0 - c) * v[i];
                r[i] = 0.0;
                nF++;
            }
            if (nF == 0) { status = 2; rounds = t; break; }
            for (int32_t i = 0; i < n; i++) {
                if (!active[i]) continue;
                int64_t deg = outdeg(out_off, i);
                for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) {
                    int32_t j = out_dst[e];
                    if (outdeg(out_off, j) == 0) continue;
                    pend[j] += c * v[i] / (double)deg;
                    nE++;
                }
            }
            if (trace_F) trace_F[t] = nF;
            if (trace_E) trace_E[t] = nE;
            t++;
            continue;
        }
        if (t >= max_rounds) { status = 1; rounds = t; break; }
        int64_t nF = 0, nE = 0;
        for (int32_t l = 0; l <= L; l++) {
            for (int32_t j = 0; j < n; j++) { /* the level's vertices receive (all at once) */
                if (outdeg(out_off, j) == 0 || level[j] != l) continue;
                r[j] += pend[j];
                pend[j] = 0.0;
            }
            for (int32_t j = 0; j < n; j++) { /* and activate together */
                active[j] = outdeg(out_off, j) > 0 && level[j] == l && fabs(r[j]) > xi_act;
                if (!active[j]) continue;
                v[j] = r[j];
                x[j] += (1.0 - c) * v[j];
                r[j] = 0.0;
                nF++;
            }
            for (int32_t j = 0; j < n; j++) {
                if (!active[j]) continue;
                int64_t deg = outdeg(out_off, j);
                for (int64_t e = out_off[j]; e < out_off[j + 1]; e++) {
                    int32_t k = out_dst[e];
                    if (outdeg(out_off, k) == 0) continue;
                    pend[k] += c * v[j] / (double)deg;
                    nE++;
                }
            }
        }
        double R = 0.0;
        for (int32_t i = 0; i < n; i++)
            if (outdeg(out_off, i) > 0) R += fabs(r[i]) + fabs(pend[i]);
        if (trace_R) trace_R[t] = R;
        if (trace_F) trace_F[t] = nF;
        if (trace_E) trace_E[t] = nE;
        if (R <= eps) { status = 0; rounds = t + 1; break; }
        if (nF == 0) { status = 2; rounds = t + 1; break; }
        t++;
    }
    if (rounds_out) *rounds_out = rounds;
    if (r_pending)
        for (int32_t i = 0; i < n; i++) r_pending[i] = pend[i];
    ifp_finalise(ORC_IFP2, n, out_off, out_dst, c, p, x, r, pi);
    free(pend);
    free(v);
    free(active);
    return status;
}

/*
 * IFP1 / IFP2 in synchronous snapshot rounds with a (1-c) reserve.
 *
 * The reserved share does not change the normalised result (Sec. 3.1, after
 * Eq. 4); with reserve x_i += (1-c) v and push c v / deg(v_i), the residual r
 * and reserve x satisfy sum x + sum r = sum p throughout (IFP1).  One round
 * (Sec. 3.3.1: all vertices scanned once):
 *
 *   R_t = sum_{i non-dangling} |r_i|; stop when R_t <= eps.
 *   F_t = { i non-dangling : |r_i| > xi_act }   (snapshot, taken before any push)
 *   for i in F_t: v_i = r_i; x_i += (1-c) v_i; r_i = 0
 *   for i in F_t, j in D(i) (IFP2: only non-dangling j): r_j += c v_i / deg(v_i)
 *
 * Mass pushed in round t is seen by its targets in round t+1.  With x, r
 * starting at 0 and p, the state after any round satisfies
 * (I - cP~) (x/(1-c)) = p - r, where P~ = P (IFP1) or P with the rows of
 * dangling vertices zeroed, i.e. the invalid edges removed (IFP2).
 *
 * IFP2 phase 2 (Alg. 3): for each dangling d, r_d = p_d + sum_{u in S(d)}
 * c * x_u / ((1-c) deg(u)).
 * Finalise: IFP1 z_i = x_i + (1-c) r_i (Alg. 2: pibar + h, scaled by 1-c);
 * IFP2 z_i = x_i for non-dangling, (1-c) r_d for dangling (Alg. 3: pibar).
 * pi = z / sum z.
 *
 * Per-round traces (optional, length >= max_rounds + 1): R_t, |F_t|, edges
 * pushed in round t, and sum x + sum r after round t (IFP1 mass).
 * Returns 0 on R <= eps, 1 if max_rounds ran out, 2 if F_t was empty while
 * R_t > eps (no progress possible with this xi_act).
 */
int orc_ifp_rounds(int algo, int32_t n, const int64_t *out_off, const int32_t *out_dst,
                   double c, double eps, double xi_act, const double *p, int32_t max_rounds,
                   double *x, double *r, double *pi, int32_t *rounds_out, double *trace_R,
                   int64_t *trace_F, int64_t *trace_E, double *trace_mass) {
    size_t N = (size_t)(n > 0 ? n : 1);
    double *v = (double *)calloc(N, sizeof(double));
    unsigned char *active = (unsigned char *)calloc(N, 1);
    for (int32_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = p[i]; }
    int32_t t = 0;
    int status = 1;
    for (;;) {
        double R = nd_residual(n, out_off, r);
        if (trace_R) trace_R[t] = R;
        if (R <= eps) { status = 0; break; }
        if (t >= max_rounds) { status = 1; break; }
        int64_t nF = 0, nE = 0;
        for (int32_t i = 0; i < n; i++) { /* snapshot */
            active[i] = outdeg(out_off, i) > 0 && fabs(r[i]) > xi_act;
            if (!active[i]) continue;
            v[i] = r[i];
            x[i] += (1.0 - c) * v[i];
            r[i] = 0.0;
            nF++;
        }
        if (nF == 0) { status = 2; break; }
        for (int32_t i = 0; i < n; i++) { /* push */
            if (!active[i]) continue;
            int64_t deg = outdeg(out_off, i);
            for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) {
                int32_t j = out_dst[e];
                if (algo == ORC_IFP2 && outdeg(out_off, j) == 0) continue;
                r[j] += c * v[i] / (double)deg;
                nE++;
            }
        }
        if (trace_F) trace_F[t] = nF;
        if (trace_E) trace_E[t] = nE;
        t++;
        if (trace_mass) {
            double s = 0.0;
            for (int32_t i = 0; i < n; i++) s += x[i] + r[i];
            trace_mass[t] = s;
        }
    }
    if (rounds_out) *rounds_out = t;
    ifp_finalise(algo, n, out_off, out_dst, c, p, x, r, pi);
    free(v);
    free(active);
    return status;
}

/*
 * IFP1 / IFP2 in scans (Alg. 2 / Alg. 3 with one Calculation thread, in id
 * order), with the (1-c) reserve and the stopping rule of the rounds.  At its
 * turn each non-dangling vertex i looks at the residual it holds now -- its
 * value at the scan's start plus everything pushed to it so far in this scan
 * -- and, if |r_i| > xi_act, keeps (1-c) of it in x_i and pushes c/deg(i) of
 * it to each out-neighbour (IFP2: non-dangling ones only), r_i = 0.
 *
 * After each scan: R_t = sum of |r| over non-dangling vertices (the exact
 * residual at the scan's end), and the upper bound the GPU's concurrent scans
 * stop on, which cannot know whether a target took a push in the same scan:
 * the residual each vertex left at its turn plus c |v| n_i / deg(i) for every
 * push v of i, n_i its pushes that can land on a non-dangling vertex.  The
 * scans stop when R_t <= eps (status 0), at max_rounds (status 1), or when a
 * scan pushed nothing while R_t > eps (status 2); ifp_finalise ends them.
 */
int orc_ifp_scan(int algo, int32_t n, const int64_t *out_off, const int32_t *out_dst, double c, double eps,
                 double xi_act, const double *p, int32_t max_rounds, double *x, double *r, double *pi,
                 int32_t *rounds_out, double *trace_R, double *trace_Rub, int64_t *trace_F) {
    for (int32_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = p[i]; }
    int32_t t = 0;
    int status = 1;
    for (;;) {
        if (t >= max_rounds) { status = 1; break; }
        int64_t nF = 0;
        double Rub = 0.0;
        for (int32_t i = 0; i < n; i++) {
            int64_t deg = outdeg(out_off, i);
            if (deg == 0) continue;
            if (!(fabs(r[i]) > xi_act)) { Rub += fabs(r[i]); continue; }
            double v = r[i]; /* everything i holds at its turn */
            r[i] = 0.0;
            x[i] = x[i] + (1.0 - c) * v;
            nF++;
            int64_t valid = 0;
            for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) {
                int32_t j = out_dst[e];
                if (outdeg(out_off, j) == 0) {
                    if (algo == ORC_IFP2) continue; /* invalid edge */
                } else {
                    valid++;
                }
                r[j] = r[j] + c * v / (double)deg;
            }
            Rub += c * fabs(v) * (double)valid / (double)deg; /* may land after its target's turn */
        }
        double R = nd_residual(n, out_off, r);
        if (trace_R) trace_R[t] = R;
        if (trace_Rub) trace_Rub[t] = Rub;
        if (trace_F) trace_F[t] = nF;
        t++;
        if (R <= eps) { status = 0; break; }
        if (nF == 0) { status = 2; break; }
    }
    if (rounds_out) *rounds_out = t;
    ifp_finalise(algo, n, out_off, out_dst, c, p, x, r, pi);
    return status;
}
