/*
 * ORACLE — test infrastructure only.
 *
 * Plain, sequential, FP64 CPU implementation of what the D-iteration hot path computes, written
 * from the paper ("Revisiting the D-iteration method: runtime comparison", Hong, Burnside,
 * Raoult). It is used by the tests, by the smoke check and by the benchmark's CPU-baseline leg,
 * and by nothing else. It shares no code with the CUDA library: no headers, no helpers, no
 * tables. It is deliberately slow and obvious: no blocking, no fusion, no reordering beyond
 * what the definitions below state.
 *
 * Problem (Section 1): X = P.X + B. P has d/out_j at (i, j) for every link j -> i, so column j
 * holds the out-links of j (Section 2.4: out-degree = non-null entries of column j, in-degree =
 * non-null entries of row i); a dangling column is zero. B >= 0.
 *
 * Contents
 *   or_build         iterator build ("Init", Section 2.1 / 2.5): validate ids, order links by
 *                    (origin, destination), drop duplicates, out-CSR = l_out (columns of P),
 *                    in-CSR = l_in (rows of P), out[], in[], loop[], L, D, O, max_in, max_out
 *                    (Section 2.4).
 *   or_zero_in       E, the recursively defined zero-in-degree set (Section 2.4), by peeling.
 *   or_zero_in_naive E by its definition, iterated to the least fixpoint (small N only).
 *   or_di            DI-CYC and DI-SOP (Section 2.3, Section 2.5), one node visit at a time.
 *   or_di_refresh    DI-SOP with r taken again every r_every node ids within a cycle.
 *   or_di_e          the same after one visit of every node of E in level order (E converges
 *                    in finitely many steps, Section 2.4).
 *   or_di_from       the same from a given state (H, F) instead of (0, B): resuming a
 *                    checkpoint, or a warm start whose fluid is the exact residual of H.
 *   or_pi            power iteration (Jacobi) on X = P.X + B (Section 2.3, Section 2.5 "PI").
 *   or_pi_push       the same iteration per column, scattering over l_out (Section 2.5 "PI'").
 *   or_pi_paper      the paper's normalised PageRank power iteration (Section 2.5 "PI").
 *   or_residual      F* = B + P.H - H, the fluid that H still owes (used for a-posteriori bounds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Iterator build                                                                              */
/* ------------------------------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Build both iterators from an edge list (origin src[e] -> destination dst[e]).
 * Output arrays are sized by the caller: rp_out/rp_in n+1, col_out/col_in m (upper bound on L),
 * outdeg/indeg n, loop n. stats[0..4] = L, D, O, max_in, max_out.
 * Returns L >= 0, or -(1 + e) where e is the first edge whose id is outside [0, n).
 */
int64_t or_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 int64_t *rp_out, int32_t *col_out, int64_t *rp_in, int32_t *col_in,
                 int32_t *outdeg, int32_t *indeg, uint8_t *loop, int64_t *stats) {
    for (int64_t e = 0; e < m; e++)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -(1 + e);

    /* group links by origin (counting sort), then sort each group by destination */
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t e = 0; e < m; e++) cnt[src[e] + 1]++;
    for (int64_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(cur, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; e++) tmp[cur[src[e]]++] = dst[e];

    /* sort each origin's destinations, drop repeats, write the out-CSR */
    int64_t L = 0;
    rp_out[0] = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t b = cnt[v], len = cnt[v + 1] - cnt[v];
        qsort(tmp + b, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int64_t k = 0; k < len; k++) {
            if (k > 0 && tmp[b + k] == tmp[b + k - 1]) continue;
            col_out[L++] = tmp[b + k];
        }
        rp_out[v + 1] = L;
    }

    /* degrees and loop flags (Section 2.4) */
    memset(indeg, 0, sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; v++) {
        outdeg[v] = (int32_t)(rp_out[v + 1] - rp_out[v]);
        loop[v] = 0;
        for (int64_t k = rp_out[v]; k < rp_out[v + 1]; k++) {
            indeg[col_out[k]]++;
            if (col_out[k] == v) loop[v] = 1;
        }
    }
    /* in-CSR: rows of P. Walking the out-CSR in (origin, destination) order keeps each row's
     * origins ascending. */
    rp_in[0] = 0;
    for (int64_t v = 0; v < n; v++) rp_in[v + 1] = rp_in[v] + indeg[v];
    memcpy(cur, rp_in, sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; v++)
        for (int64_t k = rp_out[v]; k < rp_out[v + 1]; k++) col_in[cur[col_out[k]]++] = (int32_t)v;

    int64_t D = 0, O = 0, max_in = 0, max_out = 0;
    for (int64_t v = 0; v < n; v++) {
        if (outdeg[v] == 0) D++;
        if (loop[v]) O++;
        if (indeg[v] > max_in) max_in = indeg[v];
        if (outdeg[v] > max_out) max_out = outdeg[v];
    }
    stats[0] = L; stats[1] = D; stats[2] = O; stats[3] = max_in; stats[4] = max_out;
    free(cnt); free(tmp); free(cur);
    return L;
}

/*
 * E by peeling (Section 2.4): start from nodes of in-degree 0; removing a member of E removes
 * its out-links; a node whose in-links are all gone joins E. level = 0 for in-degree 0, else
 * 1 + the largest level among its in-neighbours. e_mask[v] = 1 for members, level[v] = -1 for
 * non-members. Returns |E|; *n_levels = 1 + the largest level (0 when E is empty).
 */
int64_t or_zero_in(int64_t n, const int64_t *rp_out, const int32_t *col_out, const int32_t *indeg,
                   uint8_t *e_mask, int32_t *level, int32_t *n_levels) {
    int32_t *left = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t head = 0, tail = 0;
    for (int64_t v = 0; v < n; v++) {
        left[v] = indeg[v];
        e_mask[v] = 0;
        level[v] = -1;
        if (indeg[v] == 0) { queue[tail++] = (int32_t)v; e_mask[v] = 1; level[v] = 0; }
    }
    int32_t top = -1;
    while (head < tail) {
        int32_t u = queue[head++];
        if (level[u] > top) top = level[u];
        for (int64_t k = rp_out[u]; k < rp_out[u + 1]; k++) {
            int32_t w = col_out[k];
            if (level[u] + 1 > level[w] && !e_mask[w]) level[w] = level[u] + 1;
            left[w]--;
            if (left[w] == 0) { e_mask[w] = 1; queue[tail++] = w; }
        }
    }
    /* nodes never peeled keep level -1 */
    for (int64_t v = 0; v < n; v++) if (!e_mask[v]) level[v] = -1;
    *n_levels = top + 1;
    free(left); free(queue);
    return tail;
}

/*
 * E straight from its definition, iterated to the least fixpoint: a node joins when every one
 * of its in-neighbours is already a member (vacuously true for in-degree 0). Repeats full
 * passes until nothing changes, so it is O(N * depth) and meant for small graphs.
 */
int64_t or_zero_in_naive(int64_t n, const int64_t *rp_in, const int32_t *col_in,
                         uint8_t *e_mask, int32_t *level, int32_t *n_levels) {
    for (int64_t v = 0; v < n; v++) { e_mask[v] = 0; level[v] = -1; }
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int64_t v = 0; v < n; v++) {
            if (e_mask[v]) continue;
            int all_in = 1;
            int32_t lv = 0;
            for (int64_t k = rp_in[v]; k < rp_in[v + 1]; k++) {
                int32_t u = col_in[k];
                if (!e_mask[u]) { all_in = 0; break; }
                if (level[u] + 1 > lv) lv = level[u] + 1;
            }
            if (all_in) { e_mask[v] = 1; level[v] = lv; changed = 1; }
        }
    }
    int64_t count = 0;
    int32_t top = -1;
    for (int64_t v = 0; v < n; v++) if (e_mask[v]) { count++; if (level[v] > top) top = level[v]; }
    *n_levels = top + 1;
    return count;
}

/* ------------------------------------------------------------------------------------------ */
/* D-iteration                                                                                 */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int64_t cycles;        /* completed cycles over i = 0..N-1 */
    int64_t visits;        /* node visits (diffusions) */
    int64_t pushed_edges;  /* sum of out[i] over visits */
    int64_t fallback_cycles; /* DI-SOP cycles that selected nothing and ran as DI-CYC */
    double e;              /* fluid absorbed by dangling nodes: sum of H over out[i] == 0 */
    double residual;       /* sum of F at exit */
    double paper_error;    /* residual / (1 - d - d*e), Section 2.5 DI-CYC */
    int64_t e_visits;      /* visits of the E pre-diffusion (or_di_e) */
} or_di_info;

/*
 * One diffusion of node i (Section 2.5 DI-CYC body): the fluid F_i moves into the history H_i
 * and d/out_i of it goes to every out-neighbour other than i. A loop node (p_ii != 0) first
 * absorbs the geometric series of its own self-diffusion: transit = F_i * out_i / (out_i - d).
 * A dangling node keeps its transit in H and adds it to e.
 */
static void visit(int64_t i, double d, const int64_t *rp_out, const int32_t *col_out,
                  const uint8_t *loop, double *H, double *F, or_di_info *info) {
    int64_t o = rp_out[i + 1] - rp_out[i];
    double transit = loop[i] ? F[i] * (double)o / ((double)o - d) : F[i];
    H[i] += transit;
    F[i] = 0.0;
    if (o == 0) {
        info->e += transit;
    } else {
        double sent = transit * d / (double)o;
        for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++)
            if (col_out[k] != i) F[col_out[k]] += sent;
    }
    info->visits++;
    info->pushed_edges += o;
}

/* ||F||_1; with F >= 0 (every run from H = 0, F = B) this is the paper's sum of the fluid */
static double sum_fluid(int64_t n, const double *F) {
    double r = 0.0;
    for (int64_t i = 0; i < n; i++) r += fabs(F[i]);
    return r;
}

/*
 * D-iteration from H = 0, F = B (Section 2.5). schedule 0 = DI-CYC: in each cycle visit
 * i = 0..N-1 when F_i != 0. schedule 1 = DI-SOP: r = ||F||_1 is taken once at the start of the
 * cycle and i is visited when |F_i| > (r / L) * out_i (Section 2.3); a DI-SOP cycle that visits
 * nothing is run again as a DI-CYC cycle. The loop stops when ||F||_1 <= tol after a cycle, or
 * after max_cycles cycles (max_cycles < 0: no limit). Returns 0 when converged, 1 otherwise.
 * With F >= 0, as in every run from (0, B), the tests read exactly as the paper's F_i > 0,
 * F_i > (r / L) * out_i and sum F; a resumed state may carry negative fluid (a warm start whose
 * H overshoots X), which the visit moves like any other by linearity.
 */
static int run_cycles(int64_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out, const uint8_t *loop,
                      double d, double tol, int schedule, int64_t max_cycles, int64_t r_every, double *H, double *F,
                      or_di_info *info) {
    double r = sum_fluid(n, F);
    while (r > tol && (max_cycles < 0 || info->cycles < max_cycles)) {
        int64_t visits_before = info->visits;
        if (schedule == 1) {
            double r_cycle = r;
            for (int64_t i = 0; i < n; i++) {
                /* the refreshed variant takes r again before nodes r_every, 2 r_every, ... */
                if (r_every > 0 && i > 0 && i % r_every == 0) r_cycle = sum_fluid(n, F);
                double out_i = (double)(rp_out[i + 1] - rp_out[i]);
                if (fabs(F[i]) > (r_cycle / (double)L) * out_i) visit(i, d, rp_out, col_out, loop, H, F, info);
            }
            if (info->visits == visits_before) {
                info->fallback_cycles++;
                for (int64_t i = 0; i < n; i++)
                    if (F[i] != 0.0) visit(i, d, rp_out, col_out, loop, H, F, info);
            }
        } else {
            for (int64_t i = 0; i < n; i++)
                if (F[i] != 0.0) visit(i, d, rp_out, col_out, loop, H, F, info);
        }
        info->cycles++;
        r = sum_fluid(n, F);
    }
    info->residual = r;
    info->paper_error = r / (1.0 - d - d * info->e);
    return r <= tol ? 0 : 1;
}

int or_di(int64_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out, const uint8_t *loop,
          const double *B, double d, double tol, int schedule, int64_t max_cycles,
          double *H, double *F, or_di_info *info) {
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) { H[i] = 0.0; F[i] = B[i]; }
    return run_cycles(n, L, rp_out, col_out, loop, d, tol, schedule, max_cycles, 0, H, F, info);
}

/*
 * DI-SOP with r refreshed within the cycle (the variant of Section 2.3's threshold that takes
 * r_n' more often than once per cycle): r = ||F||_1 is taken at the start of the cycle and again
 * before node ids r_every, 2 r_every, ... Everything else is or_di's DI-SOP, including the
 * fallback of a cycle that visits nothing. r_every <= 0 or >= n is or_di itself.
 */
int or_di_refresh(int64_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out, const uint8_t *loop,
                  const double *B, double d, double tol, int64_t r_every, int64_t max_cycles,
                  double *H, double *F, or_di_info *info) {
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) { H[i] = 0.0; F[i] = B[i]; }
    return run_cycles(n, L, rp_out, col_out, loop, d, tol, 1, max_cycles, r_every, H, F, info);
}

/*
 * D-iteration from a given state (H0, F0) (copied into H, F): the identity X = H + (I - P)^-1 F
 * holds for the state of any run, so resuming a run's checkpoint continues it exactly, and
 * F0 = B + P.H0 - H0 turns any approximate solution H0 into a warm start for B.
 */
int or_di_from(int64_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out, const uint8_t *loop,
               const double *H0, const double *F0, double d, double tol, int schedule, int64_t max_cycles,
               double *H, double *F, or_di_info *info) {
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) { H[i] = H0[i]; F[i] = F0[i]; }
    return run_cycles(n, L, rp_out, col_out, loop, d, tol, schedule, max_cycles, 0, H, F, info);
}

/*
 * E-level pre-diffusion (Section 2.4: the nodes of E, the recursively zero-in-degree set,
 * converge exactly in finitely many steps). Every in-neighbour of a node of E at level l lies in
 * E at a level below l, and no node of E has a self-loop. So once every node of E below level l
 * has been visited, the fluid of a level-l node is final. Visiting E once in level order (ids
 * ascending within a level) gives every node of E its exact history, and no fluid reaches E
 * afterwards. The cycles of or_di then run from that (H, F). e_mask and e_level are or_zero_in's.
 */
int or_di_e(int64_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out, const uint8_t *loop,
            const uint8_t *e_mask, const int32_t *e_level, int32_t n_levels, const double *B, double d,
            double tol, int schedule, int64_t max_cycles, double *H, double *F, or_di_info *info) {
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) { H[i] = 0.0; F[i] = B[i]; }
    for (int32_t l = 0; l < n_levels; l++)
        for (int64_t i = 0; i < n; i++)
            if (e_mask[i] && e_level[i] == l) {
                visit(i, d, rp_out, col_out, loop, H, F, info);
                info->e_visits++;
            }
    return run_cycles(n, L, rp_out, col_out, loop, d, tol, schedule, max_cycles, 0, H, F, info);
}

/* ------------------------------------------------------------------------------------------ */
/* Power iteration                                                                             */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int64_t iterations;
    double residual;       /* ||X_k - X_{k-1}||_1 at exit */
} or_pi_info;

/*
 * Jacobi iteration on X = P.X + B over the rows of P (Section 2.5 "PI", row vectors l_in):
 * X_0 = 0, X_{k+1}[i] = B[i] + sum_{j in in(i)} d * X_k[j] / out[j]. Stops when
 * ||X_{k+1} - X_k||_1 <= tol or after max_iters. Returns 0 when converged, 1 otherwise.
 */
int or_pi(int64_t n, const int64_t *rp_in, const int32_t *col_in, const int32_t *outdeg,
          const double *B, double d, double tol, int64_t max_iters, double *X, or_pi_info *info) {
    double *Xn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) X[i] = 0.0;
    double res = INFINITY;
    while (res > tol && info->iterations < max_iters) {
        for (int64_t i = 0; i < n; i++) {
            double acc = B[i];
            for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {
                int32_t j = col_in[k];
                acc += d * X[j] / (double)outdeg[j];
            }
            Xn[i] = acc;
        }
        res = 0.0;
        for (int64_t i = 0; i < n; i++) { res += fabs(Xn[i] - X[i]); X[i] = Xn[i]; }
        info->iterations++;
    }
    info->residual = res;
    free(Xn);
    return res <= tol ? 0 : 1;
}

/*
 * Power iteration per column (Section 2.5 "PI'"): the same Jacobi iteration on X = P.X + B as
 * or_pi, formed by the columns of P: X_new = B, then every node i with out_i > 0 adds
 * d * X[i] / out_i to each of its out-neighbours (its own self-link included, as a plain entry
 * of P). Stops on PI's criterion ||X_new - X||_1 <= tol (the printed PI' scales its threshold
 * twice; the paper's tables give PI and PI' the same iteration counts).
 */
int or_pi_push(int64_t n, const int64_t *rp_out, const int32_t *col_out, const double *B, double d, double tol,
               int64_t max_iters, double *X, or_pi_info *info) {
    double *Xn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) X[i] = 0.0;
    double res = INFINITY;
    while (res > tol && info->iterations < max_iters) {
        for (int64_t i = 0; i < n; i++) Xn[i] = B[i];
        for (int64_t i = 0; i < n; i++) {
            int64_t o = rp_out[i + 1] - rp_out[i];
            if (o == 0) continue;
            double transit = d * X[i] / (double)o;
            for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++) Xn[col_out[k]] += transit;
        }
        res = 0.0;
        for (int64_t i = 0; i < n; i++) { res += fabs(Xn[i] - X[i]); X[i] = Xn[i]; }
        info->iterations++;
    }
    info->residual = res;
    free(Xn);
    return res <= tol ? 0 : 1;
}

/*
 * The paper's PI as printed (Section 2.5), with its evident slips repaired: x starts at 1/N,
 * each iteration computes x_new = (1-d)/N + sum d*x_old[j]/out[j], hands the mass lost at
 * dangling nodes back uniformly, measures error = ||x_new - x_old||_1 * d/(1-d) and then swaps
 * x_old and x_new (the listing never swaps, uses abs() on a double and leaves error unset).
 * Stops when error <= tol. Returns 0 when converged.
 */
int or_pi_paper(int64_t n, const int64_t *rp_in, const int32_t *col_in, const int32_t *outdeg,
                double d, double tol, int64_t max_iters, double *x, or_pi_info *info) {
    double *xn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memset(info, 0, sizeof(*info));
    for (int64_t i = 0; i < n; i++) x[i] = 1.0 / (double)n;
    double err = INFINITY;
    while (err > tol && info->iterations < max_iters) {
        for (int64_t i = 0; i < n; i++) {
            xn[i] = (1.0 - d) / (double)n;
            for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {
                int32_t j = col_in[k];
                xn[i] += d * x[j] / (double)outdeg[j];
            }
        }
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) s += xn[i];
        for (int64_t i = 0; i < n; i++) xn[i] += (1.0 - s) / (double)n;
        err = 0.0;
        for (int64_t i = 0; i < n; i++) err += fabs(xn[i] - x[i]);
        err *= d / (1.0 - d);
        for (int64_t i = 0; i < n; i++) x[i] = xn[i];
        info->iterations++;
    }
    info->residual = err;
    free(xn);
    return err <= tol ? 0 : 1;
}

/*
 * F* = B + P.H - H over the rows of P. By the identity X = H + (I - P)^-1 F (every diffusion
 * moves mass between H and F without changing H + (I - P)^-1 F), F* is the fluid a history H
 * still owes, and ||X - H||_1 <= ||F*||_1 / (1 - d). Returns ||F*||_1.
 */
double or_residual(int64_t n, const int64_t *rp_in, const int32_t *col_in, const int32_t *outdeg,
                   const double *B, double d, const double *H, double *Fstar) {
    double norm = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double acc = B[i];
        for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {
            int32_t j = col_in[k];
            acc += d * H[j] / (double)outdeg[j];
        }
        Fstar[i] = acc - H[i];
        norm += fabs(Fstar[i]);
    }
    return norm;
}
