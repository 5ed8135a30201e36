/*
 * FP64 CPU oracle for the Markov-chain semi-Lagrangian value iteration of the
 * 2-D second-order HJB equation of a stochastic minimum-time problem and for
 * the pre-computation of the patchy (dynamic) domain decomposition
 * (Cacace & Falcone, "A dynamic domain decomposition for a class of second
 * order semi-linear equations", Sections 3 and 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, single-threaded, slow and written to be
 * checked against the paper by eye.  Only the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark may load it; the solver
 * library never does.  It shares no source, header, table or helper with the
 * CUDA path.
 *
 * Grid: n nodes per side on [-1,1]^2, dx = 2/(n-1), node (i,j) at
 * (-1+i dx, -1+j dx), linear index k = j*n + i.  Positions inside the
 * routines are in grid units (x = -1 + xi*dx).
 *
 * Readings of the paper taken here (the paper is silent or targets a different
 * setting):
 *   - discount: the expectation is multiplied by beta = 1/(1+lambda h), the
 *     running cost h*l is added outside; lambda = 0 gives the paper's
 *     undiscounted exit-time scheme (Section 3, eq. SLscheme2);
 *   - diffusion: sigma_k = sqrt(2) sigma e_k, i.e. the four points are
 *     x_i + h f +- sqrt(2h) sigma e_k (Section 4.1, eq. const-eps with
 *     epsilon = sigma^2);
 *   - projection: every point is clamped to the square before interpolation;
 *     a point on the right/top edge uses the last cell with fraction 1;
 *   - the self weight lambda_{i0} is the Q1 weight of x_i when x_i is a vertex
 *     of the point's cell, and 0 otherwise (the stencil may reach further than
 *     the first neighbouring cells when h = dx);
 *   - general terms (Section 5.3): sigma(x) may vary per node; the diffusion is
 *     either sigma(x) I_2 (two Wiener components, 2d = 4 points along e_1, e_2)
 *     or sigma(x) a, a one-dimensional Wiener process along the control (2d = 2
 *     points x + h f +- sqrt(2h) sigma(x) a, weight 1/2 each: the k of eq.
 *     SLscheme2 runs over the columns of sigma); the running cost is
 *     l(x, a) = l(x) + m(a), which holds the paper's l_1, l_2 and l_3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MASK_FREE 0
#define MASK_TARGET 1
#define MASK_OBSTACLE 2

typedef struct {
    int32_t n;               /* nodes per side */
    int32_t n_controls;      /* N_A */
    double h;                /* time step */
    double lambda;           /* discount rate (0: undiscounted) */
    double sigma;            /* diffusion coefficient */
    double cost;             /* running cost l (constant) */
    double u_obstacle;       /* value held on obstacle nodes */
    const float *speed;      /* c(x), n*n */
    const float *drift;      /* b(x), n*n*2 interleaved, or NULL */
    const uint8_t *mask;     /* 0 free, 1 target, 2 obstacle */
    const double *controls;  /* a_m = (controls[2m], controls[2m+1]) */
    const float *sigma_field;   /* sigma(x) per node, or NULL: sigma everywhere */
    int32_t diffusion;          /* 0: sigma(x) I_2; 1: sigma(x) a (along the control) */
    const float *cost_field;    /* l(x) per node, or NULL: cost everywhere */
    const double *control_cost; /* m(a_m) per control, or NULL: m = 0 */
} orc_problem;

static double orc_dx(const orc_problem *P) { return 2.0 / (P->n - 1); }
static double orc_beta(const orc_problem *P) { return 1.0 / (1.0 + P->lambda * P->h); }

/* ------------------------------------------------------------------------
 * Q1 (bilinear) reconstruction of u at the grid-unit point (p, q) after the
 * projection onto the square (Section 3, Fig. "bilinear": the four vertices
 * x_{i_0..i_3} of the cell containing the point, with weights lambda_{i_p}).
 * The contribution of the vertex `self` is split out: *excl receives
 * sum_{v != self} w_v u_v and *selfw receives the weight of `self`
 * (0 when self is not a vertex of the cell), as in eq. self-dependency.
 * ---------------------------------------------------------------------- */
static void q1_split(const double *u, int n, double p, double q, int64_t self,
                     double *excl, double *selfw)
{
    if (p < 0.0) p = 0.0;
    if (p > n - 1) p = n - 1;
    if (q < 0.0) q = 0.0;
    if (q > n - 1) q = n - 1;
    int64_t cx = (int64_t)floor(p);
    int64_t cy = (int64_t)floor(q);
    if (cx > n - 2) cx = n - 2;
    if (cy > n - 2) cy = n - 2;
    double fx = p - (double)cx;
    double fy = q - (double)cy;
    int64_t v[4];
    double w[4];
    v[0] = cy * n + cx;           w[0] = (1.0 - fx) * (1.0 - fy);
    v[1] = cy * n + cx + 1;       w[1] = fx * (1.0 - fy);
    v[2] = (cy + 1) * n + cx;     w[2] = (1.0 - fx) * fy;
    v[3] = (cy + 1) * n + cx + 1; w[3] = fx * fy;
    *excl = 0.0;
    *selfw = 0.0;
    for (int t = 0; t < 4; t++) {
        if (v[t] == self)
            *selfw += w[t];
        else
            *excl += w[t] * u[v[t]];
    }
}

/* Full Q1 value (self included), used by the synthesis and the coarse-to-fine
 * interpolation. */
static double q1_full(const double *u, int n, double p, double q)
{
    double e, s;
    q1_split(u, n, p, q, -1, &e, &s);
    return e;
}

/* Foot of the characteristic x_i + h f(x_i, a_m), in grid units, with
 * f(x, a) = b(x) + c(x) a (Section 5, dynamics A, B, C). */
static void foot(const orc_problem *P, int64_t k, int m, double *xi, double *eta)
{
    const int n = P->n;
    const double dx = orc_dx(P);
    const int64_t i = k % n, j = k / n;
    double fx = (double)P->speed[k] * P->controls[2 * m];
    double fy = (double)P->speed[k] * P->controls[2 * m + 1];
    if (P->drift) {
        fx += (double)P->drift[2 * k];
        fy += (double)P->drift[2 * k + 1];
    }
    *xi = (double)i + P->h * fx / dx;
    *eta = (double)j + P->h * fy / dx;
}

/* The 2d points x_{i,k}^{a,s} of eq. SLscheme2 for control m at node k, in
 * grid units, and their common weight 1/(2d).  The Wiener part is
 * sqrt(h) sigma_k with sigma = sqrt(2) sigma(x) I_2 (d = 2, points along the
 * axes) or sigma = sqrt(2) sigma(x) a_m (d = 1, points along the control).
 * With sigma(x) = 0 the points coincide with the foot.  Returns 2d. */
static int scheme_points(const orc_problem *P, int64_t k, int m, double px[4], double py[4],
                         double *weight)
{
    const double dx = orc_dx(P);
    const double sig = P->sigma_field ? (double)P->sigma_field[k] : P->sigma;
    const double r = sqrt(2.0 * P->h) * sig / dx;   /* sqrt(h) |sigma_k| in grid units */
    double xi, eta;
    foot(P, k, m, &xi, &eta);
    if (P->diffusion == 1) {
        const double ax = P->controls[2 * m], ay = P->controls[2 * m + 1];
        px[0] = xi + r * ax;  py[0] = eta + r * ay;
        px[1] = xi - r * ax;  py[1] = eta - r * ay;
        *weight = 0.5;
        return 2;
    }
    px[0] = xi + r;  py[0] = eta;
    px[1] = xi - r;  py[1] = eta;
    px[2] = xi;      py[2] = eta + r;
    px[3] = xi;      py[3] = eta - r;
    *weight = 0.25;
    return 4;
}

/* h l(x_k, a_m) with l(x, a) = l(x) + m(a). */
static double running_cost(const orc_problem *P, int64_t k, int m)
{
    const double lx = P->cost_field ? (double)P->cost_field[k] : P->cost;
    const double la = P->control_cost ? P->control_cost[m] : 0.0;
    return P->h * (lx + la);
}

/* ------------------------------------------------------------------------
 * One node update (free node k).
 *   scheme 2: original scheme (Section 3, eq. SLscheme2):
 *       u_i = min_a { beta * (1/2d) sum_{k,s} u(x_{i,k}^{a,s}) + h l }
 *   scheme 3: modified scheme without self-dependency (eq. SLscheme3 and the
 *       2-D isotropic form of Section 4.1), with the discount:
 *       u_i = min_a { (beta * Lambda1'(a) + h l) / (1 - beta * Lambda0(a)) }
 *       Lambda0 = (1/2d) sum_{k,s} lambda_{i0,k}^{a,s},
 *       Lambda1' = (1/2d) sum_{k,s} sum_{p=1..3} lambda_{ip,k}^{a,s} u(x_{ip,k}^{a,s}).
 * The min is taken by direct comparison over the N_A controls; ties go to the
 * lowest control index.  Returns the new value and the argmin in *argmin.
 * ---------------------------------------------------------------------- */
double orc_node_update(const orc_problem *P, const double *u, int64_t k, int scheme,
                       int32_t *argmin)
{
    const double beta = orc_beta(P);
    double best = INFINITY;
    int32_t best_m = -1;
    for (int m = 0; m < P->n_controls; m++) {
        double px[4], py[4], w;
        const int np = scheme_points(P, k, m, px, py, &w);
        double lam1 = 0.0, lam0 = 0.0;
        for (int p = 0; p < np; p++) {           /* 2d points, weight 1/(2d) */
            double e, s;
            q1_split(u, P->n, px[p], py[p], k, &e, &s);
            lam1 += w * e;
            lam0 += w * s;
        }
        const double hl = running_cost(P, k, m);
        double v;
        if (scheme == 3) {
            double den = 1.0 - beta * lam0;
            v = den > 0.0 ? (beta * lam1 + hl) / den : INFINITY;
        } else {
            v = beta * (lam1 + lam0 * u[k]) + hl;
        }
        if (v < best) {
            best = v;
            best_m = m;
        }
    }
    if (argmin) *argmin = best_m;
    return best;
}

/* Every control's candidate value at free node k (the quantities the min of
 * eq. SLscheme2 / SLscheme3 compares), vals[m] for m < N_A.  Used to decide
 * whether a minimiser chosen elsewhere is a valid one at a near-tie. */
void orc_node_candidates(const orc_problem *P, const double *u, int64_t k, int scheme,
                         double *vals)
{
    const double beta = orc_beta(P);
    for (int m = 0; m < P->n_controls; m++) {
        double px[4], py[4], w;
        const int np = scheme_points(P, k, m, px, py, &w);
        double lam1 = 0.0, lam0 = 0.0;
        for (int p = 0; p < np; p++) {
            double e, s;
            q1_split(u, P->n, px[p], py[p], k, &e, &s);
            lam1 += w * e;
            lam0 += w * s;
        }
        const double hl = running_cost(P, k, m);
        if (scheme == 3) {
            double den = 1.0 - beta * lam0;
            vals[m] = den > 0.0 ? (beta * lam1 + hl) / den : INFINITY;
        } else {
            vals[m] = beta * (lam1 + lam0 * u[k]) + hl;
        }
    }
}

/* Values held on non-free nodes: u = g = 0 on the target, u_obstacle on obstacles. */
void orc_fix_nonfree(const orc_problem *P, double *u)
{
    const int64_t N = (int64_t)P->n * P->n;
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] == MASK_TARGET) u[k] = 0.0;
        else if (P->mask[k] == MASK_OBSTACLE) u[k] = P->u_obstacle;
    }
}

/* One application of the scheme operator to every free node (a Jacobi step):
 * out = T u.  argmin (nullable) receives the minimising control, -1 on
 * non-free nodes.  Returns max |T u - u| over free nodes. */
double orc_apply(const orc_problem *P, const double *u, double *out, int32_t *argmin, int scheme)
{
    const int64_t N = (int64_t)P->n * P->n;
    double inc = 0.0;
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] != MASK_FREE) {
            out[k] = u[k];
            if (argmin) argmin[k] = -1;
            continue;
        }
        int32_t am;
        double v = orc_node_update(P, u, k, scheme, &am);
        out[k] = v;
        if (argmin) argmin[k] = am;
        double dlt = fabs(v - u[k]);
        if (dlt > inc) inc = dlt;
    }
    return inc;
}

/* Sup-norm residual || T2 u - u ||_inf over free nodes, with the original
 * scheme SLscheme2 (the plain definition of the fixed point). */
double orc_residual(const orc_problem *P, const double *u)
{
    const int64_t N = (int64_t)P->n * P->n;
    double r = 0.0;
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] != MASK_FREE) continue;
        double v = orc_node_update(P, u, k, 2, NULL);
        double dlt = fabs(v - u[k]);
        if (dlt > r) r = dlt;
    }
    return r;
}

/* One Gauss-Seidel sweep: free nodes are updated in place in the given order
 * (row-major k = 0..N-1 when order is NULL).  Returns the sup-increment. */
double orc_sweep_gs(const orc_problem *P, double *u, int scheme, const int64_t *order,
                    int64_t n_order)
{
    const int64_t N = (int64_t)P->n * P->n;
    const int64_t cnt = order ? n_order : N;
    double inc = 0.0;
    for (int64_t t = 0; t < cnt; t++) {
        int64_t k = order ? order[t] : t;
        if (P->mask[k] != MASK_FREE) continue;
        double v = orc_node_update(P, u, k, scheme, NULL);
        double dlt = fabs(v - u[k]);
        if (dlt > inc) inc = dlt;
        u[k] = v;
    }
    return inc;
}

/* Value iteration until the sup-increment of a sweep is <= tol.
 *   method 0: Gauss-Seidel in `order` (row-major when NULL);
 *   method 1: Jacobi (u <- T u).
 * Returns the number of sweeps performed, counting the final one whose
 * increment met the tolerance (the paper counts the checking sweep too,
 * Section 5.1), or -1 if max_sweeps was reached.  *last_inc gets the last
 * sweep's increment. */
int32_t orc_solve(const orc_problem *P, double *u, int scheme, int method,
                  const int64_t *order, int64_t n_order, double tol, int32_t max_sweeps,
                  double *last_inc)
{
    const int64_t N = (int64_t)P->n * P->n;
    double *tmp = NULL;
    if (method == 1) {
        tmp = (double *)malloc(sizeof(double) * (size_t)N);
        if (!tmp) return -2;
    }
    orc_fix_nonfree(P, u);
    double inc = INFINITY;
    int32_t s;
    for (s = 1; s <= max_sweeps; s++) {
        if (method == 1) {
            inc = orc_apply(P, u, tmp, NULL, scheme);
            memcpy(u, tmp, sizeof(double) * (size_t)N);
        } else {
            inc = orc_sweep_gs(P, u, scheme, order, n_order);
        }
        if (inc <= tol) break;
    }
    free(tmp);
    if (last_inc) *last_inc = inc;
    return s > max_sweeps ? -1 : s;
}

/* ------------------------------------------------------------------------
 * Pre-computation of the patchy decomposition (Section 4.3).
 * ---------------------------------------------------------------------- */

/* Data of the coarse grid G_c nested in G (Section 2: G_c possibly contained
 * in G).  r = (n-1)/(nc-1); coarse node (I,J) is fine node (rI, rJ).  The
 * coarse speed is the fine speed there.  A coarse node is a target when some
 * fine target node lies within r/2 fine cells of it in both axes (so that a
 * small target is never lost on the coarse grid); otherwise it is an obstacle
 * when its fine node is one, and free otherwise.  Returns 0, or -1 when the
 * grids do not nest. */
int32_t orc_coarse_data(int32_t n, int32_t nc, const float *speed, const uint8_t *mask,
                        float *speed_c, uint8_t *mask_c)
{
    if (nc < 3 || (n - 1) % (nc - 1) != 0) return -1;
    const int r = (n - 1) / (nc - 1);
    const int hw = r / 2;
    for (int J = 0; J < nc; J++) {
        for (int I = 0; I < nc; I++) {
            const int64_t kf = (int64_t)(r * J) * n + r * I;
            const int64_t kc = (int64_t)J * nc + I;
            speed_c[kc] = speed[kf];
            int tgt = 0;
            for (int dj = -hw; dj <= hw && !tgt; dj++) {
                for (int di = -hw; di <= hw; di++) {
                    int fi = r * I + di, fj = r * J + dj;
                    if (fi < 0 || fj < 0 || fi >= n || fj >= n) continue;
                    if (mask[(int64_t)fj * n + fi] == MASK_TARGET) { tgt = 1; break; }
                }
            }
            mask_c[kc] = tgt ? MASK_TARGET : (mask[kf] == MASK_OBSTACLE ? MASK_OBSTACLE : MASK_FREE);
        }
    }
    return 0;
}

/* u_hat on G: Q1 interpolation of the coarse solution u_c (Section 2 and the
 * pre-computation list of Section 4.3).  Fine node i sits at coarse grid
 * coordinate i (nc-1)/(n-1).  Target nodes get g = 0 and obstacle nodes
 * u_obstacle, the values the fine scheme holds there. */
void orc_interp_coarse(int32_t nc, const double *uc, int32_t n, const uint8_t *mask,
                       double u_obstacle, double *uhat)
{
    const double s = (double)(nc - 1) / (double)(n - 1);
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < n; i++) {
            const int64_t k = j * n + i;
            double v = q1_full(uc, nc, (double)i * s, (double)j * s);
            if (mask[k] == MASK_TARGET) v = 0.0;
            else if (mask[k] == MASK_OBSTACLE) v = u_obstacle;
            uhat[k] = v;
        }
    }
}

/* Discrete feedback synthesis (Section 4.3, eq. discrete-synthesis) with the
 * discount: a*(x_i) = argmin_a { beta u_hat(x_i + h f(x_i,a)) + h l(x_i, a) },
 * sigma = 0, ties to the lowest control index.  a_out = 255 on non-free nodes. */
void orc_synthesis(const orc_problem *P, const double *uhat, uint8_t *a_out)
{
    const int64_t N = (int64_t)P->n * P->n;
    const double beta = orc_beta(P);
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] != MASK_FREE) { a_out[k] = 255; continue; }
        double best = INFINITY;
        int best_m = 0;
        for (int m = 0; m < P->n_controls; m++) {
            double xi, eta;
            foot(P, k, m, &xi, &eta);
            double v = beta * q1_full(uhat, P->n, xi, eta) + running_cost(P, k, m);
            if (v < best) { best = v; best_m = m; }
        }
        a_out[k] = (uint8_t)best_m;
    }
}

/* The synthesis objective beta u_hat(foot) + h l(x, a) for every control at the
 * listed nodes: vals[t*N_A + m].  Used to decide near-ties. */
void orc_synthesis_values(const orc_problem *P, const double *uhat, const int64_t *nodes,
                          int64_t n_nodes, double *vals)
{
    const double beta = orc_beta(P);
    for (int64_t t = 0; t < n_nodes; t++) {
        for (int m = 0; m < P->n_controls; m++) {
            double xi, eta;
            foot(P, nodes[t], m, &xi, &eta);
            vals[t * P->n_controls + m] = beta * q1_full(uhat, P->n, xi, eta) +
                                          running_cost(P, nodes[t], m);
        }
    }
}

/* Successor of each free node along the synthesised feedback: the transport
 * step phi_p(x_i) = phi_p(x_i + h f(x_i, a*(x_i))) of eq. discrete-advection
 * (Section 4.3) read winner-take-all, i.e. the node takes the patch of the cell
 * vertex carrying the largest Q1 weight at the foot, x_i itself excluded
 * (it cannot inform itself, cf. the self-dependency removal of Section 3).
 *
 * The foot is computed with a prescribed sequence of IEEE FP32 operations
 * (s = (float)(h/dx); t = c*ax; t = t + bx; t = s*t; xi = (float)i + t) so that
 * the integer result is reproducible on any IEEE machine.  The largest-weight
 * vertex rounds each coordinate (fraction 0.5 rounds down: equal weights go to
 * the lower index).  If that vertex is x_i, the second-largest is taken by
 * moving along the axis whose fraction is closer to 1/2; equal distances go to
 * the lower linear index.  A foot exactly at x_i gives succ = k (a self-loop).
 * Non-free nodes are terminal: succ = k. */
void orc_successors(const orc_problem *P, const uint8_t *a, int32_t *succ)
{
    const int n = P->n;
    const int64_t N = (int64_t)n * n;
    const float s = (float)(P->h / orc_dx(P));
    const float top = (float)(n - 1);
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] != MASK_FREE) { succ[k] = (int32_t)k; continue; }
        const int i = (int)(k % n), j = (int)(k / n);
        const int m = a[k];
        const float c = P->speed[k];
        const float ax = (float)P->controls[2 * m], ay = (float)P->controls[2 * m + 1];
        const float bx = P->drift ? P->drift[2 * k] : 0.0f;
        const float by = P->drift ? P->drift[2 * k + 1] : 0.0f;
        float tx = c * ax;
        tx = tx + bx;
        tx = s * tx;
        float ty = c * ay;
        ty = ty + by;
        ty = s * ty;
        float xi = (float)i + tx;
        float eta = (float)j + ty;
        if (xi < 0.0f) xi = 0.0f;
        if (xi > top) xi = top;
        if (eta < 0.0f) eta = 0.0f;
        if (eta > top) eta = top;
        int cx = (int)floorf(xi), cy = (int)floorf(eta);
        if (cx > n - 2) cx = n - 2;
        if (cy > n - 2) cy = n - 2;
        const float fx = xi - (float)cx, fy = eta - (float)cy;
        int vx = cx + (fx > 0.5f ? 1 : 0);
        int vy = cy + (fy > 0.5f ? 1 : 0);
        if (vx == i && vy == j) {
            if (xi == (float)i && eta == (float)j) { succ[k] = (int32_t)k; continue; }
            const float ex = fabsf(fx - 0.5f), ey = fabsf(fy - 0.5f);
            const int ox = (vx == cx) ? cx + 1 : cx;   /* other x-vertex of the cell */
            const int oy = (vy == cy) ? cy + 1 : cy;
            const int64_t kx = (int64_t)vy * n + ox;   /* flip x */
            const int64_t ky = (int64_t)oy * n + vx;   /* flip y */
            if (ex < ey) succ[k] = (int32_t)kx;
            else if (ey < ex) succ[k] = (int32_t)ky;
            else succ[k] = (int32_t)(kx < ky ? kx : ky);
        } else {
            succ[k] = (int32_t)((int64_t)vy * n + vx);
        }
    }
}

/* Patch labels (Section 4.3: Omega_p = nodes carried to Gamma_p by the
 * transport).  Every node takes the label of the end of its successor chain:
 * the sector of a target node (0..N_P-1), or N_P ("leftover") when the chain
 * ends at an obstacle, at a target node without sector, or in a cycle.
 * Memoised chain walk; labels of non-free nodes are their own terminal label. */
int32_t orc_labels(int32_t n, const int32_t *succ, const uint8_t *mask, const int8_t *sector,
                   int32_t n_patches, int8_t *label)
{
    const int64_t N = (int64_t)n * n;
    uint8_t *state = (uint8_t *)calloc((size_t)N, 1);   /* 0 new, 1 on path, 2 done */
    int64_t *path = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!state || !path) { free(state); free(path); return -1; }
    for (int64_t k0 = 0; k0 < N; k0++) {
        if (state[k0] == 2) continue;
        int64_t len = 0, k = k0;
        int8_t lab;
        for (;;) {
            if (state[k] == 2) { lab = label[k]; break; }
            if (state[k] == 1) { lab = (int8_t)n_patches; break; }        /* cycle */
            if (mask[k] != MASK_FREE) {                                    /* terminal */
                lab = (mask[k] == MASK_TARGET && sector[k] >= 0) ? sector[k] : (int8_t)n_patches;
                label[k] = lab;
                state[k] = 2;
                break;
            }
            if (succ[k] == k) { lab = (int8_t)n_patches; break; }          /* self-loop */
            state[k] = 1;
            path[len++] = k;
            k = succ[k];
        }
        for (int64_t t = 0; t < len; t++) {
            label[path[t]] = lab;
            state[path[t]] = 2;
        }
        if (state[k0] != 2) { label[k0] = lab; state[k0] = 2; }
    }
    free(state);
    free(path);
    return 0;
}

/* Causal band of each free node (Section 4.2: nodes are processed by
 * increasing u_hat).  Bands are intervals of the travel-time scale
 * T(u) = -log(1 - lambda u)/lambda (T = u when lambda = 0), on which one
 * characteristic step costs about h: band k holds T in [k w, (k+1) w).  With
 * lambda > 0 the band edges are taken on the value scale,
 * e_k = T^{-1}(k w) = (1 - exp(-(lambda (k w)))) / lambda for k = 1 .. L-1 with
 * L = min(n_bands, floor(log(1e6) / (lambda w)) + 2) (travel times beyond
 * log(1e6)/lambda, i.e. lambda u > 1 - 1e-6, share the last band), and the key of
 * u is the number of edges <= u, an exact comparison of u with FP64 edges; with
 * lambda = 0 the key is floor(u / w), capped at n_bands - 1.  u < 0 counts as 0.
 * keys = -1 on non-free nodes. */
void orc_band_keys(int64_t N, const double *uhat, const uint8_t *mask, double lambda,
                   double width, int32_t n_bands, int32_t *keys)
{
    int64_t L = 0;
    double *edge = NULL;
    if (lambda > 0.0) {
        const double span = floor(log(1e6) / (lambda * width));
        L = span + 2.0 < (double)n_bands ? (int64_t)span + 2 : n_bands;
        edge = (double *)malloc((size_t)L * sizeof(double));
        edge[0] = 0.0;
        for (int64_t k = 1; k < L; k++)
            edge[k] = (1.0 - exp(-(lambda * ((double)k * width)))) / lambda;
    }
    for (int64_t k = 0; k < N; k++) {
        if (mask[k] != MASK_FREE) { keys[k] = -1; continue; }
        const double u = uhat[k] < 0.0 ? 0.0 : uhat[k];
        if (lambda > 0.0) {
            /* number of edges e_1 .. e_{L-1} that are <= u (binary search) */
            int64_t lo = 0, hi = L - 1;       /* answer in [lo, hi] */
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                if (edge[mid] <= u) lo = mid; else hi = mid - 1;
            }
            keys[k] = (int32_t)lo;
        } else {
            const double b = floor(u / width);
            keys[k] = b >= (double)(n_bands - 1) ? n_bands - 1 : (int32_t)b;
        }
    }
    free(edge);
}
