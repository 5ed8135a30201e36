/*
 * All-core FP64 CPU baseline of the Markov-chain semi-Lagrangian value
 * iteration (Cacace & Falcone, Section 3, eq. SLscheme3 with the discount of
 * the workloads): the plain full-grid Jacobi sweep and a Gauss-Seidel sweep in
 * increasing u_hat (Section 4.3, the nodes of each patch ordered by the
 * interpolated coarse solution), both spread over every host core with OpenMP.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY: the CPU context the GPU timings are
 * set against.  It shares no source, header or helper with the CUDA path (nor
 * with the single-threaded oracle beside it, whose plain restatement it times
 * against on one core).
 *
 * Grid: n nodes per side on [-1,1]^2, dx = 2/(n-1), node k = j*n + i at
 * (-1 + i dx, -1 + j dx).  Per free node and control a_m the foot is
 * x + h (c(x) a_m + b(x)); the 2d = 4 points of the diffusion are the foot
 * +- sqrt(2h) sigma e_1, e_2 (one point, the foot, when sigma = 0), each
 * clamped to the square and read by Q1 interpolation; the node's own Q1 weight
 * Lambda0 is split out, giving the candidate (beta Lambda1' + h l)/(1 - beta Lambda0).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n, n_controls;
    double h, lambda, sigma, cost, u_obstacle;
    const float *speed;      /* n*n */
    const float *drift;      /* n*n*2 or NULL */
    const uint8_t *mask;     /* 0 free, 1 target, 2 obstacle */
    const double *controls;  /* 2 per control */
} cpb_problem;

int cpb_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static inline double rd(const double *p)
{
    double v;
    __atomic_load(p, &v, __ATOMIC_RELAXED);
    return v;
}

static inline void wr(double *p, double v)
{
    __atomic_store(p, &v, __ATOMIC_RELAXED);
}

/* Q1 value at grid-unit point (x, y) after clamping, the weight of node `self`
 * split out into *w_self (0 when it is not a vertex of the cell). */
static inline double q1(const double *u, int n, double x, double y, int64_t self,
                        double *w_self)
{
    const double top = (double)(n - 1);
    x = x < 0.0 ? 0.0 : (x > top ? top : x);
    y = y < 0.0 ? 0.0 : (y > top ? top : y);
    int64_t ci = (int64_t)x, cj = (int64_t)y;
    if (ci > n - 2) ci = n - 2;
    if (cj > n - 2) cj = n - 2;
    const double ax = x - (double)ci, ay = y - (double)cj;
    const int64_t k00 = cj * n + ci;
    const int64_t ks[4] = {k00, k00 + 1, k00 + n, k00 + n + 1};
    const double ws[4] = {(1.0 - ax) * (1.0 - ay), ax * (1.0 - ay), (1.0 - ax) * ay, ax * ay};
    double s = 0.0;
    for (int t = 0; t < 4; t++) {
        if (ks[t] == self)
            *w_self += ws[t];
        else
            s += ws[t] * rd(u + ks[t]);
    }
    return s;
}

/* min over controls of the eq. SLscheme3 candidate at free node k */
static double update(const cpb_problem *P, const double *u, int64_t k)
{
    const int n = P->n;
    const double dx = 2.0 / (n - 1);
    const double beta = 1.0 / (1.0 + P->lambda * P->h);
    const double s = P->h / dx;
    const double r = sqrt(2.0 * P->h) * P->sigma / dx;
    const double i = (double)(k % n), j = (double)(k / n);
    const double c = (double)P->speed[k];
    const double bx = P->drift ? (double)P->drift[2 * k] : 0.0;
    const double by = P->drift ? (double)P->drift[2 * k + 1] : 0.0;
    const double hl = P->h * P->cost;
    double best = INFINITY;
    for (int m = 0; m < P->n_controls; m++) {
        const double x = i + s * (c * P->controls[2 * m] + bx);
        const double y = j + s * (c * P->controls[2 * m + 1] + by);
        double w0 = 0.0, l1;
        if (r > 0.0) {
            l1 = 0.25 * (q1(u, n, x + r, y, k, &w0) + q1(u, n, x - r, y, k, &w0) +
                         q1(u, n, x, y + r, k, &w0) + q1(u, n, x, y - r, k, &w0));
            w0 *= 0.25;
        } else {
            l1 = q1(u, n, x, y, k, &w0);
        }
        const double den = 1.0 - beta * w0;
        if (den > 0.0) {
            const double v = (beta * l1 + hl) / den;
            if (v < best) best = v;
        }
    }
    return best;
}

/* Non-free nodes hold their fixed values: 0 on the target, u_obstacle on obstacles. */
void cpb_fix(const cpb_problem *P, double *u)
{
    const int64_t N = (int64_t)P->n * P->n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] == 1) u[k] = 0.0;
        else if (P->mask[k] == 2) u[k] = P->u_obstacle;
    }
}

/* One Jacobi sweep: out = T u on free nodes (others copied); returns sup |Tu - u|. */
double cpb_jacobi(const cpb_problem *P, const double *u, double *out)
{
    const int64_t N = (int64_t)P->n * P->n;
    double inc = 0.0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(max : inc)
    for (int64_t k = 0; k < N; k++) {
        if (P->mask[k] != 0) {
            out[k] = u[k];
            continue;
        }
        const double v = update(P, u, k);
        const double d = fabs(v - u[k]);
        if (d > inc) inc = d;
        out[k] = v;
    }
    return inc;
}

/* One Gauss-Seidel sweep over every thread's node list in its order (list t =
 * nodes[off[t] .. off[t+1]-1], one list per thread: e.g. the free nodes of a
 * block of rows sorted by u_hat); threads update the shared array in place, so
 * values written by one are read by the others as they appear (a chaotic
 * relaxation of the same contraction).  Returns sup |increment|. */
double cpb_gs(const cpb_problem *P, double *u, const int64_t *nodes, const int64_t *off,
              int32_t lists)
{
    double inc = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : inc)
    for (int32_t t = 0; t < lists; t++) {
        for (int64_t q = off[t]; q < off[t + 1]; q++) {
            const int64_t k = nodes[q];
            const double v = update(P, u, k);
            const double d = fabs(v - rd(u + k));
            if (d > inc) inc = d;
            wr(u + k, v);
        }
    }
    return inc;
}
