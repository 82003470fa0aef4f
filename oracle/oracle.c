/*
 * oracle.c -- plain, slow, obviously correct CPU reference (test infrastructure).
 *
 * This file is test infrastructure.  Only the tests, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares no code, header, table or
 * helper with the CUDA path.  Arithmetic is scalar IEEE double with separate
 * multiply and add (build with -O2 -ffp-contract=off, no -ffast-math), loops
 * in the order the definitions state them.  The optional thread count only
 * splits independent instances / columns across POSIX threads; it does not
 * change any arithmetic.
 *
 * Pinned functions (the CPU tests check them against closed forms, special
 * cases, brute force and library routines):
 *   oracle_update_chain   -- the batched update chain of the paper's Eigen
 *                            benchmark (Sec. 5, Listings eigen1/eigen2),
 *                            in the stable form X_{k+1} = X_k + c X_k A.
 *   oracle_update_chain_uneven -- the same chain over a work list of
 *                            instances with their own n and T.
 *   oracle_ltimes         -- Kripke's LTimes contraction (Sec. 5.2, Listing
 *                            kripold: six storage orders chosen at run time).
 *   oracle_lplustimes     -- its adjoint, in[d][g][z] += sum_m L+[d][m]
 *                            out[m][g][z], with the same storage orders.
 *   oracle_ltimes_sample  -- single output elements of LTimes, for sampled
 *                            checks at sizes the full oracle cannot finish.
 *   oracle_mlp_*, oracle_adam -- the cost model's 3-layer MLP, MSE loss,
 *                            hand-derived backward pass and Adam step (the
 *                            paper's future-work autotuning, Sec. 6).
 *   oracle_eigen_bench    -- the paper's literal Eigen recurrence
 *                            M = Ones + 5e-5 (M + M M) from
 *                            M(i, j) = i + n j (Sec. 5, Listing eigen1).
 *   oracle_eigen_recurrence -- the same recurrence over a batch of starting
 *                            matrices, for any constant c.
 *   oracle_mass           -- the mass operator of tensor-product finite
 *                            elements (the Laghos kernel of Sec. 5), from its
 *                            finite-element definition y = B^T diag(op) B x
 *                            with B a Kronecker product formed explicitly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Update chain (Sec. 5, Eigen benchmark; stable form).                      */
/*                                                                           */
/* Per instance b: c = 1/(N*T); X_0 = I;                                     */
/*   repeat T times: P[i][j] = sum_{l=0}^{N-1} X[i][l] * A[l][j] (l ascending) */
/*                   X[i][j] = X[i][j] + c * P[i][j]                         */
/* layout 0: A and X stored row-major per instance (element (r,s) at r*N+s); */
/* layout 1: column-major (element (r,s) at s*N+r).                           */
/* ------------------------------------------------------------------------ */

static void chain_one(int n, int steps, int layout, const double *A, double *X)
{
    const double c = 1.0 / ((double)n * (double)steps);
    double *x = (double *)malloc(sizeof(double) * (size_t)n * n);   /* logical row-major */
    double *p = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *a = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s)
            a[r * n + s] = (layout == 0) ? A[r * n + s] : A[s * n + r];
    for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s)
            x[r * n + s] = (r == s) ? 1.0 : 0.0;
    for (int k = 0; k < steps; ++k) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double sum = 0.0;
                for (int l = 0; l < n; ++l)
                    sum = sum + x[i * n + l] * a[l * n + j];
                p[i * n + j] = sum;
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                x[i * n + j] = x[i * n + j] + c * p[i * n + j];
    }
    for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
            if (layout == 0) X[r * n + s] = x[r * n + s];
            else             X[s * n + r] = x[r * n + s];
        }
    free(x);
    free(p);
    free(a);
}

typedef struct {
    int n, steps, layout;
    int64_t b0, b1;
    const double *A;
    double *X;
} chain_job;

static void *chain_worker(void *arg)
{
    chain_job *j = (chain_job *)arg;
    const int64_t nn = (int64_t)j->n * j->n;
    for (int64_t b = j->b0; b < j->b1; ++b)
        chain_one(j->n, j->steps, j->layout, j->A + b * nn, j->X + b * nn);
    return NULL;
}

/* Returns 0 on success, -1 on invalid arguments. */
int oracle_update_chain(int n, int steps, int layout, int64_t batch,
                        const double *A, double *X, int nthreads)
{
    if (n < 1 || steps < 1 || (layout != 0 && layout != 1) || batch < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((int64_t)nthreads > batch) nthreads = batch > 0 ? (int)batch : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    chain_job *jobs = (chain_job *)malloc(sizeof(chain_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].n = n; jobs[t].steps = steps; jobs[t].layout = layout;
        jobs[t].b0 = batch * t / nthreads;
        jobs[t].b1 = batch * (t + 1) / nthreads;
        jobs[t].A = A; jobs[t].X = X;
        pthread_create(&th[t], NULL, chain_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return 0;
}

/* Same recurrence for instances of different size and step count packed in
 * one pool: instance k has size n[k], steps t[k], and its A / X start at
 * element off[k] of the pools (row-major). */
int oracle_update_chain_uneven(int64_t count, const int64_t *n, const int64_t *t,
                               const int64_t *off, const double *A_pool, double *X_pool)
{
    for (int64_t k = 0; k < count; ++k) {
        if (n[k] < 1 || t[k] < 1) return -1;
        chain_one((int)n[k], (int)t[k], 0, A_pool + off[k], X_pool + off[k]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LTimes contraction (Sec. 5.2, Kripke; storage orders of Listing kripold). */
/*                                                                           */
/* out[m][g][z] = sum_{d=0}^{D-1} L[m][d] * in[d][g][z]   (d ascending)       */
/* on logical indices.  L is [M][D] row-major.  A storage order lists the    */
/* three logical axes (x = d or m, g, z) slowest to fastest:                 */
/*   0 XGZ, 1 XZG, 2 GXZ, 3 GZX, 4 ZXG, 5 ZGX.                                */
/* ------------------------------------------------------------------------ */

static int64_t phys_offset(int layout, int64_t ex, int64_t eg, int64_t ez,
                           int64_t x, int64_t g, int64_t z)
{
    switch (layout) {
    case 0: return (x * eg + g) * ez + z;   /* X G Z */
    case 1: return (x * ez + z) * eg + g;   /* X Z G */
    case 2: return (g * ex + x) * ez + z;   /* G X Z */
    case 3: return (g * ez + z) * ex + x;   /* G Z X */
    case 4: return (z * ex + x) * eg + g;   /* Z X G */
    case 5: return (z * eg + g) * ex + x;   /* Z G X */
    default: return -1;
    }
}

typedef struct {
    int M, D, lin, lout;
    int64_t G, Z, g0, g1;
    const double *L, *in;
    double *out;
} lt_job;

static void *ltimes_worker(void *arg)
{
    lt_job *j = (lt_job *)arg;
    for (int64_t g = j->g0; g < j->g1; ++g)
        for (int m = 0; m < j->M; ++m)
            for (int64_t z = 0; z < j->Z; ++z) {
                double sum = 0.0;
                for (int d = 0; d < j->D; ++d)
                    sum = sum + j->L[(int64_t)m * j->D + d] *
                                j->in[phys_offset(j->lin, j->D, j->G, j->Z, d, g, z)];
                j->out[phys_offset(j->lout, j->M, j->G, j->Z, m, g, z)] = sum;
            }
    return NULL;
}

int oracle_ltimes(int M, int D, int64_t G, int64_t Z, int layout_in, int layout_out,
                  const double *L, const double *in, double *out, int nthreads)
{
    if (M < 1 || D < 1 || G < 0 || Z < 0 || layout_in < 0 || layout_in > 5 ||
        layout_out < 0 || layout_out > 5) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((int64_t)nthreads > G) nthreads = G > 0 ? (int)G : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    lt_job *jobs = (lt_job *)malloc(sizeof(lt_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (lt_job){M, D, layout_in, layout_out, G, Z,
                           G * t / nthreads, G * (t + 1) / nthreads, L, in, out};
        pthread_create(&th[t], NULL, ltimes_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return 0;
}

/* LPlusTimes, the adjoint contraction named beside LTimes in Sec. 5.2:
 *   in[d][g][z] = in[d][g][z] + sum_{m=0}^{M-1} Lp[d][m] * out[m][g][z]   (m ascending)
 * Lp is [D][M] row-major; `in` (order layout_in) is accumulated into. */
int oracle_lplustimes(int M, int D, int64_t G, int64_t Z, int layout_in, int layout_out,
                      const double *Lp, const double *out, double *in)
{
    if (M < 1 || D < 1 || G < 0 || Z < 0 || layout_in < 0 || layout_in > 5 ||
        layout_out < 0 || layout_out > 5) return -1;
    for (int64_t g = 0; g < G; ++g)
        for (int d = 0; d < D; ++d)
            for (int64_t z = 0; z < Z; ++z) {
                double sum = 0.0;
                for (int m = 0; m < M; ++m)
                    sum = sum + Lp[(int64_t)d * M + m] *
                                out[phys_offset(layout_out, M, G, Z, m, g, z)];
                const int64_t o = phys_offset(layout_in, D, G, Z, d, g, z);
                in[o] = in[o] + sum;
            }
    return 0;
}

/* Sampled outputs: out at the canonical (m, g, z) triples listed in idx
 * (3 entries per sample).  Used to check full-size results one by one. */
int oracle_ltimes_sample(int M, int D, int64_t G, int64_t Z, int layout_in,
                         const double *L, const double *in,
                         int64_t nsamples, const int64_t *idx, double *vals)
{
    for (int64_t s = 0; s < nsamples; ++s) {
        int64_t m = idx[3 * s], g = idx[3 * s + 1], z = idx[3 * s + 2];
        if (m < 0 || m >= M || g < 0 || g >= G || z < 0 || z >= Z) return -1;
        double sum = 0.0;
        for (int d = 0; d < D; ++d)
            sum = sum + L[m * D + d] * in[phys_offset(layout_in, D, G, Z, d, g, z)];
        vals[s] = sum;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cost model MLP (future-work autotuning, Sec. 6): F -> H -> H -> 1, ReLU.  */
/*   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3           */
/*   loss = (1/B) sum_b (y_b - t_b)^2                                         */
/* W1 is [H][F], W2 is [H][H], row-major (output index slowest).             */
/* relu'(0) is taken as 0.                                                   */
/* ------------------------------------------------------------------------ */

static double relu(double v) { return v > 0.0 ? v : 0.0; }

void oracle_mlp_forward(int F, int H, int64_t B,
                        const double *W1, const double *b1, const double *W2,
                        const double *b2, const double *w3, const double *b3,
                        const double *X, double *y, double *h1_out, double *h2_out)
{
    double *h1 = (double *)malloc(sizeof(double) * H);
    double *h2 = (double *)malloc(sizeof(double) * H);
    for (int64_t b = 0; b < B; ++b) {
        const double *x = X + b * F;
        for (int o = 0; o < H; ++o) {
            double s = b1[o];
            for (int i = 0; i < F; ++i) s = s + W1[o * F + i] * x[i];
            h1[o] = relu(s);
        }
        for (int o = 0; o < H; ++o) {
            double s = b2[o];
            for (int i = 0; i < H; ++i) s = s + W2[o * H + i] * h1[i];
            h2[o] = relu(s);
        }
        double s = b3[0];
        for (int i = 0; i < H; ++i) s = s + w3[i] * h2[i];
        y[b] = s;
        if (h1_out) memcpy(h1_out + b * H, h1, sizeof(double) * H);
        if (h2_out) memcpy(h2_out + b * H, h2, sizeof(double) * H);
    }
    free(h1);
    free(h2);
}

/* Loss and its gradient with respect to every parameter (backward pass by
 * the chain rule, written out by hand).  Gradients are overwritten. */
double oracle_mlp_loss_grad(int F, int H, int64_t B,
                            const double *W1, const double *b1, const double *W2,
                            const double *b2, const double *w3, const double *b3,
                            const double *X, const double *t,
                            double *gW1, double *gb1, double *gW2, double *gb2,
                            double *gw3, double *gb3)
{
    memset(gW1, 0, sizeof(double) * H * F);
    memset(gb1, 0, sizeof(double) * H);
    memset(gW2, 0, sizeof(double) * H * H);
    memset(gb2, 0, sizeof(double) * H);
    memset(gw3, 0, sizeof(double) * H);
    gb3[0] = 0.0;
    double *z1 = (double *)malloc(sizeof(double) * H);
    double *h1 = (double *)malloc(sizeof(double) * H);
    double *z2 = (double *)malloc(sizeof(double) * H);
    double *h2 = (double *)malloc(sizeof(double) * H);
    double *d2 = (double *)malloc(sizeof(double) * H);
    double *d1 = (double *)malloc(sizeof(double) * H);
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        const double *x = X + b * F;
        for (int o = 0; o < H; ++o) {
            double s = b1[o];
            for (int i = 0; i < F; ++i) s = s + W1[o * F + i] * x[i];
            z1[o] = s;
            h1[o] = relu(s);
        }
        for (int o = 0; o < H; ++o) {
            double s = b2[o];
            for (int i = 0; i < H; ++i) s = s + W2[o * H + i] * h1[i];
            z2[o] = s;
            h2[o] = relu(s);
        }
        double y = b3[0];
        for (int i = 0; i < H; ++i) y = y + w3[i] * h2[i];
        double r = y - t[b];
        loss = loss + r * r;
        double dy = 2.0 * r / (double)B;          /* d loss / d y_b */
        gb3[0] = gb3[0] + dy;
        for (int i = 0; i < H; ++i) {
            gw3[i] = gw3[i] + dy * h2[i];
            d2[i] = (z2[i] > 0.0) ? dy * w3[i] : 0.0;   /* d loss / d z2 */
        }
        for (int o = 0; o < H; ++o) {
            gb2[o] = gb2[o] + d2[o];
            for (int i = 0; i < H; ++i) gW2[o * H + i] = gW2[o * H + i] + d2[o] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int o = 0; o < H; ++o) s = s + W2[o * H + i] * d2[o];
            d1[i] = (z1[i] > 0.0) ? s : 0.0;               /* d loss / d z1 */
        }
        for (int o = 0; o < H; ++o) {
            gb1[o] = gb1[o] + d1[o];
            for (int i = 0; i < F; ++i) gW1[o * F + i] = gW1[o * F + i] + d1[o] * x[i];
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(d2); free(d1);
    return loss / (double)B;
}

/* One Adam step (Kingma and Ba, 2015) on a flat parameter vector; step is
 * the 1-based step number used for bias correction. */
void oracle_adam(int64_t count, double *theta, const double *grad, double *m, double *v,
                 int64_t step, double lr, double beta1, double beta2, double eps)
{
    const double c1 = 1.0 - pow(beta1, (double)step);
    const double c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        const double mh = m[i] / c1;
        const double vh = v[i] / c2;
        theta[i] = theta[i] - lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* The paper's literal Eigen benchmark recurrence (Sec. 5, Listing eigen1):  */
/*   m(i,j) = i + size*j initially; repeat: m = Ones + 5e-5 * (m + m*m).     */
/* Output m after `repeat` iterations, row-major.                            */
/* ------------------------------------------------------------------------ */

/* The same recurrence for a batch of caller-given starts M0 (batch*n*n,     */
/* row-major) and scale c: M_{k+1} = Ones + c * (M_k + M_k * M_k).           */
void oracle_eigen_recurrence(long long batch, int n, int repeat, double c, const double *M0, double *out)
{
    double *m = (double *)malloc(sizeof(double) * n * n);
    double *q = (double *)malloc(sizeof(double) * n * n);
    for (long long b = 0; b < batch; ++b) {
        memcpy(m, M0 + b * n * n, sizeof(double) * n * n);
        for (int r = 0; r < repeat; ++r) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s = s + m[i * n + l] * m[l * n + j];
                    q[i * n + j] = s;
                }
            for (int i = 0; i < n * n; ++i) m[i] = 1.0 + c * (m[i] + q[i]);
        }
        memcpy(out + b * n * n, m, sizeof(double) * n * n);
    }
    free(m);
    free(q);
}

void oracle_eigen_bench(int n, int repeat, double *out)
{
    double *m = (double *)malloc(sizeof(double) * n * n);
    double *q = (double *)malloc(sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) m[i * n + j] = (double)(i + n * j);
    for (int r = 0; r < repeat; ++r) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int l = 0; l < n; ++l) s = s + m[i * n + l] * m[l * n + j];
                q[i * n + j] = s;
            }
        for (int i = 0; i < n * n; ++i) m[i] = 1.0 + 5e-5 * (m[i] + q[i]);
    }
    memcpy(out, m, sizeof(double) * n * n);
    free(m);
    free(q);
}

/* ------------------------------------------------------------------------ */
/* Mass operator of tensor-product finite elements (the Laghos kernel of    */
/* Sec. 5, whose specializations are keyed on the dimension, the dofs per   */
/* dimension and the quadrature points per dimension).  The paper does not  */
/* state the operator; this is its standard finite-element definition      */
/* ("partial assembly" of the mass matrix):                                 */
/*                                                                           */
/*   y_e = B^T diag(op_e) B x_e    for every element e,                     */
/*                                                                           */
/* with B the Kronecker product of DIM copies of the 1-D basis matrix       */
/* B1[q][d] = phi_d(xi_q) (Q x D, row-major): B[k][j] = prod_i B1[k_i][j_i] */
/* for quadrature multi-index k and dof multi-index j.  x_e, y_e hold D^DIM */
/* values, op_e Q^DIM values (quadrature weight x |J| x density), each with */
/* the first index fastest: j = (j_3 D + j_2) D + j_1.                      */
/* Here B is formed explicitly, entry by entry, and applied as two dense    */
/* matrix-vector products (no sum factorization).                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dim, D, Q;
    int64_t e0, e1;
    const double *B1, *op, *x;
    double *y;
} mass_job;

static void *mass_worker(void *arg)
{
    mass_job *j = (mass_job *)arg;
    const int D = j->D, Q = j->Q, dim = j->dim;
    int nd = 1, nq = 1;
    for (int i = 0; i < dim; ++i) {
        nd *= D;
        nq *= Q;
    }
    double *B = (double *)malloc(sizeof(double) * (size_t)nq * nd);
    double *u = (double *)malloc(sizeof(double) * (size_t)nq);
    for (int k = 0; k < nq; ++k)
        for (int jj = 0; jj < nd; ++jj) {
            double v = 1.0;
            int kr = k, jr = jj;
            for (int i = 0; i < dim; ++i) {
                v = v * j->B1[(kr % Q) * D + (jr % D)];
                kr /= Q;
                jr /= D;
            }
            B[(size_t)k * nd + jj] = v;
        }
    for (int64_t e = j->e0; e < j->e1; ++e) {
        const double *x = j->x + e * nd, *op = j->op + e * nq;
        double *y = j->y + e * nd;
        for (int k = 0; k < nq; ++k) {
            double s = 0.0;
            for (int jj = 0; jj < nd; ++jj) s = s + B[(size_t)k * nd + jj] * x[jj];
            u[k] = op[k] * s;
        }
        for (int jj = 0; jj < nd; ++jj) {
            double s = 0.0;
            for (int k = 0; k < nq; ++k) s = s + B[(size_t)k * nd + jj] * u[k];
            y[jj] = s;
        }
    }
    free(B);
    free(u);
    return NULL;
}

/* Returns 0 on success, -1 on invalid arguments (dim not 1..3, D or Q < 1). */
int oracle_mass(int dim, int D, int Q, int64_t ne, const double *B1, const double *op, const double *x, double *y,
                int nthreads)
{
    if (dim < 1 || dim > 3 || D < 1 || Q < 1 || ne < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((int64_t)nthreads > ne) nthreads = ne > 0 ? (int)ne : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    mass_job *jobs = (mass_job *)malloc(sizeof(mass_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        mass_job jb = {dim, D, Q, ne * t / nthreads, ne * (t + 1) / nthreads, B1, op, x, y};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, mass_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return 0;
}
