/*
 * Plain FP64 CPU oracle for the Chebyshev-interpolation butterfly.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (Poulson, Demanet, Maxwell, Ying, "A Parallel Butterfly
 * Algorithm"):
 *
 *   direct sum   f(x) = sum_y K(x,y) g(y),  K(x,y) = exp(2 pi i Phi(x,y))
 *                (the operator of Section 1, the potential f^{AB} of Eq. 1 with
 *                A = X, B = Y; kernel of Eq. "phase" written with the 2 pi
 *                outside Phi).
 *
 *   butterfly    Algorithm 1 ("Sequential butterfly algorithm"): initialise the
 *                weights w_{XB} of every leaf source box, translate them through
 *                log2 N stages (w_{A_c B_p} += T w_{AB} for every pair and every
 *                child A_c of A), evaluate f_{AY} = U_{AY} w_{AY} at the end.
 *                The translation operators are the analytic tensor-product
 *                Chebyshev interpolation of Section 1.4: column-space
 *                interpolation while source boxes are small, a switch to
 *                row-space interpolation in the middle (level m = floor(L/2)),
 *                row-space interpolation afterwards.  Section 1.4 defers the
 *                explicit formulas to the Candes-Demanet-Ying butterfly paper;
 *                they are restated here from that method's mathematics:
 *
 *     init   delta_t^{XB} = e^{-2pi i Phi(x0(X), y_t^B)} sum_{y in B} L_t^B(y) e^{2pi i Phi(x0(X), y)} g(y)
 *     column w_{A_c,B_p}(t) += e^{-2pi i Phi(x0(A_c), y_t^{B_p})}
 *                               sum_t' L_t^{B_p}(y_t'^B) e^{2pi i Phi(x0(A_c), y_t'^B)} w_{A,B}(t')
 *     switch delta_s^{AB} <- sum_t e^{2pi i Phi(x_s^A, y_t^B)} delta_t^{AB}          (level m)
 *     row    w_{A_c,B_p}(s) += e^{2pi i Phi(x_s^{A_c}, y0(B))}
 *                               sum_t L_t^A(x_s^{A_c}) e^{-2pi i Phi(x_t^A, y0(B))} w_{A,B}(t)
 *     final  f(x) = e^{2pi i Phi(x, y0(Y))} sum_t L_t^A(x) e^{-2pi i Phi(x_t^A, y0(Y))} w_{A,Y}(t)
 *
 *   adjoint      the exact conjugate transpose of the approximate operator
 *                above: every step conjugate-transposed, stages in reverse.
 *
 * Readings where the paper is silent (identical in the CUDA path):
 *   - Chebyshev-Lobatto nodes z_j = cos(j pi/(q-1))/2 on [-1/2,1/2]
 *     (node_kind 0), or first-kind nodes cos((2j+1) pi/(2q))/2 (node_kind 1);
 *   - switch level m = floor(L/2) unless given;
 *   - one point per leaf box, at offset (lower corner + off * width);
 *   - Morton order with dimension 0 in the lowest bit; node index
 *     t = sum_k t_k q^k; child index c = sum_k c_k 2^k;
 *   - e^{2 pi i Phi} is evaluated as cos/sin of 2 pi (Phi - nearbyint(Phi)).
 *
 * Everything is FP64 and written as plain loops; OpenMP only distributes
 * independent outer iterations.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORC_DOT = 0, ORC_GENRADON = 1, ORC_HYPRADON = 2, ORC_SEPARABLE = 3, ORC_GENRADON_PAPER = 4 };

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOMEM = 2 };

typedef struct {
    int32_t d;          /* dimension, 1..3                                   */
    int32_t L;          /* N = 2^L points per dimension                      */
    int32_t q;          /* Chebyshev nodes per dimension, r = q^d            */
    int32_t m;          /* switch level, 0 <= m <= L                         */
    int32_t phase;      /* ORC_* phase kind                                  */
    int32_t node_kind;  /* 0 Lobatto, 1 first kind                           */
    double scale;       /* Phi is multiplied by this                         */
    double x_lo[3], x_w[3];  /* target domain X = prod [x_lo, x_lo + x_w)    */
    double y_lo[3], y_w[3];  /* source domain Y = prod [y_lo, y_lo + y_w)    */
    double tgt_off, src_off; /* point position inside its leaf box, in widths */
} orc_problem;

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ phase */

/* Phi(x, y) in cycles: K = exp(2 pi i Phi). */
double orc_phi(const orc_problem *P, const double *x, const double *y)
{
    const int d = P->d;
    double s = 0.0;
    switch (P->phase) {
    case ORC_DOT: /* Fourier kernel, Section 3 */
        for (int k = 0; k < d; ++k) s += x[k] * y[k];
        break;
    case ORC_GENRADON: { /* generalized Radon analogue, 2-pi form, Section 3.2 */
        double xy = 0.0, q2 = 0.0;
        for (int k = 0; k < d; ++k) xy += x[k] * y[k];
        if (d == 2) {
            double a0 = (2.0 + sin(TWO_PI * x[0]) * sin(TWO_PI * x[1])) / 3.0;
            double a1 = (2.0 + cos(TWO_PI * x[0]) * cos(TWO_PI * x[1])) / 3.0;
            q2 = a0 * a0 * y[0] * y[0] + a1 * a1 * y[1] * y[1];
        } else {
            for (int k = 0; k < d; ++k) {
                double a = (2.0 + sin(TWO_PI * x[k]) * cos(TWO_PI * x[(k + 1) % d])) / 3.0;
                q2 += a * a * y[k] * y[k];
            }
        }
        s = xy + sqrt(q2);
        break;
    }
    case ORC_HYPRADON: /* hyperbolic Radon, Section 3.1: x = (w, h), y = (tau, p) */
        s = x[0] * sqrt(y[0] * y[0] + y[1] * y[1] * x[1] * x[1]);
        break;
    case ORC_SEPARABLE: { /* Phi = a(x) + b(y): the butterfly is exact for it */
        double a = 0.0, b = 0.0;
        for (int k = 0; k < d; ++k) {
            a += sin(TWO_PI * (x[k] + (k + 1) / 7.0));
            b += y[k] * y[k] / (k + 2.0);
        }
        s = a + b;
        break;
    }
    case ORC_GENRADON_PAPER: { /* Section 3.2 as printed: gamma, kappa use x0,x1,p0,p1 */
        double xy = 0.0;
        for (int k = 0; k < d; ++k) xy += x[k] * y[k];
        double g = y[0] * (2.0 + sin(TWO_PI * x[0]) * sin(TWO_PI * x[1])) / 3.0;
        double kk = y[1] * (2.0 + cos(TWO_PI * x[0]) * cos(TWO_PI * x[1])) / 3.0;
        s = xy + sqrt(g * g + kk * kk);
        break;
    }
    default:
        s = 0.0;
    }
    return P->scale * s;
}

/* exp(2 pi i theta), reduced mod 1 first (round-half-even nearest integer). */
static cplx expi2pi(double theta)
{
    double f = theta - nearbyint(theta);
    return cos(TWO_PI * f) + I * sin(TWO_PI * f);
}

static cplx kern(const orc_problem *P, const double *x, const double *y)
{
    return expi2pi(orc_phi(P, x, y));
}

/* ------------------------------------------------ Chebyshev and Lagrange */

void orc_cheb_nodes(int q, int kind, double *z)
{
    for (int j = 0; j < q; ++j) {
        if (kind == 0)
            z[j] = 0.5 * cos(j * M_PI / (q - 1));
        else
            z[j] = 0.5 * cos((2 * j + 1) * M_PI / (2.0 * q));
    }
}

/* l_t(xi) = prod_{k != t} (xi - z_k) / (z_t - z_k) */
double orc_lagrange1(int q, const double *z, int t, double xi)
{
    double v = 1.0;
    for (int k = 0; k < q; ++k)
        if (k != t) v *= (xi - z[k]) / (z[t] - z[k]);
    return v;
}

/* ------------------------------------------------------------- geometry */

static int64_t ipow(int64_t b, int e)
{
    int64_t v = 1;
    while (e-- > 0) v *= b;
    return v;
}

/* per-dimension coordinates of the box with Morton index mi (bits per dim = lev) */
static void morton_decode(int d, int bits, int64_t mi, int64_t *c)
{
    for (int k = 0; k < d; ++k) c[k] = 0;
    for (int j = 0; j < bits; ++j)
        for (int k = 0; k < d; ++k)
            c[k] |= ((mi >> (j * d + k)) & 1) << j;
}

static int64_t morton_encode(int d, int bits, const int64_t *c)
{
    int64_t mi = 0;
    for (int j = 0; j < bits; ++j)
        for (int k = 0; k < d; ++k)
            mi |= ((c[k] >> j) & 1) << (j * d + k);
    return mi;
}

/* target box at level l: centre and width per dimension */
static void tbox(const orc_problem *P, int l, int64_t A, double *ctr, double *w)
{
    int64_t a[3];
    morton_decode(P->d, l, A, a);
    for (int k = 0; k < P->d; ++k) {
        w[k] = P->x_w[k] / (double)(1LL << l);
        ctr[k] = P->x_lo[k] + (a[k] + 0.5) * w[k];
    }
}

/* source box at level l (side y_w * 2^l / N): centre and width */
static void sbox(const orc_problem *P, int l, int64_t B, double *ctr, double *w)
{
    int64_t b[3];
    morton_decode(P->d, P->L - l, B, b);
    for (int k = 0; k < P->d; ++k) {
        w[k] = P->y_w[k] * (double)(1LL << l) / (double)(1LL << P->L);
        ctr[k] = P->y_lo[k] + (b[k] + 0.5) * w[k];
    }
}

/* node t of a box: centre + width * z_{t_k} per dimension */
static void node(int d, int q, const double *z, const double *ctr, const double *w, int t, double *p)
{
    for (int k = 0; k < d; ++k) {
        int tk = t % q;
        t /= q;
        p[k] = ctr[k] + w[k] * z[tk];
    }
}

/* tensor Lagrange basis of a box evaluated at point p */
static double lag(int d, int q, const double *z, const double *ctr, const double *w, int t, const double *p)
{
    double v = 1.0;
    for (int k = 0; k < d; ++k) {
        int tk = t % q;
        t /= q;
        v *= orc_lagrange1(q, z, tk, (p[k] - ctr[k]) / w[k]);
    }
    return v;
}

/*
 * One-dimensional Lagrange factors for the tensor basis of a parent box
 * (centre cp, width wp) evaluated at the nodes of a box (centre cc, width wc):
 * l1[k][t_k][s_k] = l_{t_k}((node_{s_k} - cp_k) / wp_k).  The tensor value
 * L_t(node_s) is the product over k (see lagtab).
 */
static void lag1tab(int d, int q, const double *z, const double *cp, const double *wp,
                    const double *cc, const double *wc, double l1[3][16][16])
{
    for (int k = 0; k < d; ++k)
        for (int s = 0; s < q; ++s) {
            double pk = cc[k] + wc[k] * z[s];
            for (int t = 0; t < q; ++t) l1[k][t][s] = orc_lagrange1(q, z, t, (pk - cp[k]) / wp[k]);
        }
}

static double lagtab(int d, int q, double l1[3][16][16], int t, int s)
{
    double v = 1.0;
    for (int k = 0; k < d; ++k) {
        v *= l1[k][t % q][s % q];
        t /= q;
        s /= q;
    }
    return v;
}

/* the target (or source) point with row-major flat index j (last dim fastest) */
static void point(const orc_problem *P, int is_src, int64_t j, double *p, int64_t *mort)
{
    const int d = P->d;
    const int64_t N = 1LL << P->L;
    int64_t c[3];
    for (int k = d - 1; k >= 0; --k) {
        c[k] = j % N;
        j /= N;
    }
    for (int k = 0; k < d; ++k) {
        if (is_src)
            p[k] = P->y_lo[k] + (c[k] + P->src_off) * (P->y_w[k] / (double)N);
        else
            p[k] = P->x_lo[k] + (c[k] + P->tgt_off) * (P->x_w[k] / (double)N);
    }
    if (mort) *mort = morton_encode(d, P->L, c);
}

static int64_t flat_from_morton(const orc_problem *P, int64_t mi)
{
    const int64_t N = 1LL << P->L;
    int64_t c[3], j = 0;
    morton_decode(P->d, P->L, mi, c);
    for (int k = 0; k < P->d; ++k) j = j * N + c[k];
    return j;
}

static int check(const orc_problem *P)
{
    if (!P || P->d < 1 || P->d > 3 || P->L < 0 || P->L * P->d > 40 || P->q < 2 || P->q > 16)
        return ORC_ERR_ARG;
    if (P->m < 0 || P->m > P->L) return ORC_ERR_ARG;
    return ORC_OK;
}

/* ------------------------------------------------------------ direct sum */

/* f[i] = sum_j K(x_{tgt[i]}, y_j) g[j] for the listed targets (all if tgt == NULL). */
int orc_direct_sum(const orc_problem *P, const cplx *g, int64_t ntgt, const int64_t *tgt, cplx *f)
{
    if (check(P)) return ORC_ERR_ARG;
    const int d = P->d;
    const int64_t Nd = ipow(1LL << P->L, d);
    if (!tgt) ntgt = Nd;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ntgt; ++i) {
        double x[3], y[3];
        point(P, 0, tgt ? tgt[i] : i, x, NULL);
        cplx acc = 0.0;
        for (int64_t j = 0; j < Nd; ++j) {
            point(P, 1, j, y, NULL);
            acc += kern(P, x, y) * g[j];
        }
        f[i] = acc;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------- butterfly */

/* Is target box A at level l on the path to the restriction box R at level rl? */
static int tgt_active(int d, int l, int64_t A, int rl, int64_t R)
{
    if (rl < 0) return 1;
    if (l <= rl) return (R >> (d * (rl - l))) == A;
    return (A >> (d * (l - rl))) == R;
}

/*
 * The log2 N stages of Algorithm 1 (and the switch at level m) on the level-0 weights
 * in *W; *W holds the level-L weights afterwards (*Wn is scratch; the two may be swapped).
 */
static void stages(const orc_problem *P, cplx **Wp, cplx **Wnp, int rl, int64_t R, const double *z)
{
    const int d = P->d, L = P->L, q = P->q, m = P->m;
    const int r = (int)ipow(q, d);
    const int nc = 1 << d;
    const int64_t Nd = ipow(1LL << L, d);
    cplx *W = *Wp, *Wn = *Wnp;
    for (int l = 0; l < L; ++l) {
        if (l == m) { /* switch to row-space interpolation at level m */
            const int64_t SB = ipow(1LL << (L - l), d);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t ip = 0; ip < Nd; ++ip) {
                int64_t A = ip / SB, B = ip % SB;
                if (!tgt_active(d, l, A, rl, R)) continue;
                double ca[3], wa[3], cb[3], wb[3], xs[3], yt[3];
                cplx tmp[4096];
                tbox(P, l, A, ca, wa);
                sbox(P, l, B, cb, wb);
                for (int s = 0; s < r; ++s) {
                    node(d, q, z, ca, wa, s, xs);
                    cplx acc = 0.0;
                    for (int t = 0; t < r; ++t) {
                        node(d, q, z, cb, wb, t, yt);
                        acc += kern(P, xs, yt) * W[ip * r + t];
                    }
                    tmp[s] = acc;
                }
                for (int s = 0; s < r; ++s) W[ip * r + s] = tmp[s];
            }
        }
        /* stage l: pairs (A,B) at level l -> (A_c, B_p) at level l+1 */
        const int64_t SB = ipow(1LL << (L - l), d);       /* source boxes at level l   */
        const int64_t SBp = SB / nc;                       /* source boxes at level l+1 */
        const int64_t NA = Nd / SB;                        /* target boxes at level l   */
        memset(Wn, 0, (size_t)Nd * r * sizeof(cplx));
        /* one group per (A, B_p): its 2^d children B write only to (A_c, B_p) */
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t G = 0; G < NA * SBp; ++G) {
            const int64_t A = G / SBp, Bp = G % SBp;
            double ca[3], wa[3], cbp[3], wbp[3], cb[3], wb[3], cac[3], wac[3];
            double p[3], pt[3], l1[3][16][16];
            tbox(P, l, A, ca, wa);
            sbox(P, l + 1, Bp, cbp, wbp);
            for (int cB = 0; cB < nc; ++cB) {
                const int64_t B = Bp * nc + cB;
                const cplx *w = &W[(A * SB + B) * r];
                sbox(P, l, B, cb, wb);
                if (l < m) lag1tab(d, q, z, cbp, wbp, cb, wb, l1);
                for (int cA = 0; cA < nc; ++cA) {
                    const int64_t Ac = A * nc + cA;
                    if (!tgt_active(d, l + 1, Ac, rl, R)) continue;
                    cplx *wo = &Wn[(Ac * SBp + Bp) * r];
                    tbox(P, l + 1, Ac, cac, wac);
                    if (l < m) {
                        /* column form: sources of B at its nodes -> nodes of B_p */
                        cplx u[4096];
                        for (int tp = 0; tp < r; ++tp) {
                            node(d, q, z, cb, wb, tp, p);
                            u[tp] = kern(P, cac, p) * w[tp];
                        }
                        for (int t = 0; t < r; ++t) {
                            node(d, q, z, cbp, wbp, t, pt);
                            cplx acc = 0.0;
                            for (int tp = 0; tp < r; ++tp)
                                acc += lagtab(d, q, l1, t, tp) * u[tp];
                            wo[t] += conj(kern(P, cac, pt)) * acc;
                        }
                    } else {
                        /* row form: values at nodes of A -> values at nodes of A_c */
                        cplx u[4096];
                        lag1tab(d, q, z, ca, wa, cac, wac, l1);
                        for (int t = 0; t < r; ++t) {
                            node(d, q, z, ca, wa, t, pt);
                            u[t] = conj(kern(P, pt, cb)) * w[t];
                        }
                        for (int s = 0; s < r; ++s) {
                            node(d, q, z, cac, wac, s, p);
                            cplx acc = 0.0;
                            for (int t = 0; t < r; ++t)
                                acc += lagtab(d, q, l1, t, s) * u[t];
                            wo[s] += kern(P, p, cb) * acc;
                        }
                    }
                }
            }
        }
        cplx *tmp = W;
        W = Wn;
        Wn = tmp;
    }
    if (m == L) { /* switch at the last level (m == L, e.g. L == 0) */
        const int l = L;
        for (int64_t A = 0; A < Nd; ++A) {
            if (!tgt_active(d, l, A, rl, R)) continue;
            double ca[3], wa[3], cb[3], wb[3], xs[3], yt[3];
            cplx tmp[4096];
            tbox(P, l, A, ca, wa);
            sbox(P, l, 0, cb, wb);
            for (int s = 0; s < r; ++s) {
                node(d, q, z, ca, wa, s, xs);
                cplx acc = 0.0;
                for (int t = 0; t < r; ++t) {
                    node(d, q, z, cb, wb, t, yt);
                    acc += kern(P, xs, yt) * W[A * r + t];
                }
                tmp[s] = acc;
            }
            for (int s = 0; s < r; ++s) W[A * r + s] = tmp[s];
        }
    }

    *Wp = W;
    *Wnp = Wn;
}

/*
 * Forward butterfly, Algorithm 1.  g: N^d source values (row-major);
 * f: N^d outputs.  If rl >= 0 only target boxes on the path to box R at level
 * rl are computed (a restriction of the same arithmetic: outputs for targets
 * inside R are identical to the unrestricted run, other outputs are zero).
 */
int orc_butterfly(const orc_problem *P, const cplx *g, cplx *f, int rl, int64_t R)
{
    if (check(P)) return ORC_ERR_ARG;
    if (rl > P->L) return ORC_ERR_ARG;
    const int d = P->d, L = P->L, q = P->q;
    const int r = (int)ipow(q, d);
    const int64_t Nd = ipow(1LL << L, d);
    double z[16];
    orc_cheb_nodes(q, P->node_kind, z);

    cplx *W = calloc((size_t)Nd * r, sizeof(cplx));
    cplx *Wn = calloc((size_t)Nd * r, sizeof(cplx));
    if (!W || !Wn) {
        free(W);
        free(Wn);
        return ORC_ERR_NOMEM;
    }

    /* init: A = X, one source per leaf box B (pair index = B) */
    {
        double x0[3], wx[3];
        tbox(P, 0, 0, x0, wx);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < Nd; ++j) {
            double y[3], cb[3], wb[3], yt[3];
            int64_t B;
            point(P, 1, j, y, &B);
            sbox(P, 0, B, cb, wb);
            cplx src = kern(P, x0, y) * g[j];
            for (int t = 0; t < r; ++t) {
                node(d, q, z, cb, wb, t, yt);
                W[B * r + t] = conj(kern(P, x0, yt)) * lag(d, q, z, cb, wb, t, y) * src;
            }
        }
    }

    stages(P, &W, &Wn, rl, R, z);

    /* final: B = Y, one target per leaf box A (pair index = A) */
    {
        double y0[3], wy[3];
        sbox(P, L, 0, y0, wy);
        memset(f, 0, (size_t)Nd * sizeof(cplx));
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < Nd; ++j) {
            double x[3], ca[3], wa[3], xt[3];
            int64_t A;
            point(P, 0, j, x, &A);
            if (!tgt_active(d, L, A, rl, R)) continue;
            tbox(P, L, A, ca, wa);
            cplx acc = 0.0;
            for (int t = 0; t < r; ++t) {
                node(d, q, z, ca, wa, t, xt);
                acc += lag(d, q, z, ca, wa, t, x) * conj(kern(P, xt, y0)) * W[A * r + t];
            }
            f[j] = kern(P, x, y0) * acc;
        }
    }
    free(W);
    free(Wn);
    return ORC_OK;
}

/*
 * Adjoint butterfly: g = B^H f for the operator B computed by orc_butterfly
 * (each step conjugate-transposed, stages in reverse order).
 */
int orc_butterfly_adjoint(const orc_problem *P, const cplx *f, cplx *g)
{
    if (check(P)) return ORC_ERR_ARG;
    const int d = P->d, L = P->L, q = P->q, m = P->m;
    const int r = (int)ipow(q, d);
    const int nc = 1 << d;
    const int64_t Nd = ipow(1LL << L, d);
    double z[16];
    orc_cheb_nodes(q, P->node_kind, z);

    cplx *W = calloc((size_t)Nd * r, sizeof(cplx));
    cplx *Wn = calloc((size_t)Nd * r, sizeof(cplx));
    if (!W || !Wn) {
        free(W);
        free(Wn);
        return ORC_ERR_NOMEM;
    }

    /* final^H */
    {
        double y0[3], wy[3];
        sbox(P, L, 0, y0, wy);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < Nd; ++j) {
            double x[3], ca[3], wa[3], xt[3];
            int64_t A;
            point(P, 0, j, x, &A);
            tbox(P, L, A, ca, wa);
            cplx v = conj(kern(P, x, y0)) * f[j];
            for (int t = 0; t < r; ++t) {
                node(d, q, z, ca, wa, t, xt);
                W[A * r + t] = lag(d, q, z, ca, wa, t, x) * kern(P, xt, y0) * v;
            }
        }
    }
    if (m == L) { /* switch^H at the last level (m == L) */
        double ca[3], wa[3], cb[3], wb[3], xs[3], yt[3];
        cplx tmp[4096];
        tbox(P, L, 0, ca, wa);
        sbox(P, L, 0, cb, wb);
        for (int t = 0; t < r; ++t) {
            node(d, q, z, cb, wb, t, yt);
            cplx acc = 0.0;
            for (int s = 0; s < r; ++s) {
                node(d, q, z, ca, wa, s, xs);
                acc += conj(kern(P, xs, yt)) * W[s];
            }
            tmp[t] = acc;
        }
        for (int t = 0; t < r; ++t) W[t] = tmp[t];
    }

    for (int l = L - 1; l >= 0; --l) {
        /* stage l^H: weights at level l+1 -> level l */
        const int64_t SB = ipow(1LL << (L - l), d);
        const int64_t SBp = SB / nc;
        const int64_t NA = Nd / SB;
        memset(Wn, 0, (size_t)Nd * r * sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t ip = 0; ip < NA * SB; ++ip) {
            const int64_t A = ip / SB, B = ip % SB, Bp = B / nc;
            double ca[3], wa[3], cbp[3], wbp[3], cb[3], wb[3], cac[3], wac[3];
            double p[3], pt[3];
            tbox(P, l, A, ca, wa);
            sbox(P, l + 1, Bp, cbp, wbp);
            sbox(P, l, B, cb, wb);
            cplx *wo = &Wn[ip * r];
            for (int cA = 0; cA < nc; ++cA) {
                const int64_t Ac = A * nc + cA;
                const cplx *w = &W[(Ac * SBp + Bp) * r];
                tbox(P, l + 1, Ac, cac, wac);
                if (l < m) {
                    for (int tp = 0; tp < r; ++tp) {
                        node(d, q, z, cb, wb, tp, p);
                        cplx acc = 0.0;
                        for (int t = 0; t < r; ++t) {
                            node(d, q, z, cbp, wbp, t, pt);
                            acc += lag(d, q, z, cbp, wbp, t, p) * kern(P, cac, pt) * w[t];
                        }
                        wo[tp] += conj(kern(P, cac, p)) * acc;
                    }
                } else {
                    for (int t = 0; t < r; ++t) {
                        node(d, q, z, ca, wa, t, pt);
                        cplx acc = 0.0;
                        for (int s = 0; s < r; ++s) {
                            node(d, q, z, cac, wac, s, p);
                            acc += lag(d, q, z, ca, wa, t, p) * conj(kern(P, p, cb)) * w[s];
                        }
                        wo[t] += kern(P, pt, cb) * acc;
                    }
                }
            }
        }
        cplx *tmp = W;
        W = Wn;
        Wn = tmp;
        if (l == m) { /* switch^H at level m, after the row stages have been undone */
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t ip = 0; ip < Nd; ++ip) {
                int64_t A = ip / SB, B = ip % SB;
                double ca[3], wa[3], cb[3], wb[3], xs[3], yt[3];
                cplx tmp2[4096];
                tbox(P, l, A, ca, wa);
                sbox(P, l, B, cb, wb);
                for (int t = 0; t < r; ++t) {
                    node(d, q, z, cb, wb, t, yt);
                    cplx acc = 0.0;
                    for (int s = 0; s < r; ++s) {
                        node(d, q, z, ca, wa, s, xs);
                        acc += conj(kern(P, xs, yt)) * W[ip * r + s];
                    }
                    tmp2[t] = acc;
                }
                for (int t = 0; t < r; ++t) W[ip * r + t] = tmp2[t];
            }
        }
    }

    /* init^H */
    {
        double x0[3], wx[3];
        tbox(P, 0, 0, x0, wx);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < Nd; ++j) {
            double y[3], cb[3], wb[3], yt[3];
            int64_t B;
            point(P, 1, j, y, &B);
            sbox(P, 0, B, cb, wb);
            cplx acc = 0.0;
            for (int t = 0; t < r; ++t) {
                node(d, q, z, cb, wb, t, yt);
                acc += kern(P, x0, yt) * lag(d, q, z, cb, wb, t, y) * W[B * r + t];
            }
            g[j] = conj(kern(P, x0, y)) * acc;
        }
    }
    free(W);
    free(Wn);
    return ORC_OK;
}

/* flat row-major index of the target in leaf box with Morton index mi */
/* ------------------------------------------------ arbitrary point sets */

/* Leaf box (Morton index) of a point of the source (is_src) or target domain: the box
 * whose half-open extent holds it; points on the upper face belong to the last box. */
static int64_t leaf_of(const orc_problem *P, int is_src, const double *p)
{
    const int d = P->d;
    const int64_t N = 1LL << P->L;
    int64_t c[3];
    for (int k = 0; k < d; ++k) {
        const double lo = is_src ? P->y_lo[k] : P->x_lo[k], w = is_src ? P->y_w[k] : P->x_w[k];
        int64_t ck = (int64_t)floor((p[k] - lo) / (w / (double)N));
        c[k] = ck < 0 ? 0 : (ck >= N ? N - 1 : ck);
    }
    return morton_encode(d, P->L, c);
}

/* f[i] = sum_j K(x_i, y_j) g[j] for arbitrary points (rows of x: ntgt x d, y: nsrc x d). */
int orc_direct_sum_points(const orc_problem *P, int64_t nsrc, const double *y, const cplx *g, int64_t ntgt,
                          const double *x, cplx *f)
{
    if (check(P) || nsrc < 0 || ntgt < 0) return ORC_ERR_ARG;
    const int d = P->d;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ntgt; ++i) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < nsrc; ++j) acc += kern(P, x + i * d, y + j * d) * g[j];
        f[i] = acc;
    }
    return ORC_OK;
}

/*
 * Butterfly for arbitrary sources and targets (the field of Section 1.4 evaluated
 * anywhere; sparse and clustered point sets of the future-work discussion).  Only
 * the first and last steps change: init sums over the sources that lie in each leaf
 * box, final evaluates the interpolant of the target's leaf box at the target.  Points
 * must lie in their domains (the box of a point outside is its nearest one).
 */
int orc_butterfly_points(const orc_problem *P, int64_t nsrc, const double *y, const cplx *g, int64_t ntgt,
                         const double *x, cplx *f)
{
    if (check(P) || nsrc < 0 || ntgt < 0) return ORC_ERR_ARG;
    const int d = P->d, L = P->L, q = P->q;
    const int r = (int)ipow(q, d);
    const int64_t Nd = ipow(1LL << L, d);
    double z[16];
    orc_cheb_nodes(q, P->node_kind, z);
    cplx *W = calloc((size_t)Nd * r, sizeof(cplx));
    cplx *Wn = calloc((size_t)Nd * r, sizeof(cplx));
    if (!W || !Wn) {
        free(W);
        free(Wn);
        return ORC_ERR_NOMEM;
    }
    /* init: every source adds its interpolation weights to its leaf box (sources in order) */
    {
        double x0[3], wx[3];
        tbox(P, 0, 0, x0, wx);
        for (int64_t j = 0; j < nsrc; ++j) {
            const double *yj = y + j * d;
            double cb[3], wb[3], yt[3];
            const int64_t B = leaf_of(P, 1, yj);
            sbox(P, 0, B, cb, wb);
            cplx src = kern(P, x0, yj) * g[j];
            for (int t = 0; t < r; ++t) {
                node(d, q, z, cb, wb, t, yt);
                W[B * r + t] += conj(kern(P, x0, yt)) * lag(d, q, z, cb, wb, t, yj) * src;
            }
        }
    }
    stages(P, &W, &Wn, -1, 0, z);
    /* final: each target from the weights of its leaf box */
    {
        double y0[3], wy[3];
        sbox(P, L, 0, y0, wy);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < ntgt; ++i) {
            const double *xi = x + i * d;
            double ca[3], wa[3], xt[3];
            const int64_t A = leaf_of(P, 0, xi);
            tbox(P, L, A, ca, wa);
            cplx acc = 0.0;
            for (int t = 0; t < r; ++t) {
                node(d, q, z, ca, wa, t, xt);
                acc += lag(d, q, z, ca, wa, t, xi) * conj(kern(P, xt, y0)) * W[A * r + t];
            }
            f[i] = kern(P, xi, y0) * acc;
        }
    }
    free(W);
    free(Wn);
    return ORC_OK;
}

int64_t orc_flat_from_morton(const orc_problem *P, int64_t mi) { return flat_from_morton(P, mi); }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
